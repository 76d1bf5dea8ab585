// k_corr.cu -- multi-filter correlation, threshold and candidate keys
// (Section 4.1.1: linear classification filter and detection; Section 5.1,
// classifier and detection kernels, fused here).
//
// score_f(u, v) = sum_{a<10, b<10, c<31} W_f[a][b][c] * feat[u+a][v+b][c]
// for every window (u, v) of a level and every filter f.  A window is a
// candidate when its best score over the filters is strictly greater than
// the threshold; its suppression key ranks (score desc, level, filter, u, v).
// Windows at one position share one box, so only the best filter of a
// position can survive greedy suppression; the key therefore carries the
// best filter only (equal scores: the lowest filter index).
//
// GB300 design: FP32 FMA on the CUDA cores, bound by the FMA pipe.
//  - Each warp owns one tile of 128 windows, shaped 8x16, 4x32 or 16x8 per
//    level (the host picks the shape that pads the level's window grid
//    least); a lane owns 4 consecutive windows of one row for all filters,
//    so it keeps 4 x NF accumulators and uses every feature it loads for 4
//    windows x NF filters.  The four warps of a CTA are independent (no
//    block barrier).
//  - Features stream in half-chunks of 4 channels (one float4 per cell of
//    the internal layout [4][cy][cx][8]): the warp copies the
//    (TU+9) x (TV+9)-cell region of the next half-chunk into shared memory
//    with cp.async while it computes on the current one (double buffer).
//    The region's row stride TV+9 is odd, so the float4 loads of a
//    quarter-warp (consecutive rows, or rows x column groups) fall on
//    distinct bank groups.
//  - For a filter row a, a lane loads the 13 float4 of its feature row once
//    and slides over the 10 filter columns in registers.  Filter weights are
//    read with warp-uniform loads through L1 (62 KB for five filters).
#include "hog_internal.cuh"

namespace hogk {

namespace {
constexpr int NT = 32 * CORR_WARPS;
constexpr int WPT = 4;                  // windows per lane
constexpr int BUF4 = 544;               // float4 per region buffer (max 13 x 41 = 533)
constexpr size_t SMEM = sizeof(float4) * BUF4 * 2 * CORR_WARPS;   // 69,632 bytes
}  // namespace

template <int NF>
__global__ void __launch_bounds__(NT, 3) corr_kernel(const LevelDesc *__restrict__ descs,
                                                     const Job *__restrict__ jobs, int njobs,
                                                     const float *__restrict__ wchunks,
                                                     int nf_real, float threshold) {
    extern __shared__ float4 sm4[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int jid = blockIdx.x * CORR_WARPS + w;
    if (jid >= njobs) return;
    float4 *buf0 = sm4 + (size_t)w * 2 * BUF4;
    const Job jb = jobs[jid];
    const LevelDesc &d = descs[jb.desc];
    const int shape = (jb.tile >> 28) & 3, tile = jb.tile & 0x0fffffff;
    const int TU = corr_tu(shape), TV = corr_tv(shape);
    const int RU = TU + WIN - 1, RV = TV + WIN - 1;
    const int ntv = (d.nv + TV - 1) / TV;
    const int u0 = (tile / ntv) * TU, v0 = (tile % ntv) * TV;
    const int lr = lane % TU, lc = (lane / TU) * WPT;    // window row / first column in tile

    const float4 *feat4 = reinterpret_cast<const float4 *>(d.feat);
    const size_t plane4 = (size_t)d.cy * d.cx * 2;       // float4 per chunk plane
    const float4 *w4 = reinterpret_cast<const float4 *>(wchunks);

    // copy half-chunk h (chunk h/2, channels 4*(h&1)..+3) of the tile region
    auto stage = [&](int h, float4 *dst) {
        const float4 *src = feat4 + (size_t)(h >> 1) * plane4 + (h & 1);
        for (int k = lane; k < RU * RV; k += 32) {
            const int rr = k / RV, cc = k - rr * RV;
            const int i = u0 + rr, j = v0 + cc;
            const bool ok = i < d.cy && j < d.cx;
            cp_async16_zfill(dst + k, ok ? (const void *)(src + ((size_t)i * d.cx + j) * 2)
                                         : (const void *)src, ok);
        }
        cp_async_commit();
    };

    float acc[WPT][NF];
#pragma unroll
    for (int j = 0; j < WPT; j++)
#pragma unroll
        for (int f = 0; f < NF; f++) acc[j][f] = 0.0f;

    stage(0, buf0);
#pragma unroll 1
    for (int h = 0; h < 2 * NCHUNK; h++) {
        float4 *cur = buf0 + (h & 1) * BUF4;
        if (h + 1 < 2 * NCHUNK) {
            stage(h + 1, buf0 + ((h + 1) & 1) * BUF4);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        __syncwarp();
        const int ch = h >> 1, c4 = h & 1;
        const float4 *wch = w4 + (size_t)ch * NF * 200 + c4;
#pragma unroll 1
        for (int a = 0; a < WIN; a++) {
            const float4 *frow = cur + (lr + a) * RV + lc;
            float4 fv[WPT + WIN - 1];
#pragma unroll
            for (int j = 0; j < WPT + WIN - 1; j++) fv[j] = frow[j];
#pragma unroll
            for (int b = 0; b < WIN; b++) {
                float4 wv[NF];
#pragma unroll
                for (int f = 0; f < NF; f++) wv[f] = __ldg(wch + ((f * WIN + a) * WIN + b) * 2);
#pragma unroll
                for (int j = 0; j < WPT; j++) {
                    const float4 x = fv[j + b];
#pragma unroll
                    for (int f = 0; f < NF; f++) {
                        float s = acc[j][f];
                        s = fmaf(wv[f].x, x.x, s);
                        s = fmaf(wv[f].y, x.y, s);
                        s = fmaf(wv[f].z, x.z, s);
                        s = fmaf(wv[f].w, x.w, s);
                        acc[j][f] = s;
                    }
                }
            }
        }
        __syncwarp();   // every lane is done with `cur` before it is refilled
    }

    const int u = u0 + lr;
    if (u >= d.nu) return;
#pragma unroll
    for (int j = 0; j < WPT; j++) {
        const int v = v0 + lc + j;
        if (v >= d.nv) break;
        float best = acc[j][0];
        int fb = 0;
#pragma unroll
        for (int f = 1; f < NF; f++)
            if (f < nf_real && acc[j][f] > best) { best = acc[j][f]; fb = f; }
        if (d.scores_user) {
#pragma unroll
            for (int f = 0; f < NF; f++)
                if (f < nf_real)
                    d.scores_user[((size_t)f * d.nu + u) * d.nv + v] = acc[j][f];
        }
        if (d.keys)
            d.keys[(size_t)u * d.nv + v] =
                (d.scan && best > threshold) ? make_key(best, d.level, fb, u, v) : KEY_NONE;
    }
}

template <int NF>
static cudaError_t launch_corr_t(const LevelDesc *descs, const Job *jobs, int njobs,
                                 const float *wchunks, int nf_real, float threshold,
                                 cudaStream_t stream) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(corr_kernel<NF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (njobs <= 0) return cudaSuccess;
    const int grid = (njobs + CORR_WARPS - 1) / CORR_WARPS;
    corr_kernel<NF><<<grid, NT, SMEM, stream>>>(descs, jobs, njobs, wchunks, nf_real, threshold);
    return cudaGetLastError();
}

cudaError_t launch_corr(const LevelDesc *descs, const Job *jobs, int njobs,
                        const float *wchunks, int nf_kernel, int nf_real, float threshold,
                        cudaStream_t stream) {
    switch (nf_kernel) {
    case 1: return launch_corr_t<1>(descs, jobs, njobs, wchunks, nf_real, threshold, stream);
    case 5: return launch_corr_t<5>(descs, jobs, njobs, wchunks, nf_real, threshold, stream);
    case 8: return launch_corr_t<8>(descs, jobs, njobs, wchunks, nf_real, threshold, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hogk
