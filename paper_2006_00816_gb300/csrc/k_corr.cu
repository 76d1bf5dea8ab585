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
//  - CTA = 128 threads, tile = 16 x 32 windows; each warp owns 8 x 16, each
//    thread 4 consecutive windows of one row for all filters, so a thread
//    keeps 4 x NF accumulators and reuses every staged feature for up to 4
//    windows x NF filters.
//  - Features come in 8-channel chunks (internal layout [4][cy][cx][8]):
//    the CTA stages the 25 x 41-cell region of a chunk in shared memory
//    with a 16-byte row pad (row stride 83 float4), which makes the
//    per-lane float4 loads of a quarter-warp (8 consecutive rows) hit 8
//    different bank groups.  The filter chunk is staged beside it and read
//    with uniform (broadcast) float4 loads.
//  - For a filter row a and 4 channels, a thread loads the 13 float4 of its
//    feature row once and slides over the 10 filter columns in registers.
#include "hog_internal.cuh"

namespace hogk {

namespace {
constexpr int NT = 128;
constexpr int RU = CORR_TU + WIN - 1;        // 25 staged rows
constexpr int RV = CORR_TV + WIN - 1;        // 41 staged columns
constexpr int ROW4 = RV * 2 + 1;             // 83 float4 per staged row (incl. pad)
constexpr int WPT = 4;                       // windows per thread

template <int NF>
constexpr size_t corr_smem() {
    return sizeof(float4) * ((size_t)RU * ROW4 + (size_t)NF * WIN * WIN * 2);
}
}  // namespace

template <int NF>
__global__ void __launch_bounds__(NT, 3) corr_kernel(const LevelDesc *__restrict__ descs,
                                                     const Job *__restrict__ jobs,
                                                     const float *__restrict__ wchunks,
                                                     int nf_real, float threshold) {
    extern __shared__ float4 sm4[];
    float4 *fS = sm4;                     // [RU][ROW4]
    float4 *wS = sm4 + RU * ROW4;         // [NF][10][10][2]

    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int ntv = (d.nv + CORR_TV - 1) / CORR_TV;
    const int u0 = (jb.tile / ntv) * CORR_TU, v0 = (jb.tile % ntv) * CORR_TV;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int lr = (w >> 1) * 8 + (lane & 7);           // window row in tile
    const int lc = (w & 1) * 16 + (lane >> 3) * WPT;     // first window column in tile

    float acc[WPT][NF];
#pragma unroll
    for (int j = 0; j < WPT; j++)
#pragma unroll
        for (int f = 0; f < NF; f++) acc[j][f] = 0.0f;

    const size_t plane = (size_t)d.cy * d.cx * CHUNK;
    for (int ch = 0; ch < NCHUNK; ch++) {
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(d.feat + ch * plane);
        for (int k = t; k < RU * RV * 2; k += NT) {
            const int rr = k / (RV * 2);
            const int rem = k - rr * RV * 2;
            const int cc = rem >> 1, half = rem & 1;
            const int i = u0 + rr, j = v0 + cc;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < d.cy && j < d.cx) v = __ldg(src + ((size_t)i * d.cx + j) * 2 + half);
            fS[rr * ROW4 + cc * 2 + half] = v;
        }
        const float4 *wsrc = reinterpret_cast<const float4 *>(wchunks) + (size_t)ch * NF * 200;
        for (int k = t; k < NF * 200; k += NT) wS[k] = __ldg(wsrc + k);
        __syncthreads();

#pragma unroll 1
        for (int a = 0; a < WIN; a++) {
            const float4 *frow = fS + (lr + a) * ROW4 + lc * 2;
#pragma unroll 1
            for (int c4 = 0; c4 < 2; c4++) {
                float4 fv[WPT + WIN - 1];
#pragma unroll
                for (int j = 0; j < WPT + WIN - 1; j++) fv[j] = frow[j * 2 + c4];
#pragma unroll
                for (int b = 0; b < WIN; b++) {
                    float4 wv[NF];
#pragma unroll
                    for (int f = 0; f < NF; f++) wv[f] = wS[((f * WIN + a) * WIN + b) * 2 + c4];
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
        }
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
                                             (int)corr_smem<NF>());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (njobs <= 0) return cudaSuccess;
    corr_kernel<NF><<<njobs, NT, corr_smem<NF>(), stream>>>(descs, jobs, wchunks, nf_real,
                                                            threshold);
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
