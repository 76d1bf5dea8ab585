// k_nms.cu -- non-maximum suppression on the device (Section 4.1.1, last
// step; the paper runs it on the host because a trained detector yields few
// windows per face, Section 5.1).  Random or weak filters pass a large share
// of all windows, so here it runs on the GPU.
//
// Definition (greedy): rank the candidates of a frame by (score desc, level,
// filter, u, v); walk them in rank order and keep a box unless a kept box
// overlaps it with IoU > nms_iou.  Boxes are the windows (8v, 8u, 80, 80)
// scaled to the frame by W0/Wl, H0/Hl, in FP64.
//
// Parallel form: the greedy result is the unique set K with "p in K iff no
// member of K ranked above p overlaps p".  It is reached by rounds in which
// every undecided candidate p looks at its higher-ranked overlapping
// neighbours: one of them kept -> p suppressed; all of them suppressed ->
// p kept; otherwise p waits.  The best undecided candidate always decides,
// so the rounds terminate; decisions are final, so threads may read a
// neighbour's state while it is being updated within a round.
//
// Overlap does not depend on content, only on the frame size: a geometry
// kernel lists, once per frame size, each window position's neighbours with
// IoU > nms_iou, computed in FP64 with explicitly rounded operations (no
// fused multiply-add), so the test matches a host evaluation of the same
// formula bit for bit.
#include "hog_stages.cuh"

namespace hogk {

namespace {
constexpr int NMS_NT = 1024;
constexpr int NMS_SMEM_MAX = 200 * 1024;   // dynamic shared memory for keys and states

__device__ __forceinline__ double box_iou(const WinBox &a, const WinBox &b) {
    const double ix1 = a.x > b.x ? a.x : b.x;
    const double ax2 = __dadd_rn(a.x, a.w), bx2 = __dadd_rn(b.x, b.w);
    const double ix2 = ax2 < bx2 ? ax2 : bx2;
    const double iy1 = a.y > b.y ? a.y : b.y;
    const double ay2 = __dadd_rn(a.y, a.h), by2 = __dadd_rn(b.y, b.h);
    const double iy2 = ay2 < by2 ? ay2 : by2;
    const double iw = __dsub_rn(ix2, ix1), ih = __dsub_rn(iy2, iy1);
    if (iw <= 0.0 || ih <= 0.0) return 0.0;
    const double inter = __dmul_rn(iw, ih);
    const double uni = __dsub_rn(__dadd_rn(__dmul_rn(a.w, a.h), __dmul_rn(b.w, b.h)), inter);
    return __ddiv_rn(inter, uni);
}

__device__ __forceinline__ int level_of(const int32_t *lev_pos, int nlev, int p) {
    int l = 0;
    while (l + 1 < nlev && p >= lev_pos[l + 1]) l++;
    return l;
}
}  // namespace

__global__ void __launch_bounds__(256) nms_geometry_kernel(GeomDesc g, int32_t *nbr,
                                                           uint8_t *cnt, int *overflow) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npos) return;
    const int l = level_of(g.lev_pos, g.nlev, p);
    const int idx = p - g.lev_pos[l];
    const int u = idx / g.lev_nv[l], v = idx - (idx / g.lev_nv[l]) * g.lev_nv[l];
    const WinBox bp = window_box(g.W, g.H, g.lev_w[l], g.lev_h[l], u, v);
    int n = 0;
    for (int m = 0; m < g.nlev; m++) {
        if (!((g.pair_mask[l] >> m) & 1u)) continue;
        if (g.lev_nu[m] <= 0 || g.lev_nv[m] <= 0) continue;
        const double sx = __dmul_rn((double)CELL, __ddiv_rn((double)g.W, (double)g.lev_w[m]));
        const double sy = __dmul_rn((double)CELL, __ddiv_rn((double)g.H, (double)g.lev_h[m]));
        const double wm = (double)(CELL * WIN) / ((double)g.lev_w[m]) * (double)g.W;
        const double hm = (double)(CELL * WIN) / ((double)g.lev_h[m]) * (double)g.H;
        int vlo = (int)floor((bp.x - wm) / sx) - 1, vhi = (int)ceil((bp.x + bp.w) / sx) + 1;
        int ulo = (int)floor((bp.y - hm) / sy) - 1, uhi = (int)ceil((bp.y + bp.h) / sy) + 1;
        vlo = max(vlo, 0); ulo = max(ulo, 0);
        vhi = min(vhi, g.lev_nv[m] - 1); uhi = min(uhi, g.lev_nu[m] - 1);
        for (int uu = ulo; uu <= uhi; uu++) {
            for (int vv = vlo; vv <= vhi; vv++) {
                const int q = g.lev_pos[m] + uu * g.lev_nv[m] + vv;
                if (q == p) continue;
                const WinBox bq = window_box(g.W, g.H, g.lev_w[m], g.lev_h[m], uu, vv);
                if (box_iou(bq, bp) > g.iou) {
                    if (n < MAXN) nbr[(size_t)n * g.npos + p] = q;   // slot-major
                    n++;
                }
            }
        }
    }
    if (n > MAXN) {
        atomicOr(overflow, 1);
        n = MAXN;
    }
    cnt[p] = (uint8_t)n;
}

template <bool SM>
__global__ void __launch_bounds__(NMS_NT) nms_kernel(const FrameDesc *__restrict__ frames,
                                                     int *flags) {
    extern __shared__ __align__(16) unsigned char nsm[];
    __shared__ int sh[NMS_NT / 32 + 4];   // warp sums, total, two list sizes
    nms_frame<SM, NMS_NT, false>(frames[blockIdx.x], nsm, flags, sh);
}

__global__ void __launch_bounds__(256) pack_kernel(const hog_det *__restrict__ dets, int per_frame,
                                                   const int32_t *__restrict__ counts, int nframes,
                                                   hog_det *out, int out_cap, int32_t *counts_out) {
    const int i = blockIdx.x;
    __shared__ int off_s;
    if (threadIdx.x < 32) {
        int s = 0;
        for (int k = threadIdx.x; k < i; k += 32) s += min(counts[k], per_frame);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) off_s = s;
    }
    __syncthreads();
    const int off = off_s;
    const int n = min(counts[i], per_frame);
    // copy as 8-byte words (hog_det is 56 bytes = 7 words)
    const unsigned long long *src =
        reinterpret_cast<const unsigned long long *>(dets + (size_t)i * per_frame);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(out + off);
    const int nw = max(0, min(n, out_cap - off)) * 7;
    for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
    if (threadIdx.x == 0) counts_out[i] = counts[i];
}

cudaError_t launch_pack(const hog_det *dets, int per_frame, const int32_t *counts, int nframes,
                        hog_det *out, int out_cap, int32_t *counts_out, cudaStream_t stream) {
    if (nframes <= 0) return cudaSuccess;
    pack_kernel<<<nframes, 256, 0, stream>>>(dets, per_frame, counts, nframes, out, out_cap,
                                             counts_out);
    return cudaGetLastError();
}

cudaError_t launch_nms_geometry(const GeomDesc &g, int32_t *nbr, uint8_t *cnt, int *overflow,
                                cudaStream_t stream) {
    if (g.npos <= 0) return cudaSuccess;
    nms_geometry_kernel<<<(g.npos + 255) / 256, 256, 0, stream>>>(g, nbr, cnt, overflow);
    return cudaGetLastError();
}

cudaError_t launch_nms(const FrameDesc *frames, int nframes, int max_npos, int *flags,
                       cudaStream_t stream) {
    if (nframes <= 0) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(nms_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, NMS_SMEM_MAX);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const size_t ws = nms_ws_bytes(max_npos);
    if (ws <= (size_t)NMS_SMEM_MAX)
        nms_kernel<true><<<nframes, NMS_NT, ws, stream>>>(frames, flags);
    else
        nms_kernel<false><<<nframes, NMS_NT, 0, stream>>>(frames, flags);
    return cudaGetLastError();
}

}  // namespace hogk
