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
#include "hog_internal.cuh"

namespace hogk {

namespace {
constexpr uint8_t ST_DEAD = 0, ST_ALIVE = 1, ST_KEPT = 2;
constexpr int NMS_NT = 512;
constexpr int NMS_SMEM_MAX = 200 * 1024;   // dynamic shared memory for keys and states

struct Box {
    double x, y, w, h;
};

__device__ __forceinline__ Box window_box(int W0, int H0, int Wl, int Hl, int u, int v) {
    const double rx = __ddiv_rn((double)W0, (double)Wl);
    const double ry = __ddiv_rn((double)H0, (double)Hl);
    Box b;
    b.x = __dmul_rn((double)(CELL * v), rx);
    b.y = __dmul_rn((double)(CELL * u), ry);
    b.w = __dmul_rn((double)(CELL * WIN), rx);
    b.h = __dmul_rn((double)(CELL * WIN), ry);
    return b;
}

__device__ __forceinline__ double box_iou(const Box &a, const Box &b) {
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
    const Box bp = window_box(g.W, g.H, g.lev_w[l], g.lev_h[l], u, v);
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
                const Box bq = window_box(g.W, g.H, g.lev_w[m], g.lev_h[m], uu, vv);
                if (box_iou(bq, bp) > g.iou) {
                    if (n < MAXN) nbr[(size_t)p * MAXN + n] = q;
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

// MODE 2: keys and states in shared memory; 1: states only; 0: both global.
template <int MODE>
__global__ void __launch_bounds__(NMS_NT) nms_kernel(const FrameDesc *__restrict__ frames,
                                                     int *flags) {
    extern __shared__ __align__(16) unsigned char nsm[];
    const FrameDesc &fd = frames[blockIdx.x];
    const int t = threadIdx.x;
    const int npos = fd.npos;
    uint64_t *skeys = reinterpret_cast<uint64_t *>(nsm);
    uint8_t *sstate = MODE == 2 ? nsm + (size_t)npos * 8 : nsm;
    volatile uint8_t *state = MODE >= 1 ? sstate : fd.state;
    const uint64_t *__restrict__ gkeys = fd.keys;
    const uint64_t *keys = MODE == 2 ? skeys : gkeys;
    const int32_t *__restrict__ nbr = fd.nbr;
    const uint8_t *__restrict__ nbr_cnt = fd.nbr_cnt;

    for (int p = t; p < npos; p += NMS_NT) {
        const uint64_t k = __ldg(gkeys + p);
        if (MODE == 2) skeys[p] = k;
        state[p] = k != KEY_NONE ? ST_ALIVE : ST_DEAD;
    }
    __syncthreads();

    // rounds; each one decides at least the best undecided candidate
    int round = 0;
    for (; round <= npos; round++) {
        int undecided = 0;
        for (int p = t; p < npos; p += NMS_NT) {
            if (state[p] != ST_ALIVE) continue;
            const uint64_t kp = keys[p];
            const int n = __ldg(nbr_cnt + p);
            const int32_t *nb = nbr + (size_t)p * MAXN;
            bool dead = false, wait = false;
            for (int s = 0; s < n; s++) {
                const int q = __ldg(nb + s);
                if (keys[q] >= kp) continue;   // ranked below p (or no candidate)
                const uint8_t sq = state[q];
                if (sq == ST_KEPT) { dead = true; break; }
                if (sq == ST_ALIVE) wait = true;
            }
            if (dead) state[p] = ST_DEAD;
            else if (!wait) state[p] = ST_KEPT;
            else undecided = 1;
        }
        if (!__syncthreads_or(undecided)) break;
    }

    // compact kept positions in position order
    __shared__ int wsum[NMS_NT / 32];
    __shared__ int total;
    const int per = (npos + NMS_NT - 1) / NMS_NT;
    const int beg = min(t * per, npos), end = min(beg + per, npos);
    int mine = 0;
    for (int p = beg; p < end; p++) mine += state[p] == ST_KEPT;
    int incl = mine;
    const int lane = t & 31, wid = t >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int k = 0; k < NMS_NT / 32; k++) {
            const int x = wsum[k];
            wsum[k] = run;
            run += x;
        }
        total = run;
    }
    __syncthreads();
    int pos = wsum[wid] + incl - mine;
    for (int p = beg; p < end; p++) {
        if (state[p] != ST_KEPT) continue;
        if (pos < fd.out_cap) {
            const uint64_t k = keys[p];
            const int l = key_level(k);
            const int u = key_u(k), v = key_v(k);
            const Box b = window_box(fd.W, fd.H, fd.lev_w[l], fd.lev_h[l], u, v);
            hog_det det;
            det.frame = fd.frame;
            det.level = l;
            det.filter = key_filter(k);
            det.u = u;
            det.v = v;
            det.score = key_score(k);
            det.x = b.x; det.y = b.y; det.w = b.w; det.h = b.h;
            fd.out[pos] = det;
        }
        pos++;
    }
    if (t == 0) {
        *fd.count = total;
        if (total > fd.out_cap) atomicOr(flags, 1);
        atomicMax(flags + 1, round + 1);
    }
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
        cudaError_t e = cudaFuncSetAttribute(nms_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             NMS_SMEM_MAX);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(nms_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     NMS_SMEM_MAX);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const size_t both = (size_t)max_npos * 9 + 16, states = (size_t)max_npos + 16;
    if (both <= (size_t)NMS_SMEM_MAX)
        nms_kernel<2><<<nframes, NMS_NT, both, stream>>>(frames, flags);
    else if (states <= (size_t)NMS_SMEM_MAX)
        nms_kernel<1><<<nframes, NMS_NT, states, stream>>>(frames, flags);
    else
        nms_kernel<0><<<nframes, NMS_NT, 0, stream>>>(frames, flags);
    return cudaGetLastError();
}

}  // namespace hogk
