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
constexpr int NMS_NT = 1024;         // cluster form: threads per CTA
constexpr int NMS_BATCH_NT = 512;    // one CTA per frame: three CTAs per SM for 640x480 frames
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
                                                           int32_t *nbr_t, uint8_t *cnt,
                                                           int *overflow) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npos) return;
    const int l = level_of(g.lev_pos, g.nlev, p);
    const int idx = p - g.lev_pos[l];
    const int u = idx / g.lev_nv[l], v = idx - (idx / g.lev_nv[l]) * g.lev_nv[l];
    const WinBox bp = window_box(g.lev_rx[l], g.lev_ry[l], u, v);
    int n = 0;
    for (int m = 0; m < g.nlev; m++) {
        if (!((g.pair_mask[l] >> m) & 1u)) continue;
        if (g.lev_nu[m] <= 0 || g.lev_nv[m] <= 0) continue;
        // candidate range on level m (one cell of slack on each side; the
        // IoU test below is exact)
        const double sx = __dmul_rn((double)CELL, g.lev_rx[m]), sy = __dmul_rn((double)CELL, g.lev_ry[m]);
        const double wm = (double)(CELL * WIN) * g.lev_rx[m], hm = (double)(CELL * WIN) * g.lev_ry[m];
        // reciprocals in FP32: a relative error of 1e-7 moves a bound by far
        // less than the slack
        const double isx = (double)(1.0f / (float)sx), isy = (double)(1.0f / (float)sy);
        int vlo = (int)floor((bp.x - wm) * isx) - 1, vhi = (int)ceil((bp.x + bp.w) * isx) + 1;
        int ulo = (int)floor((bp.y - hm) * isy) - 1, uhi = (int)ceil((bp.y + bp.h) * isy) + 1;
        vlo = max(vlo, 0); ulo = max(ulo, 0);
        vhi = min(vhi, g.lev_nv[m] - 1); uhi = min(uhi, g.lev_nu[m] - 1);
        for (int uu = ulo; uu <= uhi; uu++) {
            for (int vv = vlo; vv <= vhi; vv++) {
                const int q = g.lev_pos[m] + uu * g.lev_nv[m] + vv;
                if (q == p) continue;
                const WinBox bq = window_box(g.lev_rx[m], g.lev_ry[m], uu, vv);
                if (box_iou(bq, bp) > g.iou) {
                    if (n < MAXN) {
                        nbr[(size_t)n * g.npos + p] = q;     // slot-major
                        nbr_t[(size_t)p * MAXN + n] = q;     // position-major
                    }
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

// Three CTAs per SM with the workspace in shared memory (40 registers).
template <bool SM>
__global__ void __launch_bounds__(NMS_BATCH_NT, SM ? 3 : 2)
    nms_kernel(const FrameDesc *__restrict__ frames, int *flags) {
    extern __shared__ __align__(16) unsigned char nsm[];
    __shared__ int sh[NMS_BATCH_NT / 32 + 4];   // warp sums, total
    nms_frame<SM, NMS_BATCH_NT, false>(frames[blockIdx.x], nsm, flags, sh);
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

cudaError_t launch_nms_geometry(const GeomDesc &g, int32_t *nbr, int32_t *nbr_t, uint8_t *cnt,
                                int *overflow,
                                cudaStream_t stream) {
    if (g.npos <= 0) return cudaSuccess;
    nms_geometry_kernel<<<(g.npos + 255) / 256, 256, 0, stream>>>(g, nbr, nbr_t, cnt, overflow);
    return cudaGetLastError();
}

// ---- cluster form --------------------------------------------------------
// One frame's suppression spread over a thread-block cluster of C CTAs
// (C = 2..16, one CTA per SM): CTA r owns the contiguous position range
// [r*P, r*P + P), P = ceil(npos / C), and keeps the key high words, states
// and candidate lists of its range in its own shared memory.  A neighbour's
// key and state are read from the owning CTA's shared memory through the
// cluster's distributed shared memory (mapa + ld.shared::cluster), and a
// kept candidate marks its neighbours' suppression bits in their owners'
// shared memory with remote atomics (atom.shared::cluster.or).  Each CTA
// only writes the states of its own positions; the rounds are the same as
// in the one-CTA form, with a cluster barrier (release/acquire) closing each
// round, after which every CTA reads the cluster's count of undecided
// candidates from CTA 0.  Within a round a remote state or bit may be read
// stale, which can only make a candidate wait one more round: the kept set
// is the same for every C.  This gives one frame the shared memory and L2
// bandwidth of C SMs (a 1280x1024 frame has about 55K positions, 715 KB of
// state: more than one SM holds), and cuts the latency of small batches.
namespace {
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// shared::cluster address of `p` (a shared variable) in CTA `rank`
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t cl_ld_u8(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u8 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cl_or_u32(uint32_t addr, uint32_t v) {
    asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
}  // namespace

constexpr int NMS_MAX_CLUSTER = 16;
// per CTA: key high words, two lists (4 B each), the suppression bits, and
// state and resume slot (1 B each) of its owned positions
__host__ __device__ constexpr size_t nms_cluster_ws_bytes(int npos, int c) {
    return (size_t)((npos + c - 1) / c) * 14 + 4 * (size_t)(((npos + c - 1) / c + 31) / 32) + 64;
}

__global__ void __launch_bounds__(NMS_NT, 1) nms_cluster_kernel(const FrameDesc *__restrict__ frames,
                                                                int *flags) {
    extern __shared__ __align__(16) unsigned char nsm[];
    __shared__ int sh[NMS_NT / 32 + 4];
    __shared__ int s_cnt[2][NMS_MAX_CLUSTER];     // read in CTA 0: undecided per CTA
    __shared__ int s_kept[NMS_MAX_CLUSTER];       // read in CTA 0: kept per CTA
    __shared__ uint32_t s_rkhi[NMS_MAX_CLUSTER], s_rstate[NMS_MAX_CLUSTER], s_rsupp[NMS_MAX_CLUSTER];
    __shared__ int s_total;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int C = (int)cl_size(), rank = (int)cl_rank();
    const FrameDesc &fd = frames[cl_id()];
    const int npos = fd.npos;
    const int P = (npos + C - 1) / C;
    const int lo = min(rank * P, npos), nmine = min(lo + P, npos) - lo;
    uint32_t *khi = reinterpret_cast<uint32_t *>(nsm);                       // [P]
    int32_t *list[2] = {reinterpret_cast<int32_t *>(nsm) + P,                  // local indices
                        reinterpret_cast<int32_t *>(nsm) + 2 * (size_t)P};
    const int PW = (P + 31) / 32;
    volatile uint32_t *supp = reinterpret_cast<volatile uint32_t *>(nsm + (size_t)P * 12);   // bits [P]
    volatile uint8_t *state = nsm + (size_t)P * 12 + 4 * (size_t)PW;                        // [P]
    uint8_t *resume = nsm + (size_t)P * 13 + 4 * (size_t)PW;                                 // [P]
    const uint64_t *gkeys = fd.keys;
    const int32_t *__restrict__ nbr = fd.nbr;
    const int32_t *__restrict__ nbr_t = fd.nbr_t;
    const uint8_t *__restrict__ nbr_cnt = fd.nbr_cnt;
    int *s_n = sh + NMS_NT / 32 + 1;
    const float invP = P > 0 ? 1.0f / (float)P : 0.f;
    // owner CTA of position q (float estimate, corrected)
    auto owner = [&](int q) -> int {
        int o = __float2int_rz((float)q * invP);
        const int b = o * P;
        if (b > q) o--;
        else if (q - b >= P) o++;
        return o;
    };

    auto append = [&](bool flag, int i, int which) {
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (!m) return;
        int b0 = 0;
        if (lane == __ffs(m) - 1) b0 = atomicAdd(s_n + which, __popc(m));
        b0 = __shfl_sync(0xffffffffu, b0, __ffs(m) - 1);
        if (flag) list[which][b0 + __popc(m & ((1u << lane) - 1))] = i;
    };

    if (t < C) {
        s_rkhi[t] = cl_map(khi, t);
        s_rstate[t] = cl_map((const void *)state, t);
        s_rsupp[t] = cl_map((const void *)supp, t);
    }
    if (t == 0) { s_n[0] = 0; s_n[1] = 0; }
    for (int k = t; k < PW; k += NMS_NT) supp[k] = 0u;
    __syncthreads();
    for (int i0 = 0; i0 < nmine; i0 += NMS_NT) {
        const int i = i0 + t;
        uint32_t h = NMS_NOKEY;
        if (i < nmine) {
            // positions of levels that are not scanned carry no key
            if (nms_scanned(fd, lo + i)) h = (uint32_t)(__ldg(gkeys + lo + i) >> 32);
            khi[i] = h;
            state[i] = h != NMS_NOKEY ? NMS_ALIVE : NMS_DEAD;
            resume[i] = 0;
        }
        append(h != NMS_NOKEY, i, 0);
    }
    cl_sync();   // every CTA's keys, states and bits are initialised

    int cur = 0, round = 0;
    for (; round <= npos; round++) {
        const int n_cur = s_n[cur];
        for (int i0 = 0; i0 < n_cur; i0 += NMS_NT) {
            const int i = i0 + t;
            bool undecided = false, kept = false;
            int li = -1, p = -1;
            if (i < n_cur) {
                li = list[cur][i];
                p = lo + li;
                const uint32_t hp = khi[li];
                const int n = __ldg(nbr_cnt + p);
                bool dead = (supp[li >> 5] >> (li & 31)) & 1u, wait = false;
                const int r0 = resume[li];
                int settled = r0;
                for (int s0 = r0; s0 < n && !dead && !wait; s0 += 4) {
                    int q[4];
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        q[k] = s0 + k < n ? __ldg(nbr + (size_t)(s0 + k) * npos + p) : -1;
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if (q[k] < 0 || dead || wait) continue;
                        const int o = owner(q[k]);
                        const int lq = q[k] - o * P;
                        const uint32_t hq = cl_ld_u32(s_rkhi[o] + 4u * (uint32_t)lq);
                        uint32_t sq = NMS_DEAD;   // not above p: settled like a suppressed one
                        if (hq != NMS_NOKEY &&
                            (hq != hp ? hq < hp : __ldg(gkeys + q[k]) < __ldg(gkeys + p)))
                            sq = cl_ld_u8(s_rstate[o] + (uint32_t)lq);
                        if (sq == NMS_KEPT) dead = true;
                        else if (sq == NMS_ALIVE) wait = true;
                        else settled = s0 + k + 1;
                    }
                }
                if (dead) {
                    state[li] = NMS_DEAD;
                } else if (!wait) {
                    state[li] = NMS_KEPT;
                    kept = true;
                } else {
                    undecided = true;
                    resume[li] = (uint8_t)settled;
                }
            }
            // each kept candidate marks all its neighbours' bits in their
            // owners' shared memory, the warp's lanes splitting the slots
            for (unsigned km = __ballot_sync(0xffffffffu, kept); km; km &= km - 1) {
                const int pk = __shfl_sync(0xffffffffu, p, __ffs(km) - 1);
                const int nk = __ldg(nbr_cnt + pk);
                for (int s = lane; s < nk; s += 32) {
                    const int q = __ldg(nbr_t + (size_t)pk * MAXN + s);
                    const int o = owner(q);
                    const int lq = q - o * P;
                    cl_or_u32(s_rsupp[o] + 4u * (uint32_t)(lq >> 5), 1u << (lq & 31));
                }
            }
            append(undecided, li, cur ^ 1);
        }
        __syncthreads();
        // publish this CTA's undecided count to CTA 0 (slot by round parity:
        // slot r&1 is rewritten two rounds later, after every CTA read it)
        if (t == 0) cl_st_u32(cl_map(&s_cnt[round & 1][rank], 0), (uint32_t)s_n[cur ^ 1]);
        cl_sync();
        if (wid == 0) {
            int c = lane < C ? (int)cl_ld_u32(cl_map(&s_cnt[round & 1][lane], 0)) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0) {
                s_total = c;
                s_n[cur] = 0;     // the list just processed becomes next round's output
            }
        }
        __syncthreads();
        cur ^= 1;
        if (s_total == 0) break;
    }

    // kept positions in position order: CTA r's before CTA r+1's
    int *s_warp = sh;
    const int per = (nmine + NMS_NT - 1) / NMS_NT;
    const int beg = min(t * per, nmine), end = min(beg + per, nmine);
    int mine = 0;
    for (int i = beg; i < end; i++) mine += state[i] == NMS_KEPT;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int k = 0; k < NMS_NT / 32; k++) {
            const int x = s_warp[k];
            s_warp[k] = run;
            run += x;
        }
        cl_st_u32(cl_map(&s_kept[rank], 0), (uint32_t)run);
    }
    cl_sync();
    if (wid == 0) {
        const int c = lane < C ? (int)cl_ld_u32(cl_map(&s_kept[lane], 0)) : 0;
        int before = lane < rank ? c : 0, all = c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if (lane == 0) { sh[NMS_NT / 32] = before; s_total = all; }
    }
    __syncthreads();
    const int total = s_total;
    int pos = sh[NMS_NT / 32] + s_warp[wid] + incl - mine;
    for (int i = beg; i < end; i++) {
        if (state[i] != NMS_KEPT) continue;
        if (pos < fd.out_cap) {
            const uint64_t k = __ldg(gkeys + lo + i);
            const int l = key_level(k);
            const int u = key_u(k), v = key_v(k);
            const WinBox b = window_box(fd.lev_rx[l], fd.lev_ry[l], u, v);
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
    if (rank == 0 && t == 0) {
        *fd.count = total;
        if (total > fd.out_cap) atomicOr(flags, 1);
        atomicMax(flags + 1, round + 1);
    }
    cl_sync();   // no CTA leaves while another may still read its shared memory
}

namespace {
int g_nsm = 0;             // SM count of the device
int g_cluster_max = -1;    // largest cluster size the device can run (1 = none)

int nms_cluster_max() {
    if (g_cluster_max >= 0) return g_cluster_max;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    g_cluster_max = 1;
    if (cudaFuncSetAttribute(nms_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             NMS_SMEM_MAX) != cudaSuccess ||
        cudaFuncSetAttribute(nms_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
        cudaGetLastError();
        return g_cluster_max;
    }
    for (int c = NMS_MAX_CLUSTER; c >= 2; c >>= 1) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(NMS_NT);
        cfg.dynamicSmemBytes = NMS_SMEM_MAX;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, nms_cluster_kernel, &cfg) == cudaSuccess && n > 0) {
            g_cluster_max = c;
            break;
        }
        cudaGetLastError();
    }
    return g_cluster_max;
}
}  // namespace

// Cluster size for a batch: `request` 1 = one CTA per frame, 2..16 = that
// size, 0 = automatic -- spread the batch over the SMs (SMs / frames, a
// power of two), and at least the size whose per-CTA state fits in shared
// memory.  Returns 1 for the one-CTA form.
int nms_cluster_size(int nframes, int max_npos, int request) {
    const int cmax = nms_cluster_max();
    if (cmax < 2 || request == 1 || nframes <= 0) return 1;
    int c;
    if (request >= 2) {
        c = request > cmax ? cmax : request;
    } else {
        const int want = g_nsm / nframes;
        c = 1;
        while (c * 2 <= want && c * 2 <= cmax) c *= 2;
        if ((nms_ws_bytes(max_npos, true) > (size_t)NMS_SMEM_MAX || max_npos > NMS_SMEM_MAX_NPOS) &&
            c < 2)
            c = 2;
    }
    while (c < cmax && nms_cluster_ws_bytes(max_npos, c) > (size_t)NMS_SMEM_MAX) c *= 2;
    if (c >= 2 && nms_cluster_ws_bytes(max_npos, c) > (size_t)NMS_SMEM_MAX) return 1;
    return c;
}

cudaError_t launch_nms(const FrameDesc *frames, int nframes, int max_npos, int *flags,
                       cudaStream_t stream, int cluster_request) {
    if (nframes <= 0) return cudaSuccess;
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(nms_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, NMS_SMEM_MAX);
        if (e == cudaSuccess)   // all of the unified L1 as shared memory: three frames per SM
            e = cudaFuncSetAttribute(nms_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    const int c = nms_cluster_size(nframes, max_npos, cluster_request);
    if (c >= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(nframes * c);
        cfg.blockDim = dim3(NMS_NT);
        cfg.dynamicSmemBytes = nms_cluster_ws_bytes(max_npos, c);
        cfg.stream = stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, nms_cluster_kernel, frames, flags);
    }
    const size_t ws = nms_ws_bytes(max_npos, true);
    if (ws <= (size_t)NMS_SMEM_MAX && max_npos <= NMS_SMEM_MAX_NPOS)
        nms_kernel<true><<<nframes, NMS_BATCH_NT, ws, stream>>>(frames, flags);
    else
        nms_kernel<false><<<nframes, NMS_BATCH_NT, 0, stream>>>(frames, flags);
    return cudaGetLastError();
}

}  // namespace hogk
