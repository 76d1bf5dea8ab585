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
#include <algorithm>

#include "hog_stages.cuh"

namespace hogk {

namespace {
constexpr int NMS_NT = 1024;         // cluster form: threads per CTA
constexpr int NMS_BATCH_NT = 512;    // one CTA per frame: three CTAs per SM for 640x480 frames
constexpr int NMS_KEYS_NT = 1024;    // one CTA per frame, key words in shared memory
// Automatic cluster size: clusters only when a frame would get at least this
// many SMs (on 152 SMs: up to 19 frames).  At 51-77 frames per batch one CTA
// per frame measured 1.3-1.8x faster than clusters of 2 or 4.
constexpr int NMS_AUTO_CLUSTER_MIN = 8;

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

// One CTA per frame: three per SM with the whole workspace in shared memory
// (40 registers); one per SM of 1024 threads with the key words alone in
// shared memory; two per SM with everything in global memory.
template <int WS>
__global__ void __launch_bounds__(WS == NMS_WS_KEYS ? NMS_KEYS_NT : NMS_BATCH_NT,
                                  WS == NMS_WS_SMEM ? 3 : (WS == NMS_WS_KEYS ? 1 : 2))
    nms_kernel(const FrameDesc *__restrict__ frames, int *flags) {
    constexpr int NT = WS == NMS_WS_KEYS ? NMS_KEYS_NT : NMS_BATCH_NT;
    extern __shared__ __align__(16) unsigned char nsm[];
    __shared__ int sh[NT / 32 + 4];   // warp sums, total
    nms_frame<WS, NT, false>(frames[blockIdx.x], nsm, flags, sh);
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
    // copy as 8-byte words (hog_det is 56 bytes = 7 words); the gridDim.y
    // CTAs of a frame split its words (the output may be host memory, where
    // one CTA's stores alone would be latency-bound)
    const unsigned long long *src =
        reinterpret_cast<const unsigned long long *>(dets + (size_t)i * per_frame);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(out + off);
    const int nw = max(0, min(n, out_cap - off)) * 7;
    const int per = (nw + gridDim.y - 1) / gridDim.y;
    const int k0 = blockIdx.y * per, k1 = min(nw, k0 + per);
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) dst[k] = src[k];
    if (threadIdx.x == 0 && blockIdx.y == 0) counts_out[i] = counts[i];
}

cudaError_t launch_pack(const hog_det *dets, int per_frame, const int32_t *counts, int nframes,
                        hog_det *out, int out_cap, int32_t *counts_out, cudaStream_t stream) {
    if (nframes <= 0) return cudaSuccess;
    const int split = std::max(1, std::min(16, 64 / nframes));   // CTAs per frame for small batches
    pack_kernel<<<dim3(nframes, split), 256, 0, stream>>>(dets, per_frame, counts, nframes, out, out_cap,
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
__device__ __forceinline__ void cl_st_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
}  // namespace

constexpr int NMS_MAX_CLUSTER = 16;
constexpr int NMS_MASK_WORDS = MAXN / 32;   // 192 neighbour slots: six 32-bit words
// Higher-ranked neighbours a CTA caches per owned candidate (cluster form,
// mode 2); a candidate with more keeps the rest in its global above-mask.
constexpr int NMS_LIST = 48;
constexpr int NMS_WS_WORDS = 8 + NMS_LIST / 2;   // global workspace per position (cluster form)
static_assert(NMS_WS_WORDS == HOG_NMS_WS_WORDS, "workspace stride");
// Cluster-form modes: 0 scans every neighbour slot through L2 and compares
// keys; 1 scans only the above-mask's slots (mask in shared memory); 2 checks
// a cached list of the higher-ranked neighbours' positions each round.
// Per CTA: key high words, two lists (4 B each), the suppression bits, and
// state and resume slot (1 B each) of its owned positions; mode 1 adds each
// owned position's above-mask (24 B), mode 2 its cached list (96 B), its
// length and its overflow slot (1 B each).
__host__ __device__ constexpr size_t nms_cluster_ws_bytes(int npos, int c, int mode) {
    return (size_t)((npos + c - 1) / c) * (14 + (mode == 1 ? 4 * NMS_MASK_WORDS : 0)) +
           4 * (size_t)(((npos + c - 1) / c + 31) / 32) + 64 + (mode ? 16 : 0);
}
// Replicated-state cluster form: the owned slice of P positions (a multiple
// of 32), the state of every position of the frame (C P bytes), resume
// entry, list length and overflow slot (1 B each, then 3 B of padding to
// keep the lists 16-byte aligned) and the cached list (48 entries in a
// 112-byte row) per owned position, a changed flag per 16 positions and a
// suppression bit per owned position.
__host__ __device__ constexpr int nms_rep_slice(int npos, int c) {
    return ((npos + c - 1) / c + 31) / 32 * 32;
}
// Cached list lengths of the replicated form: 48 neighbours in a 112-byte
// row (the 16-byte loads of eight consecutive positions' lists fall on
// distinct banks), or 16 in a 32-byte row for frames with more positions.
__host__ __device__ constexpr int nms_rep_stride(int list) { return list == 48 ? 56 : list; }
__host__ __device__ constexpr size_t nms_rep_ws_bytes(int npos, int c, int list) {
    return (size_t)nms_rep_slice(npos, c) * (c + 6 + 2 * nms_rep_stride(list)) + nms_rep_slice(npos, c) / 16 +
           nms_rep_slice(npos, c) / 8 + 64;
}

// Above-masks and lists for the cluster form.  For every window position p
// of every frame, bit s of the mask is set iff neighbour slot s of p holds a
// scanned candidate ranked above p (full key smaller: score, then level,
// filter, u, v), and the list holds the positions of the first NMS_LIST such
// neighbours in slot order.  One warp per position, a lane per slot; the
// whole GPU takes part, so a frame's pairwise rank tests cost one short
// launch, and the rounds that follow only look at the neighbours a mask or
// list names.  Written to the frame's workspace fd.ws, NMS_WS_WORDS words per
// position: words 0-5 the mask, word 6 the list's length, word 7 the slot
// where the mask goes on past the list (255: nowhere), words 8-31 the list
// as 16-bit positions (positions below 65536; longer frames keep the mask
// only).  Non-candidates get an empty mask and list.  fd.cand[p] records
// whether p is a candidate.
__global__ void __launch_bounds__(256) nms_above_kernel(const FrameDesc *__restrict__ frames) {
    const FrameDesc &fd = frames[blockIdx.y];
    const int p = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (p >= fd.npos) return;
    uint32_t *ws = fd.ws + (size_t)p * NMS_WS_WORDS;
    uint16_t *list = reinterpret_cast<uint16_t *>(ws + 8);
    const uint64_t kp = nms_scanned(fd, p) ? __ldg(fd.keys + p) : KEY_NONE;
    if (lane == 0) fd.cand[p] = kp != KEY_NONE;
    if (kp == KEY_NONE) {
        if (lane < 8) ws[lane] = lane == 7 ? 255u : 0u;
        return;
    }
    const int32_t *row = fd.nbr_t + (size_t)p * MAXN;
    uint32_t mine = 0u;   // lane w < 6 ends up holding word w
    bool ended = false;
    int k = 0, ovf = 255;
    for (int w = 0; w < NMS_MASK_WORDS; w++) {
        unsigned above = 0u;
        if (!ended) {
            const int q = __ldg(row + w * 32 + lane);
            const bool a = q >= 0 && nms_scanned(fd, q) && __ldg(fd.keys + q) < kp;
            above = __ballot_sync(0xffffffffu, a);
            ended = __ballot_sync(0xffffffffu, q < 0) != 0u;   // -1 past the list's end
            const int idx = k + __popc(above & ((1u << lane) - 1u));
            if (a && idx < NMS_LIST) list[idx] = (uint16_t)q;
            if (a && idx == NMS_LIST) ovf = w * 32 + lane;     // first slot past the list
            k += __popc(above);
        }
        if (lane == w) mine = above;
    }
    const unsigned has_ovf = __ballot_sync(0xffffffffu, ovf != 255);
    if (has_ovf) ovf = __shfl_sync(0xffffffffu, ovf, __ffs(has_ovf) - 1);
    if (lane < NMS_MASK_WORDS) ws[lane] = mine;
    if (lane == 6) ws[6] = (uint32_t)(k < NMS_LIST ? k : NMS_LIST);
    if (lane == 7) ws[7] = (uint32_t)ovf;
}

template <int MODE>
__global__ void __launch_bounds__(NMS_NT, 1) nms_cluster_kernel(const FrameDesc *__restrict__ frames,
                                                                int *flags) {
    constexpr bool MASK = MODE == 1;
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
    // mode 1: each owned position's above-mask (nms_above_kernel), [P][6]
    uint32_t *amask = reinterpret_cast<uint32_t *>(
        (reinterpret_cast<uintptr_t>(nsm + (size_t)P * 14 + 4 * (size_t)PW) + 15) & ~(uintptr_t)15);
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
    if (MASK)
        for (int k = t; k < nmine * NMS_MASK_WORDS; k += NMS_NT) {
            const int i = k / NMS_MASK_WORDS;
            amask[k] = __ldg(fd.ws + (size_t)(lo + i) * NMS_WS_WORDS + (k - i * NMS_MASK_WORDS));
        }
    cl_sync();   // every CTA's keys, states, bits and masks are initialised

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
                bool dead = (supp[li >> 5] >> (li & 31)) & 1u, wait = false;
                const int r0 = resume[li];
                int settled = r0;
                if (MASK) {
                    // only the higher-ranked candidates among p's neighbours (the
                    // set bits of its mask, from the resume slot on), up to four
                    // in flight: one kept -> suppressed, one undecided -> wait
                    const uint32_t *mk = amask + (size_t)li * NMS_MASK_WORDS;
                    int w = settled >> 5;
                    uint32_t bits = w < NMS_MASK_WORDS ? mk[w] & (~0u << (settled & 31)) : 0u;
                    while (!dead && !wait) {
                        int sl[4], ns = 0;
                        while (ns < 4) {
                            while (!bits && ++w < NMS_MASK_WORDS) bits = mk[w];
                            if (!bits) break;
                            sl[ns++] = w * 32 + __ffs(bits) - 1;
                            bits &= bits - 1;
                        }
                        if (ns == 0) break;   // every higher-ranked neighbour is suppressed
                        int q[4];
                        uint32_t sq[4];
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            q[k] = k < ns ? __ldg(nbr_t + (size_t)p * MAXN + sl[k]) : 0;
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            sq[k] = NMS_DEAD;
                            if (k < ns) {
                                const int o = owner(q[k]);
                                sq[k] = cl_ld_u8(s_rstate[o] + (uint32_t)(q[k] - o * P));
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            if (k >= ns || dead || wait) continue;
                            if (sq[k] == NMS_KEPT) dead = true;
                            else if (sq[k] == NMS_ALIVE) { wait = true; settled = sl[k]; }
                            else settled = sl[k] + 1;
                        }
                        if (ns < 4) break;
                    }
                }
                const uint32_t hp = khi[li];
                const int n = MODE ? 0 : __ldg(nbr_cnt + p);
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


// ---- replicated-state cluster form ------------------------------------------
// For frames of at most 65535 positions whose per-position lists fit: every
// CTA of the cluster keeps the state of EVERY position of the frame (one
// byte each: 9.5 KB for a 640x480 frame), so a candidate's checks read only
// local shared memory.  CTA r decides its own slice of P positions; each of
// its candidates checks, each round, all its higher-ranked neighbours from
// the list the pre-pass wrote (nms_above_kernel): one kept -> suppressed;
// one undecided -> wait; all suppressed -> the rest of its above-mask, if
// any (through L2), then kept.  At the end of a round every CTA copies its
// slice of states, as 32-bit words, into the other CTAs' copies, and a
// cluster barrier (release/acquire) closes the round.  A copy may receive a
// newer slice while its CTA still reads it: states only move from undecided
// to decided, so a newer value is as good as the old one.  The rounds reach
// the same fixed point as the one-CTA form.
// Slot of set bit n (0-based) of a 192-bit above-mask, 255 if there are n or fewer.
__device__ __forceinline__ int nth_set_slot(const uint32_t *mk, int n) {
    for (int w = 0; w < NMS_MASK_WORDS; w++) {
        uint32_t b = __ldg(mk + w);
        const int c = __popc(b);
        if (n < c) {
            for (int j = 0; j < n; j++) b &= b - 1;
            return w * 32 + __ffs(b) - 1;
        }
        n -= c;
    }
    return 255;
}

// LIST: cached higher-ranked neighbours per position (48 or 16); PPT: owned
// positions per thread (the slice holds at most PPT x NT positions).
template <int LIST, int PPT>
__global__ void __launch_bounds__(NMS_NT, 1) nms_cluster_rep_kernel(const FrameDesc *__restrict__ frames,
                                                                    int *flags) {
    static_assert(LIST == 48 || LIST == 16, "list length");
    constexpr int LSTR = nms_rep_stride(LIST);
    extern __shared__ __align__(16) unsigned char nsm[];
    __shared__ int sh[NMS_NT / 32 + 4];
    __shared__ int s_cnt[2][NMS_MAX_CLUSTER];
    __shared__ int s_kept[NMS_MAX_CLUSTER];
    __shared__ uint32_t s_rst[NMS_MAX_CLUSTER], s_rsupp[NMS_MAX_CLUSTER];
    __shared__ int s_total;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int C = (int)cl_size(), rank = (int)cl_rank();
    const FrameDesc &fd = frames[cl_id()];
    const int npos = fd.npos;
    const int P = nms_rep_slice(npos, C);
    const int lo = min(rank * P, npos), nmine = min(lo + P, npos) - lo;
    uint8_t *st = nsm;                                                          // [C P] all states
    uint8_t *resume = nsm + (size_t)C * P;                                      // [P]
    uint8_t *lcnt = resume + P, *lovf = lcnt + P;                               // [P], [P]
    uint16_t *alist = reinterpret_cast<uint16_t *>(lovf + P + 3 * (size_t)P);   // [P][LSTR], 16-B aligned
    // suppression bits of the owned positions, set (remote atomic OR) by a
    // kept neighbour in any CTA: such a position is suppressed without a check
    volatile uint32_t *supp = reinterpret_cast<volatile uint32_t *>(alist + (size_t)P * LSTR);  // [P / 32]
    uint8_t *dirty = reinterpret_cast<uint8_t *>(const_cast<uint32_t *>(supp) + P / 32);              // [P / 16]
    const int32_t *__restrict__ nbr_t = fd.nbr_t;
    const int base = rank * P;      // owned slice of the copy, 16-byte aligned (lo: clamped to npos)
    const int nch = P / 16;

    if (t < C) {
        s_rst[t] = cl_map(st, t);
        s_rsupp[t] = cl_map((const void *)supp, t);
    }
    for (int c = t; c < nch; c += NMS_NT) dirty[c] = 0;
    for (int c = t; c < P / 32; c += NMS_NT) supp[c] = 0u;
    const uint32_t *__restrict__ ws = fd.ws;
    // every position's initial state from the pre-pass's candidate flags, 16
    // positions per load (flags are 0 or 1: ALIVE = 1, DEAD = 0; positions
    // past npos: suppressed; the flag array has room for whole 16-byte
    // chunks up to the position slot)
    static_assert(NMS_ALIVE == 1 && NMS_DEAD == 0, "states as candidate flags");
    for (int c0 = t; c0 < C * P / 16; c0 += NMS_NT) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (16 * c0 < npos) v = __ldg(reinterpret_cast<const uint4 *>(fd.cand) + c0);
        if (16 * c0 + 16 > npos) {   // the chunk holding npos: clear bytes past it
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int b = 0; b < 16; b++)
                if (16 * c0 + b >= npos) w[b >> 2] &= ~(0xffu << (8 * (b & 3)));
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        reinterpret_cast<uint4 *>(st)[c0] = v;
    }
    // the owned candidates' lists, as the pre-pass wrote them (its first
    // LIST entries; eight loads in flight per thread)
    constexpr int LW = LIST / 2;
    for (int k0 = t; k0 < nmine * LW; k0 += 8 * NMS_NT) {
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k = k0 + j * NMS_NT, i = k / LW;
            v[j] = k < nmine * LW ? __ldg(ws + (size_t)(lo + i) * NMS_WS_WORDS + 8 + (k - i * LW)) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k = k0 + j * NMS_NT, i = k / LW;
            if (k < nmine * LW) reinterpret_cast<uint32_t *>(alist)[i * (LSTR / 2) + (k - i * LW)] = v[j];
        }
    }
    for (int i = t; i < nmine; i += NMS_NT) {
        const uint32_t c = __ldg(ws + (size_t)(lo + i) * NMS_WS_WORDS + 6);
        uint32_t o = __ldg(ws + (size_t)(lo + i) * NMS_WS_WORDS + 7);
        // a shorter cached list: the rest of the mask starts after its last entry
        if (LIST < NMS_LIST && (c > (uint32_t)LIST || o != 255u))
            o = (uint32_t)nth_set_slot(ws + (size_t)(lo + i) * NMS_WS_WORDS, LIST);
        lcnt[i] = (uint8_t)(c < (uint32_t)LIST ? c : (uint32_t)LIST);
        lovf[i] = (uint8_t)o;
        resume[i] = 0;
    }
    cl_sync();   // no CTA writes into another's copy before that one is initialised

    // Each thread owns the positions t, t + NT, ... of the slice and decides
    // its undecided ones; __syncthreads_count gives the CTA's undecided count.
    int round = 0;
    for (; round <= npos; round++) {
        bool any = false;
        int kept[PPT];   // positions this thread keeps this round
#pragma unroll
        for (int m = 0; m < PPT; m++) {
            kept[m] = -1;
            const int li = t + m * NMS_NT;
            if (li >= nmine) continue;
            const int p = lo + li;
            if (st[p] != NMS_ALIVE) continue;
            const int n2 = lcnt[li];
            const uint16_t *al = alist + (size_t)li * LSTR;   // 16-byte aligned
            bool dead = (supp[li >> 5] >> (li & 31)) & 1u, wait = false, prefix = true;
            const int r0 = resume[li];
            int settled = r0;
            // eight listed neighbours per 16-byte load, their states in flight
            // together; the check ends at a kept one (suppressed) or at the
            // eight-entry group holding the first undecided one (wait: a
            // candidate that waits looks again next round, from its first
            // undecided neighbour on)
            for (int k0 = r0 & ~7; k0 < n2 && !dead && !wait; k0 += 8) {
                const uint4 v = *reinterpret_cast<const uint4 *>(al + k0);
                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
                uint8_t sq[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int k = k0 + j;
                    sq[j] = (k >= r0 && k < n2) ? st[(w4[j >> 1] >> (16 * (j & 1))) & 0xffffu] : NMS_DEAD;
                }
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int k = k0 + j;
                    if (k < r0 || k >= n2) continue;
                    if (sq[j] == NMS_KEPT) dead = true;
                    else if (sq[j] == NMS_ALIVE) { wait = true; prefix = false; }
                    else if (prefix) settled = k + 1;
                }
            }
            int ov = lovf[li];
            if (!dead && !wait && ov != 255) {
                // the rest of the above-mask, from slot ov, through L2
                const uint32_t *mk = ws + (size_t)p * NMS_WS_WORDS;
                int w = ov >> 5;
                uint32_t bits = __ldg(mk + w) & (~0u << (ov & 31));
                for (;;) {
                    while (!bits && ++w < NMS_MASK_WORDS) bits = __ldg(mk + w);
                    if (!bits) { ov = 255; break; }
                    const int sl = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const uint8_t sq = st[__ldg(nbr_t + (size_t)p * MAXN + sl)];
                    if (sq == NMS_KEPT) { dead = true; break; }
                    if (sq == NMS_ALIVE) { wait = true; ov = sl; break; }
                }
                lovf[li] = (uint8_t)ov;
            }
            if (dead || !wait) {
                st[p] = dead ? NMS_DEAD : NMS_KEPT;
                dirty[(p - base) >> 4] = 1;
                if (!dead) kept[m] = p;
            } else {
                any = true;
                resume[li] = (uint8_t)settled;
            }
        }
        // each kept candidate marks its still-undecided neighbours in their
        // owners' suppression bits, the warp's lanes splitting the slots
#pragma unroll
        for (int m = 0; m < PPT; m++) {
            const int kp = kept[m];
            for (unsigned km = __ballot_sync(0xffffffffu, kp >= 0); km; km &= km - 1) {
                const int pk = __shfl_sync(0xffffffffu, kp, __ffs(km) - 1);
                int q[MAXN / 32];   // all six 32-slot chunks in flight (-1 past the list's end)
#pragma unroll
                for (int j = 0; j < MAXN / 32; j++) q[j] = __ldg(nbr_t + (size_t)pk * MAXN + 32 * j + lane);
#pragma unroll
                for (int j = 0; j < MAXN / 32; j++) {
                    if (q[j] >= 0 && st[q[j]] == NMS_ALIVE) {
                        const int o = q[j] / P, lq = q[j] - o * P;
                        cl_or_u32(s_rsupp[o] + 4u * (uint32_t)(lq >> 5), 1u << (lq & 31));
                    }
                }
            }
        }
        const int n_und = __syncthreads_count(any);
        // the 16-byte chunks of this CTA's slice that changed this round,
        // into every other CTA's copy (bytes [base, base + P): aligned and
        // inside the C P-byte copy), and this CTA's undecided count into
        // every CTA's count table (slot by round parity: slot r & 1 is
        // rewritten two rounds later, after every CTA has read it)
        for (int k = t; k < nch * (C - 1); k += NMS_NT) {
            const int r = k / nch, c = k - r * nch;
            if (!dirty[c]) continue;
            const int dst = r < rank ? r : r + 1;
            cl_st_v4(s_rst[dst] + (uint32_t)(base + 16 * c), *reinterpret_cast<const uint4 *>(st + base + 16 * c));
        }
        if (t < C) cl_st_u32(cl_map(&s_cnt[round & 1][rank], t), (uint32_t)n_und);
        cl_sync();
        for (int c = t; c < nch; c += NMS_NT) dirty[c] = 0;
        if (wid == 0) {
            int c = lane < C ? s_cnt[round & 1][lane] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0) s_total = c;
        }
        __syncthreads();
        if (s_total == 0) break;
    }

    // kept positions in position order: CTA r's before CTA r+1's
    int *s_warp = sh;
    const int per = (nmine + NMS_NT - 1) / NMS_NT;
    const int beg = min(t * per, nmine), end = min(beg + per, nmine);
    int mine_kept = 0;
    for (int i = beg; i < end; i++) mine_kept += st[lo + i] == NMS_KEPT;
    int incl = mine_kept;
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
    int pos = sh[NMS_NT / 32] + s_warp[wid] + incl - mine_kept;
    for (int i = beg; i < end; i++) {
        if (st[lo + i] != NMS_KEPT) continue;
        if (pos < fd.out_cap) {
            const uint64_t k = __ldg(fd.keys + lo + i);
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
    cl_sync();   // no CTA leaves while another may still write into its copy
}

namespace {
constexpr int NMS_MAX_DEVICES = 64;
int g_nsm[NMS_MAX_DEVICES];           // SM count of each device
int g_cluster_max[NMS_MAX_DEVICES];   // largest cluster size each device can run (1 = none)
PerDevice g_cluster_setup;

template <class K>
bool cluster_attrs(K kern) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, NMS_SMEM_MAX) ==
               cudaSuccess &&
           cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
}

template <class K>
int largest_cluster(K kern) {
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
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0) return c;
        cudaGetLastError();
    }
    return 1;
}

// The cluster kernels' attributes are set once per device; returns the
// largest cluster size both can run there and the device's SM count.
int nms_cluster_max(int *nsm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NMS_MAX_DEVICES) {
        cudaGetLastError();
        *nsm = 1;
        return 1;
    }
    g_cluster_setup.once([&]() -> cudaError_t {
        int n = 1;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_nsm[dev] = n > 0 ? n : 1;
        g_cluster_max[dev] = 1;
        if (!cluster_attrs(nms_cluster_kernel<0>) || !cluster_attrs(nms_cluster_kernel<1>) ||
            !cluster_attrs(nms_cluster_rep_kernel<48, 2>) || !cluster_attrs(nms_cluster_rep_kernel<16, 4>)) {
            cudaGetLastError();
            return cudaSuccess;
        }
        int m = largest_cluster(nms_cluster_kernel<0>);
        m = std::min(m, largest_cluster(nms_cluster_kernel<1>));
        m = std::min(m, largest_cluster(nms_cluster_rep_kernel<48, 2>));
        m = std::min(m, largest_cluster(nms_cluster_rep_kernel<16, 4>));
        g_cluster_max[dev] = m;
        return cudaSuccess;
    });
    *nsm = g_nsm[dev];
    return g_cluster_max[dev];
}
}  // namespace

// Cluster size for a batch: `request` 1 = one CTA per frame, 2..16 = that
// size, 0 = automatic -- a cluster of SMs / frames CTAs (a power of two) when
// that is at least NMS_AUTO_CLUSTER_MIN (a few frames: each gets many SMs),
// else one CTA per frame, whose frames then run side by side (measured
// faster from a few dozen frames on); and at least 2 for frames whose
// one-CTA workspace lives in global memory.  Returns 1 for the one-CTA form.
int nms_cluster_size(int nframes, int max_npos, int request) {
    int nsm = 1;
    const int cmax = nms_cluster_max(&nsm);
    if (cmax < 2 || request == 1 || nframes <= 0) return 1;
    int c;
    if (request >= 2) {
        c = request > cmax ? cmax : request;
    } else {
        const int want = nsm / nframes;
        c = 1;
        if (want >= NMS_AUTO_CLUSTER_MIN)
            while (c * 2 <= want && c * 2 <= cmax) c *= 2;
        if (nms_ws_class(max_npos) == NMS_WS_GLOBAL && c < 2) c = 2;
    }
    if (c < 2) return 1;
    while (c < cmax && nms_cluster_ws_bytes(max_npos, c, 0) > (size_t)NMS_SMEM_MAX) c *= 2;
    if (nms_cluster_ws_bytes(max_npos, c, 0) > (size_t)NMS_SMEM_MAX) return 1;
    return c;
}

namespace {
// The frames of one workspace class.
cudaError_t launch_nms_class(const FrameDesc *frames, int nframes, int max_npos, int cls, int *flags,
                             cudaStream_t stream, int cluster_request) {
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
        cfg.stream = stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        // with the above-masks and cached lists (16-bit positions) when they
        // fit in the CTAs' shared memory, else with the masks alone
        const size_t ws48 = nms_rep_ws_bytes(max_npos, c, 48), ws16 = nms_rep_ws_bytes(max_npos, c, 16);
        const size_t ws1 = nms_cluster_ws_bytes(max_npos, c, 1);
        const int P = nms_rep_slice(max_npos, c);
        const bool rep48 = ws48 <= (size_t)NMS_SMEM_MAX && max_npos <= 65535 && P <= 2 * NMS_NT;
        const bool rep16 = ws16 <= (size_t)NMS_SMEM_MAX && max_npos <= 65535 && P <= 4 * NMS_NT;
        if (ws1 <= (size_t)NMS_SMEM_MAX || rep48 || rep16) {
            nms_above_kernel<<<dim3((max_npos + 7) / 8, nframes), 256, 0, stream>>>(frames);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            if (rep48) {
                cfg.dynamicSmemBytes = ws48;
                return cudaLaunchKernelEx(&cfg, nms_cluster_rep_kernel<48, 2>, frames, flags);
            }
            if (rep16) {
                cfg.dynamicSmemBytes = ws16;
                return cudaLaunchKernelEx(&cfg, nms_cluster_rep_kernel<16, 4>, frames, flags);
            }
            cfg.dynamicSmemBytes = ws1;
            return cudaLaunchKernelEx(&cfg, nms_cluster_kernel<1>, frames, flags);
        }
        cfg.dynamicSmemBytes = nms_cluster_ws_bytes(max_npos, c, 0);
        return cudaLaunchKernelEx(&cfg, nms_cluster_kernel<0>, frames, flags);
    }
    if (cls == NMS_WS_SMEM)
        nms_kernel<NMS_WS_SMEM><<<nframes, NMS_BATCH_NT, nms_ws_bytes(max_npos, true), stream>>>(frames, flags);
    else if (cls == NMS_WS_KEYS)
        nms_kernel<NMS_WS_KEYS><<<nframes, NMS_KEYS_NT, nms_keys_bytes(max_npos), stream>>>(frames, flags);
    else
        nms_kernel<NMS_WS_GLOBAL><<<nframes, NMS_BATCH_NT, 0, stream>>>(frames, flags);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_nms(const FrameDesc *frames, const int *ncls, const int *max_npos, int *flags,
                       cudaStream_t stream, int cluster_request, const NmsStreams *par) {
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(nms_kernel<NMS_WS_SMEM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, NMS_SMEM_MAX);
        if (e == cudaSuccess)   // all of the unified L1 as shared memory: three frames per SM
            e = cudaFuncSetAttribute(nms_kernel<NMS_WS_SMEM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(nms_kernel<NMS_WS_KEYS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     NMS_KEYS_SMEM_MAX);
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    int off[NMS_WS_CLASSES], nonempty = 0;
    for (int k = 0, o = 0; k < NMS_WS_CLASSES; k++) {
        off[k] = o;
        o += ncls[k];
        nonempty += ncls[k] > 0;
    }
    if (!par || nonempty < 2) {
        for (int k = 0; k < NMS_WS_CLASSES; k++) {
            if (ncls[k] <= 0) continue;
            cudaError_t e = launch_nms_class(frames + off[k], ncls[k], max_npos[k], k, flags, stream,
                                             cluster_request);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // the larger classes (longer frames, one CTA or a cluster per SM) go
    // first, each on a side stream; the shared-memory class fills the SMs
    // they leave on the caller's stream
    cudaError_t e = cudaEventRecord(par->fork, stream);
    int nside = 0;
    for (int k = NMS_WS_CLASSES - 1; k >= 1 && e == cudaSuccess; k--) {
        if (ncls[k] <= 0) continue;
        cudaStream_t s = par->side[nside];
        e = cudaStreamWaitEvent(s, par->fork, 0);
        if (e == cudaSuccess)
            e = launch_nms_class(frames + off[k], ncls[k], max_npos[k], k, flags, s, cluster_request);
        if (e == cudaSuccess) e = cudaEventRecord(par->join[nside], s);
        if (e == cudaSuccess) nside++;
    }
    if (e == cudaSuccess && ncls[0] > 0)
        e = launch_nms_class(frames + off[0], ncls[0], max_npos[0], 0, flags, stream, cluster_request);
    // join every branch that was forked, also after an error (a capture
    // must end with its side streams joined)
    for (int j = 0; j < nside; j++) {
        cudaError_t ej = cudaStreamWaitEvent(stream, par->join[j], 0);
        if (e == cudaSuccess) e = ej;
    }
    return e;
}

}  // namespace hogk
