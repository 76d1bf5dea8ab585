// k_corr_tc.cu -- the multi-filter correlation (Section 4.1.1: linear
// classification filter and detection) as a tensor-core contraction on
// tcgen05, the alternative to the FP32 CUDA-core kernel of k_corr.cu.
//
// Row-shift form.  Flatten a level's cells p = i*cx + j.  For a filter row
// a and filter f define, for every cell p,
//   G[a*F + f][p] = sum_{b<10, c<32} feat[p + b][c] * W_f[a][b][c],
// a GEMM with M = cells, K = 10 cell shifts x 32 channels = 320 and N =
// 10*F (filter rows x filters, padded to a multiple of 16).  The window
// score is then
//   score_f(u, v) = sum_{a<10} G[a*F + f][(u + a)*cx + v],
// ten loads per window and filter (the reduce kernel).  Row p of the GEMM's
// A operand at cell shift b is the 32 channels of cell p + b: in a
// K-major, non-swizzled shared-memory tile laid out [channel group][cell]
// [8 channels], the operand for shift b is the same tile with its start
// moved by b cells (16 bytes), so the im2col matrix is never materialised.
// Windows whose shifted rows run into the next feature row (v >= nv) are
// computed and never read.
//
// Precision: features and weights are split into fp16 hi + lo parts
// (weights scaled by 2^6 first, so their lo parts stay normal) and three
// products are kept, hi*hi, hi*lo and lo*hi, accumulated in FP32 in tensor
// memory.  The dropped lo*lo term and the split residues are below 2^-21 of
// each product, so scores agree with the FP32 path to about 1e-6.  Per K
// step two MMAs: A_hi x [W_hi | W_lo] (N = 2 N0, the two weight planes
// side by side along N) into accumulator columns [D0 | D1], and A_lo x W_hi
// (N = N0) into D0; the epilogue takes G = D0 + D1.  The MMA count, not the
// MMA width, sets the tensor pipe's pace at these sizes (N0 = 64 for five
// filters), so two wide MMAs beat three narrow ones.
//
// One CTA (4 warps) is persistent over 128-cell tiles of all levels of the
// batch: it loads both B planes once, then per tile stages the hi and lo A
// planes (137 cells: the tile plus 9 shifted cells) with cp.async, one
// thread issues the 60 MMAs (M=128, N, K=16) into a TMEM accumulator and
// commits them to an mbarrier, and the four warps read their 32 TMEM lanes
// (cells) back with tcgen05.ld and store G column by column (coalesced
// across cells).  Every wait is bounded: on expiry the kernel sets flags[2]
// (read by the host as HOG_ETIMEOUT), stops taking tiles and still frees
// its tensor memory.
#include "hog_stages.cuh"

namespace hogk {

namespace {
constexpr int TC_NT = 128;                 // 4 warps = the 4 TMEM lane quarters
constexpr int TC_M = 128;                  // cells per tile (MMA M)
constexpr int TC_ROWS = TC_M + WIN - 1;    // 137 staged cells: shifts b = 0..9
constexpr int TC_KSTEPS = 2 * WIN;         // K = 10 shifts x 32 channels, 16 per MMA
constexpr long long TC_SPIN = 1ll << 24;   // mbarrier polls before giving up
constexpr size_t TC_A_PLANE = (size_t)4 * TC_ROWS * 16;   // [4 groups][137 cells][16 B]

// TMEM columns for one accumulator pair [D0 | D1] of 2 N0 columns
__host__ __device__ constexpr int tc_cols(int n) { return 2 * n <= 32 ? 32 : (2 * n <= 64 ? 64 : (2 * n <= 128 ? 128 : 256)); }
// One weight plane (hi or lo); the two are interleaved per (shift, channel
// group): [10 shifts][4 groups][hi, lo][N0][16 B], so hi and lo of one
// (shift, group) are 2 N0 consecutive B rows.
__host__ __device__ constexpr size_t tc_b_plane(int nf) { return (size_t)WIN * 4 * tc_n(nf) * 16; }
// Dynamic shared memory: two B planes and two A planes (99.5 KB for up to 5
// filters: two CTAs per SM, so one CTA's MMAs overlap the other's staging
// and epilogue).
__host__ __device__ constexpr size_t tc_smem(int nf) { return 2 * tc_b_plane(nf) + 2 * TC_A_PLANE; }

// tcgen05 instruction descriptor, kind::f16: D = FP32 (bits 4-5 = 1), A and
// B = FP16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address >> 4 (bits
// 0-13), leading byte offset >> 4 (bits 16-29: K-direction stride between
// 8x16-byte core matrices), stride byte offset >> 4 (bits 32-45: stride
// between 8-row groups), descriptor version 1 (bit 46), layout type 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
}  // namespace

template <int NF>
__global__ void __launch_bounds__(TC_NT) corr_tc_kernel(const LevelDesc *__restrict__ descs,
                                                        const Job *__restrict__ jobs, int njobs,
                                                        const uint16_t *__restrict__ wb,
                                                        int *flags) {
    constexpr int N = tc_n(NF), COLS = tc_cols(N);
    constexpr size_t BP = tc_b_plane(NF);
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char *Bs = sm;                       // [10 shifts][4 groups][hi, lo][N][16 B]
    unsigned char *As = sm + 2 * BP;              // [hi, lo][4 groups][137 cells][16 B]
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_abort;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t mb = smem_addr(&mbar);

    for (int k = t; k < (int)(2 * BP / 16); k += TC_NT)
        cp_async16(Bs + 16 * (size_t)k, reinterpret_cast<const unsigned char *>(wb) + 16 * (size_t)k);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(&tslot)), "r"(COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    cp_async_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = tslot;
    const uint32_t a_s = smem_addr(As), b_s = smem_addr(Bs);
    constexpr uint32_t IDESC = tc_idesc(N), IDESC2 = tc_idesc(2 * N);
    uint32_t parity = 0;

    for (int jid = blockIdx.x; jid < njobs; jid += gridDim.x) {
        const Job jb = jobs[jid];
        const LevelDesc &d = descs[jb.desc];
        const int ncells = d.cy * d.cx;
        const int q0 = jb.tile * TC_M;
        // A planes: cells q0 .. q0 + 136 (zero past the level's last cell)
        for (int k = t; k < 2 * 4 * TC_ROWS; k += TC_NT) {
            const int plane = k / (4 * TC_ROWS), rem = k - plane * 4 * TC_ROWS;
            const int g = rem / TC_ROWS, r = rem - g * TC_ROWS;
            const int cell = q0 + r;
            const bool ok = cell < ncells;
            const uint16_t *src =
                (plane ? d.feat_lo : d.feat_hi) + ((size_t)g * ncells + (ok ? cell : 0)) * 8;
            cp_async16_zfill(As + ((size_t)(plane * 4 + g) * TC_ROWS + r) * 16, src, ok);
        }
        cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
        if (t == 0) {
            fence_after();
#pragma unroll 1
            for (int s = 0; s < TC_KSTEPS; s++) {
                const int b = s >> 1, half = s & 1;
                // channel groups 2*half, 2*half + 1 of cells b .. b + 127
                const uint32_t aoff = (uint32_t)((2 * half) * TC_ROWS + b) * 16;
                const uint32_t boff = (uint32_t)((b * 4 + 2 * half) * 2 * N) * 16;
                const uint64_t ah = sdesc(a_s + aoff, TC_ROWS * 16, 128);
                const uint64_t al = sdesc(a_s + (uint32_t)TC_A_PLANE + aoff, TC_ROWS * 16, 128);
                const uint64_t bhl = sdesc(b_s + boff, 2 * N * 16, 128);   // [W_hi | W_lo]
                mma_f16(tbase, ah, bhl, IDESC2, s > 0 ? 1u : 0u);        // D0 += hh, D1 += hl
                mma_f16(tbase, al, bhl, IDESC, 1u);                      // D0 += lh
            }
            mma_commit(mb);
        }
        // every thread waits for the MMAs (bounded)
        long long spins = 0;
        bool done = false;
        while (!(done = mbar_try(mb, parity)) && ++spins < TC_SPIN) {
            if (spins > 64) __nanosleep(32);
        }
        parity ^= 1u;
        if (!done) atomicExch(&s_abort, 1);
        fence_after();
        __syncthreads();
        if (s_abort) {
            if (t == 0) atomicOr(flags + 2, 1);
            break;
        }
        // warp w holds TMEM lanes 32w .. 32w + 31 = cells q0 + 32w + lane
        const int cell = q0 + 32 * warp + lane;
        float *g = d.gmat;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t r0[16], r1[16];
            const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            tmem_ld16_nowait(ta, r0);
            tmem_ld16_nowait(ta + N, r1);
            tmem_wait_ld();
            if (cell < ncells) {
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (c0 + j < WIN * NF)
                        g[(size_t)(c0 + j) * ncells + cell] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
            }
        }
        fence_before();
        __syncthreads();   // TMEM accumulator and A planes free for the next tile
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(COLS)
                     : "memory");
}

// score_f(u, v) = (1/64) sum_a G[a F + f][(u + a) cx + v]; threshold and key
// as in the CUDA-core kernel.  One thread per window, 256 windows per job.
template <int NF>
__global__ void __launch_bounds__(256) corr_tc_reduce_kernel(const LevelDesc *__restrict__ descs,
                                                             const Job *__restrict__ jobs,
                                                             int nf_real, float threshold) {
    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int w = jb.tile * 256 + threadIdx.x;
    if (w >= d.nu * d.nv) return;
    const int u = w / d.nv, v = w - u * d.nv;
    const size_t ncells = (size_t)d.cy * d.cx;
    const size_t p = (size_t)u * d.cx + v;
    const float *g = d.gmat;
    float sc[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < WIN; a++) s += __ldg(g + (size_t)(a * NF + f) * ncells + p + (size_t)a * d.cx);
        sc[f] = s * (1.0f / 64.0f);
    }
    float best = sc[0];
    int fb = 0;
#pragma unroll
    for (int f = 1; f < NF; f++)
        if (f < nf_real && sc[f] > best) { best = sc[f]; fb = f; }
    if (d.scores_user) {
#pragma unroll
        for (int f = 0; f < NF; f++)
            if (f < nf_real) d.scores_user[((size_t)f * d.nu + u) * d.nv + v] = sc[f];
    }
    if (d.keys)
        d.keys[(size_t)u * d.nv + v] =
            (d.scan && best > threshold) ? make_key(best, d.level, fb, u, v) : KEY_NONE;
}

// B planes from the filters (host layout [f][a][b][c], 31 channels):
// element (n = a*F + f, k = b*32 + c) of plane p (0 hi, 1 lo) at
// (((b*4 + c/8)*2 + p)*N + n)*8 + c%8, value 64*W split into fp16 hi and
// lo; zero for n >= 10 F and for channel 31.
template <int NF>
__global__ void corr_tc_weights_kernel(const float *__restrict__ w, int nf_real, uint16_t *wb) {
    constexpr int N = tc_n(NF);
    constexpr size_t PLANE = (size_t)WIN * 4 * N * 8;    // halves per plane
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int)PLANE) return;
    const int c8 = idx & 7, n = (idx >> 3) % N, bg = (idx >> 3) / N;
    const int b = bg >> 2, c = (bg & 3) * 8 + c8;
    const int a = n / NF, f = n - (n / NF) * NF;
    float x = 0.0f;
    if (n < WIN * NF && f < nf_real && c < NFEAT)
        x = 64.0f * w[(((size_t)f * WIN + a) * WIN + b) * NFEAT + c];
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    // [shift b][group][hi, lo][N][8 halves]
    const size_t o = ((size_t)bg * 2 * N + n) * 8 + c8;
    wb[o] = __half_as_ushort(hi);
    wb[o + (size_t)N * 8] = __half_as_ushort(lo);
}

// ===========================================================================
// Fused form: GEMM and row-shift reduction in one kernel, G never leaves
// the SM.  A CTA owns bands of window rows (whole levels in large batches)
// and walks each band's cells in row-major order in 128-cell tiles.  For a
// tile's cell (r, v) and filter row a, G[a F + f] is the a-th term of
// window (r - a, v); a ring of partial scores in shared memory, one row per
// window row in flight, collects the terms:
//   a = 0: ring = 0 + G[f]          (window row r opens)
//   a > 0: ring += G[a F + f]
//   a = 9: the window is complete -> scores, threshold, key.
// Within one tile the ten steps are separated by barriers: cells of one
// column in consecutive rows add into the same window at consecutive steps.
// Cell rows are visited in increasing order, so every window sums its ten
// terms in the order a = 0..9 whatever the banding -- the same sum, bit for
// bit, as the two-pass reduce kernel.
//
// Warp roles (192 threads, one CTA per SM): warps 0-3 read the accumulator
// (TMEM lane quarters) and run the ring; warp 4 issues the MMAs; warp 5
// stages A tiles with bulk copies (cp.async.bulk, mbarrier complete_tx) into
// a 3-stage ring.  Two TMEM accumulators let the MMAs of tile k+1 run while
// the epilogue reads tile k.  Every wait is bounded; on expiry the CTA
// stops, drains its copies and MMAs, frees TMEM and sets flags[2].
namespace {
constexpr int TF_EPI = 128;                 // epilogue threads (warps 0-3)
constexpr int TF_NT = 192;                  // + MMA warp + producer warp
constexpr int TF_STAGES = 3;
constexpr size_t TF_A_STAGE = 2 * TC_A_PLANE;   // hi + lo planes of one tile
// ring entries per filter: max over P <= TCF_PMAX of tcf_ring_rows(P) * (P - 9)
constexpr int tf_ring_max() {
    int m = 0;
    for (int P = WIN; P <= TCF_PMAX; P++) {
        const int e = tcf_ring_rows(P) * (P - WIN + 1);
        m = e > m ? e : m;
    }
    return m;
}
constexpr int TF_RING = tf_ring_max();
// TMEM columns per accumulator pair [D0 | D1] (2 N): a power of two
// (accumulator pair 1 starts there)
__host__ __device__ constexpr int tf_acc(int n) { return tc_cols(n); }
__host__ __device__ constexpr int tf_alloc(int cols) {
    return cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
}
__host__ __device__ constexpr size_t tf_smem(int nf) {
    return 2 * tc_b_plane(nf) + TF_STAGES * TF_A_STAGE + sizeof(float) * (size_t)nf * TF_RING;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
// Bounded wait on the phase of parity `parity`; false if it gave up or
// another role of the CTA already did.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int *abort_flag) {
    long long spins = 0;
    while (!mbar_try(mbar, parity)) {
        if (*abort_flag || ++spins >= TC_SPIN) return false;
        if (spins > 64) __nanosleep(32);
    }
    return true;
}
__device__ __forceinline__ void epi_sync() {   // the four epilogue warps
    asm volatile("bar.sync 1, %0;" ::"n"(TF_EPI) : "memory");
}
__device__ __forceinline__ bool epi_all(bool ok) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.and.pred q, 1, %2, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"((uint32_t)ok), "n"(TF_EPI) : "memory");
    return r != 0;
}

// Cells [q, q + n) of a band's local row-major order that lie in one
// contiguous run of the level's cell planes: returns the run's length and
// its first cell index in the level.
__device__ __forceinline__ int band_run(const TcBand &b, int cx, int q, int n, int *gcell) {
    if (b.P == cx) {   // full width: rows are contiguous in the level
        *gcell = b.u0 * cx + q;
        return n;
    }
    const int r = q / b.P, cl = q - r * b.P;
    *gcell = (b.u0 + r) * cx + b.c0 + cl;
    return min(n, b.P - cl);
}
}  // namespace

static_assert(2 * tf_acc(tc_n(8)) <= 512 && 2 * tc_n(8) <= 256, "TMEM / MMA width for 8 filters");

template <int NF>
__global__ void __launch_bounds__(TF_NT, 1) corr_tcf_kernel(const LevelDesc *__restrict__ descs,
                                                           const TcBand *__restrict__ bands,
                                                           const int32_t *__restrict__ cta_first,
                                                           const uint16_t *__restrict__ wb,
                                                           int nf_real, float threshold, int *flags) {
    constexpr int N = tc_n(NF), ACC = tf_acc(N), COLS = tf_alloc(2 * ACC);
    constexpr size_t BP = tc_b_plane(NF);
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char *Bs = sm;                                  // [10][4][hi, lo][N][16 B]
    unsigned char *As = sm + 2 * BP;                         // [stage][hi, lo][4][137][16 B]
    float *ring = reinterpret_cast<float *>(As + TF_STAGES * TF_A_STAGE);   // [NF][TF_RING]
    __shared__ __align__(8) uint64_t bar_full[TF_STAGES], bar_empty[TF_STAGES];
    __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t tslot;
    __shared__ volatile int s_abort;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    for (int k = t; k < (int)(2 * BP / 16); k += TF_NT)
        cp_async16(Bs + 16 * (size_t)k, reinterpret_cast<const unsigned char *>(wb) + 16 * (size_t)k);
    if (t == 0) {
        for (int i = 0; i < TF_STAGES; i++) {
            mbar_init(smem_addr(&bar_full[i]), 1);    // producer's arrive.expect_tx
            mbar_init(smem_addr(&bar_empty[i]), 1);   // MMA commit
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(smem_addr(&bar_tfull[i]), 1);   // MMA commit
            mbar_init(smem_addr(&bar_tempty[i]), 4);  // one arrive per epilogue warp
        }
        mbar_init(smem_addr(&bar_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(&tslot)), "r"(COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    cp_async_wait_all();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = tslot;
    const int first = cta_first[blockIdx.x], last = cta_first[blockIdx.x + 1];
    int issued[TF_STAGES] = {0, 0, 0};   // producer: batches issued per stage

    if (warp == 5) {
        // ---- producer: A tiles (hi and lo planes, 137 cells) by bulk copies
        int stage = 0, use = 0;   // use = how many tiles went through stage so far / TF_STAGES
        bool ok = true;
        for (int bi = first; bi < last && ok; bi++) {
            const TcBand b = bands[bi];
            const LevelDesc &d = descs[b.desc];
            const int nc = d.cx * d.cy;
            const int ncl = (b.u1 + WIN - 1 - b.u0) * b.P;   // local cells of the band
            const int nt = tcf_tiles(b.u0, b.u1, b.P);
            for (int tile = 0; tile < nt; tile++) {
                // warp-uniform decision (lanes poll independently)
                ok = __all_sync(0xffffffffu,
                                mbar_wait(smem_addr(&bar_empty[stage]), (uint32_t)((use & 1) ^ 1), &s_abort));
                if (!ok) { s_abort = 1; break; }
                const int q0 = tile * TC_M, qe = min(q0 + TC_ROWS, ncl);
                // total bytes of this tile's runs (every lane computes the same)
                uint32_t bytes = 0;
                for (int q = q0; q < qe;) {
                    int gc;
                    const int n = band_run(b, d.cx, q, qe - q, &gc);
                    bytes += (uint32_t)n * 16u * 8u;
                    q += n;
                }
                const uint32_t fb = smem_addr(&bar_full[stage]);
                if (lane == 0) mbar_expect_tx(fb, bytes);
                __syncwarp();
                const uint32_t abase = smem_addr(As + stage * TF_A_STAGE);
                int k = 0;
                for (int q = q0; q < qe; k++) {
                    int gc;
                    const int n = band_run(b, d.cx, q, qe - q, &gc);
                    // lanes 8k .. 8k+7 copy (plane, group) = lane & 7 of run k
                    if ((lane >> 3) == (k & 3)) {
                        const int pg = lane & 7, plane = pg >> 2, g = pg & 3;
                        const uint16_t *src = (plane ? d.feat_lo : d.feat_hi) + ((size_t)g * nc + gc) * 8;
                        const uint32_t dst = abase + (uint32_t)(((plane * 4 + g) * TC_ROWS + (q - q0)) * 16);
                        bulk_g2s(dst, src, (uint32_t)n * 16u, fb);
                    }
                    q += n;
                }
                __syncwarp();
                issued[stage]++;
                if (++stage == TF_STAGES) { stage = 0; use++; }
            }
        }
    } else if (warp == 4) {
        // ---- MMA issuer
        int stage = 0, use = 0, acc = 0, ause = 0;
        constexpr uint32_t IDESC = tc_idesc(N), IDESC2 = tc_idesc(2 * N);
        const uint32_t b_s = smem_addr(Bs);
        bool ok = true;
        for (int bi = first; bi < last && ok; bi++) {
            const TcBand b = bands[bi];
            const int nt = tcf_tiles(b.u0, b.u1, b.P);
            for (int tile = 0; tile < nt; tile++) {
                ok = mbar_wait(smem_addr(&bar_full[stage]), (uint32_t)(use & 1), &s_abort) &&
                     mbar_wait(smem_addr(&bar_tempty[acc]), (uint32_t)((ause & 1) ^ 1), &s_abort);
                ok = __all_sync(0xffffffffu, ok);   // warp-uniform decision
                if (!ok) { s_abort = 1; break; }
                fence_after();
                if (lane == 0) {
                    // descriptors: the start-address field (bits 0-13, address
                    // >> 4) of a base descriptor plus compile-time offsets in
                    // 16-byte units (shared addresses < 256 KB: no carry)
                    const uint64_t ah0 = sdesc(smem_addr(As + stage * TF_A_STAGE), TC_ROWS * 16, 128);
                    const uint64_t b0 = sdesc(b_s, 2 * N * 16, 128);
                    const uint32_t d_t = tbase + (uint32_t)(acc * ACC);
#pragma unroll
                    for (int s = 0; s < TC_KSTEPS; s++) {
                        const int bsh = s >> 1, half = s & 1;
                        const uint64_t aoff = (uint64_t)((2 * half) * TC_ROWS + bsh);
                        const uint64_t boff = (uint64_t)((bsh * 4 + 2 * half) * 2 * N);
                        const uint64_t ah = ah0 + aoff, al = ah0 + (TC_A_PLANE >> 4) + aoff;
                        const uint64_t bhl = b0 + boff;                       // [W_hi | W_lo]
                        mma_f16(d_t, ah, bhl, IDESC2, s > 0 ? 1u : 0u);     // D0 += hh, D1 += hl
                        mma_f16(d_t, al, bhl, IDESC, 1u);                   // D0 += lh
                    }
                    mma_commit(smem_addr(&bar_empty[stage]));   // A stage free once read
                    mma_commit(smem_addr(&bar_tfull[acc]));     // accumulator ready
                }
                __syncwarp();
                if (++stage == TF_STAGES) { stage = 0; use++; }
                if (++acc == 2) { acc = 0; ause++; }
            }
        }
    } else {
        // ---- epilogue: accumulator -> ring of partial scores -> keys
        int acc = 0, ause = 0;
        bool ok = true;
        for (int bi = first; bi < last && ok; bi++) {
            const TcBand b = bands[bi];
            const LevelDesc &d = descs[b.desc];
            const int ncl = (b.u1 + WIN - 1 - b.u0) * b.P;
            const int nt = tcf_tiles(b.u0, b.u1, b.P);
            const int RS = tcf_ring_rows(b.P);
            for (int tile = 0; tile < nt; tile++) {
                ok = epi_all(mbar_wait(smem_addr(&bar_tfull[acc]), (uint32_t)(ause & 1), &s_abort));
                if (!ok) { s_abort = 1; break; }
                fence_after();
                float G[WIN * NF];
                {
                    constexpr int NL = (WIN * NF + 15) / 16;
                    const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(acc * ACC);
#pragma unroll
                    // G = D0 + D1, 16 columns at a time
#pragma unroll
                    for (int c = 0; c < NL; c++) {
                        uint32_t r0[16], r1[16];
                        tmem_ld16_nowait(ta + 16 * c, r0);
                        tmem_ld16_nowait(ta + N + 16 * c, r1);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            if (16 * c + j < WIN * NF)
                                G[16 * c + j] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&bar_tempty[acc]));
                if (++acc == 2) { acc = 0; ause++; }

                const int q = tile * TC_M + t;
                const int r = q / b.P, cl = q - r * b.P;   // local cell row / column
                const bool live = q < ncl && cl < b.nvs;
                const int v = b.c0 + cl;
                const int nwr = b.u1 - b.u0;
                // ring slot of window row r - a is (r - a) mod RS: start at
                // r mod RS and step down by one row of nvs entries per a
                int idx = (r % RS) * b.nvs + cl;
                const int wrap = RS * b.nvs;
#pragma unroll
                for (int a = 0; a < WIN; a++) {
                    const int ul = r - a;   // local window row
                    if (live && ul >= 0 && ul < nwr) {
                        if (a == 0) {
#pragma unroll
                            for (int f = 0; f < NF; f++) ring[f * TF_RING + idx] = 0.0f + G[f];
                        } else {
#pragma unroll
                            for (int f = 0; f < NF; f++) ring[f * TF_RING + idx] += G[a * NF + f];
                        }
                        if (a == WIN - 1) {
                            const int u = b.u0 + ul;
                            float sc[NF];
#pragma unroll
                            for (int f = 0; f < NF; f++) sc[f] = ring[f * TF_RING + idx] * (1.0f / 64.0f);
                            float best = sc[0];
                            int fb = 0;
#pragma unroll
                            for (int f = 1; f < NF; f++)
                                if (f < nf_real && sc[f] > best) { best = sc[f]; fb = f; }
                            if (d.scores_user) {
#pragma unroll
                                for (int f = 0; f < NF; f++)
                                    if (f < nf_real) d.scores_user[((size_t)f * d.nu + u) * d.nv + v] = sc[f];
                            }
                            if (d.keys)
                                d.keys[(size_t)u * d.nv + v] =
                                    (d.scan && best > threshold) ? make_key(best, d.level, fb, u, v) : KEY_NONE;
                        }
                    }
                    idx -= b.nvs;
                    if (idx < 0) idx += wrap;
                    epi_sync();
                }
            }
        }
    }

    // ---- teardown: no copy or MMA may still be in flight when TMEM is
    // freed and the CTA exits
    __syncthreads();
    if (warp == 5 && s_abort) {
        for (int i = 0; i < TF_STAGES; i++) {
            if (issued[i] == 0) continue;
            long long spins = 0;
            while (!mbar_try(smem_addr(&bar_full[i]), (uint32_t)((issued[i] - 1) & 1)) && ++spins < TC_SPIN)
                __nanosleep(64);
        }
    }
    if (warp == 4) {
        if (lane == 0) mma_commit(smem_addr(&bar_drain));
        __syncwarp();
        long long spins = 0;
        while (!mbar_try(smem_addr(&bar_drain), 0u) && ++spins < TC_SPIN) __nanosleep(64);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(COLS)
                     : "memory");
    if (t == 0 && s_abort) atomicOr(flags + 2, 1);
}

namespace {
template <int NF>
cudaError_t launch_tcf_t(const LevelDesc *descs, const TcBand *bands, const int32_t *cta_first, int grid,
                         const uint16_t *wb, int nf_real, float threshold, int *flags,
                         cudaStream_t stream) {
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(corr_tcf_kernel<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tf_smem(NF));
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    if (grid > 0)
        corr_tcf_kernel<NF><<<grid, TF_NT, tf_smem(NF), stream>>>(descs, bands, cta_first, wb, nf_real,
                                                                  threshold, flags);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_corr_tcf(const LevelDesc *descs, const TcBand *bands, const int32_t *cta_first,
                            int grid, const uint16_t *wb, int nf_kernel, int nf_real, float threshold,
                            int *flags, cudaStream_t stream) {
    switch (nf_kernel) {
    case 1: return launch_tcf_t<1>(descs, bands, cta_first, grid, wb, nf_real, threshold, flags, stream);
    case 5: return launch_tcf_t<5>(descs, bands, cta_first, grid, wb, nf_real, threshold, flags, stream);
    case 8: return launch_tcf_t<8>(descs, bands, cta_first, grid, wb, nf_real, threshold, flags, stream);
    default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int NF>
cudaError_t launch_tc_t(const LevelDesc *descs, const Job *jobs, int njobs, const Job *rjobs,
                        int nrjobs, const uint16_t *wb, int nf_real, float threshold, int *flags,
                        int grid, cudaStream_t stream) {
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(corr_tc_kernel<NF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc_smem(NF));
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    if (njobs > 0) {
        corr_tc_kernel<NF><<<grid < njobs ? grid : njobs, TC_NT, tc_smem(NF), stream>>>(
            descs, jobs, njobs, wb, flags);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nrjobs > 0)
        corr_tc_reduce_kernel<NF><<<nrjobs, 256, 0, stream>>>(descs, rjobs, nf_real, threshold);
    return cudaGetLastError();
}
}  // namespace

size_t corr_tc_weights_halves(int nf_kernel) { return 2 * (size_t)WIN * 4 * tc_n(nf_kernel) * 8; }

cudaError_t launch_corr_tc_weights(const float *w, int nf_kernel, int nf_real, uint16_t *wb,
                                   cudaStream_t stream) {
    const int plane = WIN * 4 * tc_n(nf_kernel) * 8;
    const int grid = (plane + 255) / 256;
    switch (nf_kernel) {
    case 1: corr_tc_weights_kernel<1><<<grid, 256, 0, stream>>>(w, nf_real, wb); break;
    case 5: corr_tc_weights_kernel<5><<<grid, 256, 0, stream>>>(w, nf_real, wb); break;
    case 8: corr_tc_weights_kernel<8><<<grid, 256, 0, stream>>>(w, nf_real, wb); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_corr_tc(const LevelDesc *descs, const Job *jobs, int njobs, const Job *rjobs,
                           int nrjobs, const uint16_t *wb, int nf_kernel, int nf_real,
                           float threshold, int *flags, int grid, cudaStream_t stream) {
    switch (nf_kernel) {
    case 1: return launch_tc_t<1>(descs, jobs, njobs, rjobs, nrjobs, wb, nf_real, threshold, flags, grid, stream);
    case 5: return launch_tc_t<5>(descs, jobs, njobs, rjobs, nrjobs, wb, nf_real, threshold, flags, grid, stream);
    case 8: return launch_tc_t<8>(descs, jobs, njobs, rjobs, nrjobs, wb, nf_real, threshold, flags, grid, stream);
    default: return cudaErrorInvalidValue;
    }
}

int corr_tc_ctas_per_sm(int nf_kernel) {
    const size_t per = tc_smem(nf_kernel) + 1024;   // plus the per-CTA reservation
    const int n = (int)((228 * 1024) / per);
    return n < 1 ? 1 : n;
}

}  // namespace hogk
