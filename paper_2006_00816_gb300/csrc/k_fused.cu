// k_fused.cu -- one persistent launch that runs the pyramid, histogram,
// feature and correlation stages of every frame and level of a batch
// (the paper batches frames along the grid's z dimension and gives each
// scale its own stream, Section 5.1; here frames of any size and all their
// levels share one launch, and the launch is replayed as a CUDA graph).
//
// Work items are (stage, frame, level, tile) or, for the correlation, a
// group of up to 8 warp tiles of one level.  The host orders them by
// dependency depth -- pyramid level l at depth l, histograms of level l at
// l+1, features at l+2, correlation at l+3 -- so every item only depends on
// items that come earlier in the list.  CTAs take items in list order from
// a global ticket counter; an item whose inputs are not complete waits on
// the completion counter of the (frame, level, stage) it needs.  An item
// that is waited on has a smaller ticket, so it has already been taken by a
// running CTA, which never waits on anything later: the schedule cannot
// deadlock, even when not every CTA is resident.
//
// Waits are bounded: after spin_limit polls (2^24 by default, set by
// hog_debug_waits) the kernel raises a global abort flag and every CTA stops
// taking items, so a fault in the schedule ends the launch with an error
// status (read by the host as HOG_ETIMEOUT) instead of a hang.  A wait is
// taken before the item's work starts, so a CTA that stops has no copy in
// flight.
//
// Completion uses release/acquire at GPU scope (__threadfence then
// atomicAdd; ld.acquire.gpu polls), and every stage reads data produced in
// this launch through L2 (cp.async.cg, ld.global.cg), never from a stale L1.
#include "hog_stages.cuh"

namespace hogk {

namespace {
constexpr int FUSED_NT = 256;
constexpr int FUSED_CORR_WARPS = FUSED_NT / 32;   // 8 warp tiles per correlation item
// 8x16 and 16x8 tiles only (17x25 = 425 cells): 110.6 KB of staging, so two
// CTAs fit on an SM
constexpr int FUSED_BUF4 = 432;
static_assert((8 + WIN - 1) * (16 + WIN - 1) <= FUSED_BUF4, "fused staging holds an 8x16 tile region");
constexpr size_t FUSED_SMEM_CORR = sizeof(float4) * FUSED_BUF4 * 2 * FUSED_CORR_WARPS;
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t FUSED_SMEM = cmax(cmax(FUSED_SMEM_CORR, hist_cfg::SMEM), feat_cfg::SMEM);

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
}  // namespace

// two CTAs per SM (128 registers) up to 5 filters; 8 filters need more registers
constexpr int fused_minb(int nf) { return nf <= 5 ? 2 : 1; }

template <int NF>
__global__ void __launch_bounds__(FUSED_NT, fused_minb(NF)) fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_ok;
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) s_item = atomicAdd(a.head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) break;
        const FusedItem item = a.items[it];
        if (t == 0) {
            int ok = 1;
            if (*((volatile int *)a.abort)) ok = 0;
            if (ok && item.wait >= 0) {
                long long spins = 0;
                while (ld_acquire(a.ctr + item.wait) < item.target) {
                    if (*((volatile int *)a.abort)) { ok = 0; break; }
                    if (++spins > a.spin_limit) {
                        atomicExch(a.abort, 1);
                        atomicOr(a.flags + 2, 1);
                        ok = 0;
                        break;
                    }
                    if (spins > 32) __nanosleep(64);
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        switch (item.kind) {
        case FUSED_PYR:
            pyramid_tile<true>(a.descs[item.a], item.b);
            break;
        case FUSED_HIST:
            hist_tile(a.descs[item.a], item.b, smem);
            break;
        case FUSED_FEAT:
            feat_tile<true>(a.descs[item.a], item.b, a.eps, a.tau, smem);
            break;
        case FUSED_CORR: {
            const int w = t >> 5;
            if (w < item.b)
                corr_warp_job<NF, FUSED_BUF4>(a.descs, a.jobs[item.a + w], a.wchunks, a.nf_real,
                                              a.threshold,
                                              reinterpret_cast<float4 *>(smem) + (size_t)w * 2 * FUSED_BUF4);
            break;
        }
        default:
            break;
        }
        __syncthreads();
        if (t == 0 && item.done >= 0) {
            __threadfence();
            atomicAdd(a.ctr + item.done, 1);
        }
    }
}

template <int NF>
static cudaError_t launch_fused_t(const FusedArgs &a, int grid, cudaStream_t stream) {
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(fused_kernel<NF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)FUSED_SMEM);
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    fused_kernel<NF><<<grid, FUSED_NT, FUSED_SMEM, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fused(const FusedArgs &a, int nf_kernel, int grid, cudaStream_t stream) {
    if (a.nitems <= 0) return cudaSuccess;
    switch (nf_kernel) {
    case 1: return launch_fused_t<1>(a, grid, stream);
    case 5: return launch_fused_t<5>(a, grid, stream);
    case 8: return launch_fused_t<8>(a, grid, stream);
    default: return cudaErrorInvalidValue;
    }
}

int fused_max_ctas_per_sm(int nf_kernel) {
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (nf_kernel) {
    case 1: e = cudaFuncSetAttribute(fused_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel<1>, FUSED_NT, FUSED_SMEM); break;
    case 5: e = cudaFuncSetAttribute(fused_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel<5>, FUSED_NT, FUSED_SMEM); break;
    case 8: e = cudaFuncSetAttribute(fused_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_kernel<8>, FUSED_NT, FUSED_SMEM); break;
    default: break;
    }
    if (e != cudaSuccess) { cudaGetLastError(); return 1; }
    return n > 0 ? n : 1;
}

}  // namespace hogk
