// k_pyramid.cu -- one 5/6 step of the scale-space pyramid (Section 4.1.1,
// first step; Section 5.1, image-scaling kernel).
//
// Output pixel (x, y) of level l+1 samples level l at the pixel-centre
// aligned coordinate ((12x+1)/10, (12y+1)/10): x0 = (12x+1) div 10 and a
// fractional weight fx = (12x+1) mod 10 in tenths, likewise y.  The value
//   ((10-fx)(10-fy) p00 + fx(10-fy) p10 + (10-fx) fy p01 + fx fy p11 + 50) / 100
// (integer division) is the exact bilinear sample rounded half up, so the
// pyramid is integer-exact: no texture unit, no float rounding.
// For x < floor(5w/6), x0 + 1 <= w - 1, so no clamping is needed.  Each
// thread computes 20 consecutive outputs (pyramid_tile in hog_stages.cuh).
#include <algorithm>

#include "hog_stages.cuh"

namespace hogk {

__global__ void __launch_bounds__(256) pyramid_step_kernel(const LevelDesc *__restrict__ descs,
                                                           const Job *__restrict__ jobs) {
    const Job jb = jobs[blockIdx.x];
    pyramid_tile<false, false>(descs[jb.desc], jb.tile);
}

// Direct-to-size levels (hog_params.direct_first): read the frame, so they
// run before the 5/6 steps.
__global__ void __launch_bounds__(256) pyramid_direct_kernel(const LevelDesc *__restrict__ descs,
                                                             const Job *__restrict__ jobs) {
    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int ntx = (d.w + PYR_TX - 1) / PYR_TX;
    const int x = (jb.tile % ntx) * PYR_TX + (threadIdx.x & 7) * PYR_GROUP;
    const int y = (jb.tile / ntx) * PYR_TY + (threadIdx.x >> 3);
    if (y < d.h && x < d.w) pyramid_direct_tile<false>(d, x, y);
}

// The steps of a small batch's pyramid in one cluster: CTA r of the cluster
// takes jobs r, r + size, ... of each step; the cluster barrier (release /
// acquire at cluster scope) makes a step's levels visible to the next, whose
// reads go through L2 (coherent loads).  Every CTA runs every step, so every
// barrier is reached by all of them.
__global__ void __launch_bounds__(256) pyramid_chain_kernel(const LevelDesc *__restrict__ descs,
                                                            const Job *__restrict__ jobs, PyrChain chain) {
    unsigned rank, size;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(size));
    for (int k = 0; k < chain.nsteps; k++) {
        for (int j = (int)rank; j < chain.count[k]; j += (int)size) {
            const Job jb = jobs[chain.first[k] + j];
            pyramid_tile<true, true>(descs[jb.desc], jb.tile);
        }
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                     ::: "memory");
    }
}

namespace {
PerDevice g_chain_setup;
int g_chain_size[64];   // cluster size the chain kernel runs with per device (0: none)
}  // namespace

int pyramid_chain_size() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    const cudaError_t e = g_chain_setup.once([&]() -> cudaError_t {
        g_chain_size[dev] = 0;
        if (cudaFuncSetAttribute(pyramid_chain_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            cudaGetLastError();
        for (int c = 16; c >= 8; c >>= 1) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(256);
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, pyramid_chain_kernel, &cfg) == cudaSuccess && n > 0) {
                g_chain_size[dev] = c;
                break;
            }
            cudaGetLastError();
        }
        return cudaSuccess;
    });
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return g_chain_size[dev];
}

cudaError_t launch_pyramid_chain(const LevelDesc *descs, const Job *jobs, const PyrChain &chain,
                                 cudaStream_t stream) {
    const int c = pyramid_chain_size();
    int max_step = 0;
    for (int k = 0; k < chain.nsteps; k++) max_step = std::max(max_step, (int)chain.count[k]);
    if (c == 0 || max_step > c) return cudaErrorNotSupported;
    if (chain.nsteps <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pyramid_chain_kernel, descs, jobs, chain);
}

cudaError_t launch_pyramid(const LevelDesc *descs, const Job *jobs, int njobs,
                           cudaStream_t stream) {
    if (njobs <= 0) return cudaSuccess;
    pyramid_step_kernel<<<njobs, 256, 0, stream>>>(descs, jobs);
    return cudaGetLastError();
}

cudaError_t launch_pyramid_direct(const LevelDesc *descs, const Job *jobs, int njobs,
                                  cudaStream_t stream) {
    if (njobs <= 0) return cudaSuccess;
    pyramid_direct_kernel<<<njobs, 256, 0, stream>>>(descs, jobs);
    return cudaGetLastError();
}

}  // namespace hogk
