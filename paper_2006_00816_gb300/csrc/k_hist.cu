// k_hist.cu -- stand-alone launch of the gradient / orientation / cell
// histogram stage (Section 4.1.1: gradient computation and
// histogramisation); the stage itself is hist_tile() in hog_stages.cuh.
#include "hog_stages.cuh"

namespace hogk {

__global__ void __launch_bounds__(hist_cfg::NT, 2) hist_kernel(const LevelDesc *__restrict__ descs,
                                                               const Job *__restrict__ jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Job jb = jobs[blockIdx.x];
    hist_tile(descs[jb.desc], jb.tile, smem);
}

cudaError_t launch_hist(const LevelDesc *descs, const Job *jobs, int njobs,
                        cudaStream_t stream) {
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)hist_cfg::SMEM);
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    if (njobs <= 0) return cudaSuccess;
    hist_kernel<<<njobs, hist_cfg::NT, hist_cfg::SMEM, stream>>>(descs, jobs);
    return cudaGetLastError();
}

}  // namespace hogk
