// k_feat.cu -- stand-alone launch of the energy / normalisation /
// truncation / 31-feature stage (Section 4.1.1: normalisation and feature
// computation); the stage itself is feat_tile() in hog_stages.cuh.
#include "hog_stages.cuh"

namespace hogk {

// Five CTAs per SM (48 registers): measured faster than four CTAs at 62
// registers with the two-cell halo staging.
__global__ void __launch_bounds__(feat_cfg::NT, 5)
    feat_kernel(const LevelDesc *__restrict__ descs, const Job *__restrict__ jobs, float eps, float tau) {
    __shared__ __align__(16) unsigned char smem[feat_cfg::SMEM];
    const Job jb = jobs[blockIdx.x];
    feat_tile<false>(descs[jb.desc], jb.tile, eps, tau, smem);
}

cudaError_t launch_feat(const LevelDesc *descs, const Job *jobs, int njobs, float eps,
                        float tau, cudaStream_t stream) {
    if (njobs <= 0) return cudaSuccess;
    feat_kernel<<<njobs, feat_cfg::NT, 0, stream>>>(descs, jobs, eps, tau);
    return cudaGetLastError();
}

}  // namespace hogk
