// k_corr.cu -- stand-alone launch of the multi-filter correlation +
// threshold + candidate-key stage (Section 4.1.1: linear classification
// filter and detection); the stage itself is corr_warp_job() in
// hog_stages.cuh.  Four independent warps per CTA, one warp tile each.
#include "hog_stages.cuh"

namespace hogk {

namespace {
constexpr int NT = 32 * CORR_WARPS;
constexpr size_t SMEM = sizeof(float4) * CORR_BUF4 * 2 * CORR_WARPS;
// 8 filters need 128 accumulator registers per lane: two CTAs per SM
constexpr int corr_minb(int nf) { return nf > 5 ? 2 : HOG_CORR_MINB; }
}  // namespace

template <int NF>
__global__ void __launch_bounds__(NT, corr_minb(NF)) corr_kernel(const LevelDesc *__restrict__ descs,
                                                                 const Job *__restrict__ jobs,
                                                                 int njobs,
                                                                 const float *__restrict__ wchunks,
                                                                 int nf_real, float threshold) {
    extern __shared__ float4 sm4[];
    const int w = threadIdx.x >> 5;
    const int jid = blockIdx.x * CORR_WARPS + w;
    if (jid >= njobs) return;
    corr_warp_job<NF>(descs, jobs[jid], wchunks, nf_real, threshold,
                      sm4 + (size_t)w * 2 * CORR_BUF4);
}

template <int NF>
static cudaError_t launch_corr_t(const LevelDesc *descs, const Job *jobs, int njobs,
                                 const float *wchunks, int nf_real, float threshold,
                                 cudaStream_t stream) {
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(corr_kernel<NF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM);
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    if (njobs <= 0) return cudaSuccess;
    const int grid = (njobs + CORR_WARPS - 1) / CORR_WARPS;
    corr_kernel<NF><<<grid, NT, SMEM, stream>>>(descs, jobs, njobs, wchunks, nf_real, threshold);
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
