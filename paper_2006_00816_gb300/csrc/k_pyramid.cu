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
