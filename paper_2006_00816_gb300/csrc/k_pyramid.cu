// k_pyramid.cu -- one 5/6 step of the scale-space pyramid (Section 4.1.1,
// first step; Section 5.1, image-scaling kernel).
//
// Output pixel (x, y) of level l+1 samples level l at the pixel-centre
// aligned coordinate ((12x+1)/10, (12y+1)/10): x0 = (12x+1) div 10 and a
// fractional weight fx = (12x+1) mod 10 in tenths, likewise y.  The value
//   ((10-fx)(10-fy) p00 + fx(10-fy) p10 + (10-fx) fy p01 + fx fy p11 + 50) / 100
// (integer division) is the exact bilinear sample rounded half up, so the
// pyramid is integer-exact: no texture unit, no float rounding.
// For x < floor(5w/6), x0 + 1 <= w - 1, so no clamping is needed.
#include "hog_stages.cuh"

namespace hogk {

__global__ void __launch_bounds__(256) pyramid_step_kernel(const LevelDesc *__restrict__ descs,
                                                           const Job *__restrict__ jobs) {
    const Job jb = jobs[blockIdx.x];
    pyramid_tile<false>(descs[jb.desc], jb.tile);
}

cudaError_t launch_pyramid(const LevelDesc *descs, const Job *jobs, int njobs,
                           cudaStream_t stream) {
    if (njobs <= 0) return cudaSuccess;
    pyramid_step_kernel<<<njobs, 256, 0, stream>>>(descs, jobs);
    return cudaGetLastError();
}

}  // namespace hogk
