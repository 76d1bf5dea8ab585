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
#include "hog_internal.cuh"

namespace hogk {

__global__ void __launch_bounds__(256) pyramid_step_kernel(const LevelDesc *__restrict__ descs,
                                                           const Job *__restrict__ jobs) {
    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int ntx = (d.w + PYR_TX - 1) / PYR_TX;
    const int tx = jb.tile % ntx, ty = jb.tile / ntx;
    const int x = tx * PYR_TX + (threadIdx.x & 31) * 4;
    const int y = ty * PYR_TY + (threadIdx.x >> 5);
    if (y >= d.h || x >= d.w) return;

    const int Y = 12 * y + 1;
    const int y0 = Y / 10, fy = Y - 10 * (Y / 10);
    const uint8_t *r0 = d.src + (size_t)y0 * d.spitch;
    const uint8_t *r1 = r0 + d.spitch;
    uint32_t packed = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int xx = x + k;
        if (xx < d.w) {
            const int X = 12 * xx + 1;
            const int x0 = X / 10, fx = X - 10 * (X / 10);
            const int p00 = __ldg(r0 + x0), p10 = __ldg(r0 + x0 + 1);
            const int p01 = __ldg(r1 + x0), p11 = __ldg(r1 + x0 + 1);
            const int acc = (10 - fx) * (10 - fy) * p00 + fx * (10 - fy) * p10 +
                            (10 - fx) * fy * p01 + fx * fy * p11;
            packed |= (uint32_t)((acc + 50) / 100) << (8 * k);
        }
    }
    uint8_t *out = d.dst + (size_t)y * d.pitch + x;
    if (x + 3 < d.w) {
        *reinterpret_cast<uint32_t *>(out) = packed;   // pitch and x are multiples of 4
    } else {
        for (int k = 0; k < 4 && x + k < d.w; k++) out[k] = (uint8_t)(packed >> (8 * k));
    }
}

cudaError_t launch_pyramid(const LevelDesc *descs, const Job *jobs, int njobs,
                           cudaStream_t stream) {
    if (njobs <= 0) return cudaSuccess;
    pyramid_step_kernel<<<njobs, 256, 0, stream>>>(descs, jobs);
    return cudaGetLastError();
}

}  // namespace hogk
