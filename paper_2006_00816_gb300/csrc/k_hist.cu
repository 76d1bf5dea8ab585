// k_hist.cu -- gradient, orientation binning and cell histograms
// (Section 4.1.1: gradient computation and histogramisation).
//
// Per pixel: central differences dx = I(x+1,y)-I(x-1,y), dy = I(x,y+1)-I(x,y-1)
// for 1 <= x <= min(w-2, 8cx-1), 1 <= y <= min(h-2, 8cy-1); magnitude
// sqrt(dx^2+dy^2); one of 18 signed orientations (centres at 20 b degrees,
// the nearest one).  Each pixel votes magnitude x tent weight into the four
// nearest 8x8 cells (cell centres at 8j+4, weight 1 - |offset|/8 per axis).
//
// GB300 design.  The paper scatters votes with fixed-point shared-memory
// atomics.  Here each thread owns one cell and gathers its 16x16-pixel
// footprint in a fixed order, so the result is deterministic and needs no
// atomics:
//   phase 1: the CTA computes (bin, magnitude) for its 264x40-pixel region
//            (32x4 cells + half-cell borders) into shared memory;
//   phase 2: each thread walks its footprint as four 8x8 quadrants at once
//            (four independent read-modify-write chains into private
//            shared-memory partial histograms), then adds the quadrants.
// Shared layouts put the 32 lanes of a warp (32 consecutive cells) on 32
// different banks: pixel column rc is stored at (rc & 7) * 33 + (rc >> 3).
//
// Orientation in exact integer arithmetic: fold (dx, dy) into the first
// quadrant; the sector there is the number of bin boundaries (10, 30, 50 and
// 70 degrees) the vector lies beyond, tested as |dy| C - |dx| S > 0 with C, S
// = round(2^20 cos, 2^20 sin) of the boundary angle.  For every 8-bit
// gradient the exact test and this one agree (the smallest |dy cos - dx sin|
// over the grid is 1.3e-3, i.e. 1340 units at 2^20, against a rounding error
// of at most 255 units), and the products fit in int32.  dx == 0 (the only
// exact tie, between 80/100 or 260/280 degrees) goes to bin 4 or 13.
#include "hog_internal.cuh"

namespace hogk {

namespace {

constexpr int RX = HIST_TX * CELL + CELL;   // 264 region columns
constexpr int RY = HIST_TY * CELL + CELL;   // 40 region rows
constexpr int SXW = RX + 4;                 // staged source row (266 used)
constexpr int SYH = RY + 2;                 // 42 staged source rows
constexpr int PLANE = 33;                   // (rc & 7) plane stride
constexpr int MROW = 8 * PLANE;             // 264 entries per region row
constexpr int NT = HIST_TX * HIST_TY;       // 128 threads = cells per CTA

constexpr size_t SMEM_MAG = sizeof(float) * RY * MROW;             // 42,240
constexpr size_t SMEM_BIN = sizeof(uint8_t) * RY * MROW;           // 10,560
constexpr size_t SMEM_SRC = sizeof(uint8_t) * SYH * SXW;           // 11,256
constexpr size_t SMEM_QH = sizeof(float) * 4 * NBIN * NT;          // 36,864
constexpr size_t SMEM_U = SMEM_QH > SMEM_SRC ? SMEM_QH : SMEM_SRC; // src and qh alias
constexpr size_t SMEM_TOTAL = SMEM_MAG + SMEM_BIN + SMEM_U;

__device__ __forceinline__ int orientation_bin_i(int dx, int dy) {
    if (dx == 0) return dy > 0 ? 4 : 13;
    const int ax = dx < 0 ? -dx : dx;
    const int ay = dy < 0 ? -dy : dy;
    const int q = (ay * 1032646 - ax * 182083 > 0) + (ay * 908093 - ax * 524288 > 0) +
                  (ay * 674012 - ax * 803256 > 0) + (ay * 358634 - ax * 985339 > 0);
    if (dx > 0) return dy >= 0 ? q : (q == 0 ? 0 : 18 - q);
    return dy >= 0 ? 9 - q : 9 + q;
}

// Tent weight of footprint offset t (0..15) in sixteenths: 16 - |2t - 15|.
__host__ __device__ constexpr float tent16(int t) {
    return (float)(16 - (2 * t - 15 < 0 ? 15 - 2 * t : 2 * t - 15)) * (1.0f / 16.0f);
}

}  // namespace

__global__ void __launch_bounds__(NT) hist_kernel(const LevelDesc *__restrict__ descs,
                                                  const Job *__restrict__ jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *magS = reinterpret_cast<float *>(smem);
    uint8_t *binS = smem + SMEM_MAG;
    unsigned char *uni = smem + SMEM_MAG + SMEM_BIN;
    uint8_t *srcS = uni;
    float *qh = reinterpret_cast<float *>(uni);

    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int ntx = (d.cx + HIST_TX - 1) / HIST_TX;
    const int j0 = (jb.tile % ntx) * HIST_TX, i0 = (jb.tile / ntx) * HIST_TY;
    const int t = threadIdx.x;
    const int X0 = CELL * j0 - 4, Y0 = CELL * i0 - 4;   // region origin (pixels)
    const int xmax = min(d.w - 2, CELL * d.cx - 1);
    const int ymax = min(d.h - 2, CELL * d.cy - 1);

    // stage source pixels [Y0-1, Y0+RY] x [X0-1, X0+RX]
    for (int p = t; p < SYH * (RX + 2); p += NT) {
        const int sy = p / (RX + 2), sx = p - sy * (RX + 2);
        const int Y = Y0 - 1 + sy, X = X0 - 1 + sx;
        uint8_t v = 0;
        if (X >= 0 && X < d.w && Y >= 0 && Y < d.h) v = __ldg(d.img + (size_t)Y * d.pitch + X);
        srcS[sy * SXW + sx] = v;
    }
    __syncthreads();

    // phase 1: (bin, magnitude) of every region pixel; non-voting pixels get 0
    for (int p = t; p < RX * RY; p += NT) {
        const int ry = p / RX, rx = p - ry * RX;
        const int X = X0 + rx, Y = Y0 + ry;
        float m = 0.0f;
        int b = 0;
        if (X >= 1 && X <= xmax && Y >= 1 && Y <= ymax) {
            const uint8_t *s = srcS + (ry + 1) * SXW + (rx + 1);
            const int dx = (int)s[1] - (int)s[-1];
            const int dy = (int)s[SXW] - (int)s[-SXW];
            if (dx != 0 || dy != 0) {
                b = orientation_bin_i(dx, dy);
                m = sqrtf((float)(dx * dx + dy * dy));
            }
        }
        const int idx = ry * MROW + (rx & 7) * PLANE + (rx >> 3);
        magS[idx] = m;
        binS[idx] = (uint8_t)b;
    }
    __syncthreads();   // srcS is dead from here on; qh reuses its space

    // phase 2: zero the private quadrant histograms, then gather
    for (int k = t; k < 4 * NBIN * NT; k += NT) qh[k] = 0.0f;
    __syncthreads();

    const int ti = t / HIST_TX, tj = t - ti * HIST_TX;
#pragma unroll
    for (int dy = 0; dy < 8; dy++) {
#pragma unroll
        for (int dx = 0; dx < 8; dx++) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int qy = q >> 1, qx = q & 1;
                const int idx = (8 * ti + 8 * qy + dy) * MROW + dx * PLANE + tj + qx;
                const float m = magS[idx];
                const int b = binS[idx];
                float *h = qh + (q * NBIN + b) * NT + t;
                *h += m * (tent16(8 * qx + dx) * tent16(8 * qy + dy));
            }
        }
    }
    __syncthreads();

    // sum quadrants, stage [cell][18] in magS, then coalesced copy out
    float *hs = magS;
#pragma unroll
    for (int b = 0; b < NBIN; b++) {
        const float s01 = qh[(0 * NBIN + b) * NT + t] + qh[(1 * NBIN + b) * NT + t];
        const float s23 = qh[(2 * NBIN + b) * NT + t] + qh[(3 * NBIN + b) * NT + t];
        hs[t * NBIN + b] = s01 + s23;
    }
    __syncthreads();
    const int ncol = min(HIST_TX, d.cx - j0);
    for (int r = 0; r < HIST_TY; r++) {
        const int i = i0 + r;
        if (i >= d.cy) break;
        float *dst = d.hist + ((size_t)i * d.cx + j0) * NBIN;
        const float *srcr = hs + r * HIST_TX * NBIN;
        for (int k = t; k < ncol * NBIN; k += NT) dst[k] = srcr[k];
    }
}

cudaError_t launch_hist(const LevelDesc *descs, const Job *jobs, int njobs,
                        cudaStream_t stream) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM_TOTAL);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (njobs <= 0) return cudaSuccess;
    hist_kernel<<<njobs, NT, SMEM_TOTAL, stream>>>(descs, jobs);
    return cudaGetLastError();
}

}  // namespace hogk
