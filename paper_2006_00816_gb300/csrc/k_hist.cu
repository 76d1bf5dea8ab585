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
// atomics.  Here the pixels between four neighbouring cell centres form an
// 8x8 "block" (block (bi, bj) spans x in [8bj-4, 8bj+4), y in [8bi-4,
// 8bi+4)); all of a block's pixels vote into the same four cells (bi-1 or
// bi) x (bj-1 or bj).  One thread owns one block: it computes its 64
// pixels' gradients, bins and magnitudes straight from the staged bytes and
// accumulates four private partial histograms (one per corner cell) in
// shared memory, laid out [corner][bin][thread] so a warp's 32 lanes always
// hit 32 banks.  A cell's histogram is then the fixed-order sum of the
// partials of its four blocks: deterministic, no atomics, and no sum longer
// than 64 terms.  A CTA owns 16x16 blocks and emits the 15x15 cells whose
// four blocks it holds.
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

constexpr int NT = HIST_BX * HIST_BY;          // 256 threads, one per block
constexpr int PX = HIST_BX * CELL + 2;         // 130 staged columns (blocks + 1-px halo)
constexpr int PY = HIST_BY * CELL + 2;         // 130 staged rows
constexpr int NCH = 10;                        // 16-byte chunks per staged row (130 + 15 <= 160)
constexpr int SROWB = NCH * 16;                // 160 bytes per staged row
constexpr size_t SMEM_SRC = (size_t)PY * SROWB;                     // 20,800
constexpr size_t SMEM_PART = sizeof(float) * 4 * NBIN * NT;         // 73,728
constexpr size_t SMEM_TOTAL = SMEM_PART + SMEM_SRC;

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

__global__ void __launch_bounds__(NT, 2) hist_kernel(const LevelDesc *__restrict__ descs,
                                                     const Job *__restrict__ jobs) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *part = reinterpret_cast<float *>(smem);             // [4][18][NT]
    uint8_t *srcS = smem + SMEM_PART;                          // [PY][SROWB]
    __shared__ int xbase[PY];

    const Job jb = jobs[blockIdx.x];
    const LevelDesc &d = descs[jb.desc];
    const int ntx = (d.cx + HIST_TX - 1) / HIST_TX;
    const int j0 = (jb.tile % ntx) * HIST_TX, i0 = (jb.tile / ntx) * HIST_TY;
    const int t = threadIdx.x;
    const int xmax = min(d.w - 2, CELL * d.cx - 1);
    const int ymax = min(d.h - 2, CELL * d.cy - 1);

    // Stage rows Ys .. Ys+PY-1, columns Xs .. Xs+PX-1 (clipped to the image)
    // with 16-byte cp.async copies of the aligned chunks covering them.  A
    // 16-byte-aligned chunk holding at least one byte of the frame lies on
    // that byte's memory page, so the copies stay in mapped memory even
    // where they reach past the clipped range; those bytes are never read.
    // xbase[r] = image column of staged byte 0 of staged row r.
    const int Xs = CELL * j0 - 5, Ys = CELL * i0 - 5;
    const int xa = max(Xs, 0), xb = min(Xs + PX, d.w);
    for (int idx = t; idx < PY * NCH; idx += NT) {
        const int r = idx / NCH, ci = idx - r * NCH;
        const int Y = Ys + r;
        if (Y < 0 || Y >= d.h || xa >= xb) continue;
        const uintptr_t rp = (uintptr_t)(d.img + (size_t)Y * d.pitch);
        const uintptr_t c0 = (rp + (uintptr_t)xa) & ~(uintptr_t)15;
        const uintptr_t a = c0 + 16 * (uintptr_t)ci;
        if (ci == 0) xbase[r] = (int)((intptr_t)c0 - (intptr_t)rp);
        if (a <= rp + (uintptr_t)(xb - 1)) cp_async16(srcS + r * SROWB + 16 * ci, (const void *)a);
    }
    for (int k = t; k < 4 * NBIN * NT; k += NT) part[k] = 0.0f;
    cp_async_wait_all();
    __syncthreads();

    // one 8x8 block per thread: pixels X = 8 bj - 4 + ox, Y = 8 bi - 4 + oy
    const int by = t / HIST_BX, bx = t - by * HIST_BX;
    const int X0 = CELL * (j0 + bx) - 4, Y0 = CELL * (i0 + by) - 4;
    float *p0 = part + t;
#pragma unroll 1
    for (int oy = 0; oy < 8; oy++) {
        const int Y = Y0 + oy;
        if (Y < 1 || Y > ymax) continue;
        const int r = Y - Ys;                       // staged row of Y
        const uint8_t *up = srcS + (r - 1) * SROWB - xbase[r - 1];
        const uint8_t *mid = srcS + r * SROWB - xbase[r];
        const uint8_t *dn = srcS + (r + 1) * SROWB - xbase[r + 1];
        const float wy1 = tent16(oy), wy0 = tent16(oy + 8);   // to cell rows bi, bi-1
#pragma unroll
        for (int ox = 0; ox < 8; ox++) {
            const int X = X0 + ox;
            if (X < 1 || X > xmax) continue;
            const int dx = (int)mid[X + 1] - (int)mid[X - 1];
            const int dy = (int)dn[X] - (int)up[X];
            if ((dx | dy) == 0) continue;
            const int b = orientation_bin_i(dx, dy);
            const float m = sqrtf((float)(dx * dx + dy * dy));
            const float wx1 = tent16(ox), wx0 = tent16(ox + 8);   // to cell cols bj, bj-1
            float *pb = p0 + b * NT;
            pb[0 * NBIN * NT] += m * (wy0 * wx0);   // cell (bi-1, bj-1)
            pb[1 * NBIN * NT] += m * (wy0 * wx1);   // cell (bi-1, bj)
            pb[2 * NBIN * NT] += m * (wy1 * wx0);   // cell (bi,   bj-1)
            pb[3 * NBIN * NT] += m * (wy1 * wx1);   // cell (bi,   bj)
        }
    }
    __syncthreads();

    // cell (ci, cj) of the tile = blocks (ci,cj) corner 3 + (ci,cj+1) corner 2
    // + (ci+1,cj) corner 1 + (ci+1,cj+1) corner 0; staged for a coalesced store
    float *outS = reinterpret_cast<float *>(srcS);   // [15*15][18] = 16,200 bytes
    if (t < HIST_TX * HIST_TY) {
        const int ci = t / HIST_TX, cj = t - ci * HIST_TX;
        const int b00 = ci * HIST_BX + cj;
#pragma unroll
        for (int b = 0; b < NBIN; b++) {
            const float s3 = part[(3 * NBIN + b) * NT + b00];
            const float s2 = part[(2 * NBIN + b) * NT + b00 + 1];
            const float s1 = part[(1 * NBIN + b) * NT + b00 + HIST_BX];
            const float s0 = part[(0 * NBIN + b) * NT + b00 + HIST_BX + 1];
            outS[t * NBIN + b] = (s3 + s2) + (s1 + s0);
        }
    }
    __syncthreads();
    const int ncol = min(HIST_TX, d.cx - j0);
    for (int r = 0; r < HIST_TY; r++) {
        const int i = i0 + r;
        if (i >= d.cy) break;
        float *dst = d.hist + ((size_t)i * d.cx + j0) * NBIN;
        const float *srcr = outS + r * HIST_TX * NBIN;
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
