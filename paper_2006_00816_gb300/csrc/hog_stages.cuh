// hog_stages.cuh -- the stages of the detection path as device functions.
//
// Each stage is written once and used by two callers: the stand-alone stage
// kernels (one launch per stage over all frames of a batch, k_*.cu) and the
// persistent fused kernel (k_fused.cu), which runs all stages of many frames
// in one launch.  Template parameter COH ("coherent"): data produced earlier
// in the same launch (pyramid levels, histograms, candidate keys) must be
// read through L2 (ld.global.cg) rather than the non-coherent read-only path;
// stand-alone kernels read data of earlier launches and may use __ldg.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "hog_internal.cuh"

namespace hogk {

template <bool COH, typename T>
__device__ __forceinline__ T ld_in(const T *p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// ===========================================================================
// Pyramid (Section 4.1.1, first step; Section 5.1, image-scaling kernel).
// Output pixel (x, y) of level l+1 samples level l at ((12x+1)/10,
// (12y+1)/10) with exact weights in tenths, rounded half up (integer-exact).
//
// The mapping repeats every 5 output pixels: x = 5k + i samples source
// column 6k + i with weight fx = 2i + 1 tenths.  So 20 consecutive outputs
// x = 20k .. 20k+19 read exactly the 24 source bytes 24k .. 24k+23 of each
// of their two source rows: six aligned 32-bit loads per row, byte offsets
// and weights known at compile time, five 32-bit stores.  Tile PYR_TX x
// PYR_TY = 160 x 32 outputs, 256 threads (8 x 20 columns, 32 rows).  A
// group at a level's right edge takes the same path with its reads kept
// inside the source row and byte stores; only unaligned sources (a
// caller's frame) take the per-pixel path.
//
// Direct-to-size level (Section 6.6, future work): level s straight from
// the frame with the ratio (6/5)^s, source coordinate ((2x+1) 6^s - 5^s) /
// (2 5^s), weights in units of 1/(2 5^s), rounded half up; 64-bit integer
// arithmetic, exact.  s = d.dpow (2..8).
constexpr int PYR_GROUP = 20;   // output pixels per thread

// n / d for 0 <= n < 2^31, 0 < d < 2^31: an FP32 reciprocal estimate
// (within a few units of the quotient), then corrected to the exact floor.
__device__ __forceinline__ unsigned udiv_exact(unsigned n, unsigned d, float rd) {
    unsigned q = __float2uint_rz((float)n * rd);
    while (q > 0 && q * d > n) q--;          // q*d <= n < 2^31: no wrap
    while ((q + 1) * d <= n) q++;
    return q;
}

template <bool COH>
__device__ __noinline__ void pyramid_direct_tile(const LevelDesc &d, int x, int y) {
    if (d.dpow <= 4) {
        // 32-bit exact: X < 2^31 for widths up to 16384 (6^4 (2x+1) <
        // 4.3e7), D^2 * 255 * 4 < 2^31 (D = 2 * 5^4 = 1250)
        unsigned p6 = 1, p5 = 1;
        for (int k = 0; k < d.dpow; k++) { p6 *= 6; p5 *= 5; }
        const unsigned D = 2 * p5, D2 = D * D;
        const float rD = 1.0f / (float)D, rD2 = 1.0f / (float)D2;
        const unsigned Y = (2 * (unsigned)y + 1) * p6 - p5;
        const unsigned y0 = udiv_exact(Y, D, rD), fy = Y - D * y0;
        const uint8_t *r0 = d.src + (size_t)y0 * d.spitch;
        const uint8_t *r1 = r0 + d.spitch;
        uint8_t *out = d.dst + (size_t)y * d.pitch;
        // X advances by 2 * 6^s per output pixel: step x0 and fx without a
        // division per pixel
        const unsigned X0 = (2 * (unsigned)x + 1) * p6 - p5;
        unsigned x0 = udiv_exact(X0, D, rD), fx = X0 - D * x0;
        const unsigned qs = (2 * p6) / D, rs = (2 * p6) - D * qs;
        for (int xx = x; xx < x + PYR_GROUP && xx < d.w; xx++) {
            const unsigned p00 = ld_in<COH>(r0 + x0), p10 = ld_in<COH>(r0 + x0 + 1);
            const unsigned p01 = ld_in<COH>(r1 + x0), p11 = ld_in<COH>(r1 + x0 + 1);
            const unsigned acc = (D - fy) * ((D - fx) * p00 + fx * p10) + fy * ((D - fx) * p01 + fx * p11);
            out[xx] = (uint8_t)udiv_exact(acc + D2 / 2, D2, rD2);
            x0 += qs;
            fx += rs;
            if (fx >= D) { fx -= D; x0++; }
        }
        return;
    }
    long long p6 = 1, p5 = 1;
    for (int k = 0; k < d.dpow; k++) { p6 *= 6; p5 *= 5; }
    const long long D = 2 * p5;
    const long long Y = (2 * (long long)y + 1) * p6 - p5;
    const long long y0 = Y / D, fy = Y - D * y0;
    const uint8_t *r0 = d.src + (size_t)y0 * d.spitch;
    const uint8_t *r1 = r0 + d.spitch;
    uint8_t *out = d.dst + (size_t)y * d.pitch;
    for (int xx = x; xx < x + PYR_GROUP && xx < d.w; xx++) {
        const long long X = (2 * (long long)xx + 1) * p6 - p5;
        const long long x0 = X / D, fx = X - D * x0;
        const long long p00 = ld_in<COH>(r0 + x0), p10 = ld_in<COH>(r0 + x0 + 1);
        const long long p01 = ld_in<COH>(r1 + x0), p11 = ld_in<COH>(r1 + x0 + 1);
        const long long acc = (D - fx) * (D - fy) * p00 + fx * (D - fy) * p10 +
                              (D - fx) * fy * p01 + fx * fy * p11;
        out[xx] = (uint8_t)((acc + D * D / 2) / (D * D));
    }
}

// Byte o (compile-time) of the 24-byte window held in six words.
__device__ __forceinline__ int pyr_byte(const uint32_t (&w)[6], int o) {
    return (int)((w[o >> 2] >> (8 * (o & 3))) & 0xffu);
}

// DIRECT: the tile may be a direct-to-size level (d.dpow >= 2); the
// stand-alone 5/6-step kernel leaves that path out (direct levels have a
// launch of their own), the persistent fused kernel keeps it.
template <bool COH, bool DIRECT = true>
__device__ __forceinline__ void pyramid_tile(const LevelDesc &d, int tile) {
    const int ntx = (d.w + PYR_TX - 1) / PYR_TX;
    const int tx = tile % ntx, ty = tile / ntx;
    const int x = tx * PYR_TX + (threadIdx.x & 7) * PYR_GROUP;
    const int y = ty * PYR_TY + (threadIdx.x >> 3);
    if (y >= d.h || x >= d.w) return;
    if constexpr (DIRECT) {
        if (d.dpow >= 2) {
            pyramid_direct_tile<COH>(d, x, y);
            return;
        }
    }
    const int Y = 12 * y + 1;
    const int y0 = Y / 10, fy = Y - 10 * y0;
    const int wy0 = 10 - fy, wy1 = fy;
    const uint8_t *r0 = d.src + (size_t)y0 * d.spitch;
    const uint8_t *r1 = r0 + d.spitch;
    uint8_t *out = d.dst + (size_t)y * d.pitch + x;
    const int sx = (x / 5) * 6;   // first source column of the group
    // word reads where the rows are 4-byte aligned.  At the right edge of a
    // level the group's last source words or outputs may lie past the row:
    // only source bytes inside the row are read (no output in range needs
    // the others: x0 + 1 <= sw - 1; a word the row's end cuts is read byte
    // by byte), outputs past the width are not written
    const bool fast = ((reinterpret_cast<uintptr_t>(r0 + sx) | (uintptr_t)d.spitch) & 3u) == 0;
    if (fast) {
        const bool edge = x + PYR_GROUP > d.w || sx + 24 > d.sw;
        uint32_t a[6], b[6];
#pragma unroll
        for (int q = 0; q < 6; q++) {
            const int c = sx + 4 * q;   // first source column of word q
            if (!edge || c + 4 <= d.sw) {
                a[q] = ld_in<COH>(reinterpret_cast<const uint32_t *>(r0 + sx) + q);
                b[q] = ld_in<COH>(reinterpret_cast<const uint32_t *>(r1 + sx) + q);
            } else {
                a[q] = 0u;
                b[q] = 0u;
                for (int k = 0; k < 4 && c + k < d.sw; k++) {
                    a[q] |= (uint32_t)ld_in<COH>(r0 + c + k) << (8 * k);
                    b[q] |= (uint32_t)ld_in<COH>(r1 + c + k) << (8 * k);
                }
            }
        }
        uint32_t packed[5] = {0u, 0u, 0u, 0u, 0u};
        const uint32_t uw0 = (uint32_t)wy0, uw1 = (uint32_t)wy1;
#pragma unroll
        for (int i = 0; i < PYR_GROUP; i++) {
            const int o = (12 * i + 1) / 10;
            const uint32_t fx = (12 * i + 1) % 10;   // constants
            const uint32_t top = (10 - fx) * (uint32_t)pyr_byte(a, o) + fx * (uint32_t)pyr_byte(a, o + 1);
            const uint32_t bot = (10 - fx) * (uint32_t)pyr_byte(b, o) + fx * (uint32_t)pyr_byte(b, o + 1);
            const uint32_t acc = uw0 * top + uw1 * bot;
            packed[i >> 2] |= ((acc + 50u) / 100u) << (8 * (i & 3));
        }
        if (!edge) {
#pragma unroll
            for (int q = 0; q < 5; q++) reinterpret_cast<uint32_t *>(out)[q] = packed[q];   // x, pitch: 4 | .
        } else {
            for (int i = 0; i < PYR_GROUP && x + i < d.w; i++)
                out[i] = (uint8_t)(packed[i >> 2] >> (8 * (i & 3)));
        }
        return;
    }
    for (int i = 0; i < PYR_GROUP && x + i < d.w; i++) {
        const int X = 12 * (x + i) + 1;
        const int x0 = X / 10, fx = X - 10 * x0;
        const int p00 = ld_in<COH>(r0 + x0), p10 = ld_in<COH>(r0 + x0 + 1);
        const int p01 = ld_in<COH>(r1 + x0), p11 = ld_in<COH>(r1 + x0 + 1);
        const int acc = (10 - fx) * (10 - fy) * p00 + fx * (10 - fy) * p10 +
                        (10 - fx) * fy * p01 + fx * fy * p11;
        out[i] = (uint8_t)((acc + 50) / 100);
    }
}

// ===========================================================================
// Gradient, orientation binning, cell histograms (Section 4.1.1: gradient
// computation and histogramisation).
//
// Per pixel: central differences for 1 <= x <= min(w-2, 8cx-1),
// 1 <= y <= min(h-2, 8cy-1); magnitude sqrt(dx^2+dy^2); one of 18 signed
// orientations (nearest centre at 20 b degrees).  Each pixel votes
// magnitude x tent weight into the four nearest 8x8 cells.
//
// The pixels between four neighbouring cell centres form an 8x8 "block"
// (block (bi, bj) spans x in [8bj-4, 8bj+4), y in [8bi-4, 8bi+4)); all of a
// block's pixels vote into the same four cells.  One thread owns one block:
// it computes its 64 pixels from the staged bytes and accumulates four
// private partial histograms (one per corner cell) in shared memory, laid
// out [corner][bin][thread] so a warp's lanes hit 32 banks.  A cell is the
// fixed-order sum of its four blocks' partials: deterministic, no atomics,
// no sum longer than 64 terms.  256 threads own bw x (256 / bw) blocks and
// emit the (bw - 1) x (256 / bw - 1) cells whose four blocks they hold; bw
// is chosen per level to waste the fewest thread slots on the level's
// ragged edges (the cells' sums do not depend on it).
//
// Orientation: fold (dx, dy) into the first quadrant; the sector q is the
// number of bin boundaries (10, 30, 50, 70 degrees) the vector lies beyond.
// Each boundary test |dy| > |dx| tan(boundary) is one saturated FMA on the
// floating-point pipe: sat(2^20 |dy| - 1024 - |dx| T), T = fl32(2^20
// tan(boundary)), is exactly 1 or 0.  For every 8-bit gradient this equals
// the exact test: |dy| - |dx| tan(boundary) is at least 2.0e-3 away from 0
// on the integer grid (2097 after scaling), the margin is 1024 and the
// error of T times |dx| at most 32, so the FMA's value is >= 1057 or <= -1024.
// dx == 0 (the only exact tie) goes to bin 4 (dy > 0) or 13.
namespace hist_cfg {
constexpr int NT = HIST_NT;                    // 256 threads, one per block
// staged rows of a bw-wide tile: its 8 * bh pixel rows + a 1-px halo; row
// bytes: 8 bw + 2 columns + up to 15 bytes of 16-byte alignment slack
__host__ __device__ constexpr int py_of(int bw) { return CELL * hist_bh(bw) + 2; }
__host__ __device__ constexpr int nch_of(int bw) { return (CELL * bw + 32) / 16; }
constexpr size_t src_bytes_max() {
    size_t m = 0;
    for (int bw = HIST_BW_MIN; bw <= HIST_BW_MAX; bw++) {
        const size_t b = (size_t)py_of(bw) * nch_of(bw) * 16;
        const size_t o = sizeof(float) * NBIN * (bw - 1) * (hist_bh(bw) - 1);   // combined cells
        m = b > m ? b : m;
        m = o > m ? o : m;
    }
    return m;
}
constexpr int PY_MAX = py_of(HIST_BW_MIN);                          // 290 rows
constexpr size_t SMEM_SRC = src_bytes_max();                        // 24,768 (bw = 8)
constexpr int PB = NBIN + 1;                   // partial rows: bins 0..17 and 18 (= bin 0)
constexpr size_t SMEM_PART = sizeof(float) * 4 * PB * NT;           // 77,824
constexpr size_t SMEM_XB = sizeof(int) * ((PY_MAX + 3) / 4 * 4);    // 1,168
constexpr size_t SMEM = SMEM_PART + SMEM_SRC + SMEM_XB;             // 103,760
static_assert(SMEM_SRC % 16 == 0, "staging must keep 16-byte alignment");
}  // namespace hist_cfg

// dxf, dyf: the gradient as floats (exact integers, +0 for a zero part).
// Returns b * S for the bin b in 0..18 (18 is bin 0, taken apart by the
// caller) and a power of two S <= 2^18: 2^23 + b S is formed exactly in a
// float and its low mantissa bits are b S.
template <uint32_t S>
__device__ __forceinline__ uint32_t orientation_bin_f(float dxf, float dyf) {
    static_assert(S > 0 && S <= (1u << 18) && (S & (S - 1)) == 0, "S: a power of two <= 2^18");
    const float ax = fabsf(dxf), ay = fabsf(dyf);
    const float y = fmaf(ay, 1048576.0f, -1024.0f);   // 2^20 |dy| - 1024, exact
    // 2^20 tan 10, 30, 50, 70 degrees rounded to FP32
    const float q = __saturatef(fmaf(ax, -184892.234f, y)) + __saturatef(fmaf(ax, -605395.625f, y)) +
                    __saturatef(fmaf(ax, -1249644.25f, y)) + __saturatef(fmaf(ax, -2880939.0f, y));
    // quadrant: right half-plane (dx > 0, or dx == 0 and dy > 0): q or
    // 18 - q; left: 9 - q (dy >= 0) or 9 + q.  With sR, sU = +-1 for right
    // and dy >= 0 that is b = 9 + sU (sR (q - 4.5) - 4.5), the signs applied
    // as sign-bit flips; dx + 2^-20 dy carries the sign of dx, or of dy
    // where dx == 0.
    const uint32_t sr = __float_as_uint(fmaf(dyf, 9.5367431640625e-07f, dxf)) & 0x80000000u;
    const uint32_t su = __float_as_uint(dyf) & 0x80000000u;
    const float t = __uint_as_float(__float_as_uint(q - 4.5f) ^ sr) - 4.5f;
    return __float_as_uint(fmaf(__uint_as_float(__float_as_uint(t) ^ su), (float)S,
                                8388608.0f + 9.0f * (float)S)) & 0x7FFFFFu;   // (9 + sU t) S
}

// Byte k (0..3) of w as the float 2^23 + byte: the difference of two such
// floats is the bytes' difference, exactly.
__device__ __forceinline__ float byte_f23(uint32_t w, int k) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (unsigned)k));
}

// Tent weight of footprint offset t (0..15) in sixteenths: 16 - |2t - 15|.
__host__ __device__ constexpr float tent16(int t) {
    return (float)(16 - (2 * t - 15 < 0 ? 15 - 2 * t : 2 * t - 15)) * (1.0f / 16.0f);
}

// 256 threads; smem >= hist_cfg::SMEM, 16-byte aligned.  Reads the level
// image with cp.async.cg (through L2), so it is coherent within a launch.
__device__ __forceinline__ void hist_tile(const LevelDesc &d, int tile, unsigned char *smem) {
    using namespace hist_cfg;
    // partials [corner pair][19][NT] of float2: .x corner 2p, .y corner 2p+1;
    // row 18 collects bin 0's votes from below the positive x axis (bin
    // 18 - q at q = 0) and is added to row 0 when the cells are combined
    float2 *part = reinterpret_cast<float2 *>(smem);
    uint8_t *srcS = smem + SMEM_PART;                          // [py][srowb]
    int *xbase = reinterpret_cast<int *>(smem + SMEM_PART + SMEM_SRC);

    const int bw = d.hist_bw, bh = hist_bh(bw), tw = bw - 1, th = bh - 1;
    const int nch = nch_of(bw), srowb = 16 * nch, py = py_of(bw);
    const int ntx = (d.cx + tw - 1) / tw;
    const int j0 = (tile % ntx) * tw, i0 = (tile / ntx) * th;
    const int t = threadIdx.x;
    const int xmax = min(d.w - 2, CELL * d.cx - 1);
    const int ymax = min(d.h - 2, CELL * d.cy - 1);

    // Stage rows Ys .. Ys+py-1, columns Xs .. Xs+8bw+1 (clipped to the
    // image) with 16-byte cp.async copies of the aligned chunks covering
    // them.  A 16-byte-aligned chunk holding at least one byte of the frame
    // lies on that byte's memory page, so the copies stay in mapped memory
    // even where they reach past the clipped range; those bytes are never
    // read.  xbase[r] = image column of staged byte 0 of staged row r.
    const int Xs = CELL * j0 - 5, Ys = CELL * i0 - 5;
    const int xa = max(Xs, 0), xb = min(Xs + CELL * bw + 2, d.w);
    {
        // idx = r nch + ci walks t, t + NT, ...: one division up front, then
        // a carry from ci into r.  Every staged row gets its xbase (rows off
        // the image take the alignment of the nearest image row and are
        // never copied), so the row loop below may read any staged row.
        const int q0 = NT / nch, rem0 = NT - q0 * nch;
        int r = t / nch, ci = t - r * nch;
        while (r < py) {
            const int Y = Ys + r;
            const int Yc = min(max(Y, 0), d.h - 1);
            const uintptr_t rp = (uintptr_t)(d.img + (size_t)Yc * d.pitch);
            const uintptr_t c0 = (rp + (uintptr_t)xa) & ~(uintptr_t)15;
            const uintptr_t a = c0 + 16 * (uintptr_t)ci;
            if (ci == 0) xbase[r] = (int)((intptr_t)c0 - (intptr_t)rp);
            if (Y >= 0 && Y < d.h && xa < xb && a <= rp + (uintptr_t)(xb - 1))
                cp_async16(srcS + r * srowb + 16 * ci, (const void *)a);
            ci += rem0;
            r += q0;
            if (ci >= nch) {
                ci -= nch;
                r++;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PB; k++) reinterpret_cast<float4 *>(part)[k * NT + t] = make_float4(0.f, 0.f, 0.f, 0.f);
    cp_async_wait_all();
    __syncthreads();

    // one 8x8 block per thread (t < bw * bh): pixels X = 8 bj - 4 + ox,
    // Y = 8 bi - 4 + oy.  A block that meets no cell of the level (bi > cy
    // or bj > cx) is skipped; its partials stay 0 and no stored cell reads
    // them.  Pixels outside the voting range (X < 1, X > xmax) read staged
    // bytes that exist but vote with weight 0 (their column's tent weights
    // are zeroed); zero gradients vote 0 as well (adding +0 leaves the
    // non-negative partials unchanged).  Magnitude sqrt(s) of the exact
    // integer s = dx^2 + dy^2 by the hardware square root (sqrt.approx, a
    // few ulp; s is 0 or >= 1, so flushing subnormals changes nothing).
    const int by = t / bw, bx = t - by * bw;
    const int X0 = CELL * (j0 + bx) - 4, Y0 = CELL * (i0 + by) - 4;
    const bool active = t < bw * bh && i0 + by <= d.cy && j0 + bx <= d.cx;
    float wx0v[8], wx1v[8];   // column tent weights to cell cols bj-1, bj (0: no vote)
#pragma unroll
    for (int ox = 0; ox < 8; ox++) {
        const bool ok = X0 + ox >= 1 && X0 + ox <= xmax;
        wx0v[ox] = ok ? tent16(ox + 8) : 0.0f;
        wx1v[ox] = ok ? tent16(ox) : 0.0f;
    }
    float2 *p0 = part + t;
    // Row reads: each pixel row's three image rows are staged rows r-1, r,
    // r+1, and each staged row is read once per block: as the floats
    // 2^23 + byte of its 10 columns X0-1 .. X0+8 (one byte permute each,
    // byte_f23), which serve as the lower row, the middle row and the upper
    // row of three successive pixel rows.  dx and dy are then float
    // subtractions.  Where the level's rows are 8-byte aligned in memory
    // (image base and pitch multiples of 8), byte X0 of every staged row lies
    // at a shared address = 4 (mod 8), so the 10 bytes come from two 8-byte
    // loads; otherwise from 10 byte loads.
    const bool words = ((uintptr_t)d.img & 7) == 0 && (d.pitch & 7) == 0;
    // Staged row r as the floats 2^23 + byte of columns X0-1 .. X0+8.
    auto load_row = [&](int r, float (&f)[10]) {
        const uint8_t *row = srcS + r * srowb - xbase[r];
        if (words) {
            const uint2 lo = *reinterpret_cast<const uint2 *>(row + X0 - 4);   // X0-4 .. X0+3
            const uint2 hi = *reinterpret_cast<const uint2 *>(row + X0 + 4);   // X0+4 .. X0+11
            const uint32_t w4[4] = {lo.x, lo.y, hi.x, hi.y};
#pragma unroll
            for (int k = 0; k < 10; k++) f[k] = byte_f23(w4[(k + 3) >> 2], (k + 3) & 3);
        } else {
#pragma unroll
            for (int k = 0; k < 10; k++) f[k] = __uint_as_float(0x4B000000u | row[X0 - 1 + k]);
        }
    };
    if (active) {
        // pixel row oy of the block is staged row r0 + oy; three rows of
        // floats rotate through f (the loop is unrolled, so the rotation
        // is register naming): up = f[oy % 3], mid, down the next two
        const int r0 = CELL * by + 1;
        float f[3][10];
        load_row(r0 - 1, f[0]);
        load_row(r0, f[1]);
#pragma unroll
        for (int oy = 0; oy < 8; oy++) {
            float(&fu)[10] = f[oy % 3];
            float(&fm)[10] = f[(oy + 1) % 3];
            float(&fd)[10] = f[(oy + 2) % 3];
            load_row(r0 + oy + 1, fd);
            const int Y = Y0 + oy;
            if (Y < 1 || Y > ymax) continue;
            const float wy1 = tent16(oy), wy0 = tent16(oy + 8);   // to cell rows bi, bi-1
#pragma unroll
            for (int ox = 0; ox < 8; ox++) {
                const float dxf = fm[ox + 2] - fm[ox], dyf = fd[ox + 1] - fu[ox + 1];
                const uint32_t boff = orientation_bin_f<NT * sizeof(float2)>(dxf, dyf);   // bytes
                const float sf = fmaf(dxf, dxf, dyf * dyf);       // dx^2 + dy^2, exact
                float m;                                          // sqrt(sf); 0 for sf = 0
                asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(m) : "f"(sf));
                const float m0 = m * wy0, m1 = m * wy1;
                float2 *pb = reinterpret_cast<float2 *>(reinterpret_cast<char *>(p0) + boff);
                float2 a = pb[0], c = pb[PB * NT];
                a.x = fmaf(m0, wx0v[ox], a.x);   // cell (bi-1, bj-1)
                a.y = fmaf(m0, wx1v[ox], a.y);   // cell (bi-1, bj)
                c.x = fmaf(m1, wx0v[ox], c.x);   // cell (bi,   bj-1)
                c.y = fmaf(m1, wx1v[ox], c.y);   // cell (bi,   bj)
                pb[0] = a;
                pb[PB * NT] = c;
            }
        }
    }
    __syncthreads();

    // cell (ci, cj) = blocks (ci,cj) corner 3 + (ci,cj+1) corner 2 + (ci+1,cj)
    // corner 1 + (ci+1,cj+1) corner 0; staged for a coalesced store
    float *outS = reinterpret_cast<float *>(srcS);   // [tw*th][18]
    if (t < tw * th) {
        const int ci = t / tw, cj = t - ci * tw;
        const int b00 = ci * bw + cj;
#pragma unroll
        for (int b = 0; b < NBIN; b++) {
            float s3 = part[(1 * PB + b) * NT + b00].y;
            float s2 = part[(1 * PB + b) * NT + b00 + 1].x;
            float s1 = part[(0 * PB + b) * NT + b00 + bw].y;
            float s0 = part[(0 * PB + b) * NT + b00 + bw + 1].x;
            if (b == 0) {   // row 18: the rest of bin 0
                s3 += part[(1 * PB + NBIN) * NT + b00].y;
                s2 += part[(1 * PB + NBIN) * NT + b00 + 1].x;
                s1 += part[(0 * PB + NBIN) * NT + b00 + bw].y;
                s0 += part[(0 * PB + NBIN) * NT + b00 + bw + 1].x;
            }
            outS[t * NBIN + b] = (s3 + s2) + (s1 + s0);
        }
    }
    __syncthreads();
    // the tile's cells, row by row, as float2 (a cell is 72 bytes and the
    // level's cells start 8-byte aligned); k = r rowf2 + c walks t, t + NT, ...
    const int nrow = min(th, d.cy - i0), ncol = min(tw, d.cx - j0);
    if (nrow > 0 && ncol > 0 && ((uintptr_t)d.hist & 7) == 0) {
        const int rowf2 = ncol * (NBIN / 2);
        const int q0 = NT / rowf2, rem0 = NT - q0 * rowf2;
        int r = t / rowf2, c = t - r * rowf2;
        const float2 *src2 = reinterpret_cast<const float2 *>(outS);
        while (r < nrow) {
            float2 *dst = reinterpret_cast<float2 *>(d.hist + ((size_t)(i0 + r) * d.cx + j0) * NBIN);
            dst[c] = src2[r * tw * (NBIN / 2) + c];
            c += rem0;
            r += q0;
            if (c >= rowf2) {
                c -= rowf2;
                r++;
            }
        }
    } else {
        for (int r = 0; r < nrow; r++) {
            float *dst = d.hist + ((size_t)(i0 + r) * d.cx + j0) * NBIN;
            const float *srcr = outS + r * tw * NBIN;
            for (int k = t; k < ncol * NBIN; k += NT) dst[k] = srcr[k];
        }
    }
    __syncthreads();   // shared memory may be reused by the caller's next tile
}

// ===========================================================================
// Energy, block normalisation, truncation, 31 features (Section 4.1.1:
// normalisation and feature computation; the paper's energy and feature
// kernels fused).  E = sum_{n<9} (h_n + h_{n+9})^2, zero outside the grid;
// blocks k toward (-1,-1), (+1,-1), (-1,+1), (+1,+1); N_k = 1/sqrt(S_k+eps);
//   f[o] = 1/2 sum_k min(h_o N_k, tau)                  o < 18
//   f[18+o] = 1/2 sum_k min((h_o + h_{o+9}) N_k, tau)    o < 9
//   f[27+k] = 0.2357 sum_o min(h_o N_k, tau)             k < 4
// Output: internal layout [4][cy][cx][8] (channel 31 = 0) and optionally
// the user layout [cy][cx][31].  256 threads, 32x8 cells.
namespace feat_cfg {
constexpr int HX = FEAT_TX + 2;   // 34 halo columns
constexpr int HY = FEAT_TY + 2;   // 10 halo rows
constexpr int NT = FEAT_TX * FEAT_TY;
// cells of 18 floats, read and written as 8-byte pairs: a warp's lanes at
// the 72-byte cell stride hit distinct banks within each half-warp
constexpr size_t SMEM = sizeof(float) * (HY * HX * NBIN + HY * HX);   // 25,840
}  // namespace feat_cfg

// (a.x * b.x, a.y * b.y) and (a.x + b.x, a.y + b.y), one packed FP32
// instruction each (two IEEE operations, RN)
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pc, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pc, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

template <bool COH>
__device__ __forceinline__ void feat_tile(const LevelDesc &d, int tile, float eps, float tau,
                                          unsigned char *smem) {
    using namespace feat_cfg;
    float2 *hS = reinterpret_cast<float2 *>(smem);                  // [HY*HX][9]
    float *eS = reinterpret_cast<float *>(smem) + HY * HX * NBIN;  // [HY*HX]
    const int ntx = (d.cx + FEAT_TX - 1) / FEAT_TX;
    const int j0 = (tile % ntx) * FEAT_TX, i0 = (tile / ntx) * FEAT_TY;
    const int t = threadIdx.x;

    // stage the tile's cells and their one-cell halo (HY * HX <= 2 NT cells):
    // a thread takes cells t and t + NT, 18 floats (72 bytes: nine 8-byte
    // loads) each, and issues all its loads before storing, so the tile's
    // loads are in flight together; zero outside the grid
    static_assert(HY * HX <= 2 * NT, "two halo cells per thread");
    float2 v[2][NBIN / 2];
    bool in[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const int k = t + s * NT;
        const int r = k / HX, c = k - r * HX;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        in[s] = k < HY * HX && i >= 0 && i < d.cy && j >= 0 && j < d.cx;
        if (in[s]) {
            const float2 *src = reinterpret_cast<const float2 *>(d.hist + ((size_t)i * d.cx + j) * NBIN);
#pragma unroll
            for (int q = 0; q < NBIN / 2; q++) v[s][q] = ld_in<COH>(src + q);
        }
    }
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const int k = t + s * NT;
        if (k >= HY * HX) continue;
        float2 *dst = hS + k * (NBIN / 2);
        float e = 0.0f;   // E = sum_{n<9} (h_n + h_{n+9})^2 of this cell
        float hv[NBIN];
#pragma unroll
        for (int q = 0; q < NBIN / 2; q++) {
            const float2 x = in[s] ? v[s][q] : make_float2(0.0f, 0.0f);
            dst[q] = x;
            hv[2 * q] = x.x;
            hv[2 * q + 1] = x.y;
        }
#pragma unroll
        for (int n = 0; n < 9; n++) {
            const float sn = hv[n] + hv[n + 9];
            e += sn * sn;
        }
        eS[k] = e;
    }
    __syncthreads();

    const int ti = t / FEAT_TX, tj = t - ti * FEAT_TX;
    const int i = i0 + ti, j = j0 + tj;
    if (i < d.cy && j < d.cx) {
        const int r = ti + 1, c = tj + 1;
        const float2 *h = hS + (r * HX + c) * (NBIN / 2);
        float hv[NBIN];
#pragma unroll
        for (int q = 0; q < NBIN / 2; q++) {
            const float2 x = h[q];
            hv[2 * q] = x.x;
            hv[2 * q + 1] = x.y;
        }
        const float e00 = eS[r * HX + c];
        const float S0 = e00 + eS[r * HX + c - 1] + eS[(r - 1) * HX + c] + eS[(r - 1) * HX + c - 1];
        const float S1 = e00 + eS[r * HX + c + 1] + eS[(r - 1) * HX + c] + eS[(r - 1) * HX + c + 1];
        const float S2 = e00 + eS[r * HX + c - 1] + eS[(r + 1) * HX + c] + eS[(r + 1) * HX + c - 1];
        const float S3 = e00 + eS[r * HX + c + 1] + eS[(r + 1) * HX + c] + eS[(r + 1) * HX + c + 1];
        // halved normalisers and cap: 1/2 min(h N, tau) = min(h N/2, tau/2)
        // exactly (scaling by 2^-1 commutes with rounding and with min), so
        // the 1/2 of the averages is folded in; N_k = rsqrt(S_k + eps), the
        // hardware reciprocal square root
        const float N0 = 0.5f * rsqrtf(S0 + eps), N1 = 0.5f * rsqrtf(S1 + eps);
        const float N2 = 0.5f * rsqrtf(S2 + eps), N3 = 0.5f * rsqrtf(S3 + eps);
        const float tauh = 0.5f * tau;

        float f[32];
        // blocks (0, 1) and (2, 3) in packed pairs (two IEEE products or
        // sums per instruction); each feature sums its four terms as
        // (a0 + a2) + (a1 + a3)
        const float2 N01 = make_float2(N0, N1), N23 = make_float2(N2, N3);
        float2 t01 = make_float2(0.0f, 0.0f), t23 = make_float2(0.0f, 0.0f);   // halved bin sums
#pragma unroll
        for (int o = 0; o < NBIN; o++) {
            const float2 p01 = fmul2(make_float2(hv[o], hv[o]), N01);
            const float2 p23 = fmul2(make_float2(hv[o], hv[o]), N23);
            const float2 a01 = make_float2(fminf(p01.x, tauh), fminf(p01.y, tauh));
            const float2 a23 = make_float2(fminf(p23.x, tauh), fminf(p23.y, tauh));
            const float2 s02 = fadd2(a01, a23);
            f[o] = s02.x + s02.y;
            t01 = fadd2(t01, a01);
            t23 = fadd2(t23, a23);
        }
#pragma unroll
        for (int o = 0; o < 9; o++) {
            const float s = hv[o] + hv[o + 9];
            const float2 p01 = fmul2(make_float2(s, s), N01);
            const float2 p23 = fmul2(make_float2(s, s), N23);
            const float2 a01 = make_float2(fminf(p01.x, tauh), fminf(p01.y, tauh));
            const float2 a23 = make_float2(fminf(p23.x, tauh), fminf(p23.y, tauh));
            const float2 s02 = fadd2(a01, a23);
            f[NBIN + o] = s02.x + s02.y;
        }
        // 0.2357 x (the unhalved sum) = (2 x 0.2357) x t, both exactly
        constexpr float k2 = 2.0f * 0.2357f;
        f[27] = k2 * t01.x;
        f[28] = k2 * t01.y;
        f[29] = k2 * t23.x;
        f[30] = k2 * t23.y;
        f[31] = 0.0f;

        const size_t plane = (size_t)d.cy * d.cx * CHUNK;
        const size_t cell = (size_t)i * d.cx + j;
        if (d.feat) {   // FP32 chunked layout (CUDA-core correlation)
#pragma unroll
            for (int ch = 0; ch < NCHUNK; ch++) {
                float4 *dst = reinterpret_cast<float4 *>(d.feat + ch * plane + cell * CHUNK);
                dst[0] = make_float4(f[8 * ch + 0], f[8 * ch + 1], f[8 * ch + 2], f[8 * ch + 3]);
                dst[1] = make_float4(f[8 * ch + 4], f[8 * ch + 5], f[8 * ch + 6], f[8 * ch + 7]);
            }
        }
        if (d.feat_user) {
            float *u = d.feat_user + cell * NFEAT;
#pragma unroll
            for (int o = 0; o < NFEAT; o++) u[o] = f[o];
        }
        if (d.feat_hi) {
            // fp16 split for the tensor-core correlation: hi = f rounded to
            // fp16, lo = (f - hi) rounded to fp16; |f - hi - lo| <= 2^-22 |f|;
            // two channels per conversion
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int o = 0; o < 16; o++) {
                const __half2 h2 = __floats2half2_rn(f[2 * o], f[2 * o + 1]);
                const float2 hf = __half22float2(h2);
                const __half2 l2 = __floats2half2_rn(f[2 * o] - hf.x, f[2 * o + 1] - hf.y);
                hw[o] = *reinterpret_cast<const uint32_t *>(&h2);
                lw[o] = *reinterpret_cast<const uint32_t *>(&l2);
            }
            // group-major planes [4 channel groups][cy*cx cells][8 channels]:
            // a run of cells of one group is contiguous (bulk-copy friendly)
            const size_t nc = (size_t)d.cy * d.cx;
            uint4 *ph = reinterpret_cast<uint4 *>(d.feat_hi) + cell;
            uint4 *pl = reinterpret_cast<uint4 *>(d.feat_lo) + cell;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                ph[q * nc] = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
                pl[q * nc] = make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
            }
        }
    }
    __syncthreads();   // shared memory may be reused by the caller's next tile
}

// ===========================================================================
// Multi-filter correlation, threshold and candidate key of one warp tile
// (Section 4.1.1: linear classification filter and detection; Section 5.1,
// classifier and detection kernels fused).
//
// score_f(u, v) = sum_{a<10, b<10, c<31} W_f[a][b][c] feat[u+a][v+b][c].  A
// window is a candidate when its best score over the filters is strictly
// greater than the threshold; its key ranks (score desc, level, filter, u,
// v).  Windows at one position share one box, so only the best filter of a
// position can survive greedy suppression; the key carries that filter
// (equal scores: the lowest index).
//
// One warp owns one tile of 128 windows (8x16, 4x32 or 16x8, chosen per
// level on the host).  Features stream in half-chunks of 4 channels (one
// float4 per cell of the internal layout): the warp copies the (TU+9) x
// (TV+9) region of the next half-chunk with cp.async.cg while computing the
// current one (double buffer, 2 x CORR_BUF4 float4 of warp-private shared
// memory).  The half-warps split the channels: lanes 0-15 take channels
// 0-1 of every float4, lanes 16-31 channels 2-3; within a half-warp a lane
// owns 8 consecutive windows of one row for all filters, and the two halves'
// partial scores are added with one shuffle at the end.  For a filter row a
// lane loads its 17 channel pairs once and slides over the 10 filter
// columns in registers; each filter weight pair (a half-warp-uniform load
// through L1) feeds 8 windows, and each accumulator is a (channel 0, channel
// 1) pair updated by one packed FMA.  Register traffic per FMA from L1 is
// what bounds this loop: 8 windows per lane halve the weight bytes written
// back per FMA against 4 windows of all 4 channels.
constexpr int CORR_WPT = 8;
constexpr int CORR_BUF4 = HOG_CORR_MINB >= 4 ? 432 : 544;   // 13x41 = 533 needs the 4x32 shape

// acc += (w0 * x0, w1 * x1), one packed FP32 FMA (two IEEE fmas, RN)
__device__ __forceinline__ void ffma2(float2 &acc, float w0, float w1, float x0, float x1) {
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(acc.x), "+f"(acc.y)
        : "f"(w0), "f"(w1), "f"(x0), "f"(x1));
}

template <int NF, int BUF4 = CORR_BUF4>
__device__ __forceinline__ void corr_warp_job(const LevelDesc *__restrict__ descs, Job jb,
                                              const float *__restrict__ wchunks, int nf_real,
                                              float threshold, float4 *buf0) {
    const int lane = threadIdx.x & 31;
    const LevelDesc &d = descs[jb.desc];
    const int shape = (jb.tile >> 28) & 3, tile = jb.tile & 0x0fffffff;
    const int TU = corr_tu(shape), TV = corr_tv(shape);
    const int RU = TU + WIN - 1, RV = TV + WIN - 1;
    const int ntv = (d.nv + TV - 1) / TV;
    const int u0 = (tile / ntv) * TU, v0 = (tile % ntv) * TV;
    const int half = lane >> 4, l16 = lane & 15;               // channel pair, lane in half
    const int lr = l16 % TU, lc = (l16 / TU) * CORR_WPT;      // window row / first column in tile

    const float4 *feat4 = reinterpret_cast<const float4 *>(d.feat);
    const size_t plane4 = (size_t)d.cy * d.cx * 2;           // float4 per chunk plane
    const float2 *w2 = reinterpret_cast<const float2 *>(wchunks);

    // copy half-chunk h (chunk h/2, channels 4*(h&1)..+3) of the tile region
    auto stage = [&](int h, float4 *dst) {
        const float4 *src = feat4 + (size_t)(h >> 1) * plane4 + (h & 1);
        for (int k = lane; k < RU * RV; k += 32) {
            const int rr = k / RV, cc = k - rr * RV;
            const int i = u0 + rr, j = v0 + cc;
            const bool ok = i < d.cy && j < d.cx;
            cp_async16_zfill(dst + k, ok ? (const void *)(src + ((size_t)i * d.cx + j) * 2)
                                         : (const void *)src, ok);
        }
        cp_async_commit();
    };

#if HOG_CORR_PACKED
    // acc[j][f] = (channel 2*half, channel 2*half + 1) partial sums
    float2 acc[CORR_WPT][NF];
#pragma unroll
    for (int j = 0; j < CORR_WPT; j++)
#pragma unroll
        for (int f = 0; f < NF; f++) acc[j][f] = make_float2(0.0f, 0.0f);
#else
    // acc[j][f] = partial sum over this half's two channels
    float acc[CORR_WPT][NF];
#pragma unroll
    for (int j = 0; j < CORR_WPT; j++)
#pragma unroll
        for (int f = 0; f < NF; f++) acc[j][f] = 0.0f;
#endif

    stage(0, buf0);
#pragma unroll 1
    for (int h = 0; h < 2 * NCHUNK; h++) {
        float4 *cur = buf0 + (h & 1) * BUF4;
        if (h + 1 < 2 * NCHUNK) {
            stage(h + 1, buf0 + ((h + 1) & 1) * BUF4);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        __syncwarp();
        const int ch = h >> 1, c4 = h & 1;
        // weights: float4 index ((chunk*NF + f)*100 + a*10 + b)*2 + c4, as
        // float2 pairs: twice that plus the half
        const float2 *wch = w2 + ((size_t)ch * NF * 200 + c4) * 2 + half;
#pragma unroll 1
        for (int a = 0; a < WIN; a++) {
            const float2 *frow =
                reinterpret_cast<const float2 *>(cur + (lr + a) * RV + lc) + half;
            float2 fv[CORR_WPT + WIN - 1];
#pragma unroll
            for (int j = 0; j < CORR_WPT + WIN - 1; j++) fv[j] = frow[2 * j];
#pragma unroll
            for (int b = 0; b < WIN; b++) {
                float2 wv[NF];
#pragma unroll
                for (int f = 0; f < NF; f++) wv[f] = __ldg(wch + ((f * WIN + a) * WIN + b) * 4);
#pragma unroll
                for (int j = 0; j < CORR_WPT; j++) {
                    const float2 x = fv[j + b];
#pragma unroll
                    for (int f = 0; f < NF; f++) {
#if HOG_CORR_PACKED
                        ffma2(acc[j][f], wv[f].x, wv[f].y, x.x, x.y);
#else
                        acc[j][f] = fmaf(wv[f].y, x.y, fmaf(wv[f].x, x.x, acc[j][f]));
#endif
                    }
                }
            }
        }
        __syncwarp();   // every lane is done with `cur` before it is refilled
    }

    // score = this half's two channels + the other half's (lane ^ 16)
    float sc[CORR_WPT][NF];
#pragma unroll
    for (int j = 0; j < CORR_WPT; j++)
#pragma unroll
        for (int f = 0; f < NF; f++) {
#if HOG_CORR_PACKED
            const float mine = acc[j][f].x + acc[j][f].y;
#else
            const float mine = acc[j][f];
#endif
            const float other = __shfl_xor_sync(0xffffffffu, mine, 16);
            sc[j][f] = half == 0 ? mine + other : other + mine;
        }
    const int u = u0 + lr;
    if (half != 0 || u >= d.nu) return;
#pragma unroll
    for (int j = 0; j < CORR_WPT; j++) {
        const int v = v0 + lc + j;
        if (v >= d.nv) break;
        float best = sc[j][0];
        int fb = 0;
#pragma unroll
        for (int f = 1; f < NF; f++)
            if (f < nf_real && sc[j][f] > best) { best = sc[j][f]; fb = f; }
        if (d.scores_user) {
#pragma unroll
            for (int f = 0; f < NF; f++)
                if (f < nf_real)
                    d.scores_user[((size_t)f * d.nu + u) * d.nv + v] = sc[j][f];
        }
        if (d.keys)
            d.keys[(size_t)u * d.nv + v] =
                (d.scan && best > threshold) ? make_key(best, d.level, fb, u, v) : KEY_NONE;
    }
}

// ===========================================================================
// Non-maximum suppression of one frame (Section 4.1.1, last step).
//
// Greedy definition: rank candidates by (score desc, level, filter, u, v);
// keep a box unless a kept, higher-ranked box overlaps it with IoU >
// nms_iou.  The greedy result is the unique set K with "p in K iff no member
// of K ranked above p overlaps p", reached here by rounds in which every
// undecided candidate p decides or waits:
//   - p's bit in the suppression bitmask is set (a kept neighbour marked
//     it) -> p is suppressed;
//   - otherwise p scans its higher-ranked overlapping neighbours from where
//     its last scan stopped: one of them kept -> suppressed; one undecided ->
//     p waits (a neighbour kept later marks p's bit); all suppressed or
//     ranked below -> p is kept and marks all its neighbours' bits.
// The best undecided candidate always decides, so the rounds end (about ten
// rounds on 640x480 frames); decisions are final, so a thread may read a
// neighbour's state or bit while it changes within a round.  Neighbours
// passed over (suppressed, or not a candidate above p) stay settled, so a
// candidate's slots are scanned about once in all.
//
// Overlap lists (IoU > nms_iou, FP64) come from the per-frame-size geometry
// twice: slot-major nbr[s * npos + p], read by one thread per candidate (a
// warp's load of slot s reads consecutive entries), and position-major
// nbr_t[p * MAXN + s], read by a warp walking one candidate's slots (a
// lane per slot: consecutive entries again).  Each round walks a
// compacted list of the still-undecided candidates, so sparse late rounds
// cost little.  Ranks compare the key's high word (the score order) held in
// shared memory; equal high words fall back to the full key in global
// memory; a decision overwrites the candidate's high word (kept: 0, above
// every key; suppressed: all ones, below every key), so no state is kept
// apart.  After each round the list of undecided candidates is rebuilt from
// the high words in position order.  Workspace (nms_ws_bytes): in shared
// memory (SM, a list of 16-bit positions) or in fd.ws (32-bit positions).
// NT threads.
// candidate states of the cluster form's state bytes
constexpr uint8_t NMS_ALIVE = 1, NMS_KEPT = 2, NMS_DEAD = 0;
constexpr uint32_t NMS_NOKEY = 0xffffffffu;   // key high word of a non-candidate (or a suppressed one)
// key high word of a kept candidate: below every real high word.  A real one
// is the complemented order of a non-NaN score, in [0x007FFFFF (+inf),
// 0xFF800000 (-inf)], so neither 0 nor NMS_NOKEY is a key.
constexpr uint32_t NMS_KEPTKEY = 0u;

struct WinBox {
    double x, y, w, h;
};

// Box of window (u, v) of a level in frame pixels: (8v, 8u, 80, 80) scaled
// by rx = W0/Wl and ry = H0/Hl.  The ratios are IEEE double quotients taken
// once per level on the host (FP64 division is slow on this GPU); every
// product is rounded once, as in the oracle.
__device__ __forceinline__ WinBox window_box(double rx, double ry, int u, int v) {
    WinBox b;
    b.x = __dmul_rn((double)(CELL * v), rx);
    b.y = __dmul_rn((double)(CELL * u), ry);
    b.w = __dmul_rn((double)(CELL * WIN), rx);
    b.h = __dmul_rn((double)(CELL * WIN), ry);
    return b;
}

// Whether window position p of a frame is scanned: at or after the first
// scanned level, and inside its level's rectangle when the frame has a
// region of interest.  Other positions carry no key.
__device__ __forceinline__ bool nms_scanned(const FrameDesc &fd, int p) {
    if (!fd.has_roi) return p >= fd.scan_from;
    int l = 0;
    while (l + 1 < fd.nlev && p >= fd.lev_pos[l + 1]) l++;
    const int idx = p - fd.lev_pos[l], u = idx / fd.lev_nv[l], v = idx - u * fd.lev_nv[l];
    return u >= fd.roi_u0[l] && u < fd.roi_u1[l] && v >= fd.roi_v0[l] && v < fd.roi_v1[l];
}

// WS: where the workspace lives (nms_ws_class): NMS_WS_SMEM all of it in
// shared memory, NMS_WS_KEYS the key words in shared memory and the rest in
// fd.ws, NMS_WS_GLOBAL all of it in fd.ws.
constexpr int NMS_SCAN_U = 4;   // candidates whose scans start together
template <int WS, int NT, bool COH>
__device__ __forceinline__ void nms_frame(const FrameDesc &fd, unsigned char *smem, int *flags,
                                          int *sh /* NT/32 + 4 ints of shared memory */) {
    using idx_t = typename std::conditional<WS == NMS_WS_SMEM, uint16_t, int32_t>::type;
    const int t = threadIdx.x;
    const int npos = fd.npos;
    unsigned char *base = WS == NMS_WS_SMEM ? smem : reinterpret_cast<unsigned char *>(fd.ws);
    // key high word of each position while it is undecided; its decision
    // overwrites it: NMS_KEPTKEY (above every key) or NMS_NOKEY (below every
    // key, as for a position that never had one)
    volatile uint32_t *khi = reinterpret_cast<volatile uint32_t *>(WS == NMS_WS_GLOBAL ? base : smem);
    idx_t *list = reinterpret_cast<idx_t *>(base + 4 * (size_t)npos);   // undecided, position order
    // suppression bitmask: bit q set once a neighbour of q has been kept, so
    // q (if ranked below it) is suppressed without scanning its neighbours
    const int nwords = (npos + 31) / 32;
    const size_t off_supp = ((size_t)npos * (4 + sizeof(idx_t)) + 3) & ~(size_t)3;
    volatile uint32_t *supp = reinterpret_cast<volatile uint32_t *>(base + off_supp);
    // per candidate: how many leading neighbour slots are settled for good
    // (not a candidate, ranked below, or suppressed); later rounds resume
    // the scan there.  Written and read by the candidate's own thread only.
    uint8_t *resume = base + off_supp + 4 * (size_t)nwords;
    const uint64_t *gkeys = fd.keys;
    const int32_t *__restrict__ nbr = fd.nbr;                        // [slot][npos]
    const int32_t *__restrict__ nbr_t = fd.nbr_t;                    // [npos][slot]
    const int lane = t & 31, wid = t >> 5;

    // q ranked above p (smaller key)
    auto above = [&](int q, int p, uint32_t hq, uint32_t hp) -> bool {
        if (hq != hp) return hq < hp;
        return ld_in<COH>(gkeys + q) < ld_in<COH>(gkeys + p);
    };
    // exclusive prefix sum of one count per thread over the block (thread
    // order); *total = the sum.  One barrier: every warp scans the warp
    // totals itself.  Two calls must be separated by a barrier (sh is
    // rewritten).
    static_assert(NT / 32 <= 32, "warp totals scanned by one warp");
    auto block_scan = [&](int mine, int *total) -> int {
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) sh[wid] = incl;
        __syncthreads();
        const int w = lane < NT / 32 ? sh[lane] : 0;
        int winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        *total = __shfl_sync(0xffffffffu, winc, NT / 32 - 1);
        return __shfl_sync(0xffffffffu, winc - w, wid) + incl - mine;
    };
    // thread t's share of the positions: [beg, end)
    const int per = (npos + NT - 1) / NT;
    const int beg = min(t * per, npos), end = min(beg + per, npos);
    auto undecided_at = [&](int p) {
        const uint32_t h = khi[p];
        return h != NMS_KEPTKEY && h != NMS_NOKEY;
    };
    // the list of undecided positions, rebuilt from the key words (a stable
    // scan: it reads khi and writes the list, so no entry is overwritten
    // before it is read); returns its length
    auto build_list = [&]() -> int {
        int mine = 0;
        for (int p = beg; p < end; p++) mine += undecided_at(p);
        int n = 0;
        int o = block_scan(mine, &n);
        for (int p = beg; p < end; p++)
            if (undecided_at(p)) list[o++] = (idx_t)p;
        __syncthreads();
        return n;
    };

    for (int k = t; k < nwords; k += NT) supp[k] = 0u;
    for (int p = t; p < npos; p += NT) {
        // positions of levels that are not scanned carry no key
        khi[p] = nms_scanned(fd, p) ? (uint32_t)(ld_in<COH>(gkeys + p) >> 32) : NMS_NOKEY;
        resume[p] = 0;
    }
    __syncthreads();
    int n_cur = build_list();

    int round = 0;
    for (; round <= npos && n_cur > 0; round++) {
        for (int i0 = 0; i0 < n_cur; i0 += NT) {     // whole warps iterate together
            const int i = i0 + t;
            bool kept = false, dead = false, wait = false, done = false;
            int p = -1, settled = 0;
            uint32_t hp = 0;
            if (i < n_cur) {
                p = list[i];
                hp = khi[p];
                dead = (supp[p >> 5] >> (p & 31)) & 1u;
                // scan the unsettled slots up to the first higher-ranked
                // neighbour that is kept (p is suppressed) or undecided (p
                // waits; a neighbour kept later marks p in the bitmask):
                // four slots here, the rest by the whole warp below
                // (a list ends at its first -1 slot: the tables are filled
                // with -1 past each position's count, so no count is read)
                const int r0 = resume[p];
                settled = r0;   // end of the settled prefix of the slots
                if (!dead) {
                    int q[4];
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        q[k] = r0 + k < MAXN ? __ldg(nbr + (size_t)(r0 + k) * npos + p) : -1;
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if (done || dead || wait) continue;
                        if (q[k] < 0) { done = true; continue; }
                        // a kept neighbour ranks above p (p could not be
                        // undecided otherwise); an undecided one above p
                        // makes p wait; the rest are settled
                        const uint32_t hq = khi[q[k]];
                        if (hq == NMS_KEPTKEY) dead = true;
                        else if (hq != NMS_NOKEY && above(q[k], p, hq, hp)) wait = true;
                        else settled = r0 + k + 1;
                    }
                }
            }
            // candidates with slots left: the warp scans them, a lane per
            // slot, and takes the first unsettled slot in order.  NMS_SCAN_U
            // candidates at a time: their first 32 slots are loaded together
            // (one wait on L2 for all of them), the rest one chunk at a time
            for (unsigned um = __ballot_sync(0xffffffffu, p >= 0 && !dead && !wait && !done); um;) {
                int srcs[NMS_SCAN_U], sbs[NMS_SCAN_U], qs[NMS_SCAN_U];
#pragma unroll
                for (int j = 0; j < NMS_SCAN_U; j++) {
                    srcs[j] = um ? __ffs(um) - 1 : -1;   // warp-uniform
                    um &= um ? um - 1 : 0u;
                    const int sj = srcs[j] < 0 ? 0 : srcs[j];
                    const int pj = __shfl_sync(0xffffffffu, p, sj);
                    sbs[j] = __shfl_sync(0xffffffffu, settled, sj);
                    const int sl = sbs[j] + lane;
                    qs[j] = srcs[j] >= 0 && sl < MAXN ? __ldg(nbr_t + (size_t)pj * MAXN + sl) : -1;
                }
#pragma unroll
                for (int j = 0; j < NMS_SCAN_U; j++) {
                    const int src = srcs[j];
                    if (src < 0) break;   // warp-uniform
                    const int pp = __shfl_sync(0xffffffffu, p, src);
                    const uint32_t hpp = __shfl_sync(0xffffffffu, hp, src);
                    int res = 0, at = 0;   // 0: all settled, 1: kept neighbour, 2: undecided one
                    int q = qs[j];
                    for (int sb = sbs[j];; sb += 32) {
                        if (sb != sbs[j]) {
                            const int sl = sb + lane;
                            q = sl < MAXN ? __ldg(nbr_t + (size_t)pp * MAXN + sl) : -1;
                        }
                        const unsigned end = __ballot_sync(0xffffffffu, q < 0);
                        uint32_t cls = 0;
                        if (q >= 0) {
                            const uint32_t hq = khi[q];
                            if (hq == NMS_KEPTKEY) cls = 1u;
                            else if (hq != NMS_NOKEY && above(q, pp, hq, hpp)) cls = 2u;
                        }
                        const unsigned hit = __ballot_sync(0xffffffffu, cls != 0);
                        if (hit) {   // slots after the list's end are -1: a hit comes first
                            const int f = __ffs(hit) - 1;
                            res = (int)__shfl_sync(0xffffffffu, cls, f);
                            at = sb + f;
                            break;
                        }
                        if (end) {
                            at = sb + __ffs(end) - 1;
                            break;
                        }
                    }
                    if (lane == src) {
                        if (res == 1) dead = true;
                        else if (res == 2) wait = true;
                        settled = at;
                    }
                }
            }
            if (p >= 0) {
                if (dead) {
                    khi[p] = NMS_NOKEY;
                } else if (!wait) {
                    khi[p] = NMS_KEPTKEY;
                    kept = true;
                } else {
                    resume[p] = (uint8_t)settled;
                }
            }
            // each kept candidate marks all its neighbours, the warp's lanes
            // splitting the slots (neighbours ranked above it are decided
            // already: it could not be kept while one was undecided)
            for (unsigned km = __ballot_sync(0xffffffffu, kept); km; km &= km - 1) {
                const int pk = __shfl_sync(0xffffffffu, p, __ffs(km) - 1);
                for (int s = lane;; s += 32) {
                    const int q = s < MAXN ? __ldg(nbr_t + (size_t)pk * MAXN + s) : -1;
                    if (q >= 0) atomicOr(const_cast<uint32_t *>(supp) + (q >> 5), 1u << (q & 31));
                    if (__ballot_sync(0xffffffffu, q < 0)) break;   // the list ended here
                }
            }
        }
        __syncthreads();
        n_cur = build_list();
    }

    // kept positions in position order
    int mine = 0;
    for (int p = beg; p < end; p++) mine += khi[p] == NMS_KEPTKEY;
    int total = 0;
    int pos = block_scan(mine, &total);
    for (int p = beg; p < end; p++) {
        if (khi[p] != NMS_KEPTKEY) continue;
        if (pos < fd.out_cap) {
            const uint64_t k = ld_in<COH>(gkeys + p);
            const int l = key_level(k);
            const int u = key_u(k), v = key_v(k);
            const WinBox b = window_box(fd.lev_rx[l], fd.lev_ry[l], u, v);
            hog_det det;
            det.frame = fd.frame;
            det.level = l;
            det.filter = key_filter(k);
            det.u = u;
            det.v = v;
            det.score = key_score(k);
            det.x = b.x; det.y = b.y; det.w = b.w; det.h = b.h;
            fd.out[pos] = det;
        }
        pos++;
    }
    if (t == 0) {
        *fd.count = total;
        if (total > fd.out_cap) atomicOr(flags, 1);
        atomicMax(flags + 1, round + 1);
    }
    __syncthreads();   // shared memory may be reused by the caller's next item
}

}  // namespace hogk
