// k_train.cu -- forward (float mode) and hand-written adjoint of a hinge
// loss on the best window score of one filter, for training the linear
// filters of Section 4.1.1 (the paper uses filters trained elsewhere; the
// adjoint has no counterpart there).
//
// Float mode: the pyramid keeps real values (the same exact bilinear weights
// in tenths, no rounding); gradients are real; the orientation bin is the
// nearest of the 18 centres, found as the largest |dot| with the nine
// unsigned directions (dx == 0 -> bin 4 or 13).  For crop i with label y_i:
// s_i = max window score over all levels (ties: first in (level, u, v)),
// L = (1/B) sum_i max(0, 1 - y_i s_i) (subgradient 0 at the kink),
// dL/dW = (1/B) sum_{active} (-y_i) feat_i[window_i], and dL/dI through
// truncation (min(x, tau) passes the gradient iff x < tau), N_k(S_k), the
// energies, the histogram (bins held fixed), the magnitude, the central
// differences and the pyramid.  Every step is a gather in a fixed order, so
// the result is deterministic.
#include "hog_stages.cuh"

namespace hogk {

namespace {

// cos / sin of 20 k degrees, k = 0..8 (the nine unsigned directions).
__constant__ float c_dir[9][2] = {
    {1.0f, 0.0f},
    {0.93969262078590838f, 0.34202014332566873f},
    {0.76604444311897804f, 0.64278760968653933f},
    {0.5f, 0.86602540378443865f},
    {0.17364817766693035f, 0.98480775301220806f},
    {-0.17364817766693035f, 0.98480775301220806f},
    {-0.5f, 0.86602540378443865f},
    {-0.76604444311897804f, 0.64278760968653933f},
    {-0.93969262078590838f, 0.34202014332566873f}};

__device__ __forceinline__ int fbin(float dx, float dy) {
    if (dx == 0.0f && dy == 0.0f) return -1;
    if (dx == 0.0f) return dy > 0.0f ? 4 : 13;
    int best = 0;
    float bestabs = -1.0f, bestdot = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const float d = c_dir[k][0] * dx + c_dir[k][1] * dy;
        if (fabsf(d) > bestabs) { bestabs = fabsf(d); bestdot = d; best = k; }
    }
    return bestdot > 0.0f ? best : best + 9;
}

// Histogram of cell (i, j) of a float level image (w x h, row stride w):
// the 16x16-pixel footprint in row-major order, tent weights in sixteenths.
// acc points to 18 floats (stride `st` between bins), zeroed by the caller.
__device__ __forceinline__ void fcell_hist(const float *img, int w, int h, int cx, int cy, int i,
                                           int j, float *acc, int st) {
    const int xmax = min(w - 2, CELL * cx - 1), ymax = min(h - 2, CELL * cy - 1);
    for (int py = 0; py < 16; py++) {
        const int Y = CELL * i - 4 + py;
        if (Y < 1 || Y > ymax) continue;
        const float wy = tent16(py);
        for (int px = 0; px < 16; px++) {
            const int X = CELL * j - 4 + px;
            if (X < 1 || X > xmax) continue;
            const float dx = img[Y * w + X + 1] - img[Y * w + X - 1];
            const float dy = img[(Y + 1) * w + X] - img[(Y - 1) * w + X];
            const int b = fbin(dx, dy);
            if (b < 0) continue;
            const float m = sqrtf(dx * dx + dy * dy);
            acc[b * st] += m * (tent16(px) * wy);
        }
    }
}

}  // namespace

// ---- forward -----------------------------------------------------------

// Level l (dw x dh) of every crop from level l-1 (sw x sh), float mode.
__global__ void fpyr_step_kernel(const float *__restrict__ src, float *__restrict__ dst, int sw,
                                 int dw, int dh, size_t crop_stride) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= dw * dh) return;
    const int y = idx / dw, x = idx - y * dw;
    const float *s = src + (size_t)blockIdx.y * crop_stride;
    const int Y = 12 * y + 1, y0 = Y / 10, fy = Y % 10;
    const int X = 12 * x + 1, x0 = X / 10, fx = X % 10;
    const float acc = (float)((10 - fx) * (10 - fy)) * s[y0 * sw + x0] +
                      (float)(fx * (10 - fy)) * s[y0 * sw + x0 + 1] +
                      (float)((10 - fx) * fy) * s[(y0 + 1) * sw + x0] +
                      (float)(fx * fy) * s[(y0 + 1) * sw + x0 + 1];
    dst[(size_t)blockIdx.y * crop_stride + idx] = acc / 100.0f;
}

// Cell histograms of one level of every crop (one thread per cell).
__global__ void __launch_bounds__(128) fhist_kernel(const float *__restrict__ lvl, int w, int h,
                                                    size_t crop_stride, float *__restrict__ hist,
                                                    size_t hist_stride) {
    __shared__ float acc[NBIN * 128];
    const int cx = w / CELL, cy = h / CELL;
    const int c = blockIdx.x * 128 + threadIdx.x;
    for (int b = 0; b < NBIN; b++) acc[b * 128 + threadIdx.x] = 0.0f;
    if (c >= cx * cy) return;
    const int i = c / cx, j = c - i * cx;
    fcell_hist(lvl + (size_t)blockIdx.y * crop_stride, w, h, cx, cy, i, j, acc + threadIdx.x, 128);
    float *o = hist + (size_t)blockIdx.y * hist_stride + (size_t)c * NBIN;
    for (int b = 0; b < NBIN; b++) o[b] = acc[b * 128 + threadIdx.x];
}

// Best window of each crop over all levels; per-crop hinge margin.
// scores: per crop, levels back to back ([nu_l][nv_l] each, one filter).
__global__ void __launch_bounds__(256) argmax_kernel(const float *__restrict__ scores,
                                                     size_t crop_stride, TrainLevels lv,
                                                     const float *__restrict__ labels,
                                                     int4 *__restrict__ best, float *__restrict__ margin) {
    __shared__ float bs[256];
    __shared__ int bp[256];
    const float *s = scores + (size_t)blockIdx.x * crop_stride;
    float mv = 0.0f;
    int mp = -1;
    for (int p = threadIdx.x; p < lv.nwin; p += 256) {
        const float v = s[p];
        if (mp < 0 || v > mv) { mv = v; mp = p; }    // strided order: p increases
    }
    bs[threadIdx.x] = mv;
    bp[threadIdx.x] = mp;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            const float v2 = bs[threadIdx.x + off];
            const int p2 = bp[threadIdx.x + off];
            const float v1 = bs[threadIdx.x];
            const int p1 = bp[threadIdx.x];
            if (p2 >= 0 && (p1 < 0 || v2 > v1 || (v2 == v1 && p2 < p1))) {
                bs[threadIdx.x] = v2;
                bp[threadIdx.x] = p2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int p = bp[0];
        int l = 0;
        while (l + 1 < lv.nlev && p >= lv.win_off[l + 1]) l++;
        const int q = p - lv.win_off[l];
        best[blockIdx.x] = make_int4(l, q / lv.nv[l], q % lv.nv[l], p);
        const float m = 1.0f - labels[blockIdx.x] * bs[0];
        margin[blockIdx.x] = (p >= 0 && m > 0.0f) ? m : 0.0f;
    }
}

// dW[a][b][c] = (1/B) sum over active crops of (-y_i) feat_i[l_i][u_i+a][v_i+b][c].
__global__ void dw_kernel(const float *__restrict__ feat, size_t crop_stride, TrainLevels lv,
                          const int4 *__restrict__ best, const float *__restrict__ margin,
                          const float *__restrict__ labels, int n, float *__restrict__ dW) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= WIN * WIN * NFEAT) return;
    const int a = k / (WIN * NFEAT), b = (k / NFEAT) % WIN, c = k % NFEAT;
    float acc = 0.0f;
    for (int i = 0; i < n; i++) {
        if (!(margin[i] > 0.0f)) continue;
        const int4 bw = best[i];
        const int l = bw.x;
        const float *f = feat + (size_t)i * crop_stride + lv.feat_off[l];
        acc += (-labels[i] / (float)n) * f[((size_t)(bw.y + a) * lv.cx[l] + (bw.z + b)) * NFEAT + c];
    }
    dW[k] = acc;
}

// ---- adjoint of one crop's best window, down to its level's pixels ------
// One CTA (256 threads) per crop.  Region: the window's 10x10 cells plus a
// one-cell ring (12x12 cells: the cells whose energies the window's
// normalisers read), and the pixels voting into them (104x104 + a 1-pixel
// ring for the central differences).  dP (the crop's level-gradient image at
// the best level, zeroed by the caller) receives the pixel gradients.
namespace bw {
constexpr int RC = WIN + 2;             // 12 region cells per side
constexpr int RP = RC * CELL + CELL;    // 104 region pixels per side
constexpr int NT = 256;
static_assert(RP == TRAIN_RP, "region size of hog_backward_state");
}  // namespace bw

// With st_bins / st_trunc (may be NULL) the kernel also records the discrete
// state it holds fixed: the bin of every region pixel ([RP][RP] per crop,
// 255 where the pixel does not vote) and, per window cell and block k, the
// 27 truncation tests x N_k < tau of its 18 signed and 9 unsigned values
// ([100][4][27] per crop, 1 = below tau: the gradient passes).
__global__ void __launch_bounds__(bw::NT) window_adjoint_kernel(
    const float *__restrict__ pyr, size_t pyr_stride, const float *__restrict__ hist,
    size_t hist_stride, TrainLevels lv, const int4 *__restrict__ best,
    const float *__restrict__ margin, const float *__restrict__ labels, int n,
    const float *__restrict__ wuser, float eps, float tau, int recompute, float *__restrict__ dP,
    uint8_t *__restrict__ st_bins, uint8_t *__restrict__ st_trunc) {
    using namespace bw;
    extern __shared__ float sm[];
    float *H = sm;                           // [RC*RC][18] region histograms
    float *dH = H + RC * RC * NBIN;          // [RC*RC][18]
    float *E = dH + RC * RC * NBIN;          // [RC*RC]
    float *dS = E + RC * RC;                 // [100][4]
    float *GX = dS + WIN * WIN * 4;          // [RP][RP] d/d(dx)
    float *GY = GX + RP * RP;                // [RP][RP] d/d(dy)
    const int i = blockIdx.x, t = threadIdx.x;
    if (!(margin[i] > 0.0f)) return;
    const int4 bwin = best[i];
    const int l = bwin.x, u0 = bwin.y, v0 = bwin.z;
    const int w = lv.w[l], h = lv.h[l], cx = lv.cx[l], cy = lv.cy[l];
    const float *img = pyr + (size_t)i * pyr_stride + lv.pyr_off[l];
    const float g = -labels[i] / (float)n;

    // 1. region histograms (stored, or recomputed from the level image)
    for (int k = t; k < RC * RC * NBIN; k += NT) { H[k] = 0.0f; dH[k] = 0.0f; }
    __syncthreads();
    for (int k = t; k < RC * RC; k += NT) {
        const int ci = u0 - 1 + k / RC, cj = v0 - 1 + k % RC;
        if (ci < 0 || cj < 0 || ci >= cy || cj >= cx) continue;
        if (recompute) {
            fcell_hist(img, w, h, cx, cy, ci, cj, H + k * NBIN, 1);
        } else {
            const float *hs = hist + (size_t)i * hist_stride + lv.hist_off[l] + ((size_t)ci * cx + cj) * NBIN;
            for (int b = 0; b < NBIN; b++) H[k * NBIN + b] = hs[b];
        }
    }
    __syncthreads();
    for (int k = t; k < RC * RC; k += NT) {
        float e = 0.0f;
        for (int o = 0; o < 9; o++) {
            const float s = H[k * NBIN + o] + H[k * NBIN + o + 9];
            e += s * s;
        }
        E[k] = e;   // zero for cells outside the grid (zero histograms)
    }
    __syncthreads();

    // 2. window cells: features -> (histogram, normalisers)
    const int bdx[4] = {-1, +1, -1, +1}, bdy[4] = {-1, -1, +1, +1};
    if (t < WIN * WIN) {
        const int a = t / WIN, b = t % WIN;
        const int r = a + 1, c = b + 1;              // region coordinates
        const float *hc = H + (r * RC + c) * NBIN;
        float *dhc = dH + (r * RC + c) * NBIN;
        const float *Wc = wuser + (a * WIN + b) * NFEAT;
        float S[4], N[4], dN[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int k = 0; k < 4; k++) {
            S[k] = E[r * RC + c] + E[r * RC + c + bdx[k]] + E[(r + bdy[k]) * RC + c] +
                   E[(r + bdy[k]) * RC + c + bdx[k]];
            N[k] = 1.0f / sqrtf(S[k] + eps);
        }
        if (st_trunc) {
            uint8_t *st = st_trunc + ((size_t)i * WIN * WIN + t) * 4 * (NBIN + 9);
            for (int k = 0; k < 4; k++) {
                for (int o = 0; o < NBIN; o++) st[k * (NBIN + 9) + o] = hc[o] * N[k] < tau;
                for (int o = 0; o < 9; o++)
                    st[k * (NBIN + 9) + NBIN + o] = (hc[o] + hc[o + 9]) * N[k] < tau;
            }
        }
        for (int o = 0; o < NBIN; o++)
            for (int k = 0; k < 4; k++)
                if (hc[o] * N[k] < tau) {
                    const float coef = 0.5f * g * Wc[o] + 0.2357f * g * Wc[27 + k];
                    dhc[o] += coef * N[k];
                    dN[k] += coef * hc[o];
                }
        for (int o = 0; o < 9; o++) {
            const float su = hc[o] + hc[o + 9];
            for (int k = 0; k < 4; k++)
                if (su * N[k] < tau) {
                    const float coef = 0.5f * g * Wc[NBIN + o];
                    dhc[o] += coef * N[k];
                    dhc[o + 9] += coef * N[k];
                    dN[k] += coef * su;
                }
        }
        for (int k = 0; k < 4; k++) {
            const float se = S[k] + eps;
            dS[t * 4 + k] = dN[k] * (-0.5f) / (se * sqrtf(se));
        }
    }
    __syncthreads();

    // 3. energies -> histograms: region cell q collects dS of every window
    // cell whose block k contains q (fixed order: k, then the block's cells)
    for (int q = t; q < RC * RC; q += NT) {
        const int qr = q / RC, qc = q % RC;
        float dE = 0.0f;
        for (int k = 0; k < 4; k++) {
            const int offr[4] = {0, 0, bdy[k], bdy[k]}, offc[4] = {0, bdx[k], 0, bdx[k]};
            for (int m = 0; m < 4; m++) {
                const int wr = qr - offr[m] - 1, wc = qc - offc[m] - 1;   // window cell of the block
                if (wr >= 0 && wc >= 0 && wr < WIN && wc < WIN) dE += dS[(wr * WIN + wc) * 4 + k];
            }
        }
        if (dE != 0.0f) {
            for (int o = 0; o < 9; o++) {
                const float t2 = 2.0f * dE * (H[q * NBIN + o] + H[q * NBIN + o + 9]);
                dH[q * NBIN + o] += t2;
                dH[q * NBIN + o + 9] += t2;
            }
        }
    }
    __syncthreads();

    // 4. histogram -> magnitude -> (dx, dy) for every pixel voting into the region
    const int X0 = CELL * (v0 - 1) - 4, Y0 = CELL * (u0 - 1) - 4;   // region pixel origin
    const int xmax = min(w - 2, CELL * cx - 1), ymax = min(h - 2, CELL * cy - 1);
    for (int k = t; k < RP * RP; k += NT) {
        const int ry = k / RP, rx = k % RP;
        const int X = X0 + rx, Y = Y0 + ry;
        float gx = 0.0f, gy = 0.0f;
        int bin_state = 255;
        if (X >= 1 && X <= xmax && Y >= 1 && Y <= ymax) {
            const float dx = img[Y * w + X + 1] - img[Y * w + X - 1];
            const float dy = img[(Y + 1) * w + X] - img[(Y - 1) * w + X];
            const int b = fbin(dx, dy);
            if (b >= 0) {
                bin_state = b;
                const float mag = sqrtf(dx * dx + dy * dy);
                // the pixel's two cells per axis, tent weights (offset t = footprint position)
                const int ix = (X + 4) / CELL - 1, iy = (Y + 4) / CELL - 1;  // lower cell
                float dm = 0.0f;
                for (int di = 0; di < 2; di++)
                    for (int dj = 0; dj < 2; dj++) {
                        const int ci = iy + di, cj = ix + dj;
                        const int rr = ci - (u0 - 1), rc = cj - (v0 - 1);
                        if (ci < 0 || cj < 0 || ci >= cy || cj >= cx) continue;
                        if (rr < 0 || rc < 0 || rr >= RC || rc >= RC) continue;
                        const float wgt = tent16(X - (CELL * cj - 4)) * tent16(Y - (CELL * ci - 4));
                        dm += wgt * dH[(rr * RC + rc) * NBIN + b];
                    }
                if (dm != 0.0f) { gx = dm * dx / mag; gy = dm * dy / mag; }
            }
        }
        GX[k] = gx;
        GY[k] = gy;
        if (st_bins) st_bins[(size_t)i * RP * RP + k] = (uint8_t)bin_state;
    }
    __syncthreads();

    // 5. central differences -> level pixels (gather over the region + ring)
    float *d = dP + (size_t)i * pyr_stride + lv.pyr_off[l];
    for (int k = t; k < (RP + 2) * (RP + 2); k += NT) {
        const int ry = k / (RP + 2) - 1, rx = k % (RP + 2) - 1;   // -1 .. RP
        const int X = X0 + rx, Y = Y0 + ry;
        if (X < 0 || Y < 0 || X >= w || Y >= h) continue;
        auto gxat = [&](int yy, int xx) { return (xx >= 0 && yy >= 0 && xx < RP && yy < RP) ? GX[yy * RP + xx] : 0.0f; };
        auto gyat = [&](int yy, int xx) { return (xx >= 0 && yy >= 0 && xx < RP && yy < RP) ? GY[yy * RP + xx] : 0.0f; };
        const float v = gxat(ry, rx - 1) - gxat(ry, rx + 1) + gyat(ry - 1, rx) - gyat(ry + 1, rx);
        if (v != 0.0f) d[Y * w + X] = v;
    }
}

// Pyramid adjoint, one level step for every crop whose best level is > q:
// dP_q(x, y) += sum over level-(q+1) pixels sampling (x, y) of weight/100 x
// dP_{q+1} (gather: the samples of column x come from x' with x0(x') in
// {x-1, x}).
__global__ void fpyr_adjoint_kernel(float *__restrict__ dP, size_t pyr_stride, TrainLevels lv, int q,
                                    const int4 *__restrict__ best, const float *__restrict__ margin) {
    const int i = blockIdx.y;
    if (!(margin[i] > 0.0f) || best[i].x <= q) return;
    const int w0 = lv.w[q], h0 = lv.h[q], w1 = lv.w[q + 1], h1 = lv.h[q + 1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= w0 * h0) return;
    const int y = idx / w0, x = idx - y * w0;
    const float *d1 = dP + (size_t)i * pyr_stride + lv.pyr_off[q + 1];
    float acc = 0.0f;
    const int ylo = max(0, (10 * (y - 1) - 1) / 12 - 1), yhi = min(h1 - 1, (10 * y - 1) / 12 + 1);
    const int xlo = max(0, (10 * (x - 1) - 1) / 12 - 1), xhi = min(w1 - 1, (10 * x - 1) / 12 + 1);
    for (int yy = ylo; yy <= yhi; yy++) {
        const int Y = 12 * yy + 1, y0 = Y / 10, fy = Y % 10;
        int wy;
        if (y0 == y) wy = 10 - fy;
        else if (y0 + 1 == y) wy = fy;
        else continue;
        for (int xx = xlo; xx <= xhi; xx++) {
            const int X = 12 * xx + 1, x0 = X / 10, fx = X % 10;
            int wx;
            if (x0 == x) wx = 10 - fx;
            else if (x0 + 1 == x) wx = fx;
            else continue;
            if (wx * wy) acc += (float)(wx * wy) * (d1[(size_t)yy * w1 + xx] / 100.0f);
        }
    }
    float *d0 = dP + (size_t)i * pyr_stride + lv.pyr_off[q];
    d0[idx] += acc;
}

// filter [10][10][31] -> one-filter chunk layout [4][1][10][10][8]
__global__ void filter_chunks_kernel(const float *__restrict__ wuser, float *__restrict__ wch) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NCHUNK * WIN * WIN * CHUNK) return;
    const int ch = k / (WIN * WIN * CHUNK), ab = (k / CHUNK) % (WIN * WIN), cc = k % CHUNK;
    const int c = ch * CHUNK + cc;
    wch[k] = c < NFEAT ? wuser[ab * NFEAT + c] : 0.0f;
}

// ---- launchers ---------------------------------------------------------

cudaError_t launch_fpyr_step(const float *src, float *dst, int sw, int dw, int dh, size_t crop_stride,
                             int n, cudaStream_t s) {
    dim3 grid((dw * dh + 255) / 256, n);
    fpyr_step_kernel<<<grid, 256, 0, s>>>(src, dst, sw, dw, dh, crop_stride);
    return cudaGetLastError();
}

cudaError_t launch_fhist(const float *lvl, int w, int h, size_t crop_stride, float *hist,
                         size_t hist_stride, int n, cudaStream_t s) {
    const int cells = (w / CELL) * (h / CELL);
    if (cells <= 0) return cudaSuccess;
    dim3 grid((cells + 127) / 128, n);
    fhist_kernel<<<grid, 128, 0, s>>>(lvl, w, h, crop_stride, hist, hist_stride);
    return cudaGetLastError();
}

cudaError_t launch_argmax(const float *scores, size_t crop_stride, const TrainLevels &lv,
                          const float *labels, int4 *best, float *margin, int n, cudaStream_t s) {
    argmax_kernel<<<n, 256, 0, s>>>(scores, crop_stride, lv, labels, best, margin);
    return cudaGetLastError();
}

cudaError_t launch_dw(const float *feat, size_t crop_stride, const TrainLevels &lv, const int4 *best,
                      const float *margin, const float *labels, int n, float *dW, cudaStream_t s) {
    dw_kernel<<<(WIN * WIN * NFEAT + 255) / 256, 256, 0, s>>>(feat, crop_stride, lv, best, margin,
                                                             labels, n, dW);
    return cudaGetLastError();
}

cudaError_t launch_window_adjoint(const float *pyr, size_t pyr_stride, const float *hist,
                                  size_t hist_stride, const TrainLevels &lv, const int4 *best,
                                  const float *margin, const float *labels, int n,
                                  const float *wuser, float eps, float tau, int recompute,
                                  float *dP, uint8_t *st_bins, uint8_t *st_trunc, cudaStream_t s) {
    using namespace bw;
    const size_t smem = sizeof(float) * (2 * RC * RC * NBIN + RC * RC + WIN * WIN * 4 + 2 * RP * RP);
    static PerDevice attr;
    cudaError_t e_attr = attr.once([&]() {
        cudaError_t e = cudaFuncSetAttribute(window_adjoint_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e;
    });
    if (e_attr != cudaSuccess) return e_attr;
    window_adjoint_kernel<<<n, NT, smem, s>>>(pyr, pyr_stride, hist, hist_stride, lv, best, margin,
                                              labels, n, wuser, eps, tau, recompute, dP, st_bins,
                                              st_trunc);
    return cudaGetLastError();
}

cudaError_t launch_fpyr_adjoint(float *dP, size_t pyr_stride, const TrainLevels &lv, int q,
                                const int4 *best, const float *margin, int n, cudaStream_t s) {
    dim3 grid((lv.w[q] * lv.h[q] + 255) / 256, n);
    fpyr_adjoint_kernel<<<grid, 256, 0, s>>>(dP, pyr_stride, lv, q, best, margin);
    return cudaGetLastError();
}

cudaError_t launch_filter_chunks(const float *wuser, float *wch, cudaStream_t s) {
    filter_chunks_kernel<<<(NCHUNK * WIN * WIN * CHUNK + 255) / 256, 256, 0, s>>>(wuser, wch);
    return cudaGetLastError();
}

}  // namespace hogk
