/*
 * hog_oracle.c -- plain, slow FP64 reference of the HOG face-detection path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * It follows the algorithm breakdown of the paper's Section 4.1.1 ("Face
 * detector"), step by step, in the paper's order:
 *   pyramid (5/6 steps down to the 80x80 window)        -> hgo_level_sizes,
 *                                                          hgo_downscale_*
 *   gradient + 18 signed orientations                   -> hgo_orientation_bin
 *   8x8 cells, each pixel voting into its 4 nearest     -> hgo_cell_hist
 *   energy of the cell and 8 neighbours, normalisation,
 *   18 + 9 + 4 = 31 features                            -> hgo_features
 *   10x10-cell linear filters, threshold                -> hgo_correlate
 *   non-maximum suppression                             -> hgo_nms
 * A window is a detection only when its score is strictly greater than the
 * threshold (Section 5.1, detection kernel).
 *
 * Where the paper is silent, this file takes these readings (the same ones
 * the CUDA path implements independently):
 *   R1 level sizes w' = floor(5w/6), h' = floor(5h/6), each level from the
 *      previous one; keep a level while min(w, h) >= min_size (80).
 *   R2 resampling: pixel-centre aligned bilinear with exact weights in
 *      tenths: source coordinate (12x+1)/10, weights (10-f)(10-g) etc.,
 *      result rounded half up to uint8 (float mode: no rounding).
 *   R3 central differences dx = I(x+1,y)-I(x-1,y), dy = I(x,y+1)-I(x,y-1)
 *      for 1 <= x <= min(w-2, 8cx-1), 1 <= y <= min(h-2, 8cy-1).
 *   R4 orientation: the bin whose centre (20 b degrees) is nearest, found as
 *      the largest |dot| with the 9 unsigned directions; dx == 0 (the only
 *      exact ties for integer gradients) resolves to bin 4 (dy > 0) or 13.
 *   R5 bilinear voting, cell centres at 8j+4, weights 1-a and a.
 *   R6 energy zero outside the cell grid; blocks k = 0..3 extend to
 *      (-1,-1), (+1,-1), (-1,+1), (+1,+1) as (dx, dy); eps = 1e-4,
 *      truncation tau = 0.2, texture weight 0.2357; channel order
 *      18 signed, 9 unsigned, 4 texture.
 *   R7 scores over "valid" windows only, no bias.
 *   R8 boxes (8v, 8u, 80, 80) in level pixels mapped to the frame by W0/Wl,
 *      H0/Hl; greedy NMS over all levels and filters of a frame in order
 *      (score desc, level, filter, u, v); suppress when IoU > nms_iou.
 *   R12 direct-to-size (Section 6.6, future work), with skip_levels = s >= 2:
 *      level s is resampled from level 0 in one step with the ratio (6/5)^s
 *      under the R2 rule generalised (weights in units of 1/(2*5^s)); the
 *      levels between are not computed; the later levels follow in 5/6
 *      steps.  For s = 1 the one step is the 5/6 step itself.
 *   R13 region of interest (Section 6.6, future work: scan only scales and
 *      locations near the previous frame's face): a window is scanned iff
 *      its level is in [lmin, lmax] and its centre, mapped to the frame in
 *      FP64 as (8v + 40) * (W0/Wl), (8u + 40) * (H0/Hl), is in [x0, x1) x
 *      [y0, y1) (hgo_in_roi).
 * Built with -ffp-contract=off so that results are identical on x86-64 and
 * aarch64 hosts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CELL 8
#define WIN 10
#define NBIN 18
#define NFEAT 31
#define TEXTURE_W 0.2357

/* ------------------------------------------------------------------------ */
/* Pyramid (Section 4.1.1: steps of a 5/6 factor until the width or height
 * is smaller than the 80x80 detection window).                             */

int hgo_level_sizes(int w, int h, int min_size, int *ws, int *hs, int cap)
{
    int n = 0;
    while (w >= min_size && h >= min_size) {
        if (n < cap) { ws[n] = w; hs[n] = h; }
        n++;
        w = 5 * w / 6;
        h = 5 * h / 6;
    }
    return n;
}

/* One 5/6 step, uint8 -> uint8, reading R2. dst is floor(5w/6) x floor(5h/6). */
void hgo_downscale_u8(const uint8_t *src, int w, int h, int sstride,
                      uint8_t *dst, int dstride)
{
    int w2 = 5 * w / 6, h2 = 5 * h / 6;
    for (int y = 0; y < h2; y++) {
        int Y = 12 * y + 1, y0 = Y / 10, fy = Y % 10;
        for (int x = 0; x < w2; x++) {
            int X = 12 * x + 1, x0 = X / 10, fx = X % 10;
            int p00 = src[y0 * sstride + x0];
            int p10 = src[y0 * sstride + x0 + 1];
            int p01 = src[(y0 + 1) * sstride + x0];
            int p11 = src[(y0 + 1) * sstride + x0 + 1];
            int acc = (10 - fx) * (10 - fy) * p00 + fx * (10 - fy) * p10
                    + (10 - fx) * fy * p01 + fx * fy * p11;
            dst[y * dstride + x] = (uint8_t)((acc + 50) / 100);
        }
    }
}

/* The same step on real-valued images (float mode, no rounding). */
void hgo_downscale_f64(const double *src, int w, int h, double *dst)
{
    int w2 = 5 * w / 6, h2 = 5 * h / 6;
    for (int y = 0; y < h2; y++) {
        int Y = 12 * y + 1, y0 = Y / 10, fy = Y % 10;
        for (int x = 0; x < w2; x++) {
            int X = 12 * x + 1, x0 = X / 10, fx = X % 10;
            double acc = (double)((10 - fx) * (10 - fy)) * src[y0 * w + x0]
                       + (double)(fx * (10 - fy)) * src[y0 * w + x0 + 1]
                       + (double)((10 - fx) * fy) * src[(y0 + 1) * w + x0]
                       + (double)(fx * fy) * src[(y0 + 1) * w + x0 + 1];
            dst[y * w2 + x] = acc / 100.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Gradient orientation (Section 4.1.1: each pixel's gradient direction is
 * quantised to one of 18 signed orientations), reading R4.  Returns -1 for a
 * zero gradient.                                                            */

int hgo_orientation_bin(double dx, double dy)
{
    const double deg = 3.14159265358979323846 / 180.0;
    if (dx == 0.0 && dy == 0.0) return -1;
    if (dx == 0.0) return dy > 0.0 ? 4 : 13;
    int best = 0;
    double bestabs = -1.0, bestdot = 0.0;
    for (int k = 0; k < 9; k++) {
        double d = cos(20.0 * k * deg) * dx + sin(20.0 * k * deg) * dy;
        if (fabs(d) > bestabs) { bestabs = fabs(d); bestdot = d; best = k; }
    }
    return bestdot > 0.0 ? best : best + 9;
}

/* ------------------------------------------------------------------------ */
/* Histogramisation (Section 4.1.1): 8x8-pixel cells, 18 bins; every pixel
 * votes into the four closest cells, weighted by gradient magnitude and by
 * distance (readings R3, R5).  hist is [cy][cx][18], cy = h/8, cx = w/8.     */

void hgo_cell_hist(const double *img, int w, int h, double *hist)
{
    int cx = w / CELL, cy = h / CELL;
    memset(hist, 0, sizeof(double) * (size_t)cx * cy * NBIN);
    int xmax = w - 2 < CELL * cx - 1 ? w - 2 : CELL * cx - 1;
    int ymax = h - 2 < CELL * cy - 1 ? h - 2 : CELL * cy - 1;
    for (int y = 1; y <= ymax; y++) {
        for (int x = 1; x <= xmax; x++) {
            double dx = img[y * w + x + 1] - img[y * w + x - 1];
            double dy = img[(y + 1) * w + x] - img[(y - 1) * w + x];
            int b = hgo_orientation_bin(dx, dy);
            if (b < 0) continue;
            double mag = sqrt(dx * dx + dy * dy);
            double xp = (x + 0.5) / CELL - 0.5, yp = (y + 0.5) / CELL - 0.5;
            int ix = (int)floor(xp), iy = (int)floor(yp);
            double ax = xp - ix, ay = yp - iy;
            for (int di = 0; di < 2; di++) {
                int i = iy + di;
                if (i < 0 || i >= cy) continue;
                double wy = di ? ay : 1.0 - ay;
                for (int dj = 0; dj < 2; dj++) {
                    int j = ix + dj;
                    if (j < 0 || j >= cx) continue;
                    double wx = dj ? ax : 1.0 - ax;
                    hist[((size_t)i * cx + j) * NBIN + b] += mag * wx * wy;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Normalisation and features (Section 4.1.1): energy
 *   E = sum_{n=0..8} (h_n + h_{n+9})^2
 * normalised with the cell and its 8 neighbours; 18 signed + 9 unsigned
 * normalised bins + 4 block-energy (texture) features (reading R6).
 * feat is [cy][cx][31].                                                     */

static double energy_at(const double *E, int cx, int cy, int i, int j)
{
    if (i < 0 || j < 0 || i >= cy || j >= cx) return 0.0;
    return E[(size_t)i * cx + j];
}

void hgo_features(const double *hist, int cx, int cy, double eps, double tau,
                  double *feat)
{
    double *E = (double *)malloc(sizeof(double) * (size_t)cx * cy + 8);
    for (int c = 0; c < cx * cy; c++) {
        const double *hc = hist + (size_t)c * NBIN;
        double e = 0.0;
        for (int n = 0; n < 9; n++) e += (hc[n] + hc[n + 9]) * (hc[n] + hc[n + 9]);
        E[c] = e;
    }
    static const int bdx[4] = {-1, +1, -1, +1};
    static const int bdy[4] = {-1, -1, +1, +1};
    for (int i = 0; i < cy; i++) {
        for (int j = 0; j < cx; j++) {
            const double *hc = hist + ((size_t)i * cx + j) * NBIN;
            double *f = feat + ((size_t)i * cx + j) * NFEAT;
            double N[4];
            for (int k = 0; k < 4; k++) {
                double S = energy_at(E, cx, cy, i, j)
                         + energy_at(E, cx, cy, i, j + bdx[k])
                         + energy_at(E, cx, cy, i + bdy[k], j)
                         + energy_at(E, cx, cy, i + bdy[k], j + bdx[k]);
                N[k] = 1.0 / sqrt(S + eps);
            }
            for (int o = 0; o < NBIN; o++) {
                double s = 0.0;
                for (int k = 0; k < 4; k++) s += fmin(hc[o] * N[k], tau);
                f[o] = 0.5 * s;
            }
            for (int o = 0; o < 9; o++) {
                double s = 0.0;
                for (int k = 0; k < 4; k++) s += fmin((hc[o] + hc[o + 9]) * N[k], tau);
                f[NBIN + o] = 0.5 * s;
            }
            for (int k = 0; k < 4; k++) {
                double s = 0.0;
                for (int o = 0; o < NBIN; o++) s += fmin(hc[o] * N[k], tau);
                f[27 + k] = TEXTURE_W * s;
            }
        }
    }
    free(E);
}

/* ------------------------------------------------------------------------ */
/* Linear classification filter (Section 4.1.1): the 10x10x31 = 3100
 * features of every 10x10-cell area times the filter weights, summed.
 * filt is [nf][10][10][31]; scores is [nf][cy-9][cx-9] (reading R7).        */

void hgo_correlate(const double *feat, int cx, int cy, const double *filt,
                   int nf, double *scores)
{
    int nu = cy - WIN + 1, nv = cx - WIN + 1;
    if (nu <= 0 || nv <= 0) return;
    for (int f = 0; f < nf; f++) {
        const double *W = filt + (size_t)f * WIN * WIN * NFEAT;
        for (int u = 0; u < nu; u++) {
            for (int v = 0; v < nv; v++) {
                double s = 0.0;
                for (int a = 0; a < WIN; a++)
                    for (int b = 0; b < WIN; b++)
                        for (int c = 0; c < NFEAT; c++)
                            s += W[(a * WIN + b) * NFEAT + c]
                               * feat[((size_t)(u + a) * cx + (v + b)) * NFEAT + c];
                scores[((size_t)f * nu + u) * nv + v] = s;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Detections and non-maximum suppression (Section 4.1.1 last step;
 * Section 5.1 "Non-maximum suppression"), reading R8.                       */

typedef struct {
    int32_t level, filter, u, v;
    double score, x, y, w, h;
} hgo_det;

static int det_rank_cmp(const void *pa, const void *pb)
{
    const hgo_det *a = (const hgo_det *)pa, *b = (const hgo_det *)pb;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->filter != b->filter) return a->filter < b->filter ? -1 : 1;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

double hgo_iou(const hgo_det *a, const hgo_det *b)
{
    double ix1 = a->x > b->x ? a->x : b->x;
    double ax2 = a->x + a->w, bx2 = b->x + b->w;
    double ix2 = ax2 < bx2 ? ax2 : bx2;
    double iy1 = a->y > b->y ? a->y : b->y;
    double ay2 = a->y + a->h, by2 = b->y + b->h;
    double iy2 = ay2 < by2 ? ay2 : by2;
    double iw = ix2 - ix1, ih = iy2 - iy1;
    if (iw <= 0.0 || ih <= 0.0) return 0.0;
    double inter = iw * ih;
    double uni = a->w * a->h + b->w * b->h - inter;
    return inter / uni;
}

/* Box of window (u, v) of level l mapped to frame pixels. */
void hgo_box(int W0, int H0, int Wl, int Hl, int u, int v, hgo_det *d)
{
    double rx = (double)W0 / (double)Wl, ry = (double)H0 / (double)Hl;
    d->x = (double)(CELL * v) * rx;
    d->y = (double)(CELL * u) * ry;
    d->w = (double)(CELL * WIN) * rx;
    d->h = (double)(CELL * WIN) * ry;
}

/* Greedy NMS.  Sorts cands[0..n) into rank order in place and sets keep[i]
 * for the survivors; returns the number kept.                              */
int hgo_nms(hgo_det *cands, int n, double iou_thr, int32_t *keep)
{
    qsort(cands, (size_t)n, sizeof(hgo_det), det_rank_cmp);
    int *kept = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int nk = 0;
    for (int i = 0; i < n; i++) {
        int sup = 0;
        for (int t = 0; t < nk && !sup; t++)
            if (hgo_iou(&cands[i], &cands[kept[t]]) > iou_thr) sup = 1;
        keep[i] = !sup;
        if (!sup) kept[nk++] = i;
    }
    free(kept);
    return nk;
}

/* ------------------------------------------------------------------------ */
/* Whole-frame helpers used by the tests.                                    */

/* uint8 pyramid of all kept levels, concatenated tightly ([h_l][w_l] each). */
/* Direct-to-size first downscale (Section 6.6, future work: scale the
 * frame straight to the largest level that is needed, then continue in 5/6
 * steps).  Level s is resampled from level 0 in one step with the ratio
 * (6/5)^s per axis, pixel-centre aligned: source coordinate
 *   (x + 1/2) (6/5)^s - 1/2 = ((2x + 1) 6^s - 5^s) / (2 * 5^s),
 * bilinear with exact weights in units of 1 / (2 * 5^s), rounded half up to
 * uint8.  For s = 1 this is the 5/6 step itself.  The output is the
 * (w_s, h_s) of the level-size rule, which never exceeds (5/6)^s of the
 * frame, so the right and lower neighbours always exist.  s <= 8.          */
void hgo_downscale_direct_u8(const uint8_t *src, int w, int h, int sstride, int s,
                             uint8_t *dst, int dw, int dh, int dstride)
{
    int64_t p6 = 1, p5 = 1;
    for (int k = 0; k < s; k++) { p6 *= 6; p5 *= 5; }
    const int64_t D = 2 * p5;           /* weight denominator per axis */
    (void)w; (void)h;
    for (int y = 0; y < dh; y++) {
        int64_t Y = (2 * (int64_t)y + 1) * p6 - p5;
        int64_t y0 = Y / D, fy = Y % D;
        for (int x = 0; x < dw; x++) {
            int64_t X = (2 * (int64_t)x + 1) * p6 - p5;
            int64_t x0 = X / D, fx = X % D;
            int64_t p00 = src[y0 * sstride + x0];
            int64_t p10 = src[y0 * sstride + x0 + 1];
            int64_t p01 = src[(y0 + 1) * sstride + x0];
            int64_t p11 = src[(y0 + 1) * sstride + x0 + 1];
            int64_t acc = (D - fx) * (D - fy) * p00 + fx * (D - fy) * p10
                        + (D - fx) * fy * p01 + fx * fy * p11;
            dst[(size_t)y * dstride + x] = (uint8_t)((acc + D * D / 2) / (D * D));
        }
    }
}

/* Pyramid with the first `skip_levels` levels skipped for detection.  With
 * direct != 0 and skip_levels = s >= 2, level s comes from level 0 by
 * hgo_downscale_direct_u8 and levels 1 .. s-1 are not computed (left 0);
 * the levels after s follow in 5/6 steps as usual.                          */
int hgo_pyramid_u8_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                      int skip_levels, int direct, uint8_t *out, size_t cap)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t need = 0, offs[64];
    for (int l = 0; l < L; l++) { offs[l] = need; need += (size_t)ws[l] * hs[l]; }
    if (need > cap) return -2;
    if (direct && skip_levels > 8) return -3;
    if (L == 0) return 0;
    memset(out, 0, need);
    for (int y = 0; y < h; y++) memcpy(out + (size_t)y * w, frame + (size_t)y * stride, (size_t)w);
    for (int l = 1; l < L; l++) {
        if (direct && skip_levels >= 2 && l < skip_levels) continue;
        if (direct && skip_levels >= 2 && l == skip_levels)
            hgo_downscale_direct_u8(out, ws[0], hs[0], ws[0], l, out + offs[l], ws[l], hs[l], ws[l]);
        else
            hgo_downscale_u8(out + offs[l - 1], ws[l - 1], hs[l - 1], ws[l - 1], out + offs[l], ws[l]);
    }
    return L;
}

int hgo_pyramid_u8(const uint8_t *frame, int w, int h, int stride, int min_size,
                   uint8_t *out, size_t cap)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t need = 0;
    for (int l = 0; l < L; l++) need += (size_t)ws[l] * hs[l];
    if (need > cap) return -2;
    size_t off = 0;
    for (int y = 0; y < h && L > 0; y++) memcpy(out + (size_t)y * w, frame + (size_t)y * stride, (size_t)w);
    for (int l = 1; l < L; l++) {
        size_t prev = off;
        off += (size_t)ws[l - 1] * hs[l - 1];
        hgo_downscale_u8(out + prev, ws[l - 1], hs[l - 1], ws[l - 1], out + off, ws[l]);
    }
    return L;
}

/* Real-valued pyramid of all kept levels ([h_l][w_l] each, concatenated). */
int hgo_pyramid_f64(const double *img, int w, int h, int min_size, double *out, size_t cap)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t need = 0;
    for (int l = 0; l < L; l++) need += (size_t)ws[l] * hs[l];
    if (need > cap) return -2;
    if (L > 0) memcpy(out, img, sizeof(double) * (size_t)w * h);
    size_t off = 0;
    for (int l = 1; l < L; l++) {
        size_t prev = off;
        off += (size_t)ws[l - 1] * hs[l - 1];
        hgo_downscale_f64(out + prev, ws[l - 1], hs[l - 1], out + off);
    }
    return L;
}

/* Features of every level, concatenated ([cy_l][cx_l][31] each).  The
 * pyramid is uint8 (float_mode 0) or real-valued (float_mode 1).           */
int hgo_frame_features_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                          int skip_levels, int direct, double eps, double tau, int float_mode,
                          double *feat, size_t cap);

int hgo_frame_features(const uint8_t *frame, int w, int h, int stride, int min_size,
                       double eps, double tau, int float_mode,
                       double *feat, size_t cap)
{
    return hgo_frame_features_ex(frame, w, h, stride, min_size, 0, 0, eps, tau, float_mode,
                                 feat, cap);
}

/* Features of every level; with direct pyramids (hgo_pyramid_u8_ex) the
 * levels that are not computed get zero features.                         */
int hgo_frame_features_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                          int skip_levels, int direct, double eps, double tau, int float_mode,
                          double *feat, size_t cap)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t npx = 0, ncell = 0;
    for (int l = 0; l < L; l++) {
        npx += (size_t)ws[l] * hs[l];
        ncell += (size_t)(ws[l] / CELL) * (hs[l] / CELL);
    }
    if (ncell * NFEAT > cap) return -2;
    double *pyr = (double *)malloc(sizeof(double) * (npx + 1));
    if (float_mode) {
        double *img = (double *)malloc(sizeof(double) * ((size_t)w * h + 1));
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) img[(size_t)y * w + x] = frame[(size_t)y * stride + x];
        hgo_pyramid_f64(img, w, h, min_size, pyr, npx);
        free(img);
    } else {
        uint8_t *p8 = (uint8_t *)malloc(npx + 1);
        hgo_pyramid_u8_ex(frame, w, h, stride, min_size, skip_levels, direct, p8, npx);
        for (size_t i = 0; i < npx; i++) pyr[i] = p8[i];
        free(p8);
    }
    size_t poff = 0, foff = 0;
    for (int l = 0; l < L; l++) {
        int cx = ws[l] / CELL, cy = hs[l] / CELL;
        if (!float_mode && direct && skip_levels >= 2 && l >= 1 && l < skip_levels) {
            memset(feat + foff, 0, sizeof(double) * (size_t)cx * cy * NFEAT);
            poff += (size_t)ws[l] * hs[l];
            foff += (size_t)cx * cy * NFEAT;
            continue;
        }
        double *hist = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NBIN + 1));
        hgo_cell_hist(pyr + poff, ws[l], hs[l], hist);
        hgo_features(hist, cx, cy, eps, tau, feat + foff);
        free(hist);
        poff += (size_t)ws[l] * hs[l];
        foff += (size_t)cx * cy * NFEAT;
    }
    free(pyr);
    return L;
}

/* Scores of every level, concatenated ([nf][cy_l-9][cx_l-9] each).         */
int hgo_frame_scores_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                        int skip_levels, int direct, double eps, double tau,
                        const double *filt, int nf, double *scores, size_t cap);

int hgo_frame_scores(const uint8_t *frame, int w, int h, int stride, int min_size,
                     double eps, double tau, const double *filt, int nf,
                     double *scores, size_t cap)
{
    return hgo_frame_scores_ex(frame, w, h, stride, min_size, 0, 0, eps, tau, filt, nf,
                               scores, cap);
}

int hgo_frame_scores_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                        int skip_levels, int direct, double eps, double tau,
                        const double *filt, int nf, double *scores, size_t cap)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t ncell = 0, nwin = 0;
    for (int l = 0; l < L; l++) {
        int cx = ws[l] / CELL, cy = hs[l] / CELL;
        ncell += (size_t)cx * cy;
        nwin += (size_t)nf * (cy - WIN + 1) * (cx - WIN + 1);
    }
    if (nwin > cap) return -2;
    double *feat = (double *)malloc(sizeof(double) * (ncell * NFEAT + 1));
    hgo_frame_features_ex(frame, w, h, stride, min_size, skip_levels, direct, eps, tau, 0, feat,
                          ncell * NFEAT);
    size_t foff = 0, soff = 0;
    for (int l = 0; l < L; l++) {
        int cx = ws[l] / CELL, cy = hs[l] / CELL;
        hgo_correlate(feat + foff, cx, cy, filt, nf, scores + soff);
        foff += (size_t)cx * cy * NFEAT;
        soff += (size_t)nf * (cy - WIN + 1) * (cx - WIN + 1);
    }
    free(feat);
    return L;
}

/* Candidates of one frame: every (level >= skip_levels, filter, u, v) whose
 * score is strictly higher than the threshold, with its frame box.  Returns
 * the candidate count (may exceed cap; only cap are written) or < 0.        */
int hgo_frame_candidates_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                            int skip_levels, int direct, double eps, double tau,
                            double threshold, const double *filt, int nf, hgo_det *out, int cap);

int hgo_frame_candidates(const uint8_t *frame, int w, int h, int stride, int min_size,
                         int skip_levels, double eps, double tau, double threshold,
                         const double *filt, int nf, hgo_det *out, int cap)
{
    return hgo_frame_candidates_ex(frame, w, h, stride, min_size, skip_levels, 0, eps, tau,
                                   threshold, filt, nf, out, cap);
}

/* As hgo_frame_candidates, the pyramid direct-to-size when direct != 0.    */
int hgo_frame_candidates_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                            int skip_levels, int direct, double eps, double tau,
                            double threshold, const double *filt, int nf, hgo_det *out, int cap)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t nwin = 0;
    for (int l = 0; l < L; l++)
        nwin += (size_t)nf * (hs[l] / CELL - WIN + 1) * (ws[l] / CELL - WIN + 1);
    double *scores = (double *)malloc(sizeof(double) * (nwin + 1));
    hgo_frame_scores_ex(frame, w, h, stride, min_size, skip_levels, direct, eps, tau, filt, nf,
                        scores, nwin);
    int n = 0;
    size_t soff = 0;
    for (int l = 0; l < L; l++) {
        int nu = hs[l] / CELL - WIN + 1, nv = ws[l] / CELL - WIN + 1;
        for (int f = 0; f < nf; f++)
            for (int u = 0; u < nu; u++)
                for (int v = 0; v < nv; v++) {
                    double s = scores[soff + ((size_t)f * nu + u) * nv + v];
                    if (l >= skip_levels && s > threshold) {
                        if (n < cap) {
                            hgo_det *d = &out[n];
                            d->level = l; d->filter = f; d->u = u; d->v = v;
                            d->score = s;
                            hgo_box(w, h, ws[l], hs[l], u, v, d);
                        }
                        n++;
                    }
                }
        soff += (size_t)nf * nu * nv;
    }
    free(scores);
    return n;
}

/* Region of interest (Section 6.6, future work: near the previous frame's
 * face only some scales and locations need a scan).  Window (u, v) of level
 * l is scanned iff lmin <= l <= lmax and its centre, (8v + 40, 8u + 40) in
 * level pixels mapped to the frame as fl((8v + 40) * fl(W0 / Wl)) and
 * fl((8u + 40) * fl(H0 / Hl)), lies in [x0, x1) x [y0, y1).               */
int hgo_in_roi(int W0, int H0, int Wl, int Hl, int l, int u, int v,
               const double *roi /* x0, y0, x1, y1, lmin, lmax */)
{
    if (l < (int)roi[4] || l > (int)roi[5]) return 0;
    double rx = (double)W0 / (double)Wl, ry = (double)H0 / (double)Hl;
    double cx = (double)(CELL * v + CELL * WIN / 2) * rx;
    double cy = (double)(CELL * u + CELL * WIN / 2) * ry;
    return cx >= roi[0] && cx < roi[2] && cy >= roi[1] && cy < roi[3];
}

/* Detection restricted to a region of interest: the candidates of
 * hgo_frame_candidates_ex whose window passes hgo_in_roi, then greedy NMS.
 * Returns the kept count; *n_candidates gets the restricted count.        */
int hgo_detect_roi(const uint8_t *frame, int w, int h, int stride, int min_size,
                   int skip_levels, int direct, double eps, double tau, double threshold,
                   double nms_iou, const double *filt, int nf, const double *roi,
                   hgo_det *out, int cap, int32_t *n_candidates)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t nwin = 0;
    for (int l = 0; l < L; l++)
        nwin += (size_t)nf * (hs[l] / CELL - WIN + 1) * (ws[l] / CELL - WIN + 1);
    hgo_det *c = (hgo_det *)malloc(sizeof(hgo_det) * (nwin + 1));
    int n = hgo_frame_candidates_ex(frame, w, h, stride, min_size, skip_levels, direct, eps, tau,
                                    threshold, filt, nf, c, (int)nwin);
    int m = 0;
    for (int i = 0; i < n; i++)
        if (hgo_in_roi(w, h, ws[c[i].level], hs[c[i].level], c[i].level, c[i].u, c[i].v, roi))
            c[m++] = c[i];
    if (n_candidates) *n_candidates = m;
    int32_t *keep = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
    hgo_nms(c, m, nms_iou, keep);
    int k = 0;
    for (int i = 0; i < m; i++)
        if (keep[i]) { if (k < cap) out[k] = c[i]; k++; }
    free(keep);
    free(c);
    return k;
}

/* Full detection of one frame: candidates then greedy NMS.  Writes the kept
 * detections in rank order; returns the kept count (or < 0).               */
int hgo_detect_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                  int skip_levels, int direct, double eps, double tau, double threshold,
                  double nms_iou, const double *filt, int nf, hgo_det *out, int cap,
                  int32_t *n_candidates);

int hgo_detect(const uint8_t *frame, int w, int h, int stride, int min_size,
               int skip_levels, double eps, double tau, double threshold,
               double nms_iou, const double *filt, int nf, hgo_det *out, int cap,
               int32_t *n_candidates)
{
    return hgo_detect_ex(frame, w, h, stride, min_size, skip_levels, 0, eps, tau, threshold,
                         nms_iou, filt, nf, out, cap, n_candidates);
}

int hgo_detect_ex(const uint8_t *frame, int w, int h, int stride, int min_size,
                  int skip_levels, int direct, double eps, double tau, double threshold,
                  double nms_iou, const double *filt, int nf, hgo_det *out, int cap,
                  int32_t *n_candidates)
{
    int ws[64], hs[64];
    int L = hgo_level_sizes(w, h, min_size, ws, hs, 64);
    if (L > 64) return -1;
    size_t nwin = 0;
    for (int l = 0; l < L; l++)
        nwin += (size_t)nf * (hs[l] / CELL - WIN + 1) * (ws[l] / CELL - WIN + 1);
    hgo_det *c = (hgo_det *)malloc(sizeof(hgo_det) * (nwin + 1));
    int n = hgo_frame_candidates_ex(frame, w, h, stride, min_size, skip_levels, direct, eps, tau,
                                    threshold, filt, nf, c, (int)nwin);
    if (n_candidates) *n_candidates = n;
    int32_t *keep = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    hgo_nms(c, n, nms_iou, keep);
    int k = 0;
    for (int i = 0; i < n; i++)
        if (keep[i]) { if (k < cap) out[k] = c[i]; k++; }
    free(keep);
    free(c);
    return k;
}

/* Many frames of one size, frames[i] at frames + i*frame_bytes, each with
 * its own output block of cap_per_frame detections; frames run in parallel
 * over the host's cores when OpenMP is available.  Returns the threads used. */
int hgo_detect_many(const uint8_t *frames, int n_frames, size_t frame_bytes, int w, int h,
                    int stride, int min_size, int skip_levels, double eps, double tau,
                    double threshold, double nms_iou, const double *filt, int nf,
                    hgo_det *out, int cap_per_frame, int32_t *counts, int n_threads)
{
    int used = 1;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
    for (int i = 0; i < n_frames; i++) {
#pragma omp atomic write
        used = omp_get_num_threads();
        counts[i] = hgo_detect(frames + (size_t)i * frame_bytes, w, h, stride, min_size,
                               skip_levels, eps, tau, threshold, nms_iou, filt, nf,
                               out + (size_t)i * cap_per_frame, cap_per_frame, NULL);
    }
#else
    (void)n_threads;
    for (int i = 0; i < n_frames; i++)
        counts[i] = hgo_detect(frames + (size_t)i * frame_bytes, w, h, stride, min_size,
                               skip_levels, eps, tau, threshold, nms_iou, filt, nf,
                               out + (size_t)i * cap_per_frame, cap_per_frame, NULL);
#endif
    return used;
}

/* ------------------------------------------------------------------------ */
/* Training adjoint (hinge loss on the best window score of one filter).
 *
 * Float mode: the pyramid is real-valued (hgo_downscale_f64, no rounding).
 * For crop i with label y_i in {-1, +1}: s_i = max over all windows of all
 * levels of the filter's score (ties: the first in (level, u, v) order);
 * L = (1/B) sum_i max(0, 1 - y_i s_i), subgradient 0 at the kink.
 * dL/dW = (1/B) sum_{active i} (-y_i) feat_i[window_i]; dL/dI follows the
 * chain feature -> (truncation, N_k(S_k), E) -> histogram -> magnitude ->
 * central differences -> pyramid, with orientation bins, the argmax window,
 * the truncation set (min(x, tau) passes the gradient iff x < tau) and the
 * hinge activity held fixed.                                               */

typedef struct {
    int L;
    int ws[64], hs[64];
    double *pyr;            /* all levels, [h_l][w_l] back to back */
    size_t off[64];
} hgo_fpyr;

static void fpyr_build(const double *img, int w, int h, int min_size, hgo_fpyr *P)
{
    P->L = hgo_level_sizes(w, h, min_size, P->ws, P->hs, 64);
    size_t n = 0;
    for (int l = 0; l < P->L; l++) { P->off[l] = n; n += (size_t)P->ws[l] * P->hs[l]; }
    P->pyr = (double *)malloc(sizeof(double) * (n + 1));
    if (P->L > 0) hgo_pyramid_f64(img, w, h, min_size, P->pyr, n);
}

/* Best window of one filter over all levels (float mode). Returns s. */
static double best_window(const hgo_fpyr *P, double eps, double tau, const double *filt,
                          int *bl, int *bu, int *bv)
{
    double best = 0.0;
    int have = 0;
    *bl = *bu = *bv = -1;
    for (int l = 0; l < P->L; l++) {
        int w = P->ws[l], h = P->hs[l], cx = w / CELL, cy = h / CELL;
        int nu = cy - WIN + 1, nv = cx - WIN + 1;
        if (nu <= 0 || nv <= 0) continue;
        double *hist = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NBIN + 1));
        double *feat = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NFEAT + 1));
        double *sc = (double *)malloc(sizeof(double) * ((size_t)nu * nv + 1));
        hgo_cell_hist(P->pyr + P->off[l], w, h, hist);
        hgo_features(hist, cx, cy, eps, tau, feat);
        hgo_correlate(feat, cx, cy, filt, 1, sc);
        for (int u = 0; u < nu; u++)
            for (int v = 0; v < nv; v++) {
                double s = sc[(size_t)u * nv + v];
                if (!have || s > best) { best = s; have = 1; *bl = l; *bu = u; *bv = v; }
            }
        free(hist); free(feat); free(sc);
    }
    return best;
}

/* Forward only: loss of a batch (float mode), best scores and windows. */
double hgo_hinge_loss(const double *imgs, int n, int w, int h, const double *labels, int min_size,
                      double eps, double tau, const double *filt, double *scores, int32_t *wins)
{
    double loss = 0.0;
    for (int i = 0; i < n; i++) {
        hgo_fpyr P;
        fpyr_build(imgs + (size_t)i * w * h, w, h, min_size, &P);
        int l, u, v;
        double s = best_window(&P, eps, tau, filt, &l, &u, &v);
        if (scores) scores[i] = s;
        if (wins) { wins[3 * i] = l; wins[3 * i + 1] = u; wins[3 * i + 2] = v; }
        double m = 1.0 - labels[i] * s;
        if (l >= 0 && m > 0.0) loss += m;
        free(P.pyr);
    }
    return loss / n;
}

/* Loss, dL/dW (3100, [a][b][c]) and optionally dL/dI ([n][h][w]). */
double hgo_hinge_backward(const double *imgs, int n, int w, int h, const double *labels,
                          int min_size, double eps, double tau, const double *filt,
                          double *dW, double *dI)
{
    double loss = 0.0;
    memset(dW, 0, sizeof(double) * WIN * WIN * NFEAT);
    if (dI) memset(dI, 0, sizeof(double) * (size_t)n * w * h);
    static const int bdx[4] = {-1, +1, -1, +1};
    static const int bdy[4] = {-1, -1, +1, +1};
    for (int i = 0; i < n; i++) {
        hgo_fpyr P;
        fpyr_build(imgs + (size_t)i * w * h, w, h, min_size, &P);
        int l, u0, v0;
        double s = best_window(&P, eps, tau, filt, &l, &u0, &v0);
        double m = 1.0 - labels[i] * s;
        if (l < 0 || !(m > 0.0)) { free(P.pyr); continue; }
        loss += m;
        const double g = -labels[i] / n;       /* dL/ds_i */
        int lw = P.ws[l], lh = P.hs[l], cx = lw / CELL, cy = lh / CELL;
        const double *img = P.pyr + P.off[l];
        double *hist = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NBIN + 1));
        double *feat = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NFEAT + 1));
        hgo_cell_hist(img, lw, lh, hist);
        hgo_features(hist, cx, cy, eps, tau, feat);
        for (int a = 0; a < WIN; a++)
            for (int b = 0; b < WIN; b++)
                for (int c = 0; c < NFEAT; c++)
                    dW[(a * WIN + b) * NFEAT + c] +=
                        g * feat[((size_t)(u0 + a) * cx + (v0 + b)) * NFEAT + c];
        if (dI) {
            /* energies and normalisers of every cell */
            double *E = (double *)calloc((size_t)cx * cy + 1, sizeof(double));
            for (int c = 0; c < cx * cy; c++) {
                const double *hc = hist + (size_t)c * NBIN;
                for (int o = 0; o < 9; o++) E[c] += (hc[o] + hc[o + 9]) * (hc[o] + hc[o + 9]);
            }
            double *dh = (double *)calloc((size_t)cx * cy * NBIN + 1, sizeof(double));
            double *dE = (double *)calloc((size_t)cx * cy + 1, sizeof(double));
            for (int a = 0; a < WIN; a++)
                for (int b = 0; b < WIN; b++) {
                    int ci = u0 + a, cj = v0 + b;
                    const double *hc = hist + ((size_t)ci * cx + cj) * NBIN;
                    const double *Wc = filt + (a * WIN + b) * NFEAT;
                    double *dhc = dh + ((size_t)ci * cx + cj) * NBIN;
                    double S[4], N[4], dN[4] = {0, 0, 0, 0};
                    for (int k = 0; k < 4; k++) {
                        S[k] = energy_at(E, cx, cy, ci, cj) + energy_at(E, cx, cy, ci, cj + bdx[k])
                             + energy_at(E, cx, cy, ci + bdy[k], cj)
                             + energy_at(E, cx, cy, ci + bdy[k], cj + bdx[k]);
                        N[k] = 1.0 / sqrt(S[k] + eps);
                    }
                    for (int o = 0; o < NBIN; o++)
                        for (int k = 0; k < 4; k++)
                            if (hc[o] * N[k] < tau) {
                                double coef = 0.5 * g * Wc[o] + TEXTURE_W * g * Wc[27 + k];
                                dhc[o] += coef * N[k];
                                dN[k] += coef * hc[o];
                            }
                    for (int o = 0; o < 9; o++) {
                        double su = hc[o] + hc[o + 9];
                        for (int k = 0; k < 4; k++)
                            if (su * N[k] < tau) {
                                double coef = 0.5 * g * Wc[NBIN + o];
                                dhc[o] += coef * N[k];
                                dhc[o + 9] += coef * N[k];
                                dN[k] += coef * su;
                            }
                    }
                    for (int k = 0; k < 4; k++) {
                        double dS = dN[k] * (-0.5) * pow(S[k] + eps, -1.5);
                        int cells[4][2] = {{ci, cj}, {ci, cj + bdx[k]}, {ci + bdy[k], cj},
                                           {ci + bdy[k], cj + bdx[k]}};
                        for (int q = 0; q < 4; q++) {
                            int ii = cells[q][0], jj = cells[q][1];
                            if (ii >= 0 && jj >= 0 && ii < cy && jj < cx) dE[(size_t)ii * cx + jj] += dS;
                        }
                    }
                }
            for (int c = 0; c < cx * cy; c++) {
                if (dE[c] == 0.0) continue;
                const double *hc = hist + (size_t)c * NBIN;
                for (int o = 0; o < 9; o++) {
                    double t2 = 2.0 * dE[c] * (hc[o] + hc[o + 9]);
                    dh[(size_t)c * NBIN + o] += t2;
                    dh[(size_t)c * NBIN + o + 9] += t2;
                }
            }
            /* histogram -> magnitude -> central differences -> level pixels */
            size_t npx = 0;
            for (int q = 0; q <= l; q++) npx += (size_t)P.ws[q] * P.hs[q];
            double *dP = (double *)calloc(npx + 1, sizeof(double));
            double *dl = dP + P.off[l];
            int xmax = lw - 2 < CELL * cx - 1 ? lw - 2 : CELL * cx - 1;
            int ymax = lh - 2 < CELL * cy - 1 ? lh - 2 : CELL * cy - 1;
            for (int y = 1; y <= ymax; y++)
                for (int x = 1; x <= xmax; x++) {
                    double dx = img[y * lw + x + 1] - img[y * lw + x - 1];
                    double dy = img[(y + 1) * lw + x] - img[(y - 1) * lw + x];
                    int bb = hgo_orientation_bin(dx, dy);
                    if (bb < 0) continue;
                    double mag = sqrt(dx * dx + dy * dy);
                    double xp = (x + 0.5) / CELL - 0.5, yp = (y + 0.5) / CELL - 0.5;
                    int ix = (int)floor(xp), iy = (int)floor(yp);
                    double ax = xp - ix, ay = yp - iy, dmag = 0.0;
                    for (int di = 0; di < 2; di++) {
                        int ii = iy + di;
                        if (ii < 0 || ii >= cy) continue;
                        double wy = di ? ay : 1.0 - ay;
                        for (int dj = 0; dj < 2; dj++) {
                            int jj = ix + dj;
                            if (jj < 0 || jj >= cx) continue;
                            double wx = dj ? ax : 1.0 - ax;
                            dmag += wx * wy * dh[((size_t)ii * cx + jj) * NBIN + bb];
                        }
                    }
                    if (dmag == 0.0) continue;
                    double ddx = dmag * dx / mag, ddy = dmag * dy / mag;
                    dl[y * lw + x + 1] += ddx;
                    dl[y * lw + x - 1] -= ddx;
                    dl[(y + 1) * lw + x] += ddy;
                    dl[(y - 1) * lw + x] -= ddy;
                }
            /* pyramid transpose: level q+1 pixel = sum of 4 taps of level q / 100 */
            for (int q = l - 1; q >= 0; q--) {
                int w1 = P.ws[q + 1], h1 = P.hs[q + 1], w0 = P.ws[q];
                const double *d1 = dP + P.off[q + 1];
                double *d0 = dP + P.off[q];
                for (int y = 0; y < h1; y++) {
                    int Y = 12 * y + 1, y0 = Y / 10, fy = Y % 10;
                    for (int x = 0; x < w1; x++) {
                        int X = 12 * x + 1, x0 = X / 10, fx = X % 10;
                        double gpx = d1[(size_t)y * w1 + x] / 100.0;
                        if (gpx == 0.0) continue;
                        d0[(size_t)y0 * w0 + x0] += (10 - fx) * (10 - fy) * gpx;
                        d0[(size_t)y0 * w0 + x0 + 1] += fx * (10 - fy) * gpx;
                        d0[(size_t)(y0 + 1) * w0 + x0] += (10 - fx) * fy * gpx;
                        d0[(size_t)(y0 + 1) * w0 + x0 + 1] += fx * fy * gpx;
                    }
                }
            }
            double *di_out = dI + (size_t)i * w * h;
            for (size_t k = 0; k < (size_t)w * h; k++) di_out[k] = dP[k];
            free(dP); free(dE); free(dh); free(E);
        }
        free(hist); free(feat);
        free(P.pyr);
    }
    return loss / n;
}

/* Discrete state of a crop's forward pass: argmax window, orientation bins
 * of the argmax level, truncation flags of the window cells -- as a hash,
 * so a finite-difference test can skip perturbations that change it.      */
uint64_t hgo_forward_signature(const double *img, int w, int h, int min_size, double eps,
                               double tau, const double *filt)
{
    hgo_fpyr P;
    fpyr_build(img, w, h, min_size, &P);
    int l, u0, v0;
    best_window(&P, eps, tau, filt, &l, &u0, &v0);
    uint64_t hsh = 1469598103934665603ull;
#define MIX(x) do { hsh ^= (uint64_t)(int64_t)(x); hsh *= 1099511628211ull; } while (0)
    MIX(l); MIX(u0); MIX(v0);
    if (l >= 0) {
        int lw = P.ws[l], lh = P.hs[l], cx = lw / CELL, cy = lh / CELL;
        const double *img2 = P.pyr + P.off[l];
        for (int y = 1; y < lh - 1; y++)
            for (int x = 1; x < lw - 1; x++)
                MIX(hgo_orientation_bin(img2[y * lw + x + 1] - img2[y * lw + x - 1],
                                        img2[(y + 1) * lw + x] - img2[(y - 1) * lw + x]));
        double *hist = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NBIN + 1));
        hgo_cell_hist(img2, lw, lh, hist);
        double *E = (double *)calloc((size_t)cx * cy + 1, sizeof(double));
        for (int c = 0; c < cx * cy; c++)
            for (int o = 0; o < 9; o++) E[c] += (hist[c * NBIN + o] + hist[c * NBIN + o + 9]) *
                                                (hist[c * NBIN + o] + hist[c * NBIN + o + 9]);
        static const int bdx[4] = {-1, +1, -1, +1};
        static const int bdy[4] = {-1, -1, +1, +1};
        for (int a = 0; a < WIN; a++)
            for (int b = 0; b < WIN; b++) {
                int ci = u0 + a, cj = v0 + b;
                const double *hc = hist + ((size_t)ci * cx + cj) * NBIN;
                for (int k = 0; k < 4; k++) {
                    double S = energy_at(E, cx, cy, ci, cj) + energy_at(E, cx, cy, ci, cj + bdx[k])
                             + energy_at(E, cx, cy, ci + bdy[k], cj)
                             + energy_at(E, cx, cy, ci + bdy[k], cj + bdx[k]);
                    double N = 1.0 / sqrt(S + eps);
                    for (int o = 0; o < NBIN; o++) MIX(hc[o] * N < tau);
                    for (int o = 0; o < 9; o++) MIX((hc[o] + hc[o + 9]) * N < tau);
                }
            }
        free(hist); free(E);
    }
#undef MIX
    free(P.pyr);
    return hsh;
}

/* ------------------------------------------------------------------------ */
/* The discrete state of the float-mode forward of one crop that the adjoint
 * holds fixed -- the quantities hgo_forward_signature hashes, as arrays, so
 * that a test can find where an adjoint computed in another precision took
 * a decision the other way: best window (level, u, v) of the filter (-1 if
 * none); the orientation bin of every pixel of that level (bins [lh][lw],
 * -1 for a zero gradient and on the one-pixel border; room for w*h
 * entries); and, per window cell (a, b) and block k, the 27 truncation
 * tests x N_k < tau for x = h_o (o < 18) and h_o + h_{o+9} (o < 9) (trunc
 * [100][4][27]).  *lw, *lh receive the level's size (0 without a window).  */

void hgo_forward_state(const double *img, int w, int h, int min_size, double eps, double tau,
                       const double *filt, int32_t *best3, int32_t *lw_out, int32_t *lh_out,
                       int8_t *bins, uint8_t *trunc)
{
    hgo_fpyr P;
    fpyr_build(img, w, h, min_size, &P);
    int l, u0, v0;
    best_window(&P, eps, tau, filt, &l, &u0, &v0);
    best3[0] = l; best3[1] = u0; best3[2] = v0;
    *lw_out = *lh_out = 0;
    if (l >= 0) {
        int lw = P.ws[l], lh = P.hs[l], cx = lw / CELL, cy = lh / CELL;
        *lw_out = lw; *lh_out = lh;
        const double *img2 = P.pyr + P.off[l];
        for (int y = 0; y < lh; y++)
            for (int x = 0; x < lw; x++) {
                int b = -1;
                if (y >= 1 && y < lh - 1 && x >= 1 && x < lw - 1)
                    b = hgo_orientation_bin(img2[y * lw + x + 1] - img2[y * lw + x - 1],
                                            img2[(y + 1) * lw + x] - img2[(y - 1) * lw + x]);
                bins[(size_t)y * lw + x] = (int8_t)b;
            }
        double *hist = (double *)malloc(sizeof(double) * ((size_t)cx * cy * NBIN + 1));
        hgo_cell_hist(img2, lw, lh, hist);
        double *E = (double *)calloc((size_t)cx * cy + 1, sizeof(double));
        for (int c = 0; c < cx * cy; c++)
            for (int o = 0; o < 9; o++) E[c] += (hist[c * NBIN + o] + hist[c * NBIN + o + 9]) *
                                                (hist[c * NBIN + o] + hist[c * NBIN + o + 9]);
        static const int bdx[4] = {-1, +1, -1, +1};
        static const int bdy[4] = {-1, -1, +1, +1};
        for (int a = 0; a < WIN; a++)
            for (int b = 0; b < WIN; b++) {
                int ci = u0 + a, cj = v0 + b;
                const double *hc = hist + ((size_t)ci * cx + cj) * NBIN;
                for (int k = 0; k < 4; k++) {
                    double S = energy_at(E, cx, cy, ci, cj) + energy_at(E, cx, cy, ci, cj + bdx[k])
                             + energy_at(E, cx, cy, ci + bdy[k], cj)
                             + energy_at(E, cx, cy, ci + bdy[k], cj + bdx[k]);
                    double N = 1.0 / sqrt(S + eps);
                    uint8_t *t = trunc + ((size_t)(a * WIN + b) * 4 + k) * (NBIN + 9);
                    for (int o = 0; o < NBIN; o++) t[o] = hc[o] * N < tau;
                    for (int o = 0; o < 9; o++) t[NBIN + o] = (hc[o] + hc[o + 9]) * N < tau;
                }
            }
        free(hist); free(E);
    }
    free(P.pyr);
}
