/*
 * hog.h -- C ABI of libhog, GB300 (sm_103a) HOG face detection.
 *
 * The library computes, for 8-bit grayscale frames, the HOG face-detection
 * path of Bakker et al., "Real-time face and landmark localization for
 * eyeblink detection" (Section 4.1.1, algorithm breakdown; Section 5.1, GPU
 * implementation):
 *   scale-space pyramid (5/6 steps down to the 80x80 window)
 *   -> per-pixel gradient, 18 signed orientation bins, 8x8-pixel cells with
 *      bilinear voting into the 4 nearest cells
 *   -> energy of each cell and its 8 neighbours, block normalisation and
 *      truncation into 31 features (18 signed + 9 unsigned + 4 energy)
 *   -> correlation with F linear filters of 10x10 cells x 31 (3100 weights)
 *   -> strict threshold, non-maximum suppression over levels and filters.
 *
 * Conventions for every call:
 *   - Return HOG_OK (0) or a negative HOG_E* code.  No C++ exception crosses
 *     the ABI.  hog_last_error(ctx) gives a message for the last failure.
 *   - "device" pointers are CUDA device memory, "host" pointers host memory.
 *     The caller owns every buffer it passes; the context owns its arenas
 *     and its copy of the filters.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream).  Calls that return host results
 *     synchronise that stream before returning.
 *   - One context is used by one host thread at a time.
 *   - Image coordinates: x = column, y = row.  Cells (i, j) = (row, col).
 *     Windows (u, v) = (row, col) of the window's top-left cell.
 *   - Frames smaller than min_size in either dimension have 0 levels and 0
 *     detections; this is not an error.
 */
#ifndef HOG_H
#define HOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define HOG_OK          0
#define HOG_EINVAL     (-1)  /* bad argument (null, size, layout, parameter)  */
#define HOG_ENOMEM     (-2)  /* device or pinned-host allocation failed        */
#define HOG_ECUDA      (-3)  /* a CUDA runtime call or kernel launch failed    */
#define HOG_ECAPACITY  (-4)  /* output truncated to its capacity; counts exact */
#define HOG_ETIMEOUT   (-5)  /* a bounded device wait gave up                  */
#define HOG_EINTERNAL  (-6)  /* a kernel's own consistency check failed        */
#define HOG_EBUSY      (-7)  /* the server's request queue is full; retry      */

/* ---- fixed sizes of the method (Section 4.1.1) ------------------------- */
#define HOG_CELL        8    /* 8x8-pixel cells                               */
#define HOG_NBIN        18   /* signed orientation bins                       */
#define HOG_NFEAT       31   /* 18 signed + 9 unsigned + 4 energy features    */
#define HOG_WIN         10   /* 10x10-cell (80x80-pixel) window               */
#define HOG_MAX_FILTERS 8    /* filters per context (the paper uses 5)        */
#define HOG_MAX_LEVELS  32   /* pyramid levels per frame                      */
/* Largest |weight| the tensor-core correlation engines accept: they store
 * 64 w in fp16, whose largest finite value is 65504.  Filters with a larger
 * weight run on the FP32 CUDA-core engine (see hog_set_corr_engine).      */
#define HOG_TC_MAX_WEIGHT 1023.5f

typedef struct hog_ctx hog_ctx;   /* opaque, owned by the library */

/* Detector parameters.  hog_default_params() fills the paper's values plus
 * the readings this library takes where the paper is silent.  cell,
 * win_cells_w/h and scale_num/den are fixed by the paper (8, 10, 10, 5/6);
 * other values are rejected with HOG_EINVAL. */
typedef struct {
    int32_t cell;               /* 8                                          */
    int32_t win_cells_w;        /* 10                                         */
    int32_t win_cells_h;        /* 10                                         */
    int32_t scale_num;          /* 5  (each level is 5/6 of the previous)     */
    int32_t scale_den;          /* 6                                          */
    int32_t min_size;           /* 80: keep a level while min(w,h) >= this    */
    int32_t skip_levels;        /* 0: levels < skip_levels are not scanned     *
                                 * (Section 5.1: a face of >= 20 % of the      *
                                 * frame needs no scan of the largest scale);  *
                                 * detection computes no histograms or         *
                                 * features for them either                    */
    float   eps;                /* 1e-4: added to block energies              */
    float   trunc;              /* 0.2: truncation of normalised bins         */
    float   threshold;          /* 0: detection iff score > threshold         */
    float   nms_iou;            /* 0.5: suppress iff IoU > nms_iou (>= 0.45)  */
    int32_t max_w, max_h;       /* largest frame the context accepts          */
    int32_t max_batch;          /* frames per internal batch                  */
    int32_t max_dets_per_frame; /* device capacity of kept boxes per frame    */
    int32_t float_pyramid;      /* 0: uint8 pyramid (detection)               */
    int32_t direct_first;       /* 0; 1 with skip_levels = s >= 2: level s is  *
                                 * resampled straight from the frame with the *
                                 * ratio (6/5)^s (Section 6.6, future work:   *
                                 * direct-to-size downscale), levels 1..s-1   *
                                 * are not computed (hog_pyramid/_features/   *
                                 * _scores return zeros there), later levels  *
                                 * follow in 5/6 steps.  s <= 8 with 1.       */
} hog_params;

/* One frame: 8-bit grayscale, row pitch in bytes (>= w).  For the device
 * entry points data is a device pointer; for hog_detect_host a host one. */
typedef struct {
    const uint8_t *data;
    int32_t w, h, pitch;
} hog_frame;

/* One kept detection.  Box (x, y, w, h) is in frame pixels: the window's
 * (8v, 8u, 80, 80) in level pixels scaled by (W0/Wl, H0/Hl) in FP64. */
typedef struct {
    int32_t frame, level, filter, u, v;
    float   score;
    double  x, y, w, h;
} hog_det;

/* Geometry of one pyramid level.  offset = element offset of this level in
 * the output buffer of the call that filled it (bytes for hog_pyramid,
 * floats for hog_features / hog_scores). */
typedef struct {
    int32_t w, h, cx, cy;
    int64_t offset;
} hog_level;

/* Fill *p with the defaults listed in the struct comments; max_w/max_h
 * 1280x1024, max_batch 64, max_dets_per_frame 16384. */
void hog_default_params(hog_params *p);

/* Level geometry for a w x h frame (host only, no GPU work).  Writes up to
 * cap levels; *n_levels = the true count.  Offsets are those hog_features
 * uses (floats, [cy][cx][31] per level, levels back to back). */
int hog_level_geometry(const hog_params *p, int32_t w, int32_t h, hog_level *levels,
                       int32_t cap, int32_t *n_levels);

/* Create a context: validates *p, copies n_filters filters from host memory
 * (layout [f][row a][col b][channel c], 10 x 10 x 31 floats each; the five
 * rotation filters of Section 4.1.1) to the device and allocates the device
 * arenas for max_batch frames of max_w x max_h.  *out is NULL on failure.
 * The weights of a trained linear filter may have any scale: every finite
 * value is accepted (HOG_EINVAL for a NaN or infinite weight).  The context
 * starts on tensor-core engine 1 when every |w| <= HOG_TC_MAX_WEIGHT, else
 * on the FP32 CUDA-core engine 0 (hog_get_corr_engine tells which;
 * hog_last_error gives the reason). */
int hog_create(const hog_params *p, const float *filters_host, int32_t n_filters,
               hog_ctx **out);

/* Replace the filters (same layout; 1 <= n_filters <= HOG_MAX_FILTERS).
 * Stream-ordered on the legacy default stream; synchronises the device.
 * HOG_EINVAL (filters unchanged) for a weight that is not finite.  If a
 * tensor engine is selected and a new weight exceeds HOG_TC_MAX_WEIGHT, the
 * context switches to engine 0 and returns HOG_OK, with the reason in
 * hog_last_error. */
int hog_set_filters(hog_ctx *ctx, const float *filters_host, int32_t n_filters);

/* Release everything the context owns.  NULL-safe. */
void hog_destroy(hog_ctx *ctx);

/* Message of the last failed call on ctx (never NULL; "" if none).  With
 * ctx == NULL, the message of the last failed hog_create on this thread. */
const char *hog_last_error(const hog_ctx *ctx);

/* Pyramid of one frame (Section 4.1.1, first step; Section 5.1 scaling
 * kernel): level 0 is the frame, level l+1 the 5/6 resample of level l
 * (exact integer bilinear, pixel-centre aligned, rounded half up).  out
 * (device, caller-owned) receives all levels back to back, [h_l][w_l]
 * bytes each; levels (host) gets sizes and byte offsets.  HOG_EINVAL if
 * cap_bytes or cap_levels is too small (*n_levels still set). */
int hog_pyramid(hog_ctx *ctx, const hog_frame *frame, uint8_t *out, size_t cap_bytes,
                hog_level *levels, int32_t cap_levels, int32_t *n_levels, void *stream);

/* 31-d features of every level of one frame (Section 4.1.1 gradient,
 * histogramisation, normalisation and feature steps).  feat_out (device,
 * caller-owned) receives [cy][cx][31] floats per level, levels back to back
 * at levels[l].offset.  HOG_EINVAL if a capacity is too small. */
int hog_features(hog_ctx *ctx, const hog_frame *frame, float *feat_out, size_t cap_floats,
                 hog_level *levels, int32_t cap_levels, int32_t *n_levels, void *stream);

/* Scores of every window of every level for every filter (Section 4.1.1,
 * linear classification filter): scores_out (device) receives
 * [F][cy-9][cx-9] floats per level at levels[l].offset. */
int hog_scores(hog_ctx *ctx, const hog_frame *frame, float *scores_out, size_t cap_floats,
               hog_level *levels, int32_t cap_levels, int32_t *n_levels, void *stream);

/* Detect faces in n_frames device frames (any mix of sizes <= max_w x
 * max_h): the whole path, batched per stage, then suppression (Section
 * 4.1.1 last step) on the device.  dets (host) receives the kept boxes of
 * all frames, frame by frame, each frame's boxes in (level, u, v) order;
 * counts (host, n_frames) the kept count per frame.  Returns HOG_ECAPACITY
 * if det_cap or max_dets_per_frame truncated the output (counts exact).
 * Synchronises the stream. */
int hog_detect(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, hog_det *dets,
               int32_t det_cap, int32_t *counts, void *stream);

/* Same result as hog_detect (bit for bit), computed the batched way: all
 * pyramid levels of all frames (any mix of sizes) in one persistent fused
 * launch -- work items in dependency order, taken from a ticket counter,
 * bounded waits on per-(frame, level, stage) completion counters -- then
 * the suppression launch; from the second call on a batch of the same
 * frame buffers, both replay as a captured CUDA graph.  This generalises
 * the paper's batching of 16 frames along the grid's z dimension and its
 * per-scale streams (Section 5.1).  hog_autotune may select the per-stage
 * launches instead, when they measure faster.  HOG_ETIMEOUT if a bounded
 * device wait gave up (outputs invalid).  Synchronises the stream. */
int hog_detect_batched(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, hog_det *dets,
                       int32_t det_cap, int32_t *counts, void *stream);

/* Execution used by hog_detect_batched and hog_detect_host: 1 = persistent
 * fused launch (default), 0 = one launch per stage (both as graphs). */
int hog_set_batched_mode(hog_ctx *ctx, int32_t mode);

/* Correlation engine.  0: FP32 CUDA cores, one warp per 128-window tile.
 * 1 (default when its buffers can be allocated at hog_create) and 2: tcgen05
 * tensor cores -- for each filter row a,
 * G[a][p] = sum over 10 cell shifts and 32 channels of feat[p + b] W[a][b]
 * is a GEMM over the level's cells (M = 128 cells per MMA, K = 320, N = 10
 * rows x F filters), with features and weights split into fp16 hi + lo parts
 * (three MMAs per step, FP32 accumulation in tensor memory), and
 * score(u, v) = sum_a G[a][(u + a) cx + v].  Engine 1 sums G on chip, in a
 * ring of partial scores in shared memory, while the next tile's MMAs run
 * (one persistent CTA per SM over bands of window rows); engine 2 writes G
 * to device memory and sums it in a second kernel.  Engines 1 and 2 give
 * bit-identical scores; they agree with engine 0 to about 1e-6 (not bit for
 * bit).  With a tensor engine the persistent fused launch covers pyramid to
 * features and the same correlation kernel follows it, so both batched
 * modes stay bit-identical to hog_detect.  Engines 1 and 2 hold 128 bytes
 * per feature cell per batch slot, engine 2 another 40 F bytes; switching
 * drops cached plans.  HOG_EINVAL for other values, and for engines 1 and 2
 * while a filter weight exceeds HOG_TC_MAX_WEIGHT (their fp16 range). */
int hog_set_corr_engine(hog_ctx *ctx, int32_t engine);
int hog_get_corr_engine(const hog_ctx *ctx, int32_t *engine);

/* Suppression launch shape.  c = 1: one CTA per frame; c = 2, 4, 8 or 16:
 * each frame's suppression on a thread-block cluster of c CTAs (positions
 * split across the CTAs' shared memory, neighbour states read through
 * distributed shared memory); c = 0 (default): automatic -- clusters of
 * about SMs / frames CTAs when that is at least 8 (batches of a few frames),
 * else one CTA per frame; at least 2 for frames too large for a one-CTA
 * shared-memory workspace (about 57,800 window positions, e.g. larger than
 * 1280x1024).  The kept boxes are the same for every c.  Drops cached plans and
 * graphs when c changes.  HOG_EINVAL for other values. */
int hog_set_nms_cluster(hog_ctx *ctx, int32_t c);

/* The cluster size the suppression of a batch of n_frames frames of w x h
 * would use under the current setting (1 = one CTA per frame). */
int hog_nms_cluster_size(hog_ctx *ctx, int32_t n_frames, int32_t w, int32_t h, int32_t *c);

/* Autotuner (no counterpart in the paper, which picks block sizes by hand,
 * Section 5.1 block-size table).  On the given sample batch (device frames)
 * it times the correlation stage under each warp-tile shape policy (least
 * padding, or prefer 8x16, 4x32 or 16x8 tiles) of the CUDA-core engine and
 * under the tensor-core engine (hog_set_corr_engine) with CUDA events, then
 * the batched call in fused and per-stage mode, and keeps the fastest of
 * each in the context.  If cache_path names a JSON file written for the same device,
 * SM count, filter count and frame sizes, its choice is loaded instead of
 * measured; otherwise the measurement is written there.  cache_path may be
 * NULL.  Synchronises the stream. */
int hog_autotune(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, const char *cache_path,
                 void *stream);

/* Current tuning: batched mode (0/1) and correlation shape policy (0..3). */
int hog_get_tuning(const hog_ctx *ctx, int32_t *batched_mode, int32_t *corr_policy);

/* Failure-path control of the bounded device waits of the persistent fused
 * launch (hog_detect_batched in mode 1; no counterpart in the paper).  A
 * work item polls the completion counter it depends on at most `polls`
 * times (0 restores the default, 2^24 polls of about 64 ns each) before the
 * launch gives up and the call returns HOG_ETIMEOUT with invalid outputs.
 * withhold = 1 makes the first dependency wait of every plan built from now
 * on expect one completion more than its producers give, so that wait runs
 * out after `polls` polls: host-side fault injection for testing the error
 * path; no GPU fault or hang is involved, and the context stays usable.
 * withhold = 0 switches it off.  Drops cached plans and graphs.  HOG_EINVAL
 * for polls < 0 or withhold not 0 or 1. */
int hog_debug_waits(hog_ctx *ctx, int64_t polls, int32_t withhold);

/* Region of interest of one frame (Section 6.6, future work: near the
 * previous frame's face, scan only some scales and locations).  Window (u, v)
 * of level l is scanned iff lmin <= l <= lmax (and l >= skip_levels) and its
 * centre, (8v + 40, 8u + 40) in level pixels mapped to the frame in FP64 as
 * (8v + 40) * (W/Wl) and (8u + 40) * (H/Hl), lies in [x0, x1) x [y0, y1). */
typedef struct {
    double x0, y0, x1, y1;
    int32_t lmin, lmax;
} hog_roi;

/* hog_detect restricted to one region of interest per frame (rois[i] for
 * frames[i], host array): the kept boxes are greedy NMS over the scanned
 * windows' candidates only.  Pyramid levels above the last scanned one, and
 * histograms and features of cells no scanned window reads, are not
 * computed.  A region covering every window gives hog_detect's result bit
 * for bit.  Arguments, outputs and errors as hog_detect; HOG_EINVAL if rois
 * is NULL or a box is not finite.  Synchronises the stream. */
int hog_detect_roi(hog_ctx *ctx, const hog_frame *frames, const hog_roi *rois, int32_t n_frames,
                   hog_det *dets, int32_t det_cap, int32_t *counts, void *stream);

/* Region of interest around a previous detection (host only): the box of
 * *prev grown by margin times its width and height on each side, clipped
 * to the W x H frame, and the levels prev->level - dlev .. prev->level +
 * dlev.  HOG_EINVAL for NULL pointers, a negative margin or dlev. */
int hog_roi_around(const hog_det *prev, int32_t W, int32_t H, double margin, int32_t dlev,
                   hog_roi *out);

/* ---- Host landmark stage and the CPU/GPU pipeline (Sections 5.2, 5.3) ----
 *
 * The paper fits 68 facial landmarks to each detected face on the CPU with
 * an ensemble of regression trees (Section 4.2) and pipelines that stage
 * against the GPU detection of the next images (Table 8).  No trained model
 * exists here, so hog_ert is a STAND-IN with the same structure and cost:
 * `cascades` levels, each sampling `features` pixels at offsets from the
 * current landmarks, and `trees` trees of depth `depth` per level whose
 * splits compare two sampled pixels' difference with a threshold and whose
 * leaves add a shape increment.  Every parameter is drawn from `seed`, so
 * the landmarks carry no meaning; the stage loads the host like the real
 * one.  From the six landmarks of each eye (68-point layout, 36-41 and
 * 42-47) it reports the eye aspect ratio, the eyelid-closure signal. */
typedef struct hog_ert hog_ert;   /* opaque, host memory */
typedef struct {
    int32_t landmarks;   /* 68 (fixed)                              */
    int32_t cascades;    /* 15 levels (Section 4.2)                 */
    int32_t trees;       /* 500 trees per level (Section 4.2)       */
    int32_t depth;       /* 4 split levels per tree                 */
    int32_t features;    /* 400 sampled pixels per level            */
    uint64_t seed;
} hog_ert_params;

void hog_default_ert_params(hog_ert_params *p);
/* HOG_EINVAL for landmarks != 68 or sizes out of range; HOG_ENOMEM. */
int hog_ert_create(const hog_ert_params *p, hog_ert **out);
void hog_ert_destroy(hog_ert *m);   /* NULL-safe */
/* Fit one face (host): img (host, w x h, pitch bytes) and the face box
 * (box->x, y, w, h in frame pixels); writes landmarks[68][2] (frame pixels)
 * and, if ear is not NULL, ear[0..1] (the two eyes).  Deterministic. */
int hog_ert_fit(const hog_ert *m, const uint8_t *img, int32_t w, int32_t h, int32_t pitch,
                const hog_det *box, float *landmarks, float *ear);

/* Detect faces on n_frames HOST frames in batches of `batch` (<= max_batch)
 * and fit landmarks to each frame's best detection (highest score) with
 * n_threads host threads.  pipelined = 0: per batch, copy in, detect, wait,
 * then fit.  pipelined = 1: the detection of batch k+1 is enqueued before
 * batch k is fitted, so the GPU and the host threads overlap (Table 8).
 * Outputs (host): landmarks [n][68][2], ear [n][2], has_face [n] (0: no
 * detection, landmarks and ear zero); *seconds (may be NULL) = wall time of
 * the run without its one device allocation.  Both orders give the same
 * outputs bit for bit.  Uses the context's batched mode; synchronises the
 * stream. */
int hog_pipeline_run(hog_ctx *ctx, const hog_ert *m, const hog_frame *frames, int32_t n_frames,
                     int32_t batch, int32_t n_threads, int32_t pipelined, float *landmarks,
                     float *ear, int32_t *has_face, double *seconds, void *stream);

/* Same result as hog_detect, from frames in HOST memory: the frames are
 * copied to the device inside the call and processed like
 * hog_detect_batched, in groups of up to max_batch frames.  All frames are
 * checked first (HOG_EINVAL, nothing copied).  A group of more than
 * max_batch / 2 frames moves in chunks of up to max_batch / 2 through two
 * halves of the device staging area on a copy stream of the context: the
 * copy of chunk k+1 overlaps the per-frame stages (pyramid .. candidate
 * keys) of chunk k, and one suppression launch then takes the whole group.
 * Frames in page-locked memory are copied directly (dense frames that
 * follow each other in one copy); others are first copied into pinned host
 * staging.  The frames must stay valid until the call returns; it
 * synchronises the stream (once per group). */
int hog_detect_host(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, hog_det *dets,
                    int32_t det_cap, int32_t *counts, void *stream);

/* Features of one frame, exactly as hog_features computes them, for callers
 * that cannot allocate device memory: a frame loop with a hard deadline
 * (cudaMalloc can block and synchronise the device) or a host application
 * whose own pool owns all device memory.  The paper has no counterpart; it
 * allocates its arrays once per image sequence.  No context is needed and
 * nothing is allocated: the scratch (pyramid, histograms, internal features,
 * launch tables) is a 4 MiB file-scope device array that every GPU loading
 * libhog keeps until exit.  Only *p's min_size, eps and trunc are used (the
 * fixed fields are still checked; direct_first must be 0: this entry point
 * computes the plain 5/6 pyramid).  frame (device) must be at most 640 x 480,
 * else HOG_EINVAL with a message in err.  feat_out (device), levels (host)
 * and the capacities behave as in hog_features; frame and feat_out must be
 * memory of the current device, where the work runs.  err (host, may be
 * NULL) receives a message on failure.  All calls on a device share the
 * array: calls whose GPU work overlaps race.  The first call on each device
 * looks up the array's address; make it before any stream capture.  The
 * address is kept for the process, so a cudaDeviceReset of that device is
 * not supported afterwards. */
int hog_features_static(const hog_params *p, const hog_frame *frame, float *feat_out,
                        size_t cap_floats, hog_level *levels, int32_t cap_levels,
                        int32_t *n_levels, char *err, size_t err_cap, void *stream);

/* Training adjoint (the paper's filters are trained offline with Dlib; this
 * entry point has no counterpart there): for n crops images (device float
 * [n][h][w], 8-bit values as floats), labels (device float [n], +1 / -1) and
 * one filter weights (device float [10][10][31], layout [row][col][channel]),
 * the hinge loss on each crop's best window score,
 *   L = (1/n) sum_i max(0, 1 - y_i s_i),  s_i = max over all windows of all
 *   levels (ties: the first in (level, u, v) order),
 * computed on a real-valued pyramid (the same exact bilinear weights, no
 * rounding) with orientation bins from the largest |dot| with the 9
 * unsigned directions.  Writes dL/dW (device float [10][10][31]) and, if dI
 * is not NULL, dL/dI (device float [n][h][w]), holding bins, best windows,
 * truncation set and hinge activity fixed (subgradient 0 at every kink);
 * *loss (host, may be NULL) gets L.  recompute = 1 rebuilds the best
 * window's histograms from the pyramid in the adjoint instead of reading
 * the forward's (same result).  Synchronises the stream when loss != NULL.
 * Deterministic: every reduction is a fixed-order gather. */
int hog_backward(hog_ctx *ctx, const float *images, int32_t n, int32_t w, int32_t h,
                 const float *labels, const float *weights, float *dW, float *dI, float *loss,
                 int32_t recompute, void *stream);

/* hog_backward plus the discrete forward state its adjoint holds fixed, for
 * checking the adjoint element by element against an independent
 * implementation: where a reference computed in another precision takes
 * one of these decisions the other way, the two gradients differ by design,
 * and the state says where.  Arguments and results as hog_backward; each
 * state output may be NULL:
 *   best_out  (host int32 [n][4]): per crop the best window's level, u, v
 *             and 1 if its hinge term is active (1 - y s > 0), else 0;
 *   bins_out  (device uint8 [n][104][104]): for active crops, the
 *             orientation bin (0..17) of every pixel of the region the
 *             window's gradient reaches at its level -- 12 x 12 cells
 *             starting at cell (u - 1, v - 1), i.e. pixels from
 *             (8 (v - 1) - 4, 8 (u - 1) - 4) -- 255 where the pixel casts
 *             no vote (zero gradient, outside the level or the voting
 *             range); inactive crops are not written;
 *   trunc_out (device uint8 [n][100][4][27]): for active crops, per window
 *             cell (a, b) and block k, 1 where the truncation test
 *             x N_k < tau holds (the gradient passes) for x = h_o
 *             (o < 18) and x = h_o + h_{o+9} (o < 9); inactive crops are
 *             not written.
 * With bins_out or trunc_out the window adjoint runs even when dI is NULL.
 * Synchronises the stream when best_out or loss is not NULL. */
int hog_backward_state(hog_ctx *ctx, const float *images, int32_t n, int32_t w, int32_t h,
                       const float *labels, const float *weights, float *dW, float *dI, float *loss,
                       int32_t recompute, int32_t *best_out, uint8_t *bins_out, uint8_t *trunc_out,
                       void *stream);

/* ---- stage timing (tracing; no counterpart in the paper, which reads its
 * kernel times from a profiler, Section 5.1) ------------------------------ */
#define HOG_NSTAGES 6   /* 0 pyramid, 1 gradient+histogram, 2 normalisation+
                           features, 3 correlation+threshold, 4 suppression,
                           5 persistent fused launch (pyramid .. correlation) */
typedef struct {
    double  ms;         /* summed GPU time between CUDA events around the stage */
    int64_t launches;   /* kernel launches of the stage                         */
    int64_t units;      /* work units: output pixels, cells, cells, window x
                           filter products, frames, window x filter products  */
} hog_stage_stat;

/* Turn per-stage CUDA-event timing on (1) or off (0).  Events are recorded
 * on the caller's stream around each stage; stats accumulate until reset. */
int hog_set_profiling(hog_ctx *ctx, int32_t on);

/* Copy the accumulated per-stage stats (HOG_NSTAGES entries) into out
 * (host); waits for the last profiled work.  reset != 0 clears them. */
int hog_stage_stats(hog_ctx *ctx, hog_stage_stat *out, int32_t cap, int32_t reset);


/* ---- serving loop (no counterpart in the paper: it processes recorded
 * videos in groups of 16 frames and leaves online processing of camera
 * batches to future work, Section 6.6; its real-time target is 500 frames/s
 * per camera) ----------------------------------------------------------- */
typedef struct hog_server hog_server;   /* opaque, owned by the library */

#define HOG_SERVER_CLASSES 4   /* lane size classes of a server */

/* Server configuration.  hog_default_server_config() fills the defaults. */
typedef struct {
    int32_t max_batch;    /* frames per device batch, 1..1024 (default 8)     */
    int32_t max_lanes;    /* batches in flight at once, 1..16 (default 3):
                             each lane is a context + stream + frame slots   */
    int32_t queue_cap;    /* frames held between submit and dispatch
                             (pinned host slots), >= max_batch (default 64)  */
    int32_t batched_mode; /* -1 context default, 0 per-stage, 1 fused       */
    int64_t mem_reserve;  /* lanes after the first are created only while
                             free device memory stays above this many bytes
                             (default 1 GiB)                                 */
    /* Lane size classes (the lanes' arenas are sized for the camera mix
     * instead of all for max_w x max_h): class k holds frames up to
     * class_w[k] x class_h[k] and gets up to class_lanes[k] lanes.  All
     * class_lanes zero (default): one class of max_w x max_h with max_lanes
     * lanes.  Otherwise some class must hold max_w x max_h, the lanes of all
     * classes number at most 16, and max_lanes is not used.  A waiting frame
     * is admitted to a free lane of the smallest class that holds it; a lane
     * of a larger class takes it only while no waiting frame needs that
     * class, so small frames keep flowing while large ones wait. */
    int32_t class_w[HOG_SERVER_CLASSES];
    int32_t class_h[HOG_SERVER_CLASSES];
    int32_t class_lanes[HOG_SERVER_CLASSES];
} hog_server_config;

/* One finished request, returned by hog_server_poll. */
typedef struct {
    uint64_t id;          /* the id hog_server_submit returned                */
    int64_t  tag;         /* the caller's tag (e.g. camera << 32 | frame no)  */
    int32_t  status;      /* HOG_OK or the HOG_E* code of its batch           */
    int32_t  count;       /* kept detections (exact)                          */
    int32_t  stored;      /* of which copied into the poll's dets buffer      */
    int32_t  lane_class;  /* size class of the lane that ran it              */
    double   latency_ms;  /* submit -> result ready (host clock)              */
    double   queue_ms;    /* submit -> dispatched to a lane                   */
    double   device_ms;   /* its batch on the lane's stream: copy-in ..
                             boxes packed (CUDA events; lanes overlap)      */
    int32_t  batch;       /* frames in its batch                              */
    int32_t  lane;        /* lane that ran it                                 */
} hog_result;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t rejected;       /* submits refused with HOG_EBUSY                 */
    int64_t batches, batched_frames;
    int64_t max_inflight;   /* most frames dispatched and not yet finished    */
    int64_t lanes;          /* lanes created (admission by free memory)       */
    int64_t lane_bytes;     /* device bytes the first lane took               */
    int64_t pending;        /* frames waiting for a lane right now            */
    int64_t class_lanes[HOG_SERVER_CLASSES];   /* lanes created per class      */
    int64_t class_bytes[HOG_SERVER_CLASSES];   /* device bytes of one lane of
                                                  each class (0: none made)    */
    int64_t class_frames[HOG_SERVER_CLASSES];  /* frames each class served    */
} hog_server_stats;

void hog_default_server_config(hog_server_config *c);

/* Create a server for frames up to p->max_w x p->max_h (p->max_batch is
 * replaced by c->max_batch) with F filters (host float [F][10][10][31]).
 * Lanes are made class by class, smallest first; each lane after the very
 * first only while free device memory minus the measured size of a lane of
 * its class stays above c->mem_reserve.  Starts one worker thread.
 * HOG_EINVAL for a bad configuration (message in hog_server_last_error
 * (NULL)), HOG_ENOMEM if a class that must serve some frames gets no lane. */
int hog_server_create(const hog_params *p, const float *filters_host, int32_t n_filters,
                      const hog_server_config *c, hog_server **out);

/* Queue one 8-bit frame (HOST memory, row pitch in bytes); the frame is
 * copied before the call returns.  *id_out (may be NULL) gets the request
 * id.  HOG_EBUSY when queue_cap frames are already waiting or in flight.
 * Thread-safe: several camera threads may submit at once.  Each result is
 * bit-identical to hog_detect on that frame alone; its boxes have frame 0. */
int hog_server_submit(hog_server *s, const uint8_t *frame, int32_t w, int32_t h, int32_t pitch,
                      int64_t tag, uint64_t *id_out);

/* Take up to cap finished results in completion order (res, host) and their
 * boxes, concatenated in result order, into dets (host, det_cap entries;
 * may be NULL with det_cap 0; each result's stored says how many of its
 * boxes were copied).  Waits up to wait_us microseconds when none is ready.
 * *n_out = results returned.  Thread-safe. */
int hog_server_poll(hog_server *s, hog_result *res, int32_t cap, hog_det *dets, int32_t det_cap,
                    int32_t *n_out, int32_t wait_us);

int hog_server_get_stats(hog_server *s, hog_server_stats *out);

/* Finish every queued request, stop the worker, free everything.  Results
 * not yet polled are dropped. */
void hog_server_destroy(hog_server *s);

/* Message of the last failure of s, or of the calling thread's last
 * hog_server_create when s is NULL. */
const char *hog_server_last_error(const hog_server *s);

#ifdef __cplusplus
}
#endif
#endif /* HOG_H */
