// hog_api.cu -- C ABI of libhog: contexts, device arenas, per-batch plans
// and the orchestration of the kernels (see include/hog.h).
//
// Memory: a context allocates, once, arenas for max_batch frames of
// max_w x max_h (pyramid levels >= 1, cell histograms, features in the
// internal [4][cy][cx][8] layout, suppression keys and states, kept boxes),
// the way the paper allocates its arrays once for a sequence of equal-size
// images (Section 5.1).  Per call the host writes a plan -- one descriptor
// per (frame, level), one per frame, and per kernel a list of (descriptor,
// tile) jobs -- copies it to the device in one transfer, and launches one
// grid per stage over all frames of the batch (the paper's grid-z batching,
// Section 5.1, generalised to frames of different sizes).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hog_internal.cuh"

using namespace hogk;

namespace {

thread_local std::string g_create_error;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Geometry {
    int W = 0, H = 0, nlev = 0;
    int lw[MAX_LEVELS], lh[MAX_LEVELS], cx[MAX_LEVELS], cy[MAX_LEVELS];
    int nu[MAX_LEVELS], nv[MAX_LEVELS], pitch[MAX_LEVELS];
    int hbw[MAX_LEVELS];           // histogram tile width in blocks
    size_t pyr_off[MAX_LEVELS];    // bytes, levels >= 1, in a slot's pyramid arena
    size_t hist_off[MAX_LEVELS];   // floats
    size_t feat_off[MAX_LEVELS];   // floats, internal layout
    size_t ufeat_off[MAX_LEVELS];  // floats, user layout [cy][cx][31]
    size_t uscore_off[MAX_LEVELS]; // floats, user layout [F][nu][nv] (F filled later)
    int pos_off[MAX_LEVELS + 1];
    int npos = 0;
    size_t pyr_bytes = 0, hist_floats = 0, feat_floats = 0, ufeat_floats = 0, pyr_px = 0;
    int32_t *d_nbr = nullptr, *d_nbr_t = nullptr;
    uint8_t *d_cnt = nullptr;
};

// Level sizes: w' = floor(5w/6), h' = floor(5h/6), kept while min(w,h) >= min_size.
int compute_geometry(const hog_params &p, int W, int H, Geometry &g) {
    g = Geometry();
    g.W = W;
    g.H = H;
    int w = W, h = H, n = 0;
    size_t pyr = 0, hist = 0, feat = 0, ufeat = 0, px = 0;
    int pos = 0;
    while (w >= p.min_size && h >= p.min_size) {
        if (n >= MAX_LEVELS) return HOG_EINVAL;
        g.lw[n] = w;
        g.lh[n] = h;
        g.cx[n] = w / CELL;
        g.cy[n] = h / CELL;
        g.hbw[n] = hist_tile_bw(g.cx[n], g.cy[n], h);
        g.nu[n] = std::max(g.cy[n] - WIN + 1, 0);
        g.nv[n] = std::max(g.cx[n] - WIN + 1, 0);
        g.pitch[n] = (int)align_up((size_t)w, 16);
        g.pyr_off[n] = pyr;
        if (n >= 1) pyr += align_up((size_t)g.pitch[n] * h, 256);
        g.hist_off[n] = hist;
        hist += align_up((size_t)g.cx[n] * g.cy[n] * NBIN, 64);
        g.feat_off[n] = feat;
        feat += align_up((size_t)g.cx[n] * g.cy[n] * CHUNK, 64) * NCHUNK;
        g.ufeat_off[n] = ufeat;
        ufeat += (size_t)g.cx[n] * g.cy[n] * NFEAT;
        px += (size_t)w * h;
        g.pos_off[n] = pos;
        pos += g.nu[n] * g.nv[n];
        n++;
        w = p.scale_num * w / p.scale_den;
        h = p.scale_num * h / p.scale_den;
    }
    g.nlev = n;
    g.pos_off[n] = pos;
    g.npos = pos;
    g.pyr_bytes = pyr;
    g.hist_floats = hist;
    g.feat_floats = feat;
    g.ufeat_floats = ufeat;
    g.pyr_px = px;
    // the internal feature layout requires each chunk plane offset to keep float4 alignment
    return HOG_OK;
}

}  // namespace

namespace {
struct PlanLayout {
    size_t items = 0;
    size_t descs = 0, frames = 0, hist = 0, feat = 0, corr = 0, corrf = 0, tc = 0, tcr = 0, total = 0;
    size_t bands = 0, cta_first = 0, pyrd = 0;
    int npyrd = 0;
    std::vector<size_t> pyr;
    std::vector<int> npyr;
};

// Sizes and per-stage work of a laid-out plan (what a launch needs).
struct PlanInfo {
    PlanLayout L;
    int nhist = 0, nfeat = 0, ncorr = 0, nframes = 0, max_npos = 0, ntc = 0, ntcr = 0;
    // suppression: frames per workspace class (the plan's frames are sorted
    // by class) and the largest npos of each
    int ncls[NMS_WS_CLASSES] = {}, cls_npos[NMS_WS_CLASSES] = {};
    int tcf_grid = 0;               // fused tensor-core correlation: CTAs (0: not used)
    int nitems = 0, nctr = 0;       // persistent fused launch: work items, counters
    int64_t px = 0, cells = 0, wins = 0;
};

// Execution of a detection batch: one launch per stage, or the persistent
// fused launch (pyramid .. correlation) followed by the suppression launch.
enum { MODE_STAGED = 0, MODE_FUSED = 1 };
// Parts of a batch to enqueue: the per-frame stages up to the candidate keys
// (pyramid .. correlation), the suppression, or both.  hog_detect_host runs
// the front of each chunk of frames as its copy arrives and the back of all
// of them at once.
enum { STAGES_FRONT = 1, STAGES_BACK = 2, STAGES_ALL = 3 };

struct CachedPlan {
    std::vector<uint64_t> sig;              // batch shape: sizes, pitches, pointer alignment, regions
    std::vector<const uint8_t *> fptr;      // the frames' data pointers the plan holds
    std::vector<LevelDesc> hdescs;          // host copy of its level descriptors (rebasing)
    PlanInfo info;
    char *d = nullptr;
    size_t cap = 0;
    uint64_t used = 0;
    int runs = 0;                           // eager runs so far (graphs are captured after one)
    cudaGraphExec_t graph[2][4] = {};       // per mode and stage set (STAGES_*)
};
}  // namespace

struct hog_ctx {
    hog_params p;
    int nf = 0, nfk = 0;
    float *d_w = nullptr;   // [4][nfk][10][10][8]
    Geometry maxg;
    size_t pyr_slot = 0, hist_slot = 0, feat_slot = 0, pos_slot = 0;
    uint8_t *d_pyr = nullptr;
    float *d_hist = nullptr, *d_feat = nullptr;
    uint64_t *d_keys = nullptr;
    uint32_t *d_nmsws = nullptr;    // suppression workspace, HOG_NMS_WS_WORDS per position
    uint8_t *d_nmscand = nullptr;   // suppression: candidate flag per position
    hog_det *d_dets = nullptr;
    int32_t *d_counts = nullptr;
    int *d_flags = nullptr;
    char *h_plan = nullptr, *d_plan = nullptr;
    size_t plan_cap = 0;
    hog_det *h_dets = nullptr;      // pinned, mapped
    int32_t *h_counts = nullptr;    // pinned, mapped
    hog_det *m_dets = nullptr;      // device view of h_dets
    int32_t *m_counts = nullptr;    // device view of h_counts
    int *h_flags = nullptr;         // pinned
    uint8_t *h_stage = nullptr, *d_stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t plan_done = nullptr;
    // stage timing
    bool prof = false, prof_pending = false;
    unsigned prof_mask = 0;         // stages whose events the last profiled batch recorded
    cudaEvent_t prof_ev[2 * HOG_NSTAGES] = {};
    hog_stage_stat stats[HOG_NSTAGES] = {};
    std::vector<Geometry *> geoms;
    std::vector<CachedPlan> plans;
    uint64_t plan_clock = 0;
    // persistent fused launch and graphs
    int *d_fctr = nullptr;          // completion counters + ticket + abort flag
    size_t fctr_cap = 0;            // ints
    int num_sms = 0, fused_grid = 0;
    int batched_mode = MODE_FUSED;  // chosen by the autotuner
    int corr_policy = 0;            // 0: least padding; 1 + s: prefer warp-tile shape s
    int nms_cluster = 0;            // 0: automatic; 1: one CTA per frame; 2..16: cluster size
    long long wait_polls = FUSED_DEFAULT_POLLS;   // fused launch: polls before a wait gives up
    int wait_withhold = 0;          // 1: each new fused plan withholds one completion (tests)
    // correlation engine: 0 FP32 CUDA cores (k_corr.cu); tensor cores
    // (k_corr_tc.cu): 1 GEMM and reduction fused, 2 two passes through G
    int corr_engine = 0;
    std::vector<float> w_host;      // the filters as given, [F][10][10][31]
    float w_absmax = 0.0f;          // largest |w| of the filters
    float *d_wuser = nullptr;       // device copy of w_host
    uint16_t *d_wtc = nullptr;      // tensor-core B planes (hi, lo)
    uint16_t *d_fh = nullptr;       // per slot: fp16 feature planes hi, lo [cells][32]
    float *d_gm = nullptr;          // per slot: row-shift matrices [10 F][cells] per level
    size_t cells_slot = 0, fh_slot = 0, gm_slot = 0;
    int plan_cache_max = 16;        // cached batch plans (a server raises it)
    cudaStream_t cap_stream = nullptr;
    NmsStreams nms_par = {};        // suppression classes side by side (created at hog_create)
    // hog_detect_host: copy stream and events of the double-buffered staging
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_done[2] = {nullptr, nullptr}, stage_free = nullptr;
    cudaEvent_t front_done[2] = {nullptr, nullptr};   // a chunk's front stages, per staging half
    // training arena (hog_backward), grown on demand
    char *d_train = nullptr;
    size_t train_cap = 0;
    std::string err;
};

namespace {

int fail(hog_ctx *ctx, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(hog_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_create_error = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((ctx), HOG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

int check_params(const hog_params *p, std::string &why) {
    if (!p) { why = "params is NULL"; return HOG_EINVAL; }
    if (p->cell != CELL || p->win_cells_w != WIN || p->win_cells_h != WIN) {
        why = "cell must be 8 and the window 10x10 cells"; return HOG_EINVAL;
    }
    if (p->scale_num != 5 || p->scale_den != 6) { why = "scale must be 5/6"; return HOG_EINVAL; }
    if (p->min_size < CELL * WIN) { why = "min_size must be >= 80"; return HOG_EINVAL; }
    if (p->skip_levels < 0) { why = "skip_levels < 0"; return HOG_EINVAL; }
    if (!(p->eps > 0.0f) || !(p->trunc > 0.0f)) { why = "eps and trunc must be > 0"; return HOG_EINVAL; }
    if (!(p->nms_iou >= 0.45f && p->nms_iou < 1.0f)) { why = "nms_iou must be in [0.45, 1)"; return HOG_EINVAL; }
    if (!std::isfinite(p->threshold)) { why = "threshold must be finite"; return HOG_EINVAL; }
    if (p->max_w < p->min_size || p->max_h < p->min_size || p->max_w > 16384 || p->max_h > 16384) {
        why = "max_w/max_h out of range"; return HOG_EINVAL;
    }
    if (p->max_batch < 1 || p->max_batch > 4096) { why = "max_batch out of range"; return HOG_EINVAL; }
    if (p->max_dets_per_frame < 1) { why = "max_dets_per_frame < 1"; return HOG_EINVAL; }
    if (p->float_pyramid != 0) { why = "float_pyramid is only used by hog_backward"; return HOG_EINVAL; }
    if (p->direct_first != 0 && p->direct_first != 1) { why = "direct_first must be 0 or 1"; return HOG_EINVAL; }
    if (p->direct_first && p->skip_levels > 8) { why = "direct_first needs skip_levels <= 8"; return HOG_EINVAL; }
    return HOG_OK;
}

int upload_filters(hog_ctx *ctx, const float *filters, int n) {
    if (!filters || n < 1 || n > HOG_MAX_FILTERS)
        return fail(ctx, HOG_EINVAL, "need 1..%d filters", HOG_MAX_FILTERS);
    // the weights of a linear filter may have any finite scale; the tensor
    // engines store 64 w as fp16, finite only while |w| <= HOG_TC_MAX_WEIGHT
    float amax = 0.0f;
    for (size_t k = 0; k < (size_t)n * WIN * WIN * NFEAT; k++) {
        if (!std::isfinite(filters[k]))
            return fail(ctx, HOG_EINVAL, "filter %d weight %zu is not finite", (int)(k / (WIN * WIN * NFEAT)),
                        k % (WIN * WIN * NFEAT));
        amax = std::max(amax, std::fabs(filters[k]));
    }
    const int nfk = n == 1 ? 1 : (n <= 5 ? 5 : 8);
    if (ctx->d_w && nfk != ctx->nfk) {
        cudaFree(ctx->d_w);
        ctx->d_w = nullptr;
    }
    std::vector<float> wc((size_t)NCHUNK * nfk * WIN * WIN * CHUNK, 0.0f);
    for (int f = 0; f < n; f++)
        for (int a = 0; a < WIN; a++)
            for (int b = 0; b < WIN; b++)
                for (int c = 0; c < NFEAT; c++) {
                    const int ch = c / CHUNK, cc = c % CHUNK;
                    wc[((((size_t)ch * nfk + f) * WIN + a) * WIN + b) * CHUNK + cc] =
                        filters[(((size_t)f * WIN + a) * WIN + b) * NFEAT + c];
                }
    if (!ctx->d_w) CUDA_TRY(ctx, cudaMalloc(&ctx->d_w, wc.size() * sizeof(float)));
    CUDA_TRY(ctx, cudaMemcpy(ctx->d_w, wc.data(), wc.size() * sizeof(float), cudaMemcpyHostToDevice));
    ctx->nf = n;
    ctx->nfk = nfk;
    ctx->w_host.assign(filters, filters + (size_t)n * WIN * WIN * NFEAT);
    ctx->w_absmax = amax;
    return HOG_OK;
}

// Whether the tensor engines can represent the current filters.
bool tc_range_ok(const hog_ctx *ctx) { return ctx->w_absmax <= HOG_TC_MAX_WEIGHT; }

// Arenas and B planes of the tensor-core correlation (allocated when the
// engine is first selected; rebuilt after a filter change).
int prepare_tc(hog_ctx *ctx, bool need_g) {
    if (!tc_range_ok(ctx))
        return fail(ctx, HOG_EINVAL,
                    "filter weight |w| = %g exceeds %g, the tensor engines' fp16 range (64 |w| <= 65504); "
                    "use the CUDA-core engine 0", (double)ctx->w_absmax, (double)HOG_TC_MAX_WEIGHT);
    auto F = [](void *p) { if (p) cudaFree(p); };
    F(ctx->d_wuser); F(ctx->d_wtc); F(ctx->d_gm);
    ctx->d_wuser = nullptr; ctx->d_wtc = nullptr; ctx->d_gm = nullptr;
    const size_t B = (size_t)ctx->p.max_batch;
    ctx->cells_slot = ctx->feat_slot / 32;
    ctx->fh_slot = align_up(ctx->cells_slot * 64, 128);                  // halves
    ctx->gm_slot = align_up(ctx->cells_slot * WIN * (size_t)ctx->nfk, 64);   // floats
    if (!ctx->d_fh) CUDA_TRY(ctx, cudaMalloc(&ctx->d_fh, B * ctx->fh_slot * sizeof(uint16_t)));
    if (need_g) CUDA_TRY(ctx, cudaMalloc(&ctx->d_gm, B * ctx->gm_slot * sizeof(float)));
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_wuser, ctx->w_host.size() * sizeof(float)));
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_wtc, corr_tc_weights_halves(ctx->nfk) * sizeof(uint16_t)));
    CUDA_TRY(ctx, cudaMemcpy(ctx->d_wuser, ctx->w_host.data(), ctx->w_host.size() * sizeof(float),
                             cudaMemcpyHostToDevice));
    CUDA_TRY(ctx, launch_corr_tc_weights(ctx->d_wuser, ctx->nfk, ctx->nf, ctx->d_wtc, nullptr));
    CUDA_TRY(ctx, cudaDeviceSynchronize());
    return HOG_OK;
}

void free_ctx(hog_ctx *ctx) {
    if (!ctx) return;
    auto F = [](void *p) { if (p) cudaFree(p); };
    auto FH = [](void *p) { if (p) cudaFreeHost(p); };
    F(ctx->d_w); F(ctx->d_pyr); F(ctx->d_hist); F(ctx->d_feat); F(ctx->d_keys);
    F(ctx->d_nmsws); F(ctx->d_nmscand); F(ctx->d_dets); F(ctx->d_counts); F(ctx->d_flags); F(ctx->d_plan);
    F(ctx->d_stage);
    FH(ctx->h_plan); FH(ctx->h_dets); FH(ctx->h_counts); FH(ctx->h_flags); FH(ctx->h_stage);
    if (ctx->plan_done) cudaEventDestroy(ctx->plan_done);
    for (cudaEvent_t e : ctx->prof_ev)
        if (e) cudaEventDestroy(e);
    for (auto &cp : ctx->plans) {
        F(cp.d);
        for (auto &gm : cp.graph)
            for (auto &g : gm) if (g) cudaGraphExecDestroy(g);
    }
    F(ctx->d_fctr);
    F(ctx->d_train);
    F(ctx->d_wuser); F(ctx->d_wtc); F(ctx->d_fh); F(ctx->d_gm);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaStream_t q : ctx->nms_par.side)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t q : ctx->nms_par.join)
        if (q) cudaEventDestroy(q);
    if (ctx->nms_par.fork) cudaEventDestroy(ctx->nms_par.fork);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t e : ctx->copy_done)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->front_done)
        if (e) cudaEventDestroy(e);
    if (ctx->stage_free) cudaEventDestroy(ctx->stage_free);
    for (Geometry *g : ctx->geoms) {
        F(g->d_nbr);
        F(g->d_nbr_t);
        F(g->d_cnt);
        delete g;
    }
    delete ctx;
}

// Geometry of a frame size, with its suppression neighbour table (built on
// the device, on `stream`, the first time the size is seen).
int get_geometry(hog_ctx *ctx, int W, int H, cudaStream_t stream, Geometry **out) {
    for (Geometry *g : ctx->geoms)
        if (g->W == W && g->H == H) { *out = g; return HOG_OK; }
    if (ctx->geoms.size() >= 64)
        return fail(ctx, HOG_EINVAL, "more than 64 distinct frame sizes in one context");
    Geometry *g = new (std::nothrow) Geometry();
    if (!g) return fail(ctx, HOG_ENOMEM, "host allocation failed");
    int rc = compute_geometry(ctx->p, W, H, *g);
    if (rc) { delete g; return fail(ctx, rc, "frame %dx%d has more than %d levels", W, H, MAX_LEVELS); }
    if (g->npos > 0) {
        cudaError_t e1 = cudaMalloc(&g->d_nbr, (size_t)g->npos * MAXN * sizeof(int32_t));
        cudaError_t e2 = cudaMalloc(&g->d_cnt, (size_t)g->npos);
        cudaError_t e3 = cudaMalloc(&g->d_nbr_t, (size_t)g->npos * MAXN * sizeof(int32_t));
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            cudaFree(g->d_nbr);
            cudaFree(g->d_nbr_t);
            cudaFree(g->d_cnt);
            delete g;
            return fail(ctx, HOG_ENOMEM, "neighbour table allocation failed");
        }
        GeomDesc gd;
        std::memset(&gd, 0, sizeof gd);
        gd.W = W; gd.H = H; gd.nlev = g->nlev; gd.npos = g->npos;
        gd.iou = (double)ctx->p.nms_iou;
        for (int l = 0; l < g->nlev; l++) {
            gd.lev_w[l] = g->lw[l]; gd.lev_h[l] = g->lh[l];
            gd.lev_rx[l] = (double)W / (double)g->lw[l];
            gd.lev_ry[l] = (double)H / (double)g->lh[l];
            gd.lev_nu[l] = g->nu[l]; gd.lev_nv[l] = g->nv[l];
            gd.lev_pos[l] = g->pos_off[l];
        }
        gd.lev_pos[g->nlev] = g->npos;
        // levels l, m can only exceed the IoU threshold if area ratio allows it
        for (int l = 0; l < g->nlev; l++) {
            const double al = (80.0 * W / g->lw[l]) * (80.0 * H / g->lh[l]);
            for (int m = 0; m < g->nlev; m++) {
                const double am = (80.0 * W / g->lw[m]) * (80.0 * H / g->lh[m]);
                const double bound = std::min(al, am) / std::max(al, am);
                if (bound > gd.iou - 1e-12) gd.pair_mask[l] |= 1u << m;
            }
        }
        *ctx->h_flags = 0;
        cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), stream);
        // slots past a position's count read -1 (the list's end)
        cudaMemsetAsync(g->d_nbr, 0xff, (size_t)g->npos * MAXN * sizeof(int32_t), stream);
        cudaMemsetAsync(g->d_nbr_t, 0xff, (size_t)g->npos * MAXN * sizeof(int32_t), stream);
        cudaError_t e = launch_nms_geometry(gd, g->d_nbr, g->d_nbr_t, g->d_cnt, ctx->d_flags, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(int),
                                                  cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            cudaFree(g->d_nbr); cudaFree(g->d_nbr_t); cudaFree(g->d_cnt); delete g;
            return fail(ctx, HOG_ECUDA, "suppression geometry: %s", cudaGetErrorString(e));
        }
        if (*ctx->h_flags) {
            cudaFree(g->d_nbr); cudaFree(g->d_nbr_t); cudaFree(g->d_cnt); delete g;
            return fail(ctx, HOG_EINVAL, "nms_iou %.3f gives more than %d overlapping windows",
                        (double)ctx->p.nms_iou, MAXN);
        }
    }
    ctx->geoms.push_back(g);
    *out = g;
    return HOG_OK;
}

// ---- plans ---------------------------------------------------------------

// Direct-to-size pyramids (hog_params.direct_first, skip_levels = s >= 2):
// level s is resampled straight from the frame, levels 1..s-1 do not exist.
bool level_absent(const hog_params &p, int l) {
    return p.direct_first && p.skip_levels >= 2 && l >= 1 && l < p.skip_levels;
}

struct PlanBuilder {
    std::vector<LevelDesc> descs;
    std::vector<FrameDesc> frames;
    std::vector<std::vector<Job>> pyr;   // per step (target level)
    std::vector<Job> pyrd;               // direct-to-size levels (read the frame)
    std::vector<Job> hist, feat, corr;
    std::vector<Job> corrf;              // correlation jobs of the fused launch (8x16, 16x8 tiles)
    std::vector<Job> tc, tcr;            // tensor-core correlation: 128-cell tiles, 256-window blocks
    struct TcRect { int desc, u0, u1, v0, v1; };
    std::vector<TcRect> tcf_rects;       // fused tensor-core correlation: window rectangles to band
    std::vector<TcBand> bands;           // ... their bands, in per-CTA order
    std::vector<int32_t> cta_first;      // ... CTA k runs bands [cta_first[k], cta_first[k+1])
    std::vector<FusedItem> items;        // persistent fused launch (built on demand)
    int nctr = 0;
};

// Work items of the persistent fused launch, in dependency-depth order:
// pyramid level l at depth l, its histograms at l+1, features at l+2,
// correlation at l+3; counters ctr[3 d + stage] count finished tiles of
// level descriptor d (stage 0 pyramid, 1 histograms, 2 features).
void build_fused_items(PlanBuilder &pb) {
    const int nd = (int)pb.descs.size();
    std::vector<int> npyr(nd, 0), nhist(nd, 0), nfeat(nd, 0);
    // every pyramid job: the 5/6 steps and the direct-to-size levels
    std::vector<const std::vector<Job> *> pyr_lists;
    for (const auto &seg : pb.pyr) pyr_lists.push_back(&seg);
    pyr_lists.push_back(&pb.pyrd);
    for (const auto *seg : pyr_lists)
        for (const Job &j : *seg) npyr[j.desc]++;
    for (const Job &j : pb.hist) nhist[j.desc]++;
    for (const Job &j : pb.feat) nfeat[j.desc]++;
    struct Keyed { int depth, kind, desc, tile; FusedItem it; };
    std::vector<Keyed> v;
    v.reserve(pb.hist.size() + pb.feat.size() + pb.corrf.size() / 4 + 1024);
    for (const auto *seg : pyr_lists)
        for (const Job &j : *seg) {
            const LevelDesc &d = pb.descs[j.desc];
            FusedItem it{FUSED_PYR, j.desc, j.tile, -1, 0, 3 * j.desc + 0};
            // a 5/6 step waits for the previous level; a direct level reads the frame
            if (d.level >= 2 && d.dpow < 2) { it.wait = 3 * (j.desc - 1) + 0; it.target = npyr[j.desc - 1]; }
            v.push_back({d.level, FUSED_PYR, j.desc, j.tile, it});
        }
    for (const Job &j : pb.hist) {
        const LevelDesc &d = pb.descs[j.desc];
        FusedItem it{FUSED_HIST, j.desc, j.tile, -1, 0, 3 * j.desc + 1};
        if (d.level >= 1) { it.wait = 3 * j.desc + 0; it.target = npyr[j.desc]; }
        v.push_back({d.level + 1, FUSED_HIST, j.desc, j.tile, it});
    }
    for (const Job &j : pb.feat) {
        const LevelDesc &d = pb.descs[j.desc];
        FusedItem it{FUSED_FEAT, j.desc, j.tile, 3 * j.desc + 1, nhist[j.desc], 3 * j.desc + 2};
        v.push_back({d.level + 2, FUSED_FEAT, j.desc, j.tile, it});
    }
    for (size_t k = 0; k < pb.corrf.size();) {
        const int desc = pb.corrf[k].desc;
        size_t e = k;
        while (e < pb.corrf.size() && pb.corrf[e].desc == desc && e - k < 8) e++;
        const LevelDesc &d = pb.descs[desc];
        FusedItem it{FUSED_CORR, (int)k, (int)(e - k), 3 * desc + 2, nfeat[desc], -1};
        v.push_back({d.level + 3, FUSED_CORR, desc, (int)k, it});
        k = e;
    }
    std::stable_sort(v.begin(), v.end(), [](const Keyed &a, const Keyed &b) {
        if (a.depth != b.depth) return a.depth < b.depth;
        if (a.kind != b.kind) return a.kind < b.kind;
        if (a.desc != b.desc) return a.desc < b.desc;
        return a.tile < b.tile;
    });
    pb.items.clear();
    for (const Keyed &k : v) pb.items.push_back(k.it);
    pb.nctr = 3 * nd;
}



// Per-frame options for plan building.
struct FrameOpts {
    float *feat_user = nullptr;     // [cy][cx][31] per level, at geometry ufeat offsets
    float *scores_user = nullptr;   // [F][nu][nv] per level
    const size_t *score_off = nullptr;
    bool corr = true, nms = true, feat = true;
    const hog_roi *roi = nullptr;   // detection restricted to a region of interest
};

// Window rectangles [u0, u1) x [v0, v1) per level that a region of interest
// scans (empty where none): level in [max(lmin, skip_levels), lmax], window
// centre fl((8v + 40) fl(W/Wl)), fl((8u + 40) fl(H/Hl)) in [x0, x1) x
// [y0, y1) -- the centre grows with v and u, so the scanned windows of a
// level are a rectangle.
void roi_rects(const hog_params &p, const Geometry &g, const hog_roi &r, int *u0, int *u1, int *v0,
               int *v1) {
    for (int l = 0; l < g.nlev; l++) {
        u0[l] = u1[l] = v0[l] = v1[l] = 0;
        if (l < r.lmin || l > r.lmax || l < p.skip_levels || g.nu[l] <= 0 || g.nv[l] <= 0) continue;
        const double rx = (double)g.W / (double)g.lw[l], ry = (double)g.H / (double)g.lh[l];
        int a = 0, b = 0;
        while (a < g.nv[l] && (double)(CELL * a + CELL * WIN / 2) * rx < r.x0) a++;
        b = a;
        while (b < g.nv[l] && (double)(CELL * b + CELL * WIN / 2) * rx < r.x1) b++;
        int c = 0, e = 0;
        while (c < g.nu[l] && (double)(CELL * c + CELL * WIN / 2) * ry < r.y0) c++;
        e = c;
        while (e < g.nu[l] && (double)(CELL * e + CELL * WIN / 2) * ry < r.y1) e++;
        if (a < b && c < e) { v0[l] = a; v1[l] = b; u0[l] = c; u1[l] = e; }
    }
}

// Tiles of a tw x th cell tiling of a cx-wide level that meet the cell
// rectangle [r0, r1) x [c0, c1).
template <typename F>
void tiles_meeting(int cx, int cy, int tw, int th, int r0, int r1, int c0, int c1, F emit) {
    const int ntx = (cx + tw - 1) / tw;
    r0 = std::max(r0, 0); c0 = std::max(c0, 0); r1 = std::min(r1, cy); c1 = std::min(c1, cx);
    if (r0 >= r1 || c0 >= c1) return;
    for (int ty = r0 / th; ty <= (r1 - 1) / th; ty++)
        for (int tx = c0 / tw; tx <= (c1 - 1) / tw; tx++) emit(ty * ntx + tx);
}

void add_frame(hog_ctx *ctx, PlanBuilder &pb, const Geometry &g, const hog_frame &f, int slot,
               int frame_index, const FrameOpts &o) {
    uint8_t *pyr = ctx->d_pyr + (size_t)slot * ctx->pyr_slot;
    float *hist = ctx->d_hist + (size_t)slot * ctx->hist_slot;
    float *feat = ctx->d_feat + (size_t)slot * ctx->feat_slot;
    uint64_t *keys = ctx->d_keys + (size_t)slot * ctx->pos_slot;
    const bool tc = ctx->corr_engine >= 1;
    uint16_t *fh = tc ? ctx->d_fh + (size_t)slot * ctx->fh_slot : nullptr;
    float *gm = ctx->corr_engine == 2 ? ctx->d_gm + (size_t)slot * ctx->gm_slot : nullptr;
    size_t cell_off = 0;
    const int first = (int)pb.descs.size();
    // region of interest: scanned window rectangles, and the last level any
    // of them needs (no pyramid, histograms or features above it)
    int ru0[MAX_LEVELS], ru1[MAX_LEVELS], rv0[MAX_LEVELS], rv1[MAX_LEVELS];
    int lneed = g.nlev - 1;
    if (o.roi) {
        roi_rects(ctx->p, g, *o.roi, ru0, ru1, rv0, rv1);
        lneed = -1;
        for (int l = 0; l < g.nlev; l++)
            if (ru0[l] < ru1[l]) lneed = l;
    }
    for (int l = 0; l < g.nlev; l++) {
        LevelDesc d;
        std::memset(&d, 0, sizeof d);
        d.w = g.lw[l]; d.h = g.lh[l];
        d.cx = g.cx[l]; d.cy = g.cy[l]; d.nu = g.nu[l]; d.nv = g.nv[l];
        d.hist_bw = g.hbw[l];
        d.frame = frame_index; d.level = l;
        d.scan = l >= ctx->p.skip_levels ? 1 : 0;
        if (o.roi) d.scan = ru0[l] < ru1[l] ? 1 : 0;
        d.pos_off = g.pos_off[l];
        const bool absent = level_absent(ctx->p, l) || l > lneed;
        if (l == 0) {
            d.img = f.data;
            d.pitch = f.pitch;
        } else {
            d.dst = pyr + g.pyr_off[l];
            d.img = d.dst;
            d.pitch = g.pitch[l];
            // a direct-to-size level reads the frame, a 5/6 step the previous level
            const bool direct = ctx->p.direct_first && ctx->p.skip_levels >= 2 && l == ctx->p.skip_levels;
            const LevelDesc &prev = pb.descs[direct ? first : first + l - 1];
            d.src = prev.img;
            d.sw = prev.w; d.sh = prev.h; d.spitch = prev.pitch;
            d.dpow = direct ? l : 0;
        }
        d.hist = hist + g.hist_off[l];
        // the FP32 feature layout feeds the CUDA-core correlation only
        d.feat = tc ? nullptr : feat + g.feat_off[l];
        d.feat_user = o.feat_user ? o.feat_user + g.ufeat_off[l] : nullptr;
        d.scores_user = o.scores_user ? o.scores_user + o.score_off[l] : nullptr;
        d.keys = keys + g.pos_off[l];
        pb.descs.push_back(d);
        const int di = first + l;
        if (l >= 1 && !absent) {
            if ((int)pb.pyr.size() < l + 1) pb.pyr.resize(l + 1);
            const int nt = ((d.w + PYR_TX - 1) / PYR_TX) * ((d.h + PYR_TY - 1) / PYR_TY);
            auto &list = d.dpow >= 2 ? pb.pyrd : pb.pyr[l];
            for (int k = 0; k < nt; k++) list.push_back({di, k});
        }
        // histograms and features: for scanned levels, and for every level
        // whose features or scores the caller asked for (not for levels a
        // direct-to-size pyramid leaves out)
        const bool want = d.scan || o.feat_user || o.scores_user;
        if (o.feat && want && !absent && o.roi) {
            // only the cells the scanned windows read: features of cell rows
            // [u0, u1 + 9) x cols [v0, v1 + 9), histograms one cell wider
            tiles_meeting(d.cx, d.cy, d.hist_bw - 1, hist_bh(d.hist_bw) - 1, ru0[l] - 1,
                          ru1[l] + WIN, rv0[l] - 1, rv1[l] + WIN,
                          [&](int k) { pb.hist.push_back({di, k}); });
            tiles_meeting(d.cx, d.cy, FEAT_TX, FEAT_TY, ru0[l], ru1[l] + WIN - 1, rv0[l],
                          rv1[l] + WIN - 1, [&](int k) { pb.feat.push_back({di, k}); });
        } else if (o.feat && want && !absent) {
            const int nh = hist_ntiles(d.cx, d.cy, d.hist_bw);
            for (int k = 0; k < nh; k++) pb.hist.push_back({di, k});
            const int nfj = ((d.cx + FEAT_TX - 1) / FEAT_TX) * ((d.cy + FEAT_TY - 1) / FEAT_TY);
            for (int k = 0; k < nfj; k++) pb.feat.push_back({di, k});
        }
        if (o.corr && d.nu > 0 && d.nv > 0 && (d.scan || o.scores_user) && !absent) {
            // warp-tile shape: the one that pads this level's window grid
            // least, or the autotuner's preferred shape
            int best = 0, best_slots = 0, best_n = 0;
            for (int sh = 0; sh < CORR_NSHAPE; sh++) {
                if (!corr_shape_ok(sh)) continue;
                const int n = ((d.nu + corr_tu(sh) - 1) / corr_tu(sh)) *
                              ((d.nv + corr_tv(sh) - 1) / corr_tv(sh));
                if (sh == 0 || n * 128 < best_slots) { best = sh; best_slots = n * 128; best_n = n; }
            }
            const int pref = ctx->corr_policy - 1;
            if (pref >= 0 && pref < CORR_NSHAPE && corr_shape_ok(pref)) {
                best = pref;
                best_n = ((d.nu + corr_tu(pref) - 1) / corr_tu(pref)) *
                         ((d.nv + corr_tv(pref) - 1) / corr_tv(pref));
            }
            if (tc) {
                // tensor cores: the level's fp16 planes and row-shift matrix
                const size_t nc = (size_t)d.cx * d.cy;
                pb.descs.back().feat_hi = fh + cell_off * 32;
                pb.descs.back().feat_lo = fh + (ctx->cells_slot + cell_off) * 32;
                if (ctx->corr_engine == 2) {
                    pb.descs.back().gmat = gm + cell_off * WIN * ctx->nfk;
                    const int nt = (int)((nc + 127) / 128), nr = (d.nu * d.nv + 255) / 256;
                    for (int k = 0; k < nt; k++) pb.tc.push_back({di, k});
                    for (int k = 0; k < nr; k++) pb.tcr.push_back({di, k});
                } else if (o.roi) {
                    pb.tcf_rects.push_back({di, ru0[l], ru1[l], rv0[l], rv1[l]});
                } else {
                    pb.tcf_rects.push_back({di, 0, d.nu, 0, d.nv});
                }
            } else {
                for (int k = 0; k < best_n; k++) pb.corr.push_back({di, (best << 28) | k});
            }
            // the fused launch stages at most 17x25 cells per warp: 8x16 or
            // 16x8 tiles, the preferred one if it is one of them (with the
            // tensor-core engine the fused launch stops after the features
            // and the GEMM above follows it)
            int fb = -1, fb_n = 0;
            for (int sh = 0; sh < CORR_NSHAPE; sh++) {
                if (!corr_shape_fused(sh)) continue;
                const int n = ((d.nu + corr_tu(sh) - 1) / corr_tu(sh)) *
                              ((d.nv + corr_tv(sh) - 1) / corr_tv(sh));
                if (fb < 0 || n < fb_n || sh == pref) { fb = sh; fb_n = n; }
                if (sh == pref) break;
            }
            if (!tc)
                for (int k = 0; k < fb_n; k++) pb.corrf.push_back({di, (fb << 28) | k});
        }
        cell_off += (size_t)d.cx * d.cy;
    }
    if (o.nms) {
        FrameDesc fd;
        std::memset(&fd, 0, sizeof fd);
        fd.W = g.W; fd.H = g.H; fd.nlev = g.nlev; fd.npos = g.npos;
        fd.frame = frame_index;
        fd.scan_from = g.pos_off[std::min(std::max(ctx->p.skip_levels, 0), g.nlev)];
        if (o.roi) {
            fd.has_roi = 1;
            for (int l = 0; l < g.nlev; l++) {
                fd.roi_u0[l] = ru0[l]; fd.roi_u1[l] = ru1[l];
                fd.roi_v0[l] = rv0[l]; fd.roi_v1[l] = rv1[l];
            }
        }
        for (int l = 0; l < g.nlev; l++) {
            fd.lev_w[l] = g.lw[l]; fd.lev_h[l] = g.lh[l];
            fd.lev_rx[l] = (double)g.W / (double)g.lw[l];
            fd.lev_ry[l] = (double)g.H / (double)g.lh[l];
            fd.lev_nu[l] = g.nu[l]; fd.lev_nv[l] = g.nv[l];
            fd.lev_pos[l] = g.pos_off[l];
        }
        fd.lev_pos[g.nlev] = g.npos;
        fd.keys = keys;
        fd.ws = ctx->d_nmsws + (size_t)slot * ctx->pos_slot * HOG_NMS_WS_WORDS;
        fd.cand = ctx->d_nmscand + (size_t)slot * ctx->pos_slot;
        fd.nbr = g.d_nbr;
        fd.nbr_t = g.d_nbr_t;
        fd.nbr_cnt = g.d_cnt;
        fd.out = ctx->d_dets + (size_t)slot * ctx->p.max_dets_per_frame;
        fd.out_cap = ctx->p.max_dets_per_frame;
        fd.count = ctx->d_counts + slot;
        pb.frames.push_back(fd);
    }
}



// Bands of the fused tensor-core correlation and their assignment to CTAs
// (one CTA per SM).  A band's cost is its number of 128-cell tiles; each
// extra band of a level re-reads 9 cell rows.  The band height is chosen
// to minimise the estimated makespan max(largest band, total / CTAs) (a
// large batch keeps whole levels, a single frame splits its big levels),
// then bands go to CTAs longest first, each to the least loaded CTA.
void build_tc_bands(PlanBuilder &pb, int num_sms) {
    pb.bands.clear();
    pb.cta_first.clear();
    if (pb.tcf_rects.empty()) return;
    // strips: window rows [ub, ub + nu), columns [c0, c0 + nvs); P cells per
    // staged row (the level's width when the strip spans every column)
    struct Strip { int desc, ub, nu, c0, nvs, P; };
    std::vector<Strip> strips;
    for (const auto &r : pb.tcf_rects) {
        const LevelDesc &d = pb.descs[r.desc];
        const int nv = r.v1 - r.v0, nu = r.u1 - r.u0;
        if (nv <= 0 || nu <= 0) continue;
        const int S = (nv + (TCF_PMAX - WIN)) / (TCF_PMAX - WIN + 1);   // ceil(nv / (PMAX - 9))
        int c0 = r.v0;
        for (int k = 0; k < S; k++) {
            const int nvs = nv / S + (k < nv % S ? 1 : 0);
            const bool full = r.v0 == 0 && nvs == d.nv;
            strips.push_back({r.desc, r.u0, nu, c0, nvs, full ? d.cx : nvs + WIN - 1});
            c0 += nvs;
        }
    }
    if (strips.empty()) return;
    // window rows per band for a tile budget M (at least one row)
    auto rows_for = [](const Strip &st, long M) {
        const long h = M * 128 / st.P - (WIN - 1);
        return (int)std::max(1L, std::min((long)st.nu, h));
    };
    const long cand[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 1L << 30};
    constexpr int NC = (int)(sizeof cand / sizeof cand[0]);
    long span[NC], total[NC], best_span = -1;
    for (int k = 0; k < NC; k++) {
        long tot = 0, maxt = 0;
        for (const Strip &st : strips) {
            const int h0 = rows_for(st, cand[k]);
            const int nb = (st.nu + h0 - 1) / h0;
            const int h = (st.nu + nb - 1) / nb;
            const long t = tcf_tiles(0, h, st.P);
            tot += (long)nb * t;
            maxt = std::max(maxt, t);
        }
        span[k] = std::max(maxt, (tot + num_sms - 1) / num_sms);
        total[k] = tot;
        if (best_span < 0 || span[k] < best_span) best_span = span[k];
    }
    // among budgets within ~15 % of the best makespan, the least total work
    // (re-read rows cost HBM traffic and energy for little latency)
    long best_M = cand[NC - 1], best_tot = -1;
    for (int k = 0; k < NC; k++)
        if (span[k] * 20 <= best_span * 23 + 20 && (best_tot < 0 || total[k] < best_tot)) {
            best_tot = total[k];
            best_M = cand[k];
        }
    std::vector<TcBand> all;
    std::vector<long> cost;
    for (const Strip &st : strips) {
        const int h0 = rows_for(st, best_M);
        const int nb = (st.nu + h0 - 1) / h0;
        for (int k = 0; k < nb; k++) {
            const int u0 = st.ub + (int)((long)st.nu * k / nb);
            const int u1 = st.ub + (int)((long)st.nu * (k + 1) / nb);
            all.push_back({st.desc, u0, u1, st.c0, st.P, st.nvs});
            cost.push_back(tcf_tiles(u0, u1, st.P));
        }
    }
    std::vector<int> order(all.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    const int grid = (int)std::min<size_t>(all.size(), (size_t)num_sms);
    std::vector<long> load(grid, 0);
    std::vector<std::vector<int>> per(grid);
    for (int i : order) {
        int c = 0;
        for (int k = 1; k < grid; k++)
            if (load[k] < load[c]) c = k;
        load[c] += cost[i];
        per[c].push_back(i);
    }
    pb.cta_first.push_back(0);
    for (int c = 0; c < grid; c++) {
        for (int i : per[c]) pb.bands.push_back(all[i]);
        pb.cta_first.push_back((int32_t)pb.bands.size());
    }
}

// The suppression launches take a batch's frames by workspace class, so the
// plan holds them sorted by class (stable: frame order within a class).
void sort_frames(PlanBuilder &pb) {
    std::stable_sort(pb.frames.begin(), pb.frames.end(), [](const FrameDesc &a, const FrameDesc &b) {
        return nms_ws_class(a.npos) < nms_ws_class(b.npos);
    });
}

void layout_plan(const PlanBuilder &pb, int nf, PlanInfo &info) {
    PlanLayout &L = info.L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.descs = take(pb.descs.size() * sizeof(LevelDesc));
    L.frames = take(pb.frames.size() * sizeof(FrameDesc));
    L.pyr.resize(pb.pyr.size());
    L.npyr.resize(pb.pyr.size());
    for (size_t s = 0; s < pb.pyr.size(); s++) {
        L.pyr[s] = take(pb.pyr[s].size() * sizeof(Job));
        L.npyr[s] = (int)pb.pyr[s].size();
    }
    L.pyrd = take(pb.pyrd.size() * sizeof(Job));
    L.npyrd = (int)pb.pyrd.size();
    L.hist = take(pb.hist.size() * sizeof(Job));
    L.feat = take(pb.feat.size() * sizeof(Job));
    L.corr = take(pb.corr.size() * sizeof(Job));
    L.corrf = take(pb.corrf.size() * sizeof(Job));
    L.tc = take(pb.tc.size() * sizeof(Job));
    L.tcr = take(pb.tcr.size() * sizeof(Job));
    L.bands = take(pb.bands.size() * sizeof(TcBand));
    L.cta_first = take(pb.cta_first.size() * sizeof(int32_t));
    L.items = take(pb.items.size() * sizeof(FusedItem));
    L.total = off;
    info.nitems = (int)pb.items.size();
    info.nctr = pb.nctr;
    info.nhist = (int)pb.hist.size();
    info.nfeat = (int)pb.feat.size();
    info.ncorr = (int)pb.corr.size();
    info.ntc = (int)pb.tc.size();
    info.ntcr = (int)pb.tcr.size();
    info.tcf_grid = pb.cta_first.empty() ? 0 : (int)pb.cta_first.size() - 1;
    info.nframes = (int)pb.frames.size();
    info.max_npos = 0;
    for (const FrameDesc &f : pb.frames) {
        info.max_npos = std::max(info.max_npos, f.npos);
        const int k = nms_ws_class(f.npos);
        info.ncls[k]++;
        info.cls_npos[k] = std::max(info.cls_npos[k], f.npos);
    }
    info.px = info.cells = info.wins = 0;
    for (const LevelDesc &ld : pb.descs) {
        if (ld.level >= 1) info.px += (int64_t)ld.w * ld.h;
        info.cells += (int64_t)ld.cx * ld.cy;
        if (ld.nu > 0 && ld.nv > 0 && (ld.scan || ld.scores_user)) info.wins += (int64_t)ld.nu * ld.nv;
    }
    info.wins *= nf;
}

int ensure_plan_capacity(hog_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->plan_cap) return HOG_OK;
    size_t cap = align_up(std::max(bytes, ctx->plan_cap * 2), 1 << 16);
    if (ctx->plan_done) cudaEventSynchronize(ctx->plan_done);
    cudaFreeHost(ctx->h_plan);
    cudaFree(ctx->d_plan);
    ctx->h_plan = nullptr;
    ctx->d_plan = nullptr;
    ctx->plan_cap = 0;
    CUDA_TRY(ctx, cudaMallocHost(&ctx->h_plan, cap));
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_plan, cap));
    ctx->plan_cap = cap;
    return HOG_OK;
}

// Fold the elapsed times of the last profiled plan into the stats.
int collect_profile(hog_ctx *ctx) {
    if (!ctx->prof_pending) return HOG_OK;
    for (int k = 0; k < HOG_NSTAGES; k++) {
        if (!((ctx->prof_mask >> k) & 1u)) continue;
        float ms = 0.0f;
        CUDA_TRY(ctx, cudaEventSynchronize(ctx->prof_ev[2 * k + 1]));
        CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]));
        ctx->stats[k].ms += ms;
    }
    ctx->prof_pending = false;
    ctx->prof_mask = 0;
    return HOG_OK;
}

// Serialise pb into the pinned staging buffer and copy it to d_dst
// (capacity >= info.L.total) on `stream`.
int upload_plan(hog_ctx *ctx, const PlanBuilder &pb, const PlanInfo &info, char *d_dst,
                cudaStream_t stream) {
    const PlanLayout &L = info.L;
    int rc = ensure_plan_capacity(ctx, L.total);
    if (rc) return rc;
    CUDA_TRY(ctx, cudaEventSynchronize(ctx->plan_done));   // previous plan copy has finished
    char *h = ctx->h_plan;
    std::memcpy(h + L.descs, pb.descs.data(), pb.descs.size() * sizeof(LevelDesc));
    std::memcpy(h + L.frames, pb.frames.data(), pb.frames.size() * sizeof(FrameDesc));
    for (size_t s = 0; s < pb.pyr.size(); s++)
        std::memcpy(h + L.pyr[s], pb.pyr[s].data(), pb.pyr[s].size() * sizeof(Job));
    std::memcpy(h + L.pyrd, pb.pyrd.data(), pb.pyrd.size() * sizeof(Job));
    std::memcpy(h + L.hist, pb.hist.data(), pb.hist.size() * sizeof(Job));
    std::memcpy(h + L.feat, pb.feat.data(), pb.feat.size() * sizeof(Job));
    std::memcpy(h + L.corr, pb.corr.data(), pb.corr.size() * sizeof(Job));
    std::memcpy(h + L.corrf, pb.corrf.data(), pb.corrf.size() * sizeof(Job));
    std::memcpy(h + L.tc, pb.tc.data(), pb.tc.size() * sizeof(Job));
    std::memcpy(h + L.tcr, pb.tcr.data(), pb.tcr.size() * sizeof(Job));
    std::memcpy(h + L.bands, pb.bands.data(), pb.bands.size() * sizeof(TcBand));
    std::memcpy(h + L.cta_first, pb.cta_first.data(), pb.cta_first.size() * sizeof(int32_t));
    std::memcpy(h + L.items, pb.items.data(), pb.items.size() * sizeof(FusedItem));
    CUDA_TRY(ctx, cudaMemcpyAsync(d_dst ? d_dst : ctx->d_plan, h, L.total, cudaMemcpyHostToDevice,
                                  stream));
    CUDA_TRY(ctx, cudaEventRecord(ctx->plan_done, stream));
    return HOG_OK;
}

// Launch every stage of a plan that is resident at d on `stream`.
int launch_plan(hog_ctx *ctx, const char *d, const PlanInfo &info, cudaStream_t stream,
                int stages = STAGES_ALL) {
    const PlanLayout &L = info.L;
    const LevelDesc *descs = reinterpret_cast<const LevelDesc *>(d + L.descs);
    int rc = collect_profile(ctx);
    if (rc) return rc;
    auto mark = [&](int i) -> cudaError_t {
        return ctx->prof ? cudaEventRecord(ctx->prof_ev[i], stream) : cudaSuccess;
    };
    if (stages & STAGES_FRONT) {
        CUDA_TRY(ctx, mark(0));
        int npyr = 0;
        if (L.npyrd > 0) {
            CUDA_TRY(ctx, launch_pyramid_direct(descs, reinterpret_cast<const Job *>(d + L.pyrd), L.npyrd,
                                                stream));
            npyr++;
        }
        for (size_t s = 1; s < L.pyr.size(); s++) {
            CUDA_TRY(ctx, launch_pyramid(descs, reinterpret_cast<const Job *>(d + L.pyr[s]),
                                         L.npyr[s], stream));
            npyr += L.npyr[s] > 0;
        }
        CUDA_TRY(ctx, mark(1));
        CUDA_TRY(ctx, mark(2));
        CUDA_TRY(ctx, launch_hist(descs, reinterpret_cast<const Job *>(d + L.hist), info.nhist, stream));
        CUDA_TRY(ctx, mark(3));
        CUDA_TRY(ctx, mark(4));
        CUDA_TRY(ctx, launch_feat(descs, reinterpret_cast<const Job *>(d + L.feat), info.nfeat,
                                  ctx->p.eps, ctx->p.trunc, stream));
        CUDA_TRY(ctx, mark(5));
        CUDA_TRY(ctx, mark(6));
        if (info.tcf_grid > 0)
            CUDA_TRY(ctx, launch_corr_tcf(descs, reinterpret_cast<const TcBand *>(d + L.bands),
                                          reinterpret_cast<const int32_t *>(d + L.cta_first), info.tcf_grid,
                                          ctx->d_wtc, ctx->nfk, ctx->nf, ctx->p.threshold, ctx->d_flags,
                                          stream));
        else if (info.ntc > 0 || info.ntcr > 0)
            CUDA_TRY(ctx, launch_corr_tc(descs, reinterpret_cast<const Job *>(d + L.tc), info.ntc,
                                         reinterpret_cast<const Job *>(d + L.tcr), info.ntcr, ctx->d_wtc,
                                         ctx->nfk, ctx->nf, ctx->p.threshold, ctx->d_flags,
                                         ctx->num_sms * corr_tc_ctas_per_sm(ctx->nfk), stream));
        else
            CUDA_TRY(ctx, launch_corr(descs, reinterpret_cast<const Job *>(d + L.corr), info.ncorr,
                                      ctx->d_w, ctx->nfk, ctx->nf, ctx->p.threshold, stream));
        CUDA_TRY(ctx, mark(7));
        if (ctx->prof) {
            hog_stage_stat *st = ctx->stats;
            st[0].launches += npyr; st[0].units += info.px;
            st[1].launches += info.nhist > 0; st[1].units += info.nhist > 0 ? info.cells : 0;
            st[2].launches += info.nfeat > 0; st[2].units += info.nfeat > 0 ? info.cells : 0;
            st[3].launches += (info.ncorr > 0) + (info.ntc > 0) + (info.ntcr > 0) + (info.tcf_grid > 0);
            st[3].units += (info.ncorr > 0 || info.ntcr > 0 || info.tcf_grid > 0) ? info.wins : 0;
        }
    }
    if (stages & STAGES_BACK) {
        CUDA_TRY(ctx, mark(8));
        if (info.nframes > 0)
            CUDA_TRY(ctx, launch_nms(reinterpret_cast<const FrameDesc *>(d + L.frames), info.ncls,
                                     info.cls_npos, ctx->d_flags, stream, ctx->nms_cluster, &ctx->nms_par));
        CUDA_TRY(ctx, mark(9));
        if (ctx->prof) {
            ctx->stats[4].launches += info.nframes > 0;
            ctx->stats[4].units += info.nframes;
        }
    }
    if (ctx->prof) {
        ctx->prof_pending = true;
        ctx->prof_mask = (stages & STAGES_FRONT ? 0xfu : 0u) | (stages & STAGES_BACK ? 0x10u : 0u);
    }
    return HOG_OK;
}

// Build, upload and launch a one-off plan (inspection entry points).
int run_plan(hog_ctx *ctx, PlanBuilder &pb, cudaStream_t stream) {
    build_tc_bands(pb, ctx->num_sms);
    sort_frames(pb);
    PlanInfo info;
    layout_plan(pb, ctx->nf, info);
    int rc = upload_plan(ctx, pb, info, nullptr, stream);
    if (rc) return rc;
    return launch_plan(ctx, ctx->d_plan, info, stream);
}

// Device-resident plans of recent detection batches, keyed by the batch's
// frames (pointer, size, pitch) and frame numbering: a repeated batch (a
// ring of camera buffers, a benchmark loop) skips plan building and upload.
// Point a cached plan at other frames of the same shape: level 0 reads the
// frame (img), and the first 5/6 step or a direct-to-size level resamples it
// (src).  The patched descriptors go to the device on the stream, after the
// plan's earlier uses; its graphs read them from there and stay valid.
int rebase_plan(hog_ctx *ctx, CachedPlan &cp, const std::vector<const uint8_t *> &ptrs,
                int frame_base, cudaStream_t stream) {
    for (LevelDesc &d : cp.hdescs) {
        const int i = d.frame - frame_base;
        if (i < 0 || i >= (int)ptrs.size()) continue;
        if (d.img == cp.fptr[i]) d.img = ptrs[i];
        if (d.src == cp.fptr[i]) d.src = ptrs[i];
    }
    const size_t bytes = cp.hdescs.size() * sizeof(LevelDesc);
    if (bytes) {
        int rc = ensure_plan_capacity(ctx, cp.info.L.descs + bytes);
        if (rc) return rc;
        CUDA_TRY(ctx, cudaEventSynchronize(ctx->plan_done));   // the staging buffer is free
        std::memcpy(ctx->h_plan + cp.info.L.descs, cp.hdescs.data(), bytes);
        CUDA_TRY(ctx, cudaMemcpyAsync(cp.d + cp.info.L.descs, ctx->h_plan + cp.info.L.descs, bytes,
                                      cudaMemcpyHostToDevice, stream));
        CUDA_TRY(ctx, cudaEventRecord(ctx->plan_done, stream));
    }
    cp.fptr = ptrs;
    return HOG_OK;
}

// Frame i of the batch works in buffer slot slot_base + i (slot_base > 0:
// one chunk of a larger batch whose suppression runs over all its slots).
int cached_plan(hog_ctx *ctx, const hog_frame *frames, int nb, int frame_base, cudaStream_t stream,
                const char **d_out, const PlanInfo **info_out, CachedPlan **entry = nullptr,
                const hog_roi *rois = nullptr, int slot_base = 0) {
    // Signature of the batch's shape (frame sizes, pitches, the data
    // pointers' alignment mod 16, regions); the pointers themselves are
    // compared apart.  A plan of the same shape and other frames is rebased:
    // only the level descriptors that point at a frame change.
    std::vector<uint64_t> sig;
    std::vector<const uint8_t *> ptrs((size_t)nb);
    sig.reserve(2 + 2 * (size_t)nb + (rois ? 5 * (size_t)nb : 0));
    sig.push_back((uint64_t)nb | (rois ? (1ull << 63) : 0ull));
    sig.push_back((uint64_t)(uint32_t)frame_base | ((uint64_t)(uint32_t)slot_base << 32));
    for (int i = 0; i < nb; i++) {
        ptrs[i] = frames[i].data;
        sig.push_back((uint64_t)(uintptr_t)frames[i].data & 15u);
        sig.push_back(((uint64_t)(uint32_t)frames[i].w << 40) ^ ((uint64_t)(uint32_t)frames[i].h << 20) ^
                      (uint64_t)(uint32_t)frames[i].pitch);
        if (rois) {
            const hog_roi &r = rois[i];
            uint64_t b[4];
            std::memcpy(b, &r.x0, sizeof b);   // x0, y0, x1, y1 bit patterns
            for (uint64_t v : b) sig.push_back(v);
            sig.push_back(((uint64_t)(uint32_t)r.lmin << 32) | (uint32_t)r.lmax);
        }
    }
    ctx->plan_clock++;
    for (auto &cp : ctx->plans)
        if (cp.d && cp.sig == sig && cp.fptr == ptrs) {
            cp.used = ctx->plan_clock;
            *d_out = cp.d;
            *info_out = &cp.info;
            if (entry) *entry = &cp;
            return HOG_OK;
        }
    // no free cache entry: rebase the least recently used plan of this shape
    if ((int)ctx->plans.size() >= ctx->plan_cache_max) {
        CachedPlan *rb = nullptr;
        for (auto &cp : ctx->plans)
            if (cp.d && cp.sig == sig && (!rb || cp.used < rb->used)) rb = &cp;
        if (rb) {
            int rc = rebase_plan(ctx, *rb, ptrs, frame_base, stream);
            if (rc) return rc;
            rb->used = ctx->plan_clock;
            *d_out = rb->d;
            *info_out = &rb->info;
            if (entry) *entry = rb;
            return HOG_OK;
        }
    }
    PlanBuilder pb;
    for (int i = 0; i < nb; i++) {
        const hog_frame &f = frames[i];
        if (f.w < ctx->p.min_size || f.h < ctx->p.min_size) continue;
        Geometry *g;
        int rc = get_geometry(ctx, f.w, f.h, stream, &g);
        if (rc) return rc;
        FrameOpts o;
        o.nms = g->npos > 0;
        o.roi = rois ? &rois[i] : nullptr;
        add_frame(ctx, pb, *g, f, slot_base + i, frame_base + i, o);
    }
    build_fused_items(pb);
    if (ctx->wait_withhold)   // failure-path test: one wait expects a completion nothing gives
        for (FusedItem &it : pb.items)
            if (it.wait >= 0) { it.target += 1; break; }
    build_tc_bands(pb, ctx->num_sms);
    sort_frames(pb);
    PlanInfo info;
    layout_plan(pb, ctx->nf, info);
    // least recently used entry (or a free one)
    if ((int)ctx->plans.size() < ctx->plan_cache_max) ctx->plans.emplace_back();
    CachedPlan *victim = &ctx->plans[0];
    for (auto &cp : ctx->plans)
        if (!cp.d || cp.used < victim->used) victim = &cp;
    for (auto &gm : victim->graph)
        for (auto &g : gm)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    victim->runs = 0;
    if (victim->cap < info.L.total) {
        if (victim->d) {
            CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            cudaFree(victim->d);
        }
        victim->d = nullptr;
        victim->cap = 0;
        victim->sig.clear();
        const size_t cap = align_up(info.L.total, 1 << 16);
        CUDA_TRY(ctx, cudaMalloc(&victim->d, cap));
        victim->cap = cap;
    }
    int rc = upload_plan(ctx, pb, info, victim->d, stream);
    if (rc) { victim->sig.clear(); return rc; }
    victim->sig = std::move(sig);
    victim->fptr = std::move(ptrs);
    victim->hdescs = pb.descs;
    victim->info = info;
    victim->used = ctx->plan_clock;
    *d_out = victim->d;
    *info_out = &victim->info;
    if (entry) *entry = victim;
    return HOG_OK;
}

// Persistent fused launch of pyramid .. correlation, then suppression.
int launch_fused_plan(hog_ctx *ctx, const char *d, const PlanInfo &info, cudaStream_t stream,
                      int stages = STAGES_ALL) {
    const PlanLayout &L = info.L;
    if ((size_t)info.nctr + 8 > ctx->fctr_cap)
        return fail(ctx, HOG_EINTERNAL, "fused counter capacity %zu < %d", ctx->fctr_cap, info.nctr + 8);
    int *head = ctx->d_fctr + info.nctr, *abort_flag = head + 1;
    FusedArgs a;
    a.items = reinterpret_cast<const FusedItem *>(d + L.items);
    a.nitems = info.nitems;
    a.descs = reinterpret_cast<const LevelDesc *>(d + L.descs);
    a.jobs = reinterpret_cast<const Job *>(d + L.corrf);
    a.wchunks = ctx->d_w;
    a.nf_real = ctx->nf;
    a.threshold = ctx->p.threshold;
    a.eps = ctx->p.eps;
    a.tau = ctx->p.trunc;
    a.ctr = ctx->d_fctr;
    a.head = head;
    a.abort = abort_flag;
    a.flags = ctx->d_flags;
    a.spin_limit = ctx->wait_polls;
    int rc = collect_profile(ctx);
    if (rc) return rc;
    auto mark = [&](int i) -> cudaError_t {
        return ctx->prof ? cudaEventRecord(ctx->prof_ev[i], stream) : cudaSuccess;
    };
    if (stages & STAGES_FRONT) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_fctr, 0, sizeof(int) * ((size_t)info.nctr + 2), stream));
        CUDA_TRY(ctx, mark(10));
        CUDA_TRY(ctx, launch_fused(a, ctx->nfk, ctx->fused_grid, stream));
        if (info.tcf_grid > 0)   // tensor-core correlation after the fused stages
            CUDA_TRY(ctx, launch_corr_tcf(a.descs, reinterpret_cast<const TcBand *>(d + L.bands),
                                          reinterpret_cast<const int32_t *>(d + L.cta_first), info.tcf_grid,
                                          ctx->d_wtc, ctx->nfk, ctx->nf, ctx->p.threshold, ctx->d_flags,
                                          stream));
        else if (info.ntc > 0 || info.ntcr > 0)
            CUDA_TRY(ctx, launch_corr_tc(a.descs, reinterpret_cast<const Job *>(d + L.tc), info.ntc,
                                         reinterpret_cast<const Job *>(d + L.tcr), info.ntcr, ctx->d_wtc,
                                         ctx->nfk, ctx->nf, ctx->p.threshold, ctx->d_flags,
                                         ctx->num_sms * corr_tc_ctas_per_sm(ctx->nfk), stream));
        CUDA_TRY(ctx, mark(11));
        if (ctx->prof) {
            ctx->stats[5].launches += (info.nitems > 0) + (info.ntc > 0) + (info.ntcr > 0) + (info.tcf_grid > 0);
            ctx->stats[5].units += info.wins;
        }
    }
    if (stages & STAGES_BACK) {
        CUDA_TRY(ctx, mark(8));
        if (info.nframes > 0)
            CUDA_TRY(ctx, launch_nms(reinterpret_cast<const FrameDesc *>(d + L.frames), info.ncls,
                                     info.cls_npos, ctx->d_flags, stream, ctx->nms_cluster, &ctx->nms_par));
        CUDA_TRY(ctx, mark(9));
        if (ctx->prof) {
            ctx->stats[4].launches += info.nframes > 0;
            ctx->stats[4].units += info.nframes;
        }
    }
    if (ctx->prof) {
        ctx->prof_pending = true;
        ctx->prof_mask = (stages & STAGES_FRONT ? 1u << 5 : 0u) | (stages & STAGES_BACK ? 1u << 4 : 0u);
    }
    return HOG_OK;
}

// Everything one detection batch enqueues before its outputs are packed
// (stages: STAGES_ALL), or one part of it.  The front alone leaves the
// flags as they are: the caller clears them once before a run of fronts.
int enqueue_batch(hog_ctx *ctx, int mode, const char *d, const PlanInfo &info, int nb,
                  cudaStream_t stream, int stages = STAGES_ALL) {
    if (stages & STAGES_BACK) CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_counts, 0, sizeof(int32_t) * nb, stream));
    if (stages == STAGES_ALL) CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int), stream));
    return mode == MODE_FUSED ? launch_fused_plan(ctx, d, info, stream, stages)
                              : launch_plan(ctx, d, info, stream, stages);
}

// Run a batch eagerly, or -- from its second use on, with use_graph and no
// profiling -- as a CUDA graph captured once per cached plan and mode.
int run_batch(hog_ctx *ctx, int mode, CachedPlan *cp, int nb, bool use_graph, cudaStream_t stream,
              int stages = STAGES_ALL) {
    if (!use_graph || ctx->prof || cp->runs < 1) {
        cp->runs++;
        return enqueue_batch(ctx, mode, cp->d, cp->info, nb, stream, stages);
    }
    cudaGraphExec_t &ge = cp->graph[mode][stages];
    if (!ge) {
        if (!ctx->cap_stream) CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_batch(ctx, mode, cp->d, cp->info, nb, ctx->cap_stream, stages);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail(ctx, HOG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge = nullptr;
            return fail(ctx, HOG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    CUDA_TRY(ctx, cudaGraphLaunch(ge, stream));
    return HOG_OK;
}

// Drop every cached plan (and its graphs), e.g. after a tuning change.
void clear_plans(hog_ctx *ctx) {
    cudaDeviceSynchronize();
    for (auto &cp : ctx->plans) {
        if (cp.d) cudaFree(cp.d);
        for (auto &gm : cp.graph)
            for (auto &g : gm) if (g) cudaGraphExecDestroy(g);
    }
    ctx->plans.clear();
}

int check_frame(hog_ctx *ctx, const hog_frame *f, bool device) {
    if (!f) return fail(ctx, HOG_EINVAL, "frame is NULL");
    if (f->w < 0 || f->h < 0 || f->w > ctx->p.max_w || f->h > ctx->p.max_h)
        return fail(ctx, HOG_EINVAL, "frame %dx%d outside 0..%dx%d", f->w, f->h, ctx->p.max_w,
                    ctx->p.max_h);
    if (f->w > 0 && f->h > 0 && (!f->data || f->pitch < f->w))
        return fail(ctx, HOG_EINVAL, "frame data NULL or pitch %d < width %d", f->pitch, f->w);
    (void)device;
    return HOG_OK;
}

// The device address of a pinned (page-locked, mapped) output buffer, which
// the device then writes directly; null for any other host buffer (filled
// from the context's staging).
hog_det *mapped_dets(hog_det *dets, int det_cap) {
    hog_det *dets_dev = nullptr;
    if (dets && det_cap > 0) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, dets) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            attr.devicePointer)
            dets_dev = static_cast<hog_det *>(attr.devicePointer);
        cudaGetLastError();
    }
    return dets_dev;
}

// After the suppression of slots 0 .. nb-1 (frames b0 .. b0+nb-1 of the
// call) is enqueued: kept boxes of all frames packed frame after frame (into
// dets_dev, or the context's mapped staging) by one kernel, then one
// synchronisation and the counts.  written and truncated accumulate.
int finish_batch(hog_ctx *ctx, int nb, int b0, hog_det *dets, hog_det *dets_dev, int det_cap, int &written,
                 bool &truncated, int32_t *counts, cudaStream_t stream) {
    const size_t D = (size_t)ctx->p.max_dets_per_frame;
    const int room = dets ? std::max(det_cap - written, 0) : 0;
    if (dets_dev)
        CUDA_TRY(ctx, launch_pack(ctx->d_dets, ctx->p.max_dets_per_frame, ctx->d_counts, nb,
                                  dets_dev + written, room, ctx->m_counts, stream));
    else
        CUDA_TRY(ctx, launch_pack(ctx->d_dets, ctx->p.max_dets_per_frame, ctx->d_counts, nb, ctx->m_dets,
                                  (int)(D * ctx->p.max_batch), ctx->m_counts, stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                                  stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    if (ctx->h_flags[2]) return fail(ctx, HOG_ETIMEOUT, "a bounded device wait gave up; results are invalid");
    size_t off = 0;
    for (int i = 0; i < nb; i++) {
        const int c = ctx->h_counts[i];
        if (counts) counts[b0 + i] = c;
        const int k = std::min(c, ctx->p.max_dets_per_frame);
        if (c > k) truncated = true;
        const int take = std::min(k, std::max(det_cap - written, 0));
        if (take > 0 && !dets_dev) std::memcpy(dets + written, ctx->h_dets + off, sizeof(hog_det) * take);
        if (take < k) truncated = true;
        written += take;
        off += k;
    }
    return HOG_OK;
}

int detect_device(hog_ctx *ctx, const hog_frame *frames, int n, int frame_base, hog_det *dets,
                  int det_cap, int *written_out, int32_t *counts, cudaStream_t stream,
                  int mode = MODE_STAGED, bool use_graph = false, const hog_roi *rois = nullptr) {
    int written = 0;
    bool truncated = false;
    hog_det *dets_dev = mapped_dets(dets, det_cap);
    for (int b0 = 0; b0 < n; b0 += ctx->p.max_batch) {
        const int nb = std::min(ctx->p.max_batch, n - b0);
        const char *dplan = nullptr;
        const PlanInfo *info = nullptr;
        CachedPlan *cp = nullptr;
        int rc = cached_plan(ctx, frames + b0, nb, frame_base + b0, stream, &dplan, &info, &cp,
                             rois ? rois + b0 : nullptr);
        if (rc) return rc;
        rc = run_batch(ctx, mode, cp, nb, use_graph, stream);
        if (rc) return rc;
        rc = finish_batch(ctx, nb, b0, dets, dets_dev, det_cap, written, truncated, counts, stream);
        if (rc) return rc;
    }
    if (written_out) *written_out = written;
    return truncated ? fail(ctx, HOG_ECAPACITY, "detections truncated (%d written)", written)
                     : HOG_OK;
}

}  // namespace

namespace hogk {

// Enqueue the detection of nb <= max_batch device frames on `stream`
// without waiting: plan (cached), launches, and the packing of kept boxes
// and counts into the context's mapped pinned buffers.
int detect_enqueue(hog_ctx *ctx, const hog_frame *frames, int nb, cudaStream_t stream, int mode,
                   bool use_graph) {
    if (nb < 1 || nb > ctx->p.max_batch) return fail(ctx, HOG_EINVAL, "batch of %d frames", nb);
    const char *dplan = nullptr;
    const PlanInfo *info = nullptr;
    CachedPlan *cp = nullptr;
    int rc = cached_plan(ctx, frames, nb, 0, stream, &dplan, &info, &cp);
    if (rc) return rc;
    rc = run_batch(ctx, mode, cp, nb, use_graph, stream);
    if (rc) return rc;
    const size_t D = (size_t)ctx->p.max_dets_per_frame;
    CUDA_TRY(ctx, launch_pack(ctx->d_dets, ctx->p.max_dets_per_frame, ctx->d_counts, nb, ctx->m_dets,
                              (int)(D * ctx->p.max_batch), ctx->m_counts, stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                                  stream));
    return HOG_OK;
}

// After the enqueued work has completed: the packed boxes of frame i start
// at *first + (sum of earlier frames' stored counts).
int detect_results(hog_ctx *ctx, const int32_t **counts, const hog_det **dets) {
    if (ctx->h_flags[2]) return fail(ctx, HOG_ETIMEOUT, "a bounded device wait gave up");
    *counts = ctx->h_counts;
    *dets = ctx->h_dets;
    return HOG_OK;
}

int ctx_max_dets(const hog_ctx *ctx) { return ctx->p.max_dets_per_frame; }
int ctx_max_batch(const hog_ctx *ctx) { return ctx->p.max_batch; }
int ctx_batched_mode(const hog_ctx *ctx) { return ctx->batched_mode; }
void ctx_set_plan_cache(hog_ctx *ctx, int n) { ctx->plan_cache_max = n < 1 ? 1 : n; }
const char *ctx_error(const hog_ctx *ctx) { return ctx->err.c_str(); }

}  // namespace hogk

// ==== C ABI ===============================================================

extern "C" {

void hog_default_params(hog_params *p) {
    if (!p) return;
    p->cell = CELL;
    p->win_cells_w = WIN;
    p->win_cells_h = WIN;
    p->scale_num = 5;
    p->scale_den = 6;
    p->min_size = 80;
    p->skip_levels = 0;
    p->eps = 1e-4f;
    p->trunc = 0.2f;
    p->threshold = 0.0f;
    p->nms_iou = 0.5f;
    p->max_w = 1280;
    p->max_h = 1024;
    p->max_batch = 64;
    p->max_dets_per_frame = 16384;
    p->float_pyramid = 0;
    p->direct_first = 0;
}

int hog_level_geometry(const hog_params *p, int32_t w, int32_t h, hog_level *levels, int32_t cap,
                       int32_t *n_levels) {
    std::string why;
    if (check_params(p, why)) return HOG_EINVAL;
    if (w < 0 || h < 0 || !n_levels || (cap > 0 && !levels)) return HOG_EINVAL;
    Geometry g;
    if (compute_geometry(*p, w, h, g)) return HOG_EINVAL;
    *n_levels = g.nlev;
    for (int l = 0; l < g.nlev && l < cap; l++)
        levels[l] = hog_level{g.lw[l], g.lh[l], g.cx[l], g.cy[l], (int64_t)g.ufeat_off[l]};
    return g.nlev > cap ? HOG_EINVAL : HOG_OK;
}

int hog_create(const hog_params *p, const float *filters_host, int32_t n_filters, hog_ctx **out) {
    if (!out) { g_create_error = "out is NULL"; return HOG_EINVAL; }
    *out = nullptr;
    std::string why;
    if (check_params(p, why)) { g_create_error = why; return HOG_EINVAL; }
    hog_ctx *ctx = new (std::nothrow) hog_ctx();
    if (!ctx) { g_create_error = "host allocation failed"; return HOG_ENOMEM; }
    ctx->p = *p;
    int rc = upload_filters(ctx, filters_host, n_filters);
    if (rc) { g_create_error = ctx->err; free_ctx(ctx); return rc; }
    if (compute_geometry(ctx->p, ctx->p.max_w, ctx->p.max_h, ctx->maxg)) {
        g_create_error = "max frame has too many levels";
        free_ctx(ctx);
        return HOG_EINVAL;
    }
    const Geometry &g = ctx->maxg;
    ctx->pyr_slot = align_up(std::max<size_t>(g.pyr_bytes, 256), 256);
    ctx->hist_slot = align_up(std::max<size_t>(g.hist_floats, 64), 64);
    ctx->feat_slot = align_up(std::max<size_t>(g.feat_floats, 64), 64);
    ctx->pos_slot = align_up(std::max<size_t>(g.npos, 1), 32);
    const size_t B = (size_t)ctx->p.max_batch;
    const size_t D = (size_t)ctx->p.max_dets_per_frame;
    cudaError_t e = cudaSuccess;
    auto M = [&](void **ptr, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(ptr, bytes); };
    M((void **)&ctx->d_pyr, B * ctx->pyr_slot);
    M((void **)&ctx->d_hist, B * ctx->hist_slot * sizeof(float));
    M((void **)&ctx->d_feat, B * ctx->feat_slot * sizeof(float));
    M((void **)&ctx->d_keys, B * ctx->pos_slot * sizeof(uint64_t));
    M((void **)&ctx->d_nmsws, B * ctx->pos_slot * HOG_NMS_WS_WORDS * sizeof(uint32_t));
    M((void **)&ctx->d_nmscand, B * ctx->pos_slot);
    M((void **)&ctx->d_dets, B * D * sizeof(hog_det));
    M((void **)&ctx->d_counts, B * sizeof(int32_t));
    M((void **)&ctx->d_flags, sizeof(int) * 4);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&ctx->h_dets, B * D * sizeof(hog_det), cudaHostAllocMapped);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&ctx->h_counts, B * sizeof(int32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&ctx->m_dets, ctx->h_dets, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&ctx->m_counts, ctx->h_counts, 0);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->h_flags, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->plan_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->nms_par.fork, cudaEventDisableTiming);
    for (int k = 0; k < NMS_WS_CLASSES - 1 && e == cudaSuccess; k++) {
        e = cudaStreamCreateWithFlags(&ctx->nms_par.side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->nms_par.join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("allocation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_ctx(ctx);
        return HOG_ENOMEM;
    }
    rc = ensure_plan_capacity(ctx, 1 << 20);
    if (rc) { g_create_error = ctx->err; free_ctx(ctx); return rc; }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (ctx->num_sms <= 0) ctx->num_sms = 1;
        ctx->fused_grid = ctx->num_sms * fused_max_ctas_per_sm(ctx->nfk);
        ctx->fctr_cap = B * MAX_LEVELS * 3 + 16;
        if (cudaMalloc(&ctx->d_fctr, ctx->fctr_cap * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            g_create_error = "counter allocation failed";
            free_ctx(ctx);
            return HOG_ENOMEM;
        }
    }
    // tensor-core correlation by default; the CUDA-core engine if its
    // buffers cannot be had or the filters exceed its fp16 range (the
    // message stays in hog_last_error)
    if (prepare_tc(ctx, false) == HOG_OK) {
        ctx->corr_engine = 1;
    } else {
        cudaGetLastError();
        if (tc_range_ok(ctx)) ctx->err.clear();
    }
    *out = ctx;
    return HOG_OK;
}

int hog_set_filters(hog_ctx *ctx, const float *filters_host, int32_t n_filters) {
    if (!ctx) return HOG_EINVAL;
    cudaDeviceSynchronize();
    const int nfk0 = ctx->nfk;
    int rc = upload_filters(ctx, filters_host, n_filters);
    if (rc == HOG_OK && ctx->corr_engine >= 1) {
        if (!tc_range_ok(ctx)) {
            // outside the tensor engines' fp16 range: the CUDA-core engine
            // takes over (hog_get_corr_engine reports 0, hog_last_error why)
            clear_plans(ctx);
            ctx->corr_engine = 0;
            prepare_tc(ctx, false);   // records the reason, allocates nothing
            return HOG_OK;
        }
        if (ctx->nfk != nfk0) clear_plans(ctx);   // row-shift matrices change size
        rc = prepare_tc(ctx, ctx->corr_engine == 2);
    }
    return rc;
}

void hog_destroy(hog_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx);
}

const char *hog_last_error(const hog_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int hog_set_profiling(hog_ctx *ctx, int32_t on) {
    if (!ctx) return HOG_EINVAL;
    if (on && !ctx->prof_ev[0])
        for (cudaEvent_t &e : ctx->prof_ev) CUDA_TRY(ctx, cudaEventCreate(&e));
    int rc = collect_profile(ctx);
    if (rc) return rc;
    ctx->prof = on != 0;
    return HOG_OK;
}

int hog_stage_stats(hog_ctx *ctx, hog_stage_stat *out, int32_t cap, int32_t reset) {
    if (!ctx || (cap > 0 && !out)) return HOG_EINVAL;
    int rc = collect_profile(ctx);
    if (rc) return rc;
    for (int k = 0; k < HOG_NSTAGES && k < cap; k++) out[k] = ctx->stats[k];
    if (reset) std::memset(ctx->stats, 0, sizeof ctx->stats);
    return HOG_OK;
}

int hog_pyramid(hog_ctx *ctx, const hog_frame *frame, uint8_t *out, size_t cap_bytes,
                hog_level *levels, int32_t cap_levels, int32_t *n_levels, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    int rc = check_frame(ctx, frame, true);
    if (rc) return rc;
    if (!n_levels) return fail(ctx, HOG_EINVAL, "n_levels is NULL");
    Geometry g;
    if (compute_geometry(ctx->p, frame->w, frame->h, g)) return fail(ctx, HOG_EINVAL, "too many levels");
    *n_levels = g.nlev;
    if (g.nlev > cap_levels || (g.nlev > 0 && !levels))
        return fail(ctx, HOG_EINVAL, "level capacity %d < %d", cap_levels, g.nlev);
    size_t off = 0;
    for (int l = 0; l < g.nlev; l++) {
        levels[l] = hog_level{g.lw[l], g.lh[l], g.cx[l], g.cy[l], (int64_t)off};
        off += (size_t)g.lw[l] * g.lh[l];
    }
    if (g.nlev == 0) return HOG_OK;
    if (!out || off > cap_bytes) return fail(ctx, HOG_EINVAL, "output capacity %zu < %zu", cap_bytes, off);
    PlanBuilder pb;
    FrameOpts o;
    o.corr = false; o.nms = false; o.feat = false;
    add_frame(ctx, pb, g, *frame, 0, 0, o);
    rc = run_plan(ctx, pb, stream);
    if (rc) return rc;
    for (int l = 0; l < g.nlev; l++) {
        const LevelDesc &d = pb.descs[l];
        if (level_absent(ctx->p, l))
            CUDA_TRY(ctx, cudaMemsetAsync(out + levels[l].offset, 0, (size_t)d.w * d.h, stream));
        else
            CUDA_TRY(ctx, cudaMemcpy2DAsync(out + levels[l].offset, (size_t)d.w, d.img, (size_t)d.pitch,
                                            (size_t)d.w, (size_t)d.h, cudaMemcpyDeviceToDevice, stream));
    }
    return HOG_OK;
}

int hog_features(hog_ctx *ctx, const hog_frame *frame, float *feat_out, size_t cap_floats,
                 hog_level *levels, int32_t cap_levels, int32_t *n_levels, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    int rc = check_frame(ctx, frame, true);
    if (rc) return rc;
    if (!n_levels) return fail(ctx, HOG_EINVAL, "n_levels is NULL");
    Geometry g;
    if (compute_geometry(ctx->p, frame->w, frame->h, g)) return fail(ctx, HOG_EINVAL, "too many levels");
    *n_levels = g.nlev;
    if (g.nlev > cap_levels || (g.nlev > 0 && !levels))
        return fail(ctx, HOG_EINVAL, "level capacity %d < %d", cap_levels, g.nlev);
    for (int l = 0; l < g.nlev; l++)
        levels[l] = hog_level{g.lw[l], g.lh[l], g.cx[l], g.cy[l], (int64_t)g.ufeat_off[l]};
    if (g.nlev == 0) return HOG_OK;
    if (!feat_out || g.ufeat_floats > cap_floats)
        return fail(ctx, HOG_EINVAL, "feature capacity %zu < %zu floats", cap_floats, g.ufeat_floats);
    PlanBuilder pb;
    FrameOpts o;
    o.corr = false; o.nms = false;
    o.feat_user = feat_out;
    add_frame(ctx, pb, g, *frame, 0, 0, o);
    for (int l = 0; l < g.nlev; l++)
        if (level_absent(ctx->p, l))
            CUDA_TRY(ctx, cudaMemsetAsync(feat_out + g.ufeat_off[l], 0,
                                          sizeof(float) * (size_t)g.cx[l] * g.cy[l] * NFEAT, stream));
    return run_plan(ctx, pb, stream);
}

int hog_scores(hog_ctx *ctx, const hog_frame *frame, float *scores_out, size_t cap_floats,
               hog_level *levels, int32_t cap_levels, int32_t *n_levels, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    int rc = check_frame(ctx, frame, true);
    if (rc) return rc;
    if (!n_levels) return fail(ctx, HOG_EINVAL, "n_levels is NULL");
    Geometry g;
    if (compute_geometry(ctx->p, frame->w, frame->h, g)) return fail(ctx, HOG_EINVAL, "too many levels");
    *n_levels = g.nlev;
    if (g.nlev > cap_levels || (g.nlev > 0 && !levels))
        return fail(ctx, HOG_EINVAL, "level capacity %d < %d", cap_levels, g.nlev);
    size_t off = 0, soff[MAX_LEVELS];
    for (int l = 0; l < g.nlev; l++) {
        soff[l] = off;
        levels[l] = hog_level{g.lw[l], g.lh[l], g.cx[l], g.cy[l], (int64_t)off};
        off += (size_t)ctx->nf * g.nu[l] * g.nv[l];
    }
    if (g.nlev == 0 || off == 0) return HOG_OK;
    if (!scores_out || off > cap_floats)
        return fail(ctx, HOG_EINVAL, "score capacity %zu < %zu floats", cap_floats, off);
    PlanBuilder pb;
    FrameOpts o;
    o.nms = false;
    o.scores_user = scores_out;
    o.score_off = soff;
    add_frame(ctx, pb, g, *frame, 0, 0, o);
    for (int l = 0; l < g.nlev; l++)
        if (level_absent(ctx->p, l))
            CUDA_TRY(ctx, cudaMemsetAsync(scores_out + soff[l], 0,
                                          sizeof(float) * (size_t)ctx->nf * g.nu[l] * g.nv[l], stream));
    return run_plan(ctx, pb, stream);
}

int hog_detect(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, hog_det *dets,
               int32_t det_cap, int32_t *counts, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    if (n_frames < 0 || (n_frames > 0 && !frames) || det_cap < 0 || (det_cap > 0 && !dets))
        return fail(ctx, HOG_EINVAL, "bad frames/dets arguments");
    for (int i = 0; i < n_frames; i++) {
        int rc = check_frame(ctx, &frames[i], true);
        if (rc) return rc;
    }
    return detect_device(ctx, frames, n_frames, 0, dets, det_cap, nullptr, counts,
                         (cudaStream_t)stream_, MODE_STAGED, true);
}

int hog_detect_batched(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, hog_det *dets,
                       int32_t det_cap, int32_t *counts, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    if (n_frames < 0 || (n_frames > 0 && !frames) || det_cap < 0 || (det_cap > 0 && !dets))
        return fail(ctx, HOG_EINVAL, "bad frames/dets arguments");
    for (int i = 0; i < n_frames; i++) {
        int rc = check_frame(ctx, &frames[i], true);
        if (rc) return rc;
    }
    return detect_device(ctx, frames, n_frames, 0, dets, det_cap, nullptr, counts,
                         (cudaStream_t)stream_, ctx->batched_mode, true);
}

int hog_roi_around(const hog_det *prev, int32_t W, int32_t H, double margin, int32_t dlev,
                   hog_roi *out) {
    if (!prev || !out || !(margin >= 0.0) || dlev < 0) return HOG_EINVAL;
    const double mx = margin * prev->w, my = margin * prev->h;
    out->x0 = std::max(0.0, prev->x - mx);
    out->y0 = std::max(0.0, prev->y - my);
    out->x1 = std::min((double)W, prev->x + prev->w + mx);
    out->y1 = std::min((double)H, prev->y + prev->h + my);
    out->lmin = std::max(0, prev->level - dlev);
    out->lmax = prev->level + dlev;
    return HOG_OK;
}

int hog_detect_roi(hog_ctx *ctx, const hog_frame *frames, const hog_roi *rois, int32_t n_frames,
                   hog_det *dets, int32_t det_cap, int32_t *counts, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    if (n_frames < 0 || (n_frames > 0 && (!frames || !rois)) || det_cap < 0 || (det_cap > 0 && !dets))
        return fail(ctx, HOG_EINVAL, "bad frames/rois/dets arguments");
    for (int i = 0; i < n_frames; i++) {
        int rc = check_frame(ctx, &frames[i], true);
        if (rc) return rc;
        const hog_roi &r = rois[i];
        if (!std::isfinite(r.x0) || !std::isfinite(r.y0) || !std::isfinite(r.x1) || !std::isfinite(r.y1))
            return fail(ctx, HOG_EINVAL, "region of interest %d is not finite", i);
    }
    return detect_device(ctx, frames, n_frames, 0, dets, det_cap, nullptr, counts,
                         (cudaStream_t)stream_, MODE_STAGED, false, rois);
}

int hog_set_corr_engine(hog_ctx *ctx, int32_t engine) {
    if (!ctx || engine < 0 || engine > 2) return HOG_EINVAL;
    if (engine == ctx->corr_engine) return HOG_OK;
    clear_plans(ctx);   // plans hold the engine's jobs and buffers
    if (engine >= 1) {
        const int rc = prepare_tc(ctx, engine == 2);
        if (rc) return rc;
    }
    ctx->corr_engine = engine;
    return HOG_OK;
}

int hog_get_corr_engine(const hog_ctx *ctx, int32_t *engine) {
    if (!ctx || !engine) return HOG_EINVAL;
    *engine = ctx->corr_engine;
    return HOG_OK;
}

int hog_set_nms_cluster(hog_ctx *ctx, int32_t c) {
    if (!ctx || !(c == 0 || c == 1 || c == 2 || c == 4 || c == 8 || c == 16)) return HOG_EINVAL;
    if (c != ctx->nms_cluster) {
        clear_plans(ctx);   // captured graphs hold the old launch shape
        ctx->nms_cluster = c;
    }
    return HOG_OK;
}

int hog_nms_cluster_size(hog_ctx *ctx, int32_t n_frames, int32_t w, int32_t h, int32_t *c) {
    if (!ctx || !c || n_frames < 1 || w < 0 || h < 0) return HOG_EINVAL;
    Geometry g;   // host-side level geometry only
    if (compute_geometry(ctx->p, w, h, g)) return HOG_EINVAL;
    *c = nms_cluster_size(n_frames, g.npos, ctx->nms_cluster);
    return HOG_OK;
}

int hog_set_batched_mode(hog_ctx *ctx, int32_t mode) {
    if (!ctx || (mode != MODE_STAGED && mode != MODE_FUSED)) return HOG_EINVAL;
    ctx->batched_mode = mode;
    return HOG_OK;
}

int hog_detect_host(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, hog_det *dets,
                    int32_t det_cap, int32_t *counts, void *stream_) {
    if (!ctx) return HOG_EINVAL;
    if (n_frames < 0 || (n_frames > 0 && !frames) || det_cap < 0 || (det_cap > 0 && !dets))
        return fail(ctx, HOG_EINVAL, "bad frames/dets arguments");
    for (int i = 0; i < n_frames; i++) {
        int rc = check_frame(ctx, &frames[i], false);
        if (rc) return rc;
    }
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t fbytes = (size_t)ctx->p.max_w * ctx->p.max_h;
    if (!ctx->d_stage) {
        ctx->stage_cap = fbytes * ctx->p.max_batch;
        CUDA_TRY(ctx, cudaMalloc(&ctx->d_stage, ctx->stage_cap));
        CUDA_TRY(ctx, cudaMallocHost(&ctx->h_stage, ctx->stage_cap));
    }
    if (!ctx->copy_stream) {
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; k++) {
            CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->copy_done[k], cudaEventDisableTiming));
            CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->front_done[k], cudaEventDisableTiming));
        }
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->stage_free, cudaEventDisableTiming));
    }
    // Groups of up to max_batch frames.  A group of more than max_batch / 2
    // frames goes in chunks of up to max_batch / 2 through two halves of the
    // staging area: the host-to-device copy of chunk k+1 (on the copy
    // stream) overlaps the front stages of chunk k (pyramid .. correlation,
    // in buffer slots of their own), and one suppression launch then takes
    // the whole group, as a batch of the group's size would.  The first
    // chunk is a quarter of the others: its copy is the one nothing hides.
    const int half = std::max(1, ctx->p.max_batch / 2);
    std::vector<hog_frame> dev((size_t)ctx->p.max_batch);
    hog_det *dets_dev = mapped_dets(dets, det_cap);
    int written = 0;
    bool truncated = false;

    // the copy stream may only overwrite staging that no earlier work on
    // `stream` still reads
    CUDA_TRY(ctx, cudaEventRecord(ctx->stage_free, stream));
    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->stage_free, 0));
    int rc = HOG_OK;
    for (int g0 = 0; g0 < n_frames && !rc; g0 += ctx->p.max_batch) {
        const int ng = std::min(ctx->p.max_batch, n_frames - g0);
        const int chunk = ng > half ? std::min(half, (ng + 3) / 4) : ng;
        std::vector<int> cbeg(1, 0);   // first frame of each chunk in the group, then ng
        for (int at = ng > half ? std::max(1, chunk / 4) : ng; at < ng; at += chunk) cbeg.push_back(at);
        cbeg.push_back(ng);
        const int nchunks = (int)cbeg.size() - 1;
        auto staged = [&](int k, int i) {   // staging slot of frame i of chunk k
            return (size_t)(nchunks > 1 ? (k & 1) * chunk : 0) + (size_t)i;
        };

        // enqueue the copy of chunk k into its staging half on the copy
        // stream.  Frames that are dense (pitch = w), follow each other in
        // pinned host memory and fill their device slot exactly (w * h =
        // fbytes) move as one copy.
        auto copy_chunk = [&](int k) -> int {
            const int b0 = g0 + cbeg[k], nb = cbeg[k + 1] - cbeg[k];
            cudaStream_t cs = ctx->copy_stream;
            for (int i = 0; i < nb;) {
                const hog_frame &f = frames[b0 + i];
                uint8_t *d = ctx->d_stage + staged(k, i) * fbytes;
                if (f.w == 0 || f.h == 0) { i++; continue; }
                cudaPointerAttributes attr;
                const bool pinned = cudaPointerGetAttributes(&attr, f.data) == cudaSuccess &&
                                    attr.type == cudaMemoryTypeHost;
                cudaGetLastError();
                const size_t fb = (size_t)f.w * f.h;
                int run = 1;
                if (pinned && f.pitch == f.w && fb == fbytes) {
                    while (i + run < nb) {
                        const hog_frame &g = frames[b0 + i + run];
                        if (g.w != f.w || g.h != f.h || g.pitch != f.pitch || g.data != f.data + run * fb) break;
                        run++;
                    }
                    CUDA_TRY(ctx, cudaMemcpyAsync(d, f.data, fb * run, cudaMemcpyHostToDevice, cs));
                    i += run;
                    continue;
                }
                const uint8_t *srcp = f.data;
                size_t spitch = (size_t)f.pitch;
                if (!pinned) {   // stage through pinned memory so the copy is asynchronous
                    uint8_t *h = ctx->h_stage + staged(k, i) * fbytes;
                    for (int y = 0; y < f.h; y++)
                        std::memcpy(h + (size_t)y * f.w, f.data + (size_t)y * f.pitch, f.w);
                    srcp = h;
                    spitch = (size_t)f.w;
                }
                CUDA_TRY(ctx, cudaMemcpy2DAsync(d, (size_t)f.w, srcp, spitch, (size_t)f.w, (size_t)f.h,
                                                cudaMemcpyHostToDevice, cs));
                i++;
            }
            CUDA_TRY(ctx, cudaEventRecord(ctx->copy_done[k & 1], cs));
            return HOG_OK;
        };

        // the fronts leave the flags alone: clear them once for the group
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_flags, 0, 4 * sizeof(int), stream));
        rc = copy_chunk(0);
        for (int k = 0; k < nchunks && !rc; k++) {
            if (k + 1 < nchunks) {
                // chunk k+1 goes into the half chunk k-1 read: after its front
                if (k >= 1)
                    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->front_done[(k + 1) & 1], 0));
                rc = copy_chunk(k + 1);
                if (rc) break;
            }
            const int c0 = cbeg[k], nb = cbeg[k + 1] - c0;
            for (int i = 0; i < nb; i++) {
                const hog_frame &f = frames[g0 + c0 + i];
                dev[c0 + i] = hog_frame{ctx->d_stage + staged(k, i) * fbytes, f.w, f.h, f.w};
            }
            CUDA_TRY(ctx, cudaStreamWaitEvent(stream, ctx->copy_done[k & 1], 0));
            const char *dplan = nullptr;
            const PlanInfo *info = nullptr;
            CachedPlan *cp = nullptr;
            rc = cached_plan(ctx, dev.data() + c0, nb, g0 + c0, stream, &dplan, &info, &cp, nullptr, c0);
            if (rc) break;
            rc = run_batch(ctx, ctx->batched_mode, cp, nb, true, stream,
                           nchunks > 1 ? STAGES_FRONT : STAGES_ALL);
            if (rc) break;
            CUDA_TRY(ctx, cudaEventRecord(ctx->front_done[k & 1], stream));
        }
        if (!rc && nchunks > 1) {   // suppression of the whole group
            const char *dplan = nullptr;
            const PlanInfo *info = nullptr;
            CachedPlan *cp = nullptr;
            rc = cached_plan(ctx, dev.data(), ng, g0, stream, &dplan, &info, &cp);
            if (!rc) rc = run_batch(ctx, ctx->batched_mode, cp, ng, true, stream, STAGES_BACK);
        }
        if (!rc) rc = finish_batch(ctx, ng, g0, dets, dets_dev, det_cap, written, truncated, counts, stream);
    }
    if (rc) {
        cudaStreamSynchronize(ctx->copy_stream);   // no copy still writes the staging area
        cudaStreamSynchronize(stream);             // nor a front still reads it
        return rc;
    }
    return truncated ? fail(ctx, HOG_ECAPACITY, "detections truncated (%d written)", written) : HOG_OK;
}

int hog_autotune(hog_ctx *ctx, const hog_frame *frames, int32_t n_frames, const char *cache_path,
                 void *stream_) {
    if (!ctx || n_frames < 1 || !frames) return HOG_EINVAL;
    for (int i = 0; i < n_frames; i++) {
        int rc = check_frame(ctx, &frames[i], true);
        if (rc) return rc;
    }
    cudaStream_t stream = (cudaStream_t)stream_;
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    CUDA_TRY(ctx, cudaGetDeviceProperties(&prop, dev));
    // key: device, SM count, filters, frame sizes of the sample
    std::string key = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount) +
                      "|nf" + std::to_string(ctx->nf) + "|";
    {   // distinct frame sizes with their counts, in first-seen order
        std::vector<std::pair<std::pair<int, int>, int>> sizes;
        for (int i = 0; i < n_frames; i++) {
            bool found = false;
            for (auto &sz : sizes)
                if (sz.first.first == frames[i].w && sz.first.second == frames[i].h) { sz.second++; found = true; }
            if (!found) sizes.push_back({{frames[i].w, frames[i].h}, 1});
        }
        for (auto &sz : sizes)
            key += std::to_string(sz.first.first) + "x" + std::to_string(sz.first.second) + "*" +
                   std::to_string(sz.second) + ",";
    }
    if (cache_path && *cache_path) {
        FILE *f = std::fopen(cache_path, "r");
        if (f) {
            char buf[8192] = {0};
            const size_t nread = std::fread(buf, 1, sizeof buf - 1, f);
            std::fclose(f);
            buf[nread] = 0;
            const std::string txt(buf);
            const std::string kq = "\"key\": \"" + key + "\"";
            if (txt.find(kq) != std::string::npos) {
                int mode = -1, pol = -1, eng = 0;
                const size_t a = txt.find("\"batched_mode\": ");
                const size_t b = txt.find("\"corr_policy\": ");
                const size_t c = txt.find("\"corr_engine\": ");
                if (a != std::string::npos) mode = std::atoi(txt.c_str() + a + 16);
                if (b != std::string::npos) pol = std::atoi(txt.c_str() + b + 15);
                if (c != std::string::npos) eng = std::atoi(txt.c_str() + c + 15);
                if ((mode == MODE_STAGED || mode == MODE_FUSED) && pol >= 0 && pol <= CORR_NSHAPE &&
                    eng >= 0 && eng <= 2 && (eng == 0 || tc_range_ok(ctx))) {
                    if (pol != ctx->corr_policy) { ctx->corr_policy = pol; clear_plans(ctx); }
                    const int rc = hog_set_corr_engine(ctx, eng);
                    if (rc) return rc;
                    ctx->batched_mode = mode;
                    return HOG_OK;
                }
            }
        }
    }
    std::vector<hog_det> scratch((size_t)n_frames * ctx->p.max_dets_per_frame);
    std::vector<int32_t> counts(n_frames);
    cudaEvent_t e0, e1;
    CUDA_TRY(ctx, cudaEventCreate(&e0));
    CUDA_TRY(ctx, cudaEventCreate(&e1));
    auto timed = [&](int mode, bool graph, int reps, float *ms) -> int {
        for (int r = 0; r < 2; r++) {   // eager run, then (for graphs) capture
            int rc = detect_device(ctx, frames, n_frames, 0, scratch.data(), (int)scratch.size(), nullptr,
                                   counts.data(), stream, mode, graph);
            if (rc && rc != HOG_ECAPACITY) return rc;
        }
        CUDA_TRY(ctx, cudaEventRecord(e0, stream));
        for (int r = 0; r < reps; r++) {
            int rc = detect_device(ctx, frames, n_frames, 0, scratch.data(), (int)scratch.size(), nullptr,
                                   counts.data(), stream, mode, graph);
            if (rc && rc != HOG_ECAPACITY) return rc;
        }
        CUDA_TRY(ctx, cudaEventRecord(e1, stream));
        CUDA_TRY(ctx, cudaEventSynchronize(e1));
        CUDA_TRY(ctx, cudaEventElapsedTime(ms, e0, e1));
        *ms /= reps;
        return HOG_OK;
    };
    // 1. correlation tile-shape policy of the CUDA-core engine, then the
    //    tensor-core engine: time the correlation stage (events)
    const bool was_prof = ctx->prof;
    int rc = hog_set_corr_engine(ctx, 0);
    if (!rc) rc = hog_set_profiling(ctx, 1);
    double best_corr = 1e30;
    int best_pol = 0;
    double pol_ms[CORR_NSHAPE + 1];
    for (int pol = 0; pol <= CORR_NSHAPE && rc == HOG_OK; pol++) {
        pol_ms[pol] = -1.0;
        if (pol >= 1 && !corr_shape_ok(pol - 1)) continue;
        ctx->corr_policy = pol;
        clear_plans(ctx);
        float ms = 0.0f;
        rc = timed(MODE_STAGED, false, 1, &ms);
        hog_stage_stat st[HOG_NSTAGES];
        hog_stage_stats(ctx, st, HOG_NSTAGES, 1);
        if (rc) break;
        rc = timed(MODE_STAGED, false, 3, &ms);
        if (rc) break;
        hog_stage_stats(ctx, st, HOG_NSTAGES, 1);
        pol_ms[pol] = st[3].ms / 5.0;   // 2 warm + 3 timed calls
        if (st[3].ms < best_corr) { best_corr = st[3].ms; best_pol = pol; }
    }
    ctx->corr_policy = best_pol;
    clear_plans(ctx);
    // tensor-core engines: 2 (two passes through G), then 1 (fused)
    double tc_ms = -1.0, tc2_ms = -1.0;
    int best_engine = 0;
    for (int eng = 2; eng >= 1 && rc == HOG_OK; eng--) {
        if (hog_set_corr_engine(ctx, eng) != HOG_OK) {
            ctx->err.clear();   // no tensor-core buffers: the CUDA-core engine stays
            continue;
        }
        float ms = 0.0f;
        hog_stage_stat st[HOG_NSTAGES];
        rc = timed(MODE_STAGED, false, 1, &ms);
        hog_stage_stats(ctx, st, HOG_NSTAGES, 1);
        if (!rc) rc = timed(MODE_STAGED, false, 3, &ms);
        hog_stage_stats(ctx, st, HOG_NSTAGES, 1);
        if (rc) break;
        (eng == 1 ? tc_ms : tc2_ms) = st[3].ms / 5.0;
        if (st[3].ms < best_corr) { best_corr = st[3].ms; best_engine = eng; }
    }
    if (rc == HOG_OK && ctx->corr_engine != best_engine) rc = hog_set_corr_engine(ctx, best_engine);
    hog_set_profiling(ctx, was_prof ? 1 : 0);
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    // 2. batched execution mode (both as graphs)
    float ms_staged = 0.0f, ms_fused = 0.0f;
    rc = timed(MODE_STAGED, true, 5, &ms_staged);
    if (!rc) rc = timed(MODE_FUSED, true, 5, &ms_fused);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    ctx->batched_mode = ms_fused < ms_staged ? MODE_FUSED : MODE_STAGED;
    if (cache_path && *cache_path) {
        FILE *f = std::fopen(cache_path, "w");
        if (f) {
            std::fprintf(f, "{\n  \"key\": \"%s\",\n  \"batched_mode\": %d,\n  \"corr_policy\": %d,\n",
                         key.c_str(), ctx->batched_mode, ctx->corr_policy);
            std::fprintf(f, "  \"corr_engine\": %d,\n  \"corr_ms_tensor\": %.4f,\n", ctx->corr_engine,
                         tc_ms);
            std::fprintf(f, "  \"corr_ms_tensor_two_pass\": %.4f,\n", tc2_ms);
            std::fprintf(f, "  \"ms_per_batch\": {\"staged\": %.4f, \"fused\": %.4f},\n",
                         ms_staged, ms_fused);
            std::fprintf(f, "  \"corr_ms_by_policy\": [");
            for (int pol = 0; pol <= CORR_NSHAPE; pol++)
                std::fprintf(f, "%s%.4f", pol ? ", " : "", pol_ms[pol]);
            std::fprintf(f, "]\n}\n");
            std::fclose(f);
        }
    }
    return HOG_OK;
}

int hog_debug_waits(hog_ctx *ctx, int64_t polls, int32_t withhold) {
    if (!ctx) return HOG_EINVAL;
    if (polls < 0 || (withhold != 0 && withhold != 1))
        return fail(ctx, HOG_EINVAL, "polls must be >= 0 and withhold 0 or 1");
    clear_plans(ctx);   // plans carry the wait targets; graphs carry the budget
    ctx->wait_polls = polls == 0 ? FUSED_DEFAULT_POLLS : (long long)polls;
    ctx->wait_withhold = withhold;
    return HOG_OK;
}

int hog_get_tuning(const hog_ctx *ctx, int32_t *batched_mode, int32_t *corr_policy) {
    if (!ctx) return HOG_EINVAL;
    if (batched_mode) *batched_mode = ctx->batched_mode;
    if (corr_policy) *corr_policy = ctx->corr_policy;
    return HOG_OK;
}

int hog_backward(hog_ctx *ctx, const float *images, int32_t n, int32_t w, int32_t h,
                 const float *labels, const float *weights, float *dW, float *dI, float *loss,
                 int32_t recompute, void *stream_) {
    return hog_backward_state(ctx, images, n, w, h, labels, weights, dW, dI, loss, recompute,
                              nullptr, nullptr, nullptr, stream_);
}

int hog_backward_state(hog_ctx *ctx, const float *images, int32_t n, int32_t w, int32_t h,
                       const float *labels, const float *weights, float *dW, float *dI, float *loss,
                       int32_t recompute, int32_t *best_out, uint8_t *bins_out, uint8_t *trunc_out,
                       void *stream_) {
    if (!ctx) return HOG_EINVAL;
    if (n < 1 || !images || !labels || !weights || !dW)
        return fail(ctx, HOG_EINVAL, "hog_backward: NULL argument or n < 1");
    if (w < ctx->p.min_size || h < ctx->p.min_size || w > ctx->p.max_w || h > ctx->p.max_h)
        return fail(ctx, HOG_EINVAL, "hog_backward: crop %dx%d outside %d..%dx%d", w, h,
                    ctx->p.min_size, ctx->p.max_w, ctx->p.max_h);
    cudaStream_t stream = (cudaStream_t)stream_;
    Geometry g;
    if (compute_geometry(ctx->p, w, h, g)) return fail(ctx, HOG_EINVAL, "too many levels");
    TrainLevels lv;
    std::memset(&lv, 0, sizeof lv);
    lv.nlev = g.nlev;
    size_t pyr = 0, hist = 0, featu = 0;
    int nwin = 0;
    for (int l = 0; l < g.nlev; l++) {
        lv.w[l] = g.lw[l]; lv.h[l] = g.lh[l]; lv.cx[l] = g.cx[l]; lv.cy[l] = g.cy[l];
        lv.nu[l] = g.nu[l]; lv.nv[l] = g.nv[l];
        lv.pyr_off[l] = pyr;
        pyr += (size_t)g.lw[l] * g.lh[l];
        lv.hist_off[l] = hist;
        hist += (size_t)g.cx[l] * g.cy[l] * NBIN;
        lv.feat_off[l] = featu;
        featu += (size_t)g.cx[l] * g.cy[l] * NFEAT;
        lv.win_off[l] = nwin;
        nwin += g.nu[l] * g.nv[l];
    }
    lv.win_off[g.nlev] = nwin;
    lv.nwin = nwin;
    // per-crop slot sizes (floats), each rounded to keep 16-byte alignment
    const size_t s_pyr = align_up(pyr, 4), s_hist = align_up(hist, 4), s_featu = align_up(featu, 4);
    const size_t s_feati = g.feat_floats, s_sc = align_up((size_t)nwin, 4);
    const size_t N = (size_t)n;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_pyr = take(4 * N * s_pyr), o_dp = take(4 * N * s_pyr), o_hist = take(4 * N * s_hist);
    const size_t o_fi = take(4 * N * s_feati), o_fu = take(4 * N * s_featu), o_sc = take(4 * N * s_sc);
    const size_t o_best = take(sizeof(int4) * N), o_marg = take(4 * N), o_wch = take(4 * NCHUNK * WIN * WIN * CHUNK);
    const size_t o_descs = take(sizeof(LevelDesc) * N * g.nlev);
    std::vector<LevelDesc> descs;
    std::vector<Job> fjobs, cjobs;
    for (int i = 0; i < n; i++)
        for (int l = 0; l < g.nlev; l++) {
            const int di = (int)descs.size();
            const int nf = ((g.cx[l] + FEAT_TX - 1) / FEAT_TX) * ((g.cy[l] + FEAT_TY - 1) / FEAT_TY);
            for (int k = 0; k < nf; k++) fjobs.push_back({di, k});
            if (g.nu[l] > 0 && g.nv[l] > 0) {
                const int nc = ((g.nu[l] + corr_tu(0) - 1) / corr_tu(0)) * ((g.nv[l] + corr_tv(0) - 1) / corr_tv(0));
                for (int k = 0; k < nc; k++) cjobs.push_back({di, k});
            }
            descs.push_back(LevelDesc());
        }
    const size_t o_fj = take(sizeof(Job) * fjobs.size()), o_cj = take(sizeof(Job) * cjobs.size());
    if (off > ctx->train_cap) {
        if (ctx->d_train) { cudaStreamSynchronize(stream); cudaFree(ctx->d_train); }
        ctx->d_train = nullptr;
        ctx->train_cap = 0;
        CUDA_TRY(ctx, cudaMalloc(&ctx->d_train, off));
        ctx->train_cap = off;
    }
    char *T = ctx->d_train;
    float *d_pyr = reinterpret_cast<float *>(T + o_pyr), *d_dp = reinterpret_cast<float *>(T + o_dp);
    float *d_hist = reinterpret_cast<float *>(T + o_hist), *d_fi = reinterpret_cast<float *>(T + o_fi);
    float *d_fu = reinterpret_cast<float *>(T + o_fu), *d_sc = reinterpret_cast<float *>(T + o_sc);
    int4 *d_best = reinterpret_cast<int4 *>(T + o_best);
    float *d_marg = reinterpret_cast<float *>(T + o_marg), *d_wch = reinterpret_cast<float *>(T + o_wch);
    for (int i = 0, di = 0; i < n; i++)
        for (int l = 0; l < g.nlev; l++, di++) {
            LevelDesc &d = descs[di];
            std::memset(&d, 0, sizeof d);
            d.w = g.lw[l]; d.h = g.lh[l]; d.cx = g.cx[l]; d.cy = g.cy[l]; d.nu = g.nu[l]; d.nv = g.nv[l];
            d.frame = i; d.level = l;
            d.hist = d_hist + (size_t)i * s_hist + lv.hist_off[l];
            d.feat = d_fi + (size_t)i * s_feati + g.feat_off[l];
            d.feat_user = d_fu + (size_t)i * s_featu + lv.feat_off[l];
            d.scores_user = d_sc + (size_t)i * s_sc + lv.win_off[l];
        }
    // tables: descriptors and jobs through the pinned staging buffer
    const size_t tbytes = o_cj + sizeof(Job) * cjobs.size() - o_descs;
    int rc = ensure_plan_capacity(ctx, tbytes);
    if (rc) return rc;
    CUDA_TRY(ctx, cudaEventSynchronize(ctx->plan_done));
    std::memcpy(ctx->h_plan, descs.data(), sizeof(LevelDesc) * descs.size());
    std::memcpy(ctx->h_plan + (o_fj - o_descs), fjobs.data(), sizeof(Job) * fjobs.size());
    std::memcpy(ctx->h_plan + (o_cj - o_descs), cjobs.data(), sizeof(Job) * cjobs.size());
    CUDA_TRY(ctx, cudaMemcpyAsync(T + o_descs, ctx->h_plan, tbytes, cudaMemcpyHostToDevice, stream));
    CUDA_TRY(ctx, cudaEventRecord(ctx->plan_done, stream));
    const LevelDesc *dd = reinterpret_cast<const LevelDesc *>(T + o_descs);

    // forward: float pyramid, histograms, features, scores of the filter, best windows
    CUDA_TRY(ctx, cudaMemcpy2DAsync(d_pyr, s_pyr * 4, images, (size_t)w * h * 4, (size_t)w * h * 4, N,
                                    cudaMemcpyDeviceToDevice, stream));
    for (int l = 1; l < g.nlev; l++)
        CUDA_TRY(ctx, launch_fpyr_step(d_pyr + lv.pyr_off[l - 1], d_pyr + lv.pyr_off[l], g.lw[l - 1],
                                       g.lw[l], g.lh[l], s_pyr, n, stream));
    for (int l = 0; l < g.nlev; l++)
        CUDA_TRY(ctx, launch_fhist(d_pyr + lv.pyr_off[l], g.lw[l], g.lh[l], s_pyr, d_hist + lv.hist_off[l],
                                   s_hist, n, stream));
    CUDA_TRY(ctx, launch_feat(dd, reinterpret_cast<const Job *>(T + o_fj), (int)fjobs.size(),
                              ctx->p.eps, ctx->p.trunc, stream));
    CUDA_TRY(ctx, launch_filter_chunks(weights, d_wch, stream));
    CUDA_TRY(ctx, launch_corr(dd, reinterpret_cast<const Job *>(T + o_cj), (int)cjobs.size(), d_wch, 1, 1,
                              0.0f, stream));
    CUDA_TRY(ctx, launch_argmax(d_sc, s_sc, lv, labels, d_best, d_marg, n, stream));
    // adjoint
    CUDA_TRY(ctx, launch_dw(d_fu, s_featu, lv, d_best, d_marg, labels, n, dW, stream));
    if (dI || bins_out || trunc_out) {
        CUDA_TRY(ctx, cudaMemsetAsync(d_dp, 0, sizeof(float) * N * s_pyr, stream));
        CUDA_TRY(ctx, launch_window_adjoint(d_pyr, s_pyr, d_hist, s_hist, lv, d_best, d_marg, labels, n,
                                            weights, ctx->p.eps, ctx->p.trunc, recompute ? 1 : 0,
                                            d_dp, bins_out, trunc_out, stream));
    }
    if (dI) {
        for (int q = g.nlev - 2; q >= 0; q--)
            CUDA_TRY(ctx, launch_fpyr_adjoint(d_dp, s_pyr, lv, q, d_best, d_marg, n, stream));
        CUDA_TRY(ctx, cudaMemcpy2DAsync(dI, (size_t)w * h * 4, d_dp, s_pyr * 4, (size_t)w * h * 4, N,
                                        cudaMemcpyDeviceToDevice, stream));
    }
    if (best_out) {
        std::vector<int4> b(n);
        std::vector<float> m(n);
        CUDA_TRY(ctx, cudaMemcpyAsync(b.data(), d_best, sizeof(int4) * n, cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(m.data(), d_marg, sizeof(float) * n, cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        for (int i = 0; i < n; i++) {
            best_out[4 * i] = b[i].x;
            best_out[4 * i + 1] = b[i].y;
            best_out[4 * i + 2] = b[i].z;
            best_out[4 * i + 3] = m[i] > 0.0f;
        }
    }
    if (loss) {
        std::vector<float> m(n);
        CUDA_TRY(ctx, cudaMemcpyAsync(m.data(), d_marg, sizeof(float) * n, cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        double acc = 0.0;
        for (int i = 0; i < n; i++) acc += m[i];
        *loss = (float)(acc / n);
    }
    return HOG_OK;
}

}  // extern "C"
