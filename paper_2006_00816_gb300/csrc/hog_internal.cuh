// hog_internal.cuh -- descriptors and kernel entry points shared by the
// translation units of libhog.  Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "hog.h"

namespace hogk {

// One-time set-up per device.  A kernel's attributes (the opt-in dynamic
// shared-memory limit) belong to the function on each device, so a process
// that launches on a second GPU must set them there too.  once(f) runs f()
// the first time it is called with a given device current, and again after
// a failure; callers on several host threads (a server's worker and its
// callers) are serialised by the lock, and a finished device costs one
// atomic load.
class PerDevice {
  public:
    template <class F>
    cudaError_t once(F &&f) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return f();   // untracked: every call
        if (done_[dev].load(std::memory_order_acquire)) return cudaSuccess;
        std::lock_guard<std::mutex> lock(mu_);
        if (done_[dev].load(std::memory_order_relaxed)) return cudaSuccess;
        e = f();
        if (e == cudaSuccess) done_[dev].store(1, std::memory_order_release);
        return e;
    }

  private:
    static constexpr int kMaxDevices = 64;
    std::atomic<unsigned char> done_[kMaxDevices] = {};
    std::mutex mu_;
};

constexpr int CELL = 8;
constexpr int NBIN = 18;
constexpr int NFEAT = 31;
constexpr int WIN = 10;
constexpr int CHUNK = 8;            // channels per chunk of the internal feature layout
constexpr int NCHUNK = 4;           // 4 x 8 = 32 channels (31 + one zero pad)
constexpr int MAX_LEVELS = HOG_MAX_LEVELS;
constexpr int MAXN = 192;           // suppression neighbours per window position (<= 150 seen at IoU 0.45)
// 32-bit words of suppression workspace per window position and frame slot
// (cluster form: above-mask, list length and overflow slot, 48 listed
// neighbours; the one-CTA global-memory form uses 9 bytes of it)
#define HOG_NMS_WS_WORDS 32

// Tile shapes of the plain kernels.
constexpr int PYR_TX = 160, PYR_TY = 32;         // output pixels per CTA (256 threads x 20)
// Histogram tiles: bw x (256 / bw) blocks of 8x8 pixels (one per thread)
// emit (bw - 1) x (256 / bw - 1) cells; bw is chosen per level (hist_tile_bw).
constexpr int HIST_NT = 256;
constexpr int HIST_BW_MIN = 7, HIST_BW_MAX = 32;
__host__ __device__ constexpr int hist_bh(int bw) { return HIST_NT / bw; }
inline int hist_ntiles(int cx, int cy, int bw) {
    return ((cx + bw - 2) / (bw - 1)) * ((cy + hist_bh(bw) - 2) / (hist_bh(bw) - 1));
}
constexpr int FEAT_TX = 32, FEAT_TY = 8;         // cells per CTA (256 threads)
// Correlation warp tiles (windows): shape id 0: 8x16, 1: 4x32, 2: 16x8; the
// shape is stored in bits 28..29 of the job's tile field.
// CTAs per SM the correlation kernel is built for: 3 (all three shapes) or 4
// (shapes 8x16 and 16x8 only, smaller staging buffers).
#ifndef HOG_CORR_MINB
#define HOG_CORR_MINB 3
#endif
// Correlation accumulators: 1 = (even, odd) channel pairs updated by packed
// FP32 FMAs, 0 = one FP32 sum per window and filter (fewer registers).
#ifndef HOG_CORR_PACKED
#define HOG_CORR_PACKED 0
#endif
constexpr int CORR_NSHAPE = 3;
__host__ __device__ constexpr bool corr_shape_ok(int s) { return HOG_CORR_MINB < 4 || s != 1; }
// shapes the persistent fused launch runs (its staging buffers hold 17x25 cells)
__host__ __device__ constexpr bool corr_shape_fused(int s) { return s != 1; }
__host__ __device__ constexpr int corr_tu(int s) { return s == 0 ? 8 : (s == 1 ? 4 : 16); }
__host__ __device__ constexpr int corr_tv(int s) { return s == 0 ? 16 : (s == 1 ? 32 : 8); }
constexpr int CORR_WARPS = 4;                    // warps (independent tiles) per CTA

// A key ranks suppression candidates: smaller key = higher rank.  High word
// = score mapped to a descending unsigned order, low word = (level, filter,
// u, v) so that equal scores fall back to ascending (level, filter, u, v).
constexpr uint64_t KEY_NONE = ~0ull;

__host__ __device__ inline uint32_t float_to_ascending(float s) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(s);
#else
    uint32_t u;
    static_assert(sizeof(float) == 4, "");
    __builtin_memcpy(&u, &s, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ inline float ascending_to_float(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, 4);
    return f;
#endif
}

__host__ __device__ inline uint64_t make_key(float score, int level, int filter, int u, int v) {
    score = score + 0.0f;   // -0 -> +0: equal scores must share a key prefix
    uint32_t hi = ~float_to_ascending(score);
    uint32_t lo = ((uint32_t)level << 27) | ((uint32_t)filter << 24) |
                  ((uint32_t)u << 12) | (uint32_t)v;
    return ((uint64_t)hi << 32) | lo;
}

__host__ __device__ inline float key_score(uint64_t k) {
    return ascending_to_float(~(uint32_t)(k >> 32));
}
__host__ __device__ inline int key_level(uint64_t k) { return (int)((k >> 27) & 31); }
__host__ __device__ inline int key_filter(uint64_t k) { return (int)((k >> 24) & 7); }
__host__ __device__ inline int key_u(uint64_t k) { return (int)((k >> 12) & 4095); }
__host__ __device__ inline int key_v(uint64_t k) { return (int)(k & 4095); }

// One (frame, level) of a batch.
struct LevelDesc {
    const uint8_t *img;     // this level's image (level 0: the caller's frame)
    uint8_t *dst;           // where a pyramid job writes this level (levels >= 1)
    const uint8_t *src;     // previous level (pyramid jobs)
    int32_t w, h, pitch;    // this level
    int32_t sw, sh, spitch; // previous level
    int32_t cx, cy, nu, nv; // cells, windows
    int32_t frame, level;   // batch-relative frame index, level index
    int32_t scan;           // 1: this level takes part in detection
    int32_t dpow;           // pyramid job: 0 = 5/6 step from src; s >= 2 = direct
                            // from the frame (src) with the ratio (6/5)^s
    int32_t pos_off;        // first window position of this level in the frame
    int32_t hist_bw;        // histogram tile width in blocks (hist_tile_bw)
    float *hist;            // [cy][cx][18]
    float *feat;            // [4][cy][cx][8] internal layout
    float *feat_user;       // optional [cy][cx][31] copy (hog_features)
    float *scores_user;     // optional [F][nu][nv] (hog_scores)
    uint64_t *keys;         // [nu][nv] suppression keys of this level
    // tensor-core correlation (when enabled): features as fp16 hi + lo parts,
    // each [4 channel groups][cy*cx][8], and (two-pass form only) the
    // row-shift matrix G [10*F][cy*cx] (fp32)
    uint16_t *feat_hi, *feat_lo;
    float *gmat;
};

// Per-frame suppression work.
struct FrameDesc {
    int32_t W, H, nlev, npos;
    int32_t frame;                    // batch-relative frame index
    int32_t scan_from;                // first position of a scanned level (earlier ones: no key)
    int32_t has_roi;                  // 1: only windows in the per-level rectangles below
    int32_t roi_u0[MAX_LEVELS], roi_u1[MAX_LEVELS], roi_v0[MAX_LEVELS], roi_v1[MAX_LEVELS];
    int32_t lev_w[MAX_LEVELS], lev_h[MAX_LEVELS];
    int32_t lev_nu[MAX_LEVELS], lev_nv[MAX_LEVELS];
    int32_t lev_pos[MAX_LEVELS + 1];
    double lev_rx[MAX_LEVELS], lev_ry[MAX_LEVELS];   // W/Wl, H/Hl (FP64, host-divided)
    const uint64_t *keys;             // [npos]
    uint32_t *ws;                     // one-CTA global-memory form: workspace, 9 B per position;
                                      // cluster form: masks and lists, HOG_NMS_WS_WORDS per position
    const int32_t *nbr;               // [MAXN][npos] neighbour lists, slot-major
    const int32_t *nbr_t;             // [npos][MAXN] the same lists, position-major
    const uint8_t *nbr_cnt;           // [npos]
    uint8_t *cand;                    // [npos] 1 = scanned candidate (written by the cluster
                                      // form's pre-pass; room for the position slot)
    hog_det *out;                     // [out_cap]
    int32_t out_cap;
    int32_t *count;                   // kept count (exact)
};

struct Job {
    int32_t desc;
    int32_t tile;
};

// Geometry of one frame size for suppression: window positions of all
// levels, neighbour lists (IoU > nms_iou), built once per frame size.
struct GeomDesc {
    int32_t W, H, nlev, npos;
    double iou;
    int32_t lev_w[MAX_LEVELS], lev_h[MAX_LEVELS];
    int32_t lev_nu[MAX_LEVELS], lev_nv[MAX_LEVELS];
    int32_t lev_pos[MAX_LEVELS + 1];
    double lev_rx[MAX_LEVELS], lev_ry[MAX_LEVELS];   // W/Wl, H/Hl (FP64, host-divided)
    uint32_t pair_mask[MAX_LEVELS];   // bit m set: levels (l, m) can exceed the IoU
};

// ---- persistent fused launch (k_fused.cu) ---------------------------------
enum FusedKind : int32_t { FUSED_PYR = 0, FUSED_HIST = 1, FUSED_FEAT = 2, FUSED_CORR = 3 };

// One work item: PYR/HIST/FEAT: a = level descriptor, b = tile; CORR: a =
// first job in the correlation job list, b = number of jobs (<= 8).  The item
// starts once ctr[wait] >= target (wait < 0: no dependency) and adds 1 to
// ctr[done] when it has finished (done < 0: nothing).
struct FusedItem {
    int32_t kind, a, b, wait, target, done;
};

struct FusedArgs {
    const FusedItem *items;
    int nitems;
    const LevelDesc *descs;
    const Job *jobs;               // correlation warp-tile jobs
    const float *wchunks;
    int nf_real;
    float threshold, eps, tau;
    int *ctr;                      // completion counters (zeroed before the launch)
    int *head;                     // ticket counter (zeroed before the launch)
    int *abort;                    // set when a bounded wait gave up (zeroed before)
    int *flags;                    // flags[2] |= 1 on a timeout
    long long spin_limit;          // polls of one dependency wait before it gives up
};
constexpr long long FUSED_DEFAULT_POLLS = 1ll << 24;

cudaError_t launch_fused(const FusedArgs &a, int nf_kernel, int grid, cudaStream_t stream);
int fused_max_ctas_per_sm(int nf_kernel);

// ---- training (k_train.cu): geometry of a crop size, per-crop layouts ----
struct TrainLevels {
    int nlev, nwin;
    int w[MAX_LEVELS], h[MAX_LEVELS], cx[MAX_LEVELS], cy[MAX_LEVELS], nu[MAX_LEVELS], nv[MAX_LEVELS];
    size_t pyr_off[MAX_LEVELS];    // floats, in a crop's pyramid (and pyramid-gradient) slot
    size_t hist_off[MAX_LEVELS];   // floats, [cy][cx][18]
    size_t feat_off[MAX_LEVELS];   // floats, user layout [cy][cx][31]
    int win_off[MAX_LEVELS + 1];   // windows (one filter), [nu][nv] per level
};

cudaError_t launch_fpyr_step(const float *src, float *dst, int sw, int dw, int dh, size_t crop_stride,
                             int n, cudaStream_t s);
cudaError_t launch_fhist(const float *lvl, int w, int h, size_t crop_stride, float *hist,
                         size_t hist_stride, int n, cudaStream_t s);
cudaError_t launch_argmax(const float *scores, size_t crop_stride, const TrainLevels &lv,
                          const float *labels, int4 *best, float *margin, int n, cudaStream_t s);
cudaError_t launch_dw(const float *feat, size_t crop_stride, const TrainLevels &lv, const int4 *best,
                      const float *margin, const float *labels, int n, float *dW, cudaStream_t s);
cudaError_t launch_window_adjoint(const float *pyr, size_t pyr_stride, const float *hist,
                                  size_t hist_stride, const TrainLevels &lv, const int4 *best,
                                  const float *margin, const float *labels, int n,
                                  const float *wuser, float eps, float tau, int recompute,
                                  float *dP, uint8_t *st_bins, uint8_t *st_trunc, cudaStream_t s);
// region of the window adjoint: pixels per side of the best window's
// region (12 x 12 cells), whose bins hog_backward_state reports
constexpr int TRAIN_RP = (WIN + 2) * CELL + CELL;
cudaError_t launch_fpyr_adjoint(float *dP, size_t pyr_stride, const TrainLevels &lv, int q,
                                const int4 *best, const float *margin, int n, cudaStream_t s);
cudaError_t launch_filter_chunks(const float *wuser, float *wch, cudaStream_t s);

// Tensor-core correlation (k_corr_tc.cu): GEMM N = 10 filter rows x F
// filters padded to a multiple of 16.
__host__ __device__ constexpr int tc_n(int nf) { return (10 * nf + 15) / 16 * 16; }
// fp16 halves of the two (hi, lo) B planes for an nf_kernel-filter build
size_t corr_tc_weights_halves(int nf_kernel);
cudaError_t launch_corr_tc_weights(const float *w_user, int nf_kernel, int nf_real, uint16_t *wb,
                                   cudaStream_t stream);
// GEMM over `njobs` 128-cell tiles (Job = level descriptor, tile), then the
// row-shift reduction, threshold and keys over `nrjobs` 256-window blocks
cudaError_t launch_corr_tc(const LevelDesc *descs, const Job *jobs, int njobs, const Job *rjobs,
                           int nrjobs, const uint16_t *wb, int nf_kernel, int nf_real,
                           float threshold, int *flags, int grid, cudaStream_t stream);
int corr_tc_ctas_per_sm(int nf_kernel);

// Fused tensor-core correlation (GEMM and row-shift reduction in one
// kernel).  A band is a block of window rows [u0, u1) and window columns
// [c0, c0 + nvs) of one level; it reads cell rows [u0, u1 + 9) and cell
// columns [c0, c0 + P), P = nvs + 9 <= TCF_PMAX (P = cx: the full width).
constexpr int TCF_PMAX = 168;
struct TcBand {
    int32_t desc, u0, u1, c0, P, nvs;
};
__host__ __device__ constexpr int tcf_ring_rows(int P) { return (128 + P - 1) / P + WIN; }
__host__ __device__ constexpr int tcf_tiles(int u0, int u1, int P) {
    return ((u1 + WIN - 1 - u0) * P + 127) / 128;
}
// Bands in per-CTA order: CTA k runs bands[cta_first[k] .. cta_first[k+1]).
cudaError_t launch_corr_tcf(const LevelDesc *descs, const TcBand *bands, const int32_t *cta_first,
                            int grid, const uint16_t *wb, int nf_kernel, int nf_real,
                            float threshold, int *flags, cudaStream_t stream);

// ---- asynchronous detection for the serving runtime (hog_api.cu) ---------
int detect_enqueue(hog_ctx *ctx, const hog_frame *frames, int nb, cudaStream_t stream, int mode,
                   bool use_graph);
int detect_results(hog_ctx *ctx, const int32_t **counts, const hog_det **dets);
int ctx_max_dets(const hog_ctx *ctx);
int ctx_max_batch(const hog_ctx *ctx);
int ctx_batched_mode(const hog_ctx *ctx);
void ctx_set_plan_cache(hog_ctx *ctx, int n);
const char *ctx_error(const hog_ctx *ctx);

// ---- cp.async helpers (16-byte global -> shared copies, sm_80+) -----------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
// Copies 16 bytes when valid, else writes 16 zero bytes (gmem is not read).
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- launchers (each enqueues on `stream`; return cudaGetLastError()) ----
cudaError_t launch_pyramid(const LevelDesc *descs, const Job *jobs, int njobs,
                           cudaStream_t stream);
cudaError_t launch_pyramid_direct(const LevelDesc *descs, const Job *jobs, int njobs,
                                  cudaStream_t stream);
cudaError_t launch_hist(const LevelDesc *descs, const Job *jobs, int njobs,
                        cudaStream_t stream);
cudaError_t launch_feat(const LevelDesc *descs, const Job *jobs, int njobs, float eps,
                        float tau, cudaStream_t stream);
cudaError_t launch_corr(const LevelDesc *descs, const Job *jobs, int njobs,
                        const float *wchunks, int nf_kernel, int nf_real, float threshold,
                        cudaStream_t stream);
cudaError_t launch_nms_geometry(const GeomDesc &g, int32_t *nbr, int32_t *nbr_t, uint8_t *cnt,
                                int *overflow, cudaStream_t stream);
// Gather the kept boxes of nframes frames (slot i holds counts[i] boxes at
// dets + i*per_frame, at most per_frame) into out[0..out_cap) frame after
// frame, and copy the exact counts to counts_out; out and counts_out may be
// mapped host memory.
cudaError_t launch_pack(const hog_det *dets, int per_frame, const int32_t *counts, int nframes,
                        hog_det *out, int out_cap, int32_t *counts_out, cudaStream_t stream);

// Cluster size launch_nms uses for such a batch (1 = one CTA per frame).
int nms_cluster_size(int nframes, int max_npos, int request);

// Suppression workspace of the one-CTA form, per frame: key high words,
// which also record decisions (4 B per position), the candidate list (2 B
// per position in shared memory, 4 B in global memory), the suppression
// bitmask (1 bit) and the resume slot (1 B).  640x480 frames (9,537
// positions) take 68 KB: three CTAs per SM.
__host__ __device__ constexpr size_t nms_ws_bytes(int npos, bool in_smem) {
    return (size_t)npos * (in_smem ? 7 : 9) + 4 * (size_t)((npos + 31) / 32) + 64;
}
// Positions a shared-memory workspace can index (16-bit list entries).
constexpr int NMS_SMEM_MAX_NPOS = 65535;
constexpr int NMS_SMEM_MAX = 200 * 1024;        // all of the workspace in shared memory
constexpr int NMS_KEYS_SMEM_MAX = 226 * 1024;   // the key words alone in shared memory (227 KB less static)
// Where a frame's one-CTA suppression keeps its workspace: everything in
// shared memory (three CTAs per SM at 640x480), the key words alone in
// shared memory (the list, bitmask and resume slots in global memory; one
// CTA of 1024 threads per SM, frames up to about 57,800 positions, e.g.
// 1280x1024), or everything in global memory.
enum { NMS_WS_SMEM = 0, NMS_WS_KEYS = 1, NMS_WS_GLOBAL = 2, NMS_WS_CLASSES = 3 };
__host__ __device__ constexpr size_t nms_keys_bytes(int npos) { return 4 * (size_t)npos + 64; }
__host__ __device__ constexpr int nms_ws_class(int npos) {
    return nms_ws_bytes(npos, true) <= (size_t)NMS_SMEM_MAX && npos <= NMS_SMEM_MAX_NPOS ? NMS_WS_SMEM
           : nms_keys_bytes(npos) <= (size_t)NMS_KEYS_SMEM_MAX                          ? NMS_WS_KEYS
                                                                                         : NMS_WS_GLOBAL;
}

// Streams and events for running a batch's suppression classes side by side:
// the larger classes on side streams forked from and joined back into the
// caller's stream (also under graph capture, as parallel branches).
struct NmsStreams {
    cudaStream_t side[NMS_WS_CLASSES - 1];
    cudaEvent_t fork, join[NMS_WS_CLASSES - 1];
};
// frames: sorted by workspace class (nms_ws_class of npos); ncls[k] frames
// of class k with at most max_npos[k] positions, each class its own launch
// (concurrent through par when it is given and several classes have frames).
// flags[0] |= 1 on capacity overflow; flags[2] |= 1 if a bounded wait gave up.
cudaError_t launch_nms(const FrameDesc *frames, const int *ncls, const int *max_npos, int *flags,
                       cudaStream_t stream, int cluster_request, const NmsStreams *par = nullptr);

// Histogram tile width (blocks) for a level of cx x cy cells and height h
// pixels: the bw in [HIST_BW_MIN, HIST_BW_MAX] whose tiles issue the fewest
// warp row steps over the level, plus 3 per tile for staging, zeroing and
// the combine.  A thread runs its block's 8 pixel rows in [1, min(h - 2,
// 8 cy - 1)] if the block meets a cell of the level; a warp takes a row
// step if one of its threads does.  Tiles of one row class (first, inner,
// last tile row) and column class (inner, last) cost the same, so one
// tile of each class is counted.  Ties keep the smaller bw.
inline int hist_tile_bw(int cx, int cy, int h) {
    const int ymax = (h - 2 < CELL * cy - 1) ? h - 2 : CELL * cy - 1;
    long best_cost = -1;
    int best_bw = 16;
    for (int bw = HIST_BW_MIN; bw <= HIST_BW_MAX; bw++) {
        const int bh = hist_bh(bw), tw = bw - 1, th = bh - 1;
        const int ntx = (cx + tw - 1) / tw, nty = (cy + th - 1) / th;
        auto tile_cost = [&](int ti, int tj) {
            const int i0 = ti * th, j0 = tj * tw;
            long c = 3;
            for (int w0 = 0; w0 < HIST_NT; w0 += 32) {
                unsigned rows = 0;
                const int t1 = (w0 + 32 < bw * bh ? w0 + 32 : bw * bh) - 1;
                for (int t = w0; t <= t1; t++) {
                    const int by = t / bw, bx = t - by * bw;
                    if (i0 + by > cy || j0 + bx > cx) continue;
                    for (int oy = 0; oy < CELL; oy++) {
                        const int Y = CELL * (i0 + by) - 4 + oy;
                        if (Y >= 1 && Y <= ymax) rows |= 1u << oy;
                    }
                }
                c += __builtin_popcount(rows);
            }
            return c;
        };
        long cost = 0;
        const int ti_rep[3] = {0, 1, nty - 1};
        const long ti_mul[3] = {1, nty > 2 ? nty - 2 : 0, nty > 1 ? 1 : 0};
        for (int a = 0; a < 3; a++) {
            if (!ti_mul[a]) continue;
            if (ntx > 1) cost += ti_mul[a] * (ntx - 1) * tile_cost(ti_rep[a], 0);
            cost += ti_mul[a] * tile_cost(ti_rep[a], ntx - 1);
        }
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best_bw = bw; }
    }
    return best_bw;
}

}  // namespace hogk
