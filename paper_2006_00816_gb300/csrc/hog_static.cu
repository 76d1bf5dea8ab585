// hog_static.cu -- hog_features_static: the 31-d features of one frame
// without any device allocation.
//
// Some callers cannot allocate device memory: a frame loop with a hard
// per-frame deadline cannot afford cudaMalloc (it may block and synchronise
// the whole device), and a host application that hands all device memory to
// its own pool leaves the library no allocator to call.  hog_create
// allocates its arenas with cudaMalloc, so such callers cannot use it.  This
// entry point needs no context: its scratch (pyramid levels, cell
// histograms, internal-layout features and the launch tables) lives in the
// file-scope device array below, which every GPU that loads libhog holds
// until the process exits.  The caller still passes the frame and the output
// buffer.
//
// Limits and sharing: frames up to 640 x 480 pixels (the paper's camera
// frames); the array is 4 MiB.  Every call on a device uses the same array
// and leaves its contents behind; nothing in it needs to start at zero,
// because each call overwrites every scratch element it later reads.  Calls
// whose work overlaps on the GPU (on different streams, or from different
// threads) race on the array.  The first call on each device resolves the
// array's device address (cudaGetSymbolAddress); make that first call before
// any stream capture.  The address is kept for the life of the process, so
// a cudaDeviceReset of that device is not supported afterwards.
//
// The launch tables (level descriptors and job lists) are written into the
// array by a small kernel that receives them by value as its parameter, so
// no host memory is read after the call returns.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hog_internal.cuh"

using namespace hogk;

namespace {

constexpr int STATIC_MAX_W = 640;
constexpr int STATIC_MAX_H = 480;
constexpr size_t STATIC_SCRATCH_BYTES = size_t(4) << 20;
constexpr int STATIC_MAX_JOBS = 2048;
constexpr int STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Levels of a frame of at most 640 x 480 with min_size >= 80: 480 (5/6)^9 <
// 80, so at most 10; the table holds a few more.
constexpr int STATIC_MAX_LEVELS = 12;
constexpr int STATIC_MAX_SEGS = 3 * STATIC_MAX_LEVELS;

// Everything the launch tables hold, passed by value: the level descriptors
// and the job list as segments of consecutive tiles of one level.
struct StaticTables {
    LevelDesc descs[STATIC_MAX_LEVELS];
    int32_t nlev, nseg, njobs;
    int32_t seg_first[STATIC_MAX_SEGS];   // first job of the segment
    int32_t seg_level[STATIC_MAX_SEGS];   // its level (descriptor index)
    LevelDesc *d_descs;
    Job *d_jobs;
};
static_assert(sizeof(StaticTables) <= 4096, "kernel parameter block");

__global__ void static_tables_kernel(const StaticTables t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < t.nlev) t.d_descs[k] = t.descs[k];
    if (k >= t.njobs) return;
    int s = 0;
    while (s + 1 < t.nseg && t.seg_first[s + 1] <= k) s++;
    t.d_jobs[k] = Job{t.seg_level[s], k - t.seg_first[s]};
}

std::mutex g_static_mu;
unsigned char *g_static_addr[STATIC_MAX_DEVICES];

inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int put_error(char *err, size_t cap, int code, const char *msg) {
    if (err && cap > 0) std::snprintf(err, cap, "%s", msg);
    return code;
}

// Address of the scratch array on the current device (resolved once per device).
int scratch_address(unsigned char **out, char *err, size_t cap) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= STATIC_MAX_DEVICES)
        return put_error(err, cap, HOG_ECUDA, "hog_features_static: no usable current device");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            std::snprintf(buf, sizeof buf, "hog_features_static: cudaGetSymbolAddress: %s",
                          cudaGetErrorString(e));
            return put_error(err, cap, HOG_ECUDA, buf);
        }
        g_static_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_addr[dev];
    return HOG_OK;
}

}  // namespace

extern "C" int hog_features_static(const hog_params *p, const hog_frame *frame, float *feat_out,
                                   size_t cap_floats, hog_level *levels, int32_t cap_levels,
                                   int32_t *n_levels, char *err, size_t err_cap, void *stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!p || !frame || !n_levels)
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: NULL argument");
    if (p->cell != CELL || p->win_cells_w != WIN || p->win_cells_h != WIN || p->scale_num != 5 ||
        p->scale_den != 6 || p->min_size < CELL * WIN || !(p->eps > 0.0f) || !(p->trunc > 0.0f) ||
        p->direct_first != 0)
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: invalid parameters");
    if (frame->w < 0 || frame->h < 0 || frame->w > STATIC_MAX_W || frame->h > STATIC_MAX_H) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "hog_features_static: frame %dx%d exceeds the static limit %dx%d",
                      frame->w, frame->h, STATIC_MAX_W, STATIC_MAX_H);
        return put_error(err, err_cap, HOG_EINVAL, buf);
    }
    if (frame->w > 0 && frame->h > 0 && (!frame->data || frame->pitch < frame->w))
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: bad frame data or pitch");

    // level geometry: w' = floor(5w/6), h' = floor(5h/6), while min(w, h) >= min_size
    int lw[STATIC_MAX_LEVELS], lh[STATIC_MAX_LEVELS], L = 0;
    for (int w = frame->w, h = frame->h; w >= p->min_size && h >= p->min_size;
         w = 5 * w / 6, h = 5 * h / 6) {
        if (L >= STATIC_MAX_LEVELS) return put_error(err, err_cap, HOG_EINVAL, "too many levels");
        lw[L] = w;
        lh[L] = h;
        L++;
    }
    *n_levels = L;
    if (L > cap_levels || (L > 0 && !levels))
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: level capacity too small");
    size_t uoff = 0;
    for (int l = 0; l < L; l++) {
        levels[l] = hog_level{lw[l], lh[l], lw[l] / CELL, lh[l] / CELL, (int64_t)uoff};
        uoff += (size_t)(lw[l] / CELL) * (lh[l] / CELL) * NFEAT;
    }
    if (L == 0) return HOG_OK;
    if (!feat_out || uoff > cap_floats)
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: output capacity too small");

    // scratch layout: [descs][jobs][pyramid][hist][feat]
    const size_t off_desc = 0;
    const size_t off_jobs = up(sizeof(LevelDesc) * STATIC_MAX_LEVELS, 256);
    size_t off = up(off_jobs + sizeof(Job) * STATIC_MAX_JOBS, 256);
    size_t pyr_off[STATIC_MAX_LEVELS], hist_off[STATIC_MAX_LEVELS], feat_off[STATIC_MAX_LEVELS];
    for (int l = 1; l < L; l++) {
        pyr_off[l] = off;
        off = up(off + up((size_t)lw[l], 16) * lh[l], 256);
    }
    for (int l = 0; l < L; l++) {
        hist_off[l] = off;
        off = up(off + sizeof(float) * (size_t)(lw[l] / CELL) * (lh[l] / CELL) * NBIN, 256);
    }
    for (int l = 0; l < L; l++) {
        feat_off[l] = off;
        off = up(off + sizeof(float) * (size_t)(lw[l] / CELL) * (lh[l] / CELL) * CHUNK * NCHUNK, 256);
    }
    if (off > STATIC_SCRATCH_BYTES)
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: scratch too small");

    // job segments: pyramid levels 1..L-1, then histogram and feature tiles of every level
    StaticTables t;
    std::memset(&t, 0, sizeof t);
    int nj = 0, pyr_beg[STATIC_MAX_LEVELS], pyr_n[STATIC_MAX_LEVELS];
    auto segment = [&](int l, int ntiles) {
        t.seg_first[t.nseg] = nj;
        t.seg_level[t.nseg] = l;
        t.nseg++;
        nj += ntiles;
    };
    for (int l = 1; l < L; l++) {
        pyr_beg[l] = nj;
        pyr_n[l] = ((lw[l] + PYR_TX - 1) / PYR_TX) * ((lh[l] + PYR_TY - 1) / PYR_TY);
        segment(l, pyr_n[l]);
    }
    const int hist_beg = nj;
    for (int l = 0; l < L; l++)
        segment(l, hist_ntiles(lw[l] / CELL, lh[l] / CELL, hist_tile_bw(lw[l] / CELL, lh[l] / CELL, lh[l])));
    const int feat_beg = nj;
    for (int l = 0; l < L; l++)
        segment(l, ((lw[l] / CELL + FEAT_TX - 1) / FEAT_TX) * ((lh[l] / CELL + FEAT_TY - 1) / FEAT_TY));
    if (nj > STATIC_MAX_JOBS)
        return put_error(err, err_cap, HOG_EINVAL, "hog_features_static: job table too small");

    unsigned char *base = nullptr;
    int rc = scratch_address(&base, err, err_cap);
    if (rc) return rc;

    for (int l = 0; l < L; l++) {
        LevelDesc &d = t.descs[l];
        d.w = lw[l];
        d.h = lh[l];
        d.cx = lw[l] / CELL;
        d.cy = lh[l] / CELL;
        d.hist_bw = hist_tile_bw(d.cx, d.cy, d.h);
        d.level = l;
        if (l == 0) {
            d.img = frame->data;
            d.pitch = frame->pitch;
        } else {
            d.dst = base + pyr_off[l];
            d.img = d.dst;
            d.pitch = (int)up((size_t)lw[l], 16);
            d.src = t.descs[l - 1].img;
            d.sw = t.descs[l - 1].w;
            d.sh = t.descs[l - 1].h;
            d.spitch = t.descs[l - 1].pitch;
        }
        d.hist = reinterpret_cast<float *>(base + hist_off[l]);
        d.feat = reinterpret_cast<float *>(base + feat_off[l]);
        d.feat_user = feat_out + levels[l].offset;
    }
    LevelDesc *d_descs = reinterpret_cast<LevelDesc *>(base + off_desc);
    Job *d_jobs = reinterpret_cast<Job *>(base + off_jobs);
    t.nlev = L;
    t.njobs = nj;
    t.d_descs = d_descs;
    t.d_jobs = d_jobs;

    static_tables_kernel<<<(nj + 255) / 256, 256, 0, stream>>>(t);
    cudaError_t e = cudaGetLastError();
    for (int l = 1; l < L && e == cudaSuccess; l++)
        e = launch_pyramid(d_descs, d_jobs + pyr_beg[l], pyr_n[l], stream);
    if (e == cudaSuccess) e = launch_hist(d_descs, d_jobs + hist_beg, feat_beg - hist_beg, stream);
    if (e == cudaSuccess)
        e = launch_feat(d_descs, d_jobs + feat_beg, nj - feat_beg, p->eps, p->trunc, stream);
    if (e != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "hog_features_static: %s", cudaGetErrorString(e));
        return put_error(err, err_cap, HOG_ECUDA, buf);
    }
    return HOG_OK;
}
