// hog_server.cu -- continuous-batching request loop for camera streams.
//
// The paper processes recorded videos in fixed groups of 16 frames and
// names online processing of camera batches as future work (Section 6.6);
// its real-time target is 500 frames/s per camera.  This runtime serves
// frames as they arrive from several cameras:
//   - hog_server_submit copies a frame into a pinned host slot (the queue
//     holds queue_cap frames; a full queue refuses with HOG_EBUSY);
//   - a worker thread forms a batch whenever a lane is free: the oldest
//     waiting frame and the other waiting frames of its size, copied to
//     that lane's device frame slots, detection enqueued on the lane's
//     stream; several lanes (each a context with its own arenas and
//     stream) keep batches in flight at once, so requests that arrive while others are on the GPU join the
//     next batch and their work overlaps on the device;
//   - completion is signalled by a host callback on the lane's stream; the
//     worker moves the lane's results to the completed queue, frees the
//     slots, and the lane takes the next batch;
//   - lanes belong to size classes (arenas sized for the camera mix, not
//     all for the largest frame) and are created at start-up only while
//     free device memory stays above mem_reserve bytes (admission by
//     memory): the number of frames in flight is what the device can hold;
//   - a waiting frame is admitted to a free lane of the smallest class that
//     holds it; a lane of a larger class takes it only while no waiting frame
//     needs that class, so small frames are admitted while large ones wait.
// Each result is bit-identical to hog_detect on the same frame alone: the
// kernels are deterministic and frames of a batch never interact.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hog_internal.cuh"

using namespace hogk;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id;
    int64_t tag;
    int w, h, slot;
    double t_submit, t_dispatch;
};

struct Result {
    hog_result r;
    std::vector<hog_det> dets;
};

struct Lane {
    hog_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    uint8_t *d_frames = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int index = 0;
    int cls = 0, cw = 0, ch = 0;   // size class and the largest frame it holds
    std::vector<Request> batch;
    bool busy = false;
    volatile bool completed = false;
    struct hog_server *srv = nullptr;
};

}  // namespace

struct hog_server {
    hog_server_config cfg;
    hog_params p;
    size_t fbytes = 0;
    std::vector<Lane *> lanes;
    uint8_t *h_slots = nullptr;
    std::vector<int> free_slots;
    std::deque<Request> pending;
    std::deque<Result> done;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    hog_server_stats st = {};
    std::string err;
    int mode = 0;
    int ncls = 1;
    int cls_w[HOG_SERVER_CLASSES] = {}, cls_h[HOG_SERVER_CLASSES] = {};   // by increasing area
};

namespace {

thread_local std::string g_server_error;

void CUDART_CB lane_done(void *arg) {
    Lane *ln = static_cast<Lane *>(arg);
    hog_server *s = ln->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        ln->completed = true;
    }
    s->cv_work.notify_one();
}

void harvest(hog_server *s, Lane *ln) {
    const int32_t *counts = nullptr;
    const hog_det *dets = nullptr;
    const int rc = detect_results(ln->ctx, &counts, &dets);
    const double t = now_ms();
    const int maxd = ctx_max_dets(ln->ctx);
    float dev_ms = 0.f;
    if (cudaEventElapsedTime(&dev_ms, ln->ev0, ln->ev1) != cudaSuccess) {
        cudaGetLastError();
        dev_ms = 0.f;
    }
    std::vector<Result> out;
    out.reserve(ln->batch.size());
    size_t off = 0;
    for (size_t k = 0; k < ln->batch.size(); k++) {
        const Request &q = ln->batch[k];
        Result r;
        r.r.id = q.id;
        r.r.tag = q.tag;
        r.r.status = rc;
        r.r.count = rc ? 0 : counts[k];
        const int stored = rc ? 0 : std::min(counts[k], maxd);
        r.r.latency_ms = t - q.t_submit;
        r.r.queue_ms = q.t_dispatch - q.t_submit;
        r.r.device_ms = dev_ms;
        r.r.batch = (int32_t)ln->batch.size();
        r.r.lane = ln->index;
        r.r.lane_class = ln->cls;
        if (stored > 0) {
            r.dets.assign(dets + off, dets + off + stored);
            for (auto &d : r.dets) d.frame = 0;
        }
        r.r.stored = stored;
        off += (size_t)stored;
        out.push_back(std::move(r));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &r : out) {
        s->done.push_back(std::move(r));
        s->st.completed++;
        if (s->done.back().r.status) s->st.failed++;
    }
    for (const Request &q : ln->batch) s->free_slots.push_back(q.slot);
    ln->batch.clear();
    ln->busy = false;
    ln->completed = false;
    s->cv_done.notify_all();
}

void dispatch(hog_server *s, Lane *ln, std::vector<Request> &&batch) {
    const int nb = (int)batch.size();
    std::vector<hog_frame> frames(nb);
    const double t = now_ms();
    cudaError_t e = cudaEventRecord(ln->ev0, ln->stream);
    for (int k = 0; k < nb; k++) {
        Request &q = batch[k];
        q.t_dispatch = t;
        uint8_t *dst = ln->d_frames + (size_t)k * ln->cw * ln->ch;
        const uint8_t *src = s->h_slots + (size_t)q.slot * s->fbytes;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst, src, (size_t)q.w * q.h, cudaMemcpyHostToDevice, ln->stream);
        frames[k] = hog_frame{dst, q.w, q.h, q.w};
    }
    ln->batch = std::move(batch);
    ln->busy = true;
    int rc = e == cudaSuccess ? HOG_OK : HOG_ECUDA;
    if (!rc) rc = detect_enqueue(ln->ctx, frames.data(), nb, ln->stream, s->mode, true);
    if (!rc && cudaEventRecord(ln->ev1, ln->stream) != cudaSuccess) rc = HOG_ECUDA;
    if (!rc && cudaLaunchHostFunc(ln->stream, lane_done, ln) != cudaSuccess) rc = HOG_ECUDA;
    if (rc) {   // report the failure on every request of the batch
        cudaStreamSynchronize(ln->stream);
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Request &q : ln->batch) {
            Result r;
            std::memset(&r.r, 0, sizeof r.r);
            r.r.id = q.id;
            r.r.tag = q.tag;
            r.r.status = rc;
            r.r.latency_ms = now_ms() - q.t_submit;
            r.r.batch = (int32_t)ln->batch.size();
            r.r.lane = ln->index;
            s->done.push_back(std::move(r));
            s->st.completed++;
            s->st.failed++;
            s->free_slots.push_back(q.slot);
        }
        s->err = ctx_error(ln->ctx);
        ln->batch.clear();
        ln->busy = false;
        s->cv_done.notify_all();
        return;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.batches++;
    s->st.batched_frames += nb;
    s->st.class_frames[ln->cls] += nb;
}

// Smallest class that holds a w x h frame (ncls if none).
int class_of(const hog_server *s, int w, int h) {
    for (int k = 0; k < s->ncls; k++)
        if (w <= s->cls_w[k] && h <= s->cls_h[k]) return k;
    return s->ncls;
}

void worker_loop(hog_server *s) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completed lanes first
        for (Lane *ln : s->lanes)
            if (ln->busy && ln->completed) {
                lk.unlock();
                harvest(s, ln);
                lk.lock();
            }
        // admission: the waiting frame sizes in order of their oldest
        // request; the first size with a free lane it may use forms a batch.
        // A size uses the smallest free lane class that holds it, and a
        // larger class only while no waiting frame needs that class.
        Lane *free_lane = nullptr;
        int bw = 0, bh = 0;
        if (!s->pending.empty()) {
            bool wanted[HOG_SERVER_CLASSES + 1] = {};
            for (const Request &q : s->pending) wanted[class_of(s, q.w, q.h)] = true;
            std::vector<std::pair<int, int>> sizes;
            for (const Request &q : s->pending) {
                bool seen = false;
                for (auto &z : sizes) seen |= z.first == q.w && z.second == q.h;
                if (!seen) sizes.push_back({q.w, q.h});
            }
            for (auto &z : sizes) {
                const int c0 = class_of(s, z.first, z.second);
                for (int c = c0; c < s->ncls && !free_lane; c++) {
                    if (c > c0 && wanted[c]) break;   // that class is needed by its own frames
                    for (Lane *ln : s->lanes)
                        if (!ln->busy && ln->cls == c) { free_lane = ln; break; }
                }
                if (free_lane) { bw = z.first; bh = z.second; break; }
            }
        }
        if (free_lane) {
            // the waiting requests of that frame size, in arrival order: one
            // size per batch, so a lane's cached plans and graphs stay few
            // (size x count) and small frames never wait for a large frame's
            // suppression in the same batch
            std::vector<Request> batch;
            for (auto it = s->pending.begin();
                 it != s->pending.end() && (int)batch.size() < s->cfg.max_batch;) {
                if (it->w == bw && it->h == bh) {
                    batch.push_back(*it);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
            int inflight = 0;
            for (Lane *ln : s->lanes) inflight += ln->busy ? (int)ln->batch.size() : 0;
            s->st.max_inflight = std::max<int64_t>(s->st.max_inflight, inflight + (int64_t)batch.size());
            lk.unlock();
            dispatch(s, free_lane, std::move(batch));
            lk.lock();
            continue;
        }
        bool any_busy = false;
        for (Lane *ln : s->lanes) any_busy |= ln->busy;
        if (s->stop && !any_busy && s->pending.empty()) break;
        s->cv_work.wait(lk);
    }
}

int validate(const hog_server_config *c, std::string &why) {
    if (!c) { why = "config is NULL"; return HOG_EINVAL; }
    if (c->max_batch < 1 || c->max_batch > 1024) { why = "max_batch out of 1..1024"; return HOG_EINVAL; }
    int classed = 0;
    for (int k = 0; k < HOG_SERVER_CLASSES; k++) {
        if (c->class_lanes[k] < 0) { why = "class_lanes < 0"; return HOG_EINVAL; }
        classed += c->class_lanes[k];
        if (c->class_lanes[k] > 0 && (c->class_w[k] < 1 || c->class_h[k] < 1)) {
            why = "a lane class needs a frame size";
            return HOG_EINVAL;
        }
    }
    if (classed > 16) { why = "more than 16 lanes over the classes"; return HOG_EINVAL; }
    if (!classed && (c->max_lanes < 1 || c->max_lanes > 16)) { why = "max_lanes out of 1..16"; return HOG_EINVAL; }
    if (c->queue_cap < c->max_batch) { why = "queue_cap < max_batch"; return HOG_EINVAL; }
    if (c->batched_mode < -1 || c->batched_mode > 1) { why = "batched_mode out of -1..1"; return HOG_EINVAL; }
    if (c->mem_reserve < 0) { why = "mem_reserve < 0"; return HOG_EINVAL; }
    return HOG_OK;
}

void destroy_server(hog_server *s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    for (Lane *ln : s->lanes) {
        if (ln->stream) cudaStreamSynchronize(ln->stream);
        if (ln->d_frames) cudaFree(ln->d_frames);
        if (ln->ev0) cudaEventDestroy(ln->ev0);
        if (ln->ev1) cudaEventDestroy(ln->ev1);
        if (ln->stream) cudaStreamDestroy(ln->stream);
        hog_destroy(ln->ctx);
        delete ln;
    }
    if (s->h_slots) cudaFreeHost(s->h_slots);
    delete s;
}

}  // namespace

extern "C" {

void hog_default_server_config(hog_server_config *c) {
    if (!c) return;
    c->max_batch = 8;
    c->max_lanes = 3;
    c->queue_cap = 64;
    c->batched_mode = -1;
    c->mem_reserve = (int64_t)1 << 30;
    for (int k = 0; k < HOG_SERVER_CLASSES; k++) c->class_w[k] = c->class_h[k] = c->class_lanes[k] = 0;
}

int hog_server_create(const hog_params *p, const float *filters_host, int32_t n_filters,
                      const hog_server_config *cfg, hog_server **out) {
    if (!out) return HOG_EINVAL;
    *out = nullptr;
    std::string why;
    if (validate(cfg, why)) { g_server_error = why; return HOG_EINVAL; }
    if (!p) { g_server_error = "params is NULL"; return HOG_EINVAL; }
    hog_server *s = new hog_server();
    s->cfg = *cfg;
    s->p = *p;
    s->p.max_batch = cfg->max_batch;
    s->fbytes = (size_t)p->max_w * p->max_h;
    // lane classes by increasing area (one class of the largest frame when
    // none is configured); some class must hold p->max_w x p->max_h
    struct Cls { int w, h, lanes; };
    std::vector<Cls> cls;
    for (int k = 0; k < HOG_SERVER_CLASSES; k++)
        if (cfg->class_lanes[k] > 0)
            cls.push_back({std::min(cfg->class_w[k], p->max_w), std::min(cfg->class_h[k], p->max_h),
                           cfg->class_lanes[k]});
    if (cls.empty()) cls.push_back({p->max_w, p->max_h, cfg->max_lanes});
    std::stable_sort(cls.begin(), cls.end(),
                     [](const Cls &a, const Cls &b) { return (int64_t)a.w * a.h < (int64_t)b.w * b.h; });
    bool covers = false;
    for (const Cls &c : cls) covers |= c.w >= p->max_w && c.h >= p->max_h;
    if (!covers) {
        g_server_error = "no lane class holds max_w x max_h";
        delete s;
        return HOG_EINVAL;
    }
    s->ncls = (int)cls.size();
    for (int k = 0; k < s->ncls; k++) { s->cls_w[k] = cls[k].w; s->cls_h[k] = cls[k].h; }
    int index = 0;
    for (int k = 0; k < s->ncls; k++) {
        for (int j = 0; j < cls[k].lanes; j++) {
            size_t free0 = 0, total = 0;
            cudaMemGetInfo(&free0, &total);
            // each lane after the very first: only while free memory minus the
            // measured size of a lane of its class stays above the reserve
            // (a class's first lane is estimated by the largest class measured)
            int64_t est = s->st.class_bytes[k];
            for (int m = 0; m < k && !est; m++) est = std::max(est, s->st.class_bytes[m]);
            if (index > 0 && (int64_t)free0 - est < cfg->mem_reserve) break;
            Lane *ln = new Lane();
            ln->srv = s;
            hog_params lp = s->p;
            lp.max_w = cls[k].w;
            lp.max_h = cls[k].h;
            int rc = hog_create(&lp, filters_host, n_filters, &ln->ctx);
            if (rc) {
                g_server_error = hog_last_error(nullptr);
                delete ln;
                if (index == 0) { destroy_server(s); return rc; }
                break;
            }
            ctx_set_plan_cache(ln->ctx, 64);
            if (cfg->batched_mode >= 0) hog_set_batched_mode(ln->ctx, cfg->batched_mode);
            ln->index = index;
            ln->cls = k;
            ln->cw = cls[k].w;
            ln->ch = cls[k].h;
            const size_t fb = (size_t)cls[k].w * cls[k].h;
            if (cudaStreamCreateWithFlags(&ln->stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreate(&ln->ev0) != cudaSuccess || cudaEventCreate(&ln->ev1) != cudaSuccess ||
                cudaMalloc(&ln->d_frames, fb * cfg->max_batch) != cudaSuccess) {
                cudaGetLastError();
                hog_destroy(ln->ctx);
                if (ln->stream) cudaStreamDestroy(ln->stream);
                if (ln->ev0) cudaEventDestroy(ln->ev0);
                if (ln->ev1) cudaEventDestroy(ln->ev1);
                delete ln;
                if (index == 0) { g_server_error = "lane allocation failed"; destroy_server(s); return HOG_ENOMEM; }
                break;
            }
            s->lanes.push_back(ln);
            index++;
            s->st.class_lanes[k]++;
            if (!s->st.class_bytes[k]) {
                size_t free1 = 0;
                cudaMemGetInfo(&free1, &total);
                s->st.class_bytes[k] = free0 > free1 ? (int64_t)(free0 - free1) : 0;
                if (index == 1) s->st.lane_bytes = s->st.class_bytes[k];
            }
        }
    }
    if (!s->st.class_lanes[s->ncls - 1]) {
        g_server_error = "no lane of the largest class fits in device memory";
        destroy_server(s);
        return HOG_ENOMEM;
    }
    s->st.lanes = (int64_t)s->lanes.size();
    s->mode = ctx_batched_mode(s->lanes[0]->ctx);
    if (cudaMallocHost(&s->h_slots, s->fbytes * cfg->queue_cap) != cudaSuccess) {
        cudaGetLastError();
        g_server_error = "pinned slot allocation failed";
        destroy_server(s);
        return HOG_ENOMEM;
    }
    for (int k = cfg->queue_cap - 1; k >= 0; k--) s->free_slots.push_back(k);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return HOG_OK;
}

int hog_server_submit(hog_server *s, const uint8_t *frame, int32_t w, int32_t h, int32_t pitch,
                      int64_t tag, uint64_t *id_out) {
    if (!s || !frame || w < 0 || h < 0 || w > s->p.max_w || h > s->p.max_h || pitch < w)
        return HOG_EINVAL;
    const double t0 = now_ms();
    int slot;
    uint64_t id;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return HOG_EINVAL;
        if (s->free_slots.empty()) {
            s->st.rejected++;
            return HOG_EBUSY;
        }
        slot = s->free_slots.back();
        s->free_slots.pop_back();
        id = s->next_id++;
    }
    uint8_t *dst = s->h_slots + (size_t)slot * s->fbytes;
    for (int y = 0; y < h; y++) std::memcpy(dst + (size_t)y * w, frame + (size_t)y * pitch, (size_t)w);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->pending.push_back(Request{id, tag, w, h, slot, t0, 0.0});
        s->st.submitted++;
    }
    s->cv_work.notify_one();
    if (id_out) *id_out = id;
    return HOG_OK;
}

int hog_server_poll(hog_server *s, hog_result *res, int32_t cap, hog_det *dets, int32_t det_cap,
                    int32_t *n_out, int32_t wait_us) {
    if (!s || !n_out || (cap > 0 && !res) || det_cap < 0) return HOG_EINVAL;
    *n_out = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !s->done.empty(); });
    int n = 0, used = 0;
    while (n < cap && !s->done.empty()) {
        Result &r = s->done.front();
        const int room = dets ? std::max(det_cap - used, 0) : 0;
        const int take = std::min(r.r.stored, room);
        if (take > 0) std::memcpy(dets + used, r.dets.data(), sizeof(hog_det) * take);
        res[n] = r.r;
        res[n].stored = take;
        used += take;
        n++;
        s->done.pop_front();
    }
    *n_out = n;
    return HOG_OK;
}

int hog_server_get_stats(hog_server *s, hog_server_stats *out) {
    if (!s || !out) return HOG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->pending = (int64_t)s->pending.size();
    return HOG_OK;
}

void hog_server_destroy(hog_server *s) { destroy_server(s); }

const char *hog_server_last_error(const hog_server *s) {
    return s ? s->err.c_str() : g_server_error.c_str();
}

}  // extern "C"
