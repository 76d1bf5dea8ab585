// hog_pipeline.cu -- face detection on the GPU pipelined with a host
// landmark stage (Section 5.2: the landmark detector runs on the CPU, one
// OpenMP thread per image; Section 5.3 / Table 8: detecting the next images
// on the GPU while the CPU fits landmarks to the current ones).
//
// The paper's landmark stage is an ensemble of regression trees (Section
// 4.2) trained on 300-W; no trained model is available here, so the host
// stage is a stand-in with the same structure and cost model: a cascade of
// levels, each sampling feature pixels at offsets from the current shape's
// landmarks, and a forest of depth-D trees whose splits compare two feature
// pixels' difference with a threshold and whose leaves add a shape
// increment.  Its parameters are drawn from a seed (splitmix64), so its
// landmarks carry no meaning; it exists to load the host like the real
// stage and to show the overlap.  From the six landmarks of each eye it
// computes the eye aspect ratio (EAR), the eyelid-closure signal of the
// eyeblink use case.
//
// hog_pipeline_run: frames in host memory, in batches.  Sequential: copy a
// batch in, detect, wait, fit landmarks on all frames of the batch (host
// threads), next batch.  Pipelined: the detection of batch k+1 is enqueued
// before the host threads fit batch k, and waited for afterwards, so the
// two overlap.  Both orders give the same landmarks, bit for bit.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "hog_internal.cuh"

using namespace hogk;

struct hog_ert {
    hog_ert_params p;
    std::vector<float> mean;        // [L][2], unit box
    std::vector<int32_t> anchor;    // [T][P] landmark index of each feature pixel
    std::vector<float> offset;      // [T][P][2], in box units
    std::vector<int32_t> split;     // [T][K][nodes][2] feature pair
    std::vector<float> thresh;      // [T][K][nodes]
    std::vector<float> leaf;        // [T][K][leaves][L][2], in box units
};

namespace {

struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }   // [0, 1)
    int below(int n) { return (int)(uniform() * n); }
};

constexpr int EYE_R = 36, EYE_L = 42;   // first landmark of each eye (68-point layout)

// Eye aspect ratio of landmarks e[0..5]: (|p2 - p6| + |p3 - p5|) / (2 |p1 - p4|).
float eye_aspect(const float *s, int first) {
    auto d = [&](int a, int b) {
        const float dx = s[2 * (first + a)] - s[2 * (first + b)];
        const float dy = s[2 * (first + a) + 1] - s[2 * (first + b) + 1];
        return std::sqrt(dx * dx + dy * dy);
    };
    const float w = d(0, 3);
    return w > 0.0f ? (d(1, 5) + d(2, 4)) / (2.0f * w) : 0.0f;
}

}  // namespace

extern "C" {

void hog_default_ert_params(hog_ert_params *p) {
    if (!p) return;
    p->landmarks = 68;
    p->cascades = 15;
    p->trees = 500;
    p->depth = 4;
    p->features = 400;
    p->seed = 20060816ull;
}

int hog_ert_create(const hog_ert_params *p, hog_ert **out) {
    if (!p || !out) return HOG_EINVAL;
    *out = nullptr;
    if (p->landmarks != 68 || p->cascades < 1 || p->cascades > 64 || p->trees < 1 || p->trees > 4096 ||
        p->depth < 1 || p->depth > 8 || p->features < 2 || p->features > 4096)
        return HOG_EINVAL;
    hog_ert *m = new (std::nothrow) hog_ert();
    if (!m) return HOG_ENOMEM;
    m->p = *p;
    const int L = p->landmarks, T = p->cascades, K = p->trees, P = p->features;
    const int nodes = (1 << p->depth) - 1, leaves = 1 << p->depth;
    SplitMix r{p->seed};
    try {
        m->mean.resize((size_t)L * 2);
        for (int l = 0; l < L; l++) {
            m->mean[2 * l] = (float)(0.15 + 0.7 * r.uniform());
            m->mean[2 * l + 1] = (float)(0.15 + 0.7 * r.uniform());
        }
        // the two eyes: hexagons at eye height (corner, two upper, corner,
        // two lower points in the 68-point order), mean EAR 0.3
        for (int e = 0; e < 2; e++) {
            const float cx = e == 0 ? 0.3f : 0.7f, cy = 0.38f, rx = 0.08f, ry = 0.024f;
            const float px[6] = {-1.0f, -0.5f, 0.5f, 1.0f, 0.5f, -0.5f};
            const float py[6] = {0.0f, -1.0f, -1.0f, 0.0f, 1.0f, 1.0f};
            for (int k = 0; k < 6; k++) {
                m->mean[2 * ((e == 0 ? EYE_R : EYE_L) + k)] = cx + rx * px[k];
                m->mean[2 * ((e == 0 ? EYE_R : EYE_L) + k) + 1] = cy + ry * py[k];
            }
        }
        m->anchor.resize((size_t)T * P);
        m->offset.resize((size_t)T * P * 2);
        for (int i = 0; i < T * P; i++) {
            m->anchor[i] = r.below(L);
            m->offset[2 * (size_t)i] = (float)(0.2 * r.uniform() - 0.1);
            m->offset[2 * (size_t)i + 1] = (float)(0.2 * r.uniform() - 0.1);
        }
        m->split.resize((size_t)T * K * nodes * 2);
        m->thresh.resize((size_t)T * K * nodes);
        for (size_t i = 0; i < (size_t)T * K * nodes; i++) {
            m->split[2 * i] = r.below(P);
            m->split[2 * i + 1] = r.below(P);
            m->thresh[i] = (float)(60.0 * r.uniform() - 30.0);
        }
        m->leaf.resize((size_t)T * K * leaves * L * 2);
        for (auto &x : m->leaf) x = (float)(0.001 * r.uniform() - 0.0005);
    } catch (const std::bad_alloc &) {
        delete m;
        return HOG_ENOMEM;
    }
    *out = m;
    return HOG_OK;
}

void hog_ert_destroy(hog_ert *m) { delete m; }

int hog_ert_fit(const hog_ert *m, const uint8_t *img, int32_t w, int32_t h, int32_t pitch,
                const hog_det *box, float *landmarks, float *ear) {
    if (!m || !img || !box || !landmarks || w < 1 || h < 1 || pitch < w) return HOG_EINVAL;
    const int L = m->p.landmarks, T = m->p.cascades, K = m->p.trees, P = m->p.features, D = m->p.depth;
    const int nodes = (1 << D) - 1, leaves = 1 << D;
    const float bx = (float)box->x, by = (float)box->y, bw = (float)box->w, bh = (float)box->h;
    float *s = landmarks;
    for (int l = 0; l < L; l++) {
        s[2 * l] = bx + bw * m->mean[2 * l];
        s[2 * l + 1] = by + bh * m->mean[2 * l + 1];
    }
    std::vector<float> px((size_t)P);
    for (int t = 0; t < T; t++) {
        // feature pixels at offsets from the current landmarks (nearest pixel,
        // clamped to the frame)
        const int32_t *an = &m->anchor[(size_t)t * P];
        const float *of = &m->offset[(size_t)t * P * 2];
        for (int i = 0; i < P; i++) {
            const float x = s[2 * an[i]] + bw * of[2 * i], y = s[2 * an[i] + 1] + bh * of[2 * i + 1];
            const int xi = std::min(std::max((int)std::lround(x), 0), w - 1);
            const int yi = std::min(std::max((int)std::lround(y), 0), h - 1);
            px[i] = (float)img[(size_t)yi * pitch + xi];
        }
        for (int k = 0; k < K; k++) {
            const size_t tree = (size_t)t * K + k;
            const int32_t *sp = &m->split[tree * nodes * 2];
            const float *th = &m->thresh[tree * nodes];
            int n = 0;
            for (int d = 0; d < D; d++)
                n = 2 * n + 1 + (px[sp[2 * n]] - px[sp[2 * n + 1]] > th[n] ? 1 : 0);
            const float *lf = &m->leaf[(tree * leaves + (n - nodes)) * L * 2];
            for (int l = 0; l < L; l++) {
                s[2 * l] += bw * lf[2 * l];
                s[2 * l + 1] += bh * lf[2 * l + 1];
            }
        }
    }
    if (ear) {
        ear[0] = eye_aspect(s, EYE_R);
        ear[1] = eye_aspect(s, EYE_L);
    }
    return HOG_OK;
}

int hog_pipeline_run(hog_ctx *ctx, const hog_ert *m, const hog_frame *frames, int32_t n_frames,
                     int32_t batch, int32_t n_threads, int32_t pipelined, float *landmarks, float *ear,
                     int32_t *has_face, double *seconds, void *stream_) {
    if (!ctx || !m || (n_frames > 0 && (!frames || !landmarks || !ear || !has_face)) || n_frames < 0 ||
        batch < 1 || batch > ctx_max_batch(ctx) || n_threads < 1 || n_threads > 1024)
        return HOG_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    const int L = m->p.landmarks;
    int maxw = 0, maxh = 0;
    for (int i = 0; i < n_frames; i++) {
        if (!frames[i].data || frames[i].w < 1 || frames[i].h < 1 || frames[i].pitch < frames[i].w)
            return HOG_EINVAL;
        maxw = std::max(maxw, frames[i].w);
        maxh = std::max(maxh, frames[i].h);
    }
    const size_t fbytes = (size_t)maxw * maxh;
    uint8_t *d_frames = nullptr;
    if (n_frames > 0 && cudaMalloc(&d_frames, fbytes * batch) != cudaSuccess) {
        cudaGetLastError();
        return HOG_ENOMEM;
    }
    const auto t0 = std::chrono::steady_clock::now();   // after the allocation
    const int nb_total = (n_frames + batch - 1) / batch;
    std::vector<hog_det> best((size_t)std::max(n_frames, 1));
    std::vector<hog_frame> dev((size_t)batch);
    int rc = HOG_OK;

    // copy batch b in and enqueue its detection (asynchronous)
    auto enqueue = [&](int b) -> int {
        const int f0 = b * batch, nb = std::min(batch, n_frames - f0);
        for (int i = 0; i < nb; i++) {
            const hog_frame &f = frames[f0 + i];
            uint8_t *d = d_frames + (size_t)i * fbytes;
            dev[i] = hog_frame{d, f.w, f.h, f.w};
            if (cudaMemcpy2DAsync(d, (size_t)f.w, f.data, (size_t)f.pitch, (size_t)f.w, (size_t)f.h,
                                  cudaMemcpyHostToDevice, stream) != cudaSuccess)
                return HOG_ECUDA;
        }
        return detect_enqueue(ctx, dev.data(), nb, stream, ctx_batched_mode(ctx), true);
    };
    // wait for batch b and keep each frame's best detection
    auto collect = [&](int b) -> int {
        if (cudaStreamSynchronize(stream) != cudaSuccess) return HOG_ECUDA;
        const int32_t *counts = nullptr;
        const hog_det *dets = nullptr;
        int r = detect_results(ctx, &counts, &dets);
        if (r) return r;
        const int f0 = b * batch, nb = std::min(batch, n_frames - f0);
        size_t off = 0;
        for (int i = 0; i < nb; i++) {
            const int k = std::min(counts[i], ctx_max_dets(ctx));
            int arg = -1;
            for (int j = 0; j < k; j++)
                if (arg < 0 || dets[off + j].score > dets[off + arg].score) arg = j;
            has_face[f0 + i] = arg >= 0 ? 1 : 0;
            if (arg >= 0) best[f0 + i] = dets[off + arg];
            off += k;
        }
        return HOG_OK;
    };
    // fit landmarks on all frames of batch b with n_threads host threads
    auto fit = [&](int b) {
        const int f0 = b * batch, nb = std::min(batch, n_frames - f0);
        std::atomic<int> next{0};
        auto work = [&]() {
            for (int i; (i = next.fetch_add(1)) < nb;) {
                const int f = f0 + i;
                float *lm = landmarks + (size_t)f * L * 2;
                if (has_face[f])
                    hog_ert_fit(m, frames[f].data, frames[f].w, frames[f].h, frames[f].pitch, &best[f],
                                lm, ear + 2 * (size_t)f);
                else {
                    std::fill(lm, lm + (size_t)L * 2, 0.0f);
                    ear[2 * (size_t)f] = ear[2 * (size_t)f + 1] = 0.0f;
                }
            }
        };
        std::vector<std::thread> pool;
        for (int k = 1; k < n_threads && k < nb; k++) pool.emplace_back(work);
        work();
        for (auto &th : pool) th.join();
    };

    if (nb_total > 0) {
        rc = enqueue(0);
        if (!rc) rc = collect(0);
        for (int b = 0; b < nb_total && !rc; b++) {
            const bool more = b + 1 < nb_total;
            if (pipelined && more) rc = enqueue(b + 1);   // GPU: next batch
            if (rc) break;
            fit(b);                                        // host: this batch
            if (more) {
                if (!pipelined) rc = enqueue(b + 1);
                if (!rc) rc = collect(b + 1);
            }
        }
    }
    if (d_frames) {
        cudaStreamSynchronize(stream);
        cudaFree(d_frames);
    }
    if (seconds)
        *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // extern "C"
