"""The benchmarked batched configurations against the FP64 oracle.

The batching of many frames into one launch (Section 5.1, image
combinations along the grid's z dimension) is what the throughput figures
measure, and the batched plan differs with the batch: the fused tensor-core
correlation bands whole levels for a large batch and splits them for a
small one.  So the two batches that are timed are checked themselves, with
the call the benchmark makes:
  - 1000 frames of the 640x480 eyeblink stream, 5 filters, one
    hog_detect_batched call on the [n, h, w] tensor after the autotuner;
  - 256 frames of the seeded mix of 320x240, 640x480, 1280x720 and
    1280x1024, 5 filters.
In both batched modes (the persistent fused launch and the per-stage
launches), eager and replayed as a graph:
  - every frame's kept boxes equal the per-frame call's bit for bit;
  - on a seeded sample of frames spread over the batch, every level's scores
    are within 1e-4 of the oracle's, and the oracle's greedy NMS run on the
    GPU's own scores keeps exactly the batched call's boxes (FP64 boxes bit
    for bit).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCORE_ATOL = 1e-4
N_SAMPLE = 8


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog
    return hog


@pytest.fixture(scope="module")
def synth():
    from paper_2006_00816_gb300 import synth as S
    return S


def _frame_rows(dets, counts, i):
    """Rows of frame i in a batched result (frames back to back)."""
    off = int(counts[:i].sum())
    return dets[off:off + int(counts[i])]


def _kept(rows):
    return sorted((int(r["level"]), int(r["u"]), int(r["v"]), int(r["filter"]),
                   float(np.float32(r["score"])), r["x"], r["y"], r["w"], r["h"]) for r in rows)


def _oracle_kept_on_gpu_scores(oracle, scores, W0, H0):
    """The oracle's greedy NMS (IoU 0.5) over candidates built from the
    GPU's own per-level scores (score > 0), with the oracle's FP64 boxes."""
    sizes = oracle.level_sizes(W0, H0)
    rows = []
    for l, s in enumerate(scores):
        s = s.cpu().numpy()
        for f, u, v in zip(*np.nonzero(s > 0.0)):
            rows.append((l, int(f), int(u), int(v), float(s[f, u, v])))
    c = np.zeros(len(rows), oracle.DET_DTYPE)
    for k, (l, f, u, v, sc) in enumerate(rows):
        c[k]["level"], c[k]["filter"], c[k]["u"], c[k]["v"], c[k]["score"] = l, f, u, v, sc
        c[k]["x"], c[k]["y"], c[k]["w"], c[k]["h"] = oracle.box(W0, H0, *sizes[l], u, v)
    srt, keep = oracle.nms(c, 0.5)
    return srt[keep]


def _check_config(H, oracle, det, frames_dev, frames_host, W, batch_arg, sample, per_frame_cap):
    n = len(frames_host)
    out, _keep = H.pinned_dets(n * per_frame_cap)
    tuned_mode, _ = det.tuning()
    # per-frame call: one hog_detect per frame on the same context
    per_frame = []
    for i in range(n):
        d, c = det.detect([frames_dev[i]])
        assert len(d) == int(c[0])
        per_frame.append(d.copy())
    for mode in (tuned_mode, 1 - tuned_mode):
        det.set_batched_mode(mode)
        first = None
        for call in range(3):                 # eager, graph capture, graph replay
            dets, counts = det.detect(batch_arg, out=out, batched=True)
            dets = dets.copy()
            if first is None:
                first = (dets, counts)
            else:
                assert np.array_equal(counts, first[1]) and dets.tobytes() == first[0].tobytes(), \
                    (mode, call)
        for i in range(n):
            rows = _frame_rows(dets, counts, i)
            assert (rows["frame"] == i).all()
            want = per_frame[i].copy()
            want["frame"] = i
            assert rows.tobytes() == want.tobytes(), (mode, i)
        for i in sample:
            f = frames_host[i]
            h, w = f.shape
            scores = det.scores(frames_dev[i])
            osc = oracle.frame_scores(f, W)
            assert len(scores) == len(osc)
            for l, (g, o) in enumerate(zip(scores, osc)):
                assert g.shape == o.shape, (i, l)
                err = np.abs(g.cpu().numpy().astype(np.float64) - o).max() if o.size else 0.0
                assert err <= SCORE_ATOL, (mode, i, l, err)
            assert _kept(_frame_rows(dets, counts, i)) == _kept(
                _oracle_kept_on_gpu_scores(oracle, scores, w, h)), (mode, i)


def test_bench_stream_1000_frames(H, oracle, synth):
    """The headline batch: 1000 frames of 640x480, one [n, h, w] tensor,
    max_batch 1000, autotuned first as the benchmark does."""
    W = synth.filters(5)
    host = synth.eyeblink_stream(1000)
    fd = torch.from_numpy(host).cuda()
    frames = [fd[i] for i in range(len(host))]
    det = H.Detector(W, max_w=640, max_h=480, max_batch=1000)
    det.autotune(frames)
    rng = np.random.default_rng(1000)
    sample = [0, 999] + sorted((1 + rng.choice(998, N_SAMPLE - 2, replace=False)).tolist())
    _check_config(H, oracle, det, frames, list(host), W, fd, sample, 1536)
    det.close()


def test_bench_mixed_256_frames(H, oracle, synth):
    """The mixed-resolution batch: 256 frames, a list of tensors of four
    sizes, max_batch 256, autotuned first.  The sample takes two frames of
    each size."""
    W = synth.filters(5)
    host = synth.mixed_frames(256)
    frames = [torch.from_numpy(f).cuda() for f in host]
    det = H.Detector(W, max_w=1280, max_h=1024, max_batch=256)
    det.autotune(frames)
    by_size = {}
    for i, f in enumerate(host):
        by_size.setdefault(f.shape, []).append(i)
    assert len(by_size) == 4
    rng = np.random.default_rng(256)
    sample = sorted(j for idx in by_size.values() for j in rng.choice(idx, 2, replace=False).tolist())
    _check_config(H, oracle, det, frames, host, W, frames, sample, 4096)
    det.close()
