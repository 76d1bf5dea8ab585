"""Region-of-interest detection on the GPU (hog_detect_roi; Section 6.6,
future work: scan only the scales and locations near the previous frame's
face) against the FP64 oracle's definition (oracle.in_roi): suppression
exact over the GPU's own scores of the scanned windows, on every
correlation engine; an all-covering region equal to hog_detect bit for bit;
several frames with different regions in one call equal to one call per
frame; empty regions; the helper that grows a previous box into a region."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIG = 1e9


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog
    return hog


@pytest.fixture(scope="module")
def S():
    from paper_2006_00816_gb300 import synth
    return synth


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _kept(rows):
    return sorted((int(r["level"]), int(r["u"]), int(r["v"]), int(r["filter"]),
                   float(np.float32(r["score"]))) for r in rows)


def _oracle_nms_roi(oracle, scores, w, h, roi):
    sizes = oracle.level_sizes(w, h)
    rows = []
    for l, s in enumerate(scores):
        s = s.cpu().numpy()
        fi, ui, vi = np.nonzero(s > 0.0)
        for a, b, c in zip(fi, ui, vi):
            if oracle.in_roi(w, h, *sizes[l], l, int(b), int(c), roi):
                rows.append((l, a, b, c, float(s[a, b, c])))
    cands = np.zeros(len(rows), oracle.DET_DTYPE)
    for i, (l, fi, ui, vi, sc) in enumerate(rows):
        cands[i]["level"], cands[i]["filter"], cands[i]["u"], cands[i]["v"] = l, fi, ui, vi
        cands[i]["score"] = sc
        cands[i]["x"], cands[i]["y"], cands[i]["w"], cands[i]["h"] = oracle.box(w, h, *sizes[l],
                                                                                 int(ui), int(vi))
    return oracle.nms(cands, 0.5)


ROIS = [(150.3, 90.7, 470.1, 390.9, 1, 4), (0.0, 0.0, 320.0, 480.0, 0, 9),
        (333.3, 17.9, 640.0, 301.1, 3, 3), (200.0, 100.0, 330.0, 260.0, 0, 1)]


@pytest.mark.parametrize("engine", [1, 2, 0])
def test_roi_exact_on_gpu_scores(H, S, oracle, engine):
    f = S.eyeblink_frame(6)
    W = S.filters(5)
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=4)
    det.set_corr_engine(engine)
    ft = dev(f)
    scores = det.scores(ft)
    for roi in ROIS:
        srt, keep = _oracle_nms_roi(oracle, scores, w, h, roi)
        dets, counts = det.detect_roi([ft], [roi])
        assert counts[0] == keep.sum() == len(dets), roi
        assert _kept(dets) == _kept(srt[keep]), roi


def test_roi_all_covering_is_plain(H, S):
    frames = [dev(S.eyeblink_frame(i)) for i in range(3)] + [dev(S.camera_frame(4, 1))]
    det = H.Detector(S.filters(5), max_w=1280, max_h=1024, max_batch=4)
    ref, rc = det.detect(frames)
    got, gc = det.detect_roi(frames, [(-BIG, -BIG, BIG, BIG, 0, 99)] * len(frames))
    assert gc.tolist() == rc.tolist()
    assert got.tobytes() == ref.tobytes()


def test_roi_batch_equals_per_frame_and_empty(H, S):
    frames = [dev(S.eyeblink_frame(i)) for i in range(4)]
    rois = [ROIS[0], ROIS[2], (300.5, 200.5, 300.5, 400.0, 0, 99), ROIS[3]]
    det = H.Detector(S.filters(5), max_w=640, max_h=480, max_batch=4)
    got, gc = det.detect_roi(frames, rois)
    assert gc[2] == 0
    off = 0
    for i, (f, r) in enumerate(zip(frames, rois)):
        one, oc = det.detect_roi([f], [r])
        assert oc[0] == gc[i]
        part = got[off:off + gc[i]].copy()
        part["frame"] = 0
        assert part.tobytes() == one.tobytes(), i
        off += gc[i]
    # repeated call: the cached plan gives the same result
    again, ac = det.detect_roi(frames, rois)
    assert ac.tolist() == gc.tolist() and again.tobytes() == got.tobytes()


def test_roi_around_previous_detection(H, S, oracle):
    f0, f1 = S.eyeblink_frame(10), S.eyeblink_frame(11)
    W = S.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=2)
    d0, c0 = det.detect([dev(f0)])
    best = d0[np.argmax(d0["score"])]
    roi = H.roi_around(best, 640, 480, margin=0.5, dlev=1)
    assert roi.lmin == max(0, int(best["level"]) - 1) and roi.lmax == int(best["level"]) + 1
    assert roi.x0 == max(0.0, best["x"] - 0.5 * best["w"])
    assert roi.x1 == min(640.0, best["x"] + best["w"] + 0.5 * best["w"])
    assert roi.y1 == min(480.0, best["y"] + best["h"] + 0.5 * best["h"])
    t = (roi.x0, roi.y0, roi.x1, roi.y1, roi.lmin, roi.lmax)
    ft1 = dev(f1)
    srt, keep = _oracle_nms_roi(oracle, det.scores(ft1), 640, 480, t)
    d1, c1 = det.detect_roi([ft1], [roi])
    assert c1[0] == keep.sum() and _kept(d1) == _kept(srt[keep])
