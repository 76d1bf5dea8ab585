"""Skipping the largest scales and the direct-to-size pyramid on the GPU
(Section 5.1: with a face of at least 20 % of the frame the largest scale
need not be scanned; Section 6.6, future work: scale straight to the largest
needed level, then continue in 5/6 steps), against the FP64 oracle
implementing the same definitions.

Bars: pyramid bit-exact (the direct step is exact integer arithmetic),
features 1e-5 relative, scores 1e-4, suppression exact on the GPU's own
scores of the scanned levels, batched (both modes) equal to per-frame.  A
fresh context detects with skip_levels before any other call: the skipped
levels' positions must not be read as candidates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FEAT_RTOL, FEAT_FLOOR, SCORE_ATOL = 1e-5, 1e-6, 1e-4


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


def _nms_on(oracle, scores, w, h, skip):
    sizes = oracle.level_sizes(w, h)
    rows = []
    for l, s in enumerate(scores):
        if l < skip:
            continue
        s = s.cpu().numpy() if hasattr(s, "cpu") else s
        fi, ui, vi = np.nonzero(s > 0.0)
        for a, b, c in zip(fi, ui, vi):
            rows.append((l, a, b, c, float(s[a, b, c])))
    cands = np.zeros(len(rows), oracle.DET_DTYPE)
    for i, (l, fi, ui, vi, sc) in enumerate(rows):
        cands[i]["level"], cands[i]["filter"], cands[i]["u"], cands[i]["v"] = l, fi, ui, vi
        cands[i]["score"] = sc
        cands[i]["x"], cands[i]["y"], cands[i]["w"], cands[i]["h"] = oracle.box(w, h, *sizes[l],
                                                                                 int(ui), int(vi))
    return oracle.nms(cands, 0.5)


@pytest.mark.parametrize("skip", [1, 2])
def test_skip_levels_fresh_context(H, S, oracle, skip):
    f = S.eyeblink_frame(8)
    W = S.filters(5)
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=2, skip_levels=skip)
    ft = dev(f)
    dets, counts = det.detect([ft])            # first call on the context
    assert len(dets) == counts[0] > 0
    assert int(dets["level"].min()) >= skip
    srt, keep = _nms_on(oracle, det.scores(ft), w, h, skip)
    assert counts[0] == keep.sum()
    assert _kept(dets) == _kept(srt[keep])


CASES = [("eyeblink_640x480", 2), ("eyeblink_640x480", 3), ("ragged_333x211", 2),
         ("sxga_1280x1024", 4)]


def _frame(S, name):
    if name == "eyeblink_640x480":
        return S.eyeblink_frame(5)
    if name == "sxga_1280x1024":
        return S.camera_frame(4, 1)
    return S.single_frame(333, 211, config=13)


@pytest.mark.parametrize("name,s", CASES)
def test_direct_pyramid_features_scores(H, S, oracle, name, s):
    f = _frame(S, name)
    W = S.filters(5)
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=2, skip_levels=s, direct_first=1)
    ft = dev(f)
    gp = det.pyramid(ft)
    op = oracle.pyramid_u8(f, skip_levels=s, direct=True)
    assert len(gp) == len(op)
    for l, (a, b) in enumerate(zip(gp, op)):
        assert np.array_equal(a.cpu().numpy(), b), l          # absent levels: zeros on both
    for l, (a, b) in enumerate(zip(det.features(ft), oracle.frame_features(f, skip_levels=s,
                                                                           direct=True))):
        a = a.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(a - b) <= FEAT_RTOL * np.maximum(np.abs(b), FEAT_FLOOR)), l
    got = det.scores(ft)
    ref = oracle.frame_scores(f, W, skip_levels=s, direct=True)
    for l, (a, b) in enumerate(zip(got, ref)):
        assert np.abs(a.cpu().numpy() - b).max() <= SCORE_ATOL, l
    # suppression exact on the GPU's scores of the scanned levels
    srt, keep = _nms_on(oracle, got, w, h, s)
    dets, counts = det.detect([ft])
    assert counts[0] == keep.sum() == len(dets)
    assert _kept(dets) == _kept(srt[keep])
    # the direct pyramid changes the scanned levels against the 5/6 chain
    chain = oracle.pyramid_u8(f)
    assert not np.array_equal(op[s], chain[s])


def test_direct_batched_modes_equal_per_frame(H, S):
    frames = [dev(S.eyeblink_frame(i)) for i in range(3)] + [dev(S.camera_frame(5, 2))] + [
        dev(np.full((90, 100), 7, np.uint8))]
    det = H.Detector(S.filters(5), max_w=1280, max_h=1024, max_batch=5, skip_levels=2,
                     direct_first=1)
    ref, rc = det.detect(frames)
    for mode in (0, 1):
        det.set_batched_mode(mode)
        for _ in range(3):                 # eager, graph capture, graph replay
            got, gc = det.detect(frames, batched=True)
            assert gc.tolist() == rc.tolist(), mode
            assert got.tobytes() == ref.tobytes(), mode


def test_direct_params_checked(H, S):
    with pytest.raises(H.HogError):
        H.Detector(S.filters(1), max_w=640, max_h=480, skip_levels=9, direct_first=1)
    with pytest.raises(H.HogError):
        H.Detector(S.filters(1), max_w=640, max_h=480, direct_first=2)
