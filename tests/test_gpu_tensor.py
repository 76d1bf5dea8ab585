"""GPU tests of the correlation engines (hog_set_corr_engine): the tcgen05
tensor-core contraction (fp16 hi/lo split, three MMAs per K step) with the
row-shift reduction fused on chip (engine 1) or in a second pass (engine
2), and the FP32 CUDA-core kernel (engine 0), each against the FP64 oracle
(scores |g-o| <= 1e-4, the bar of Section 4.1.1's linear filter); engines 1
and 2 bit-identical; suppression exact on each engine's own scores; batched
modes bit-identical to the per-frame call under each engine (the fused
engine bands levels differently for one frame and for a batch); ragged
levels smaller than one 128-cell tile; frames wider than one band strip;
engine and filter-count changes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCORE_ATOL = 1e-4


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


CASES = [("cfg1_320x240", 1), ("eyeblink_640x480", 5), ("eyeblink_640x480", 8),
         ("sxga_1280x1024", 5), ("odd_81x97", 5), ("ragged_333x211", 1),
         ("wide_2000x120", 5), ("wide_2000x120", 8)]


def _frame(S, name):
    if name == "cfg1_320x240":
        return S.single_frame(320, 240)
    if name == "eyeblink_640x480":
        return S.eyeblink_frame(3)
    if name == "sxga_1280x1024":
        return S.camera_frame(4, 2)
    if name == "odd_81x97":
        return np.random.default_rng(77).integers(0, 256, (97, 81), dtype=np.uint8)
    if name == "wide_2000x120":       # 250 cells wide: two band strips at level 0
        return S.single_frame(2000, 120, config=14)
    return S.single_frame(333, 211, config=13)


@pytest.mark.parametrize("name,nf", CASES)
def test_scores_both_engines_vs_oracle(H, S, oracle, name, nf):
    f = _frame(S, name)
    W = S.filters(nf, config=2)
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=2)
    ref = oracle.frame_scores(f, W)
    got = {}
    for e in (1, 2, 0):
        det.set_corr_engine(e)
        assert det.corr_engine() == e
        got[e] = [s.cpu().numpy() for s in det.scores(dev(f))]
        assert len(got[e]) == len(ref)
        for a, b in zip(got[e], ref):
            assert a.shape == b.shape
            assert np.abs(a - b).max() <= SCORE_ATOL, (e, np.abs(a - b).max())
    for a, b in zip(got[0], got[1]):
        assert np.abs(a - b).max() <= 1e-5
    for a, b in zip(got[1], got[2]):
        assert a.tobytes() == b.tobytes()      # same MMAs, same summation order


def _kept(rows):
    return sorted((int(r["level"]), int(r["u"]), int(r["v"]), int(r["filter"]),
                   float(np.float32(r["score"]))) for r in rows)


@pytest.mark.parametrize("engine", [1, 2, 0])
def test_nms_exact_on_each_engines_scores(H, S, oracle, engine):
    f = S.camera_frame(5, 1)
    W = S.filters(5)
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=1)
    det.set_corr_engine(engine)
    ft = dev(f)
    sizes = oracle.level_sizes(w, h)
    rows = []
    for l, s in enumerate(det.scores(ft)):
        s = s.cpu().numpy()
        for fi, ui, vi in zip(*np.nonzero(s > 0.0)):
            rows.append((l, fi, ui, vi, float(s[fi, ui, vi])))
    c = np.zeros(len(rows), oracle.DET_DTYPE)
    for i, (l, fi, ui, vi, sc) in enumerate(rows):
        c[i]["level"], c[i]["filter"], c[i]["u"], c[i]["v"], c[i]["score"] = l, fi, ui, vi, sc
        c[i]["x"], c[i]["y"], c[i]["w"], c[i]["h"] = oracle.box(w, h, *sizes[l], int(ui), int(vi))
    srt, keep = oracle.nms(c, 0.5)
    dets, counts = det.detect([ft])
    assert counts[0] == keep.sum() == len(dets)
    assert _kept(dets) == _kept(srt[keep])


@pytest.mark.parametrize("engine", [1, 2, 0])
def test_batched_modes_identical_per_engine(H, S, engine):
    frames = [dev(f) for f in S.mixed_frames(7)] + [
        dev(np.full((90, 100), 7, np.uint8)), dev(np.full((60, 300), 9, np.uint8)),
        dev(np.random.default_rng(5).integers(0, 256, (97, 81), dtype=np.uint8))]
    det = H.Detector(S.filters(5), max_w=1280, max_h=1024, max_batch=10)
    det.set_corr_engine(engine)
    ref, rc = det.detect(frames)
    for mode in (0, 1):
        det.set_batched_mode(mode)
        for _ in range(3):                 # eager, graph capture, graph replay
            got, gc = det.detect(frames, batched=True)
            assert gc.tolist() == rc.tolist(), (engine, mode)
            assert got.tobytes() == ref.tobytes(), (engine, mode)


def test_engine_switch_and_filter_change(H, S, oracle):
    f = S.eyeblink_frame(9)
    det = H.Detector(S.filters(5), max_w=640, max_h=480, max_batch=4)
    assert det.corr_engine() == 1              # tensor cores by default
    a = det.detect([dev(f)])
    det.set_corr_engine(0)
    det.set_corr_engine(1)
    b = det.detect([dev(f)])
    assert a[0].tobytes() == b[0].tobytes()
    W1 = S.filters(1, config=7)
    det.set_filters(W1)                        # 5 -> 1 filter: smaller GEMM (N = 16)
    s = det.scores(dev(f))
    for x, o in zip(s, oracle.frame_scores(f, W1)):
        assert np.abs(x.cpu().numpy() - o).max() <= SCORE_ATOL
    det.set_corr_engine(2)                     # two-pass form: same scores and boxes
    s2 = det.scores(dev(f))
    assert all(x.cpu().numpy().tobytes() == y.cpu().numpy().tobytes() for x, y in zip(s, s2))
    c = det.detect([dev(f)])
    det.set_corr_engine(1)
    with pytest.raises(H.HogError):
        det.set_corr_engine(3)
    assert det.corr_engine() == 1
    assert c[0].tobytes() == det.detect([dev(f)])[0].tobytes()


def test_autotune_records_engine(H, S, tmp_path):
    import json
    frames = [dev(f) for f in S.eyeblink_stream(8)]
    det = H.Detector(S.filters(5), max_w=640, max_h=480, max_batch=8)
    ref, rc = det.detect(frames)
    path = str(tmp_path / "tune.json")
    det.autotune(frames, cache_path=path)
    rec = json.load(open(path))
    assert rec["corr_engine"] in (0, 1, 2) and rec["corr_engine"] == det.corr_engine()
    assert rec["corr_ms_tensor"] > 0 and rec["corr_ms_tensor_two_pass"] > 0
    det2 = H.Detector(S.filters(5), max_w=640, max_h=480, max_batch=8)
    det2.set_corr_engine((rec["corr_engine"] + 1) % 3)
    det2.autotune(frames, cache_path=path)     # loaded from the file, not measured
    assert det2.corr_engine() == rec["corr_engine"]


# Filter weights are trained SVM weights (Section 4.1.1, linear
# classification), so their scale is not fixed.  A score is a dot product of
# 3100 weights with features in [0, 0.85]; its rounding error grows with the
# filter's l1 norm, so the score bar is 1e-4 at the scale of the N(0, 0.01)
# workload filters (l1 norm 3100 x 0.01 x sqrt(2/pi) = 24.7) and scales with
# the l1 norm above it.
L1_REF = 3100 * 0.01 * np.sqrt(2 / np.pi)


def _score_bar(W):
    return SCORE_ATOL * np.maximum(1.0, np.abs(W).reshape(len(W), -1).sum(1) / L1_REF)


@pytest.mark.parametrize("std", [1e-3, 1.0, 100.0])
def test_filter_scales_every_engine(H, S, oracle, std):
    f = S.eyeblink_frame(6)
    W = S.filters(5, config=31, std=std)
    assert np.abs(W).max() <= 1023.5                 # inside the tensor engines' fp16 range
    det = H.Detector(W, max_w=640, max_h=480, max_batch=1)
    assert det.corr_engine() == 1
    ref = oracle.frame_scores(f, W)
    bar = _score_bar(W)[:, None, None]
    for e in (1, 2, 0):
        det.set_corr_engine(e)
        got = det.scores(dev(f))
        for a, b in zip(got, ref):
            err = np.abs(a.cpu().numpy().astype(np.float64) - b)
            assert np.isfinite(a.cpu().numpy()).all()
            assert (err <= bar).all(), (std, e, float(err.max()), bar.ravel().tolist())


def test_filters_beyond_fp16_range_run_on_cuda_cores(H, S, oracle):
    """A weight above HOG_TC_MAX_WEIGHT (64 w would overflow fp16) puts the
    context on the FP32 CUDA-core engine, whose scores stay finite and
    within the scaled bar; the tensor engines refuse those filters; a
    non-finite weight is refused outright."""
    f = S.eyeblink_frame(6)
    W = S.filters(5, config=32, std=1.0)
    W[2, 4, 4, 7] = 2000.0
    W[0, 0, 0, 0] = -1500.0
    det = H.Detector(W, max_w=640, max_h=480, max_batch=2)
    assert det.corr_engine() == 0
    assert "fp16" in det.last_error()
    for e in (1, 2):
        with pytest.raises(H.HogError) as ei:
            det.set_corr_engine(e)
        assert ei.value.code == H.HOG_EINVAL
    assert det.corr_engine() == 0
    bar = _score_bar(W)[:, None, None]
    for a, b in zip(det.scores(dev(f)), oracle.frame_scores(f, W)):
        a = a.cpu().numpy()
        assert np.isfinite(a).all() and (np.abs(a.astype(np.float64) - b) <= bar).all()
    dets, counts = det.detect([dev(f)])
    assert counts[0] == len(dets) > 0 and np.isfinite(dets["score"]).all()
    # back to in-range filters: the tensor engine can be selected again
    W_ok = S.filters(5, config=33)
    det.set_filters(W_ok)
    det.set_corr_engine(1)
    assert det.corr_engine() == 1
    # a context on a tensor engine given out-of-range filters moves to engine 0
    det.set_filters(W)
    assert det.corr_engine() == 0
    for bad in (np.nan, np.inf, -np.inf):
        Wb = W_ok.copy()
        Wb[1, 2, 3, 4] = bad
        with pytest.raises(H.HogError) as ei:
            det.set_filters(Wb)
        assert ei.value.code == H.HOG_EINVAL
        with pytest.raises(H.HogError):
            H.Detector(Wb, max_w=640, max_h=480, max_batch=1)
    assert det.corr_engine() == 0                    # the rejected call changed nothing
