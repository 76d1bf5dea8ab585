"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars: pyramid bit-exact; features |g-o| <= 1e-5 * max(|o|, 1e-6); scores
|g-o| <= 1e-4; suppression exact when run on the GPU's own scores; end to
end, candidate sets equal except windows within 1e-4 of the threshold.
"""
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
def synth():
    from paper_2006_00816_gb300 import synth as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def frames_zoo(S):
    rng = np.random.default_rng(77)
    return {
        "cfg1_320x240": S.single_frame(320, 240),
        "eyeblink_640x480": S.eyeblink_frame(3),
        "odd_81x97": rng.integers(0, 256, (97, 81), dtype=np.uint8),
        "odd_250x123": S.single_frame(250, 123, config=11, axes=(60, 70)),
        "exact_80x80": S.single_frame(80, 80, config=12, axes=(40, 50)),
        "ragged_333x211": S.single_frame(333, 211, config=13),
    }


def test_pyramid_bit_exact(H, oracle, synth):
    det = H.Detector(synth.filters(1), max_w=640, max_h=480, max_batch=2)
    for name, f in frames_zoo(synth).items():
        g = det.pyramid(dev(f))
        o = oracle.pyramid_u8(f)
        assert len(g) == len(o), name
        for l, (a, b) in enumerate(zip(g, o)):
            assert np.array_equal(a.cpu().numpy(), b), (name, l)


def _feat_check(g, o, name):
    g = g.cpu().numpy().astype(np.float64)
    assert g.shape == o.shape, name
    err = np.abs(g - o)
    bound = FEAT_RTOL * np.maximum(np.abs(o), FEAT_FLOOR)
    bad = err > bound
    assert not bad.any(), "%s: %d bad, worst rel %.3g" % (name, bad.sum(),
                                                         (err / np.maximum(np.abs(o), 1e-30)).max())


def test_features_parity(H, oracle, synth):
    det = H.Detector(synth.filters(1), max_w=640, max_h=480, max_batch=2)
    for name, f in frames_zoo(synth).items():
        g = det.features(dev(f))
        o = oracle.frame_features(f)
        assert len(g) == len(o)
        for l, (a, b) in enumerate(zip(g, o)):
            _feat_check(a, b, "%s level %d" % (name, l))


def test_features_constant_and_tiny(H, oracle, synth):
    det = H.Detector(synth.filters(1), max_w=640, max_h=480, max_batch=2)
    for v in (0, 128, 255):
        for g in det.features(dev(np.full((100, 120), v, np.uint8))):
            assert not g.any()
    assert det.features(dev(np.zeros((79, 200), np.uint8))) == []


def test_scores_parity_one_filter(H, oracle, synth):
    f = synth.single_frame(320, 240)
    W = synth.filters(1, config=1)
    det = H.Detector(W, max_w=320, max_h=240, max_batch=1)
    g = det.scores(dev(f))
    o = oracle.frame_scores(f, W)
    assert len(g) == len(o) == 6
    for a, b in zip(g, o):
        assert a.shape == b.shape
        assert np.abs(a.cpu().numpy() - b).max() <= SCORE_ATOL


@pytest.mark.parametrize("nf", [2, 5, 7])
def test_scores_parity_filter_banks(H, oracle, synth, nf):
    f = synth.eyeblink_frame(5)
    W = synth.filters(nf, config=20 + nf)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=1)
    for a, b in zip(det.scores(dev(f)), oracle.frame_scores(f, W)):
        assert a.shape == b.shape
        assert np.abs(a.cpu().numpy() - b).max() <= SCORE_ATOL


def _gpu_candidates(oracle, scores, W0, H0, skip=0, thr=0.0):
    """Candidates built from the GPU's own scores, with oracle boxes."""
    sizes = oracle.level_sizes(W0, H0)
    rows = []
    for l, s in enumerate(scores):
        if l < skip:
            continue
        s = s.cpu().numpy()
        fi, ui, vi = np.nonzero(s > thr)
        for f, u, v in zip(fi, ui, vi):
            rows.append((l, f, u, v, float(s[f, u, v])))
    c = np.zeros(len(rows), oracle.DET_DTYPE)
    for i, (l, f, u, v, sc) in enumerate(rows):
        c[i]["level"], c[i]["filter"], c[i]["u"], c[i]["v"], c[i]["score"] = l, f, u, v, sc
        c[i]["x"], c[i]["y"], c[i]["w"], c[i]["h"] = oracle.box(W0, H0, *sizes[l], int(u), int(v))
    return c


def _kept_set(rows):
    return sorted((int(r["level"]), int(r["u"]), int(r["v"]), int(r["filter"]),
                   float(np.float32(r["score"]))) for r in rows)


@pytest.mark.parametrize("case", ["cfg1", "eyeblink5", "skip1", "hd720", "sxga"])
def test_nms_exact_on_gpu_scores(H, oracle, synth, case):
    """Every suppression launch shape (one CTA per frame, clusters of 2..16
    CTAs, automatic) keeps exactly the oracle's greedy set.  hd720 (35k
    window positions) and sxga (55k) do not fit one CTA's shared memory: the
    one-CTA form runs from global memory there."""
    if case == "cfg1":
        f, W, skip = synth.single_frame(320, 240), synth.filters(1, config=1), 0
    elif case == "hd720":
        f, W, skip = synth.eyeblink_frame(2, 1280, 720, config=3), synth.filters(5), 0
    elif case == "sxga":
        f, W, skip = synth.camera_frame(4, 3), synth.filters(5), 0
    else:
        f, W = synth.eyeblink_frame(7), synth.filters(5)
        skip = 1 if case == "skip1" else 0
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=2, skip_levels=skip)
    ft = dev(f)
    scores = det.scores(ft)
    cands = _gpu_candidates(oracle, scores, w, h, skip=skip)
    srt, keep = oracle.nms(cands, 0.5)
    ob = {(int(r["level"]), int(r["u"]), int(r["v"])): (r["x"], r["y"], r["w"], r["h"])
          for r in srt[keep]}
    for c in (1, 2, 4, 8, 16, 0):
        det.set_nms_cluster(c)
        dets, counts = det.detect([ft])
        assert counts[0] == keep.sum() == len(dets), c
        assert _kept_set(dets) == _kept_set(srt[keep]), c
        # boxes are the FP64 mapping, bit for bit
        for r in dets:
            assert ob[(int(r["level"]), int(r["u"]), int(r["v"]))] == (r["x"], r["y"], r["w"], r["h"])
        # output order: (level, u, v)
        key = [(int(r["level"]), int(r["u"]), int(r["v"])) for r in dets]
        assert key == sorted(key), c


@pytest.mark.parametrize("batched", [False, True])
def test_nms_cluster_sizes_agree_on_batches(H, synth, batched):
    """Mixed batches (including frames with no level and single-level
    frames): every cluster size gives the one-CTA result bit for bit."""
    frames = [dev(f) for f in synth.mixed_frames(7)] + [
        dev(synth.camera_frame(5, 1)), dev(np.full((60, 300), 7, np.uint8)),
        dev(synth.single_frame(100, 90))]
    det = H.Detector(synth.filters(5), max_w=1280, max_h=1024, max_batch=10)
    det.set_nms_cluster(1)
    ref, rc = det.detect(frames, batched=batched)
    assert det.nms_cluster_size(10, 1280, 1024) == 1
    for c in (2, 4, 8, 16, 0):
        det.set_nms_cluster(c)
        for _ in range(2):                      # eager, then graph capture when batched
            got, gc = det.detect(frames, batched=batched)
            assert gc.tolist() == rc.tolist(), c
            assert got.tobytes() == ref.tobytes(), c
    det.set_nms_cluster(0)
    assert det.nms_cluster_size(1, 1280, 1024) >= 2
    cmax = det.nms_cluster_size(1, 640, 480)
    assert det.nms_cluster_size(4, 640, 480) == cmax    # a few frames: many SMs each
    assert det.nms_cluster_size(64, 1280, 1024) == 1    # dozens: one CTA per frame
    assert det.nms_cluster_size(152, 640, 480) == 1
    with pytest.raises(H.HogError):
        det.set_nms_cluster(3)


def test_candidates_match_oracle(H, oracle, synth):
    f, W = synth.eyeblink_frame(11), synth.filters(5)
    h, w = f.shape
    det = H.Detector(W, max_w=w, max_h=h, max_batch=1)
    gs = _gpu_candidates(oracle, det.scores(dev(f)), w, h)
    oc = oracle.frame_candidates(f, W)
    osc = oracle.frame_scores(f, W)
    a = {(int(r["level"]), int(r["filter"]), int(r["u"]), int(r["v"])) for r in gs}
    b = {(int(r["level"]), int(r["filter"]), int(r["u"]), int(r["v"])) for r in oc}
    for (l, fi, u, v) in a ^ b:
        assert abs(osc[l][fi, u, v] - 0.0) <= SCORE_ATOL, (l, fi, u, v)


def test_constant_and_small_frames_detect(H, synth):
    det = H.Detector(synth.filters(5), max_w=640, max_h=480, max_batch=4)
    frames = [dev(np.full((240, 320), 90, np.uint8)), dev(np.zeros((60, 300), np.uint8)),
              dev(np.full((80, 80), 3, np.uint8))]
    dets, counts = det.detect(frames)
    assert counts.tolist() == [0, 0, 0] and len(dets) == 0


def test_pitched_frame(H, oracle, synth):
    f = synth.single_frame(320, 240)
    W = synth.filters(1, config=1)
    det = H.Detector(W, max_w=320, max_h=240, max_batch=1)
    wide = torch.zeros((240, 400), dtype=torch.uint8, device="cuda")
    wide[:, 37:357] = dev(f)
    view = wide[:, 37:357]
    assert view.stride(0) == 400
    for a, b in zip(det.features(view), det.features(dev(f))):
        assert torch.equal(a, b)
    d1, c1 = det.detect([view])
    d2, c2 = det.detect([dev(f)])
    assert c1.tolist() == c2.tolist() and _kept_set(d1) == _kept_set(d2)


def test_batch_mixed_sizes_equals_alone(H, synth):
    W = synth.filters(5)
    det = H.Detector(W, max_w=1280, max_h=1024, max_batch=8)
    frames = [synth.eyeblink_frame(i, w, h, config=3) for i, (w, h) in
              enumerate([(320, 240), (640, 480), (1280, 720), (1280, 1024), (640, 480),
                         (101, 89), (79, 79)])]
    dfr = [dev(f) for f in frames]
    dets, counts = det.detect(dfr)
    off = 0
    for i, f in enumerate(dfr):
        alone, c = det.detect([f])
        assert c[0] == counts[i]
        mine = dets[off:off + counts[i]]
        off += counts[i]
        assert _kept_set(alone) == _kept_set(mine), i
        assert (mine["frame"] == i).all()


def test_detect_host_equals_device(H, synth):
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=3)
    frames = [synth.eyeblink_frame(i) for i in range(5)]
    d1, c1 = det.detect([dev(f) for f in frames])
    d2, c2 = det.detect_host(frames)
    assert c1.tolist() == c2.tolist()
    assert np.array_equal(d1, d2)


def test_capacity_truncation(H, synth):
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=2)
    f = dev(synth.eyeblink_frame(2))
    full, counts = det.detect([f])
    assert counts[0] > 10
    part, counts2 = det.detect([f], det_cap=10, allow_capacity=True)
    assert counts2[0] == counts[0] and len(part) == 10
    assert np.array_equal(part, full[:10])
    small = H.Detector(W, max_w=640, max_h=480, max_batch=2, max_dets_per_frame=7)
    d3, c3 = small.detect([f], allow_capacity=True)
    assert c3[0] == counts[0] and len(d3) == 7


def test_full_size_workload_sampled(H, oracle, synth):
    """640x480, 5 filters, a batch of 16 frames in one call: three sampled
    frames against the oracle (features and scores) and suppression exact on
    the GPU scores for one of them."""
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=16)
    frames = synth.eyeblink_stream(16)
    dfr = [dev(f) for f in frames]
    dets, counts = det.detect(dfr)
    assert (counts > 0).all()
    for i in (0, 7, 15):
        for a, b in zip(det.scores(dfr[i]), oracle.frame_scores(frames[i], W)):
            assert np.abs(a.cpu().numpy() - b).max() <= SCORE_ATOL
    i = 7
    cands = _gpu_candidates(oracle, det.scores(dfr[i]), 640, 480)
    srt, keep = oracle.nms(cands, 0.5)
    off = int(counts[:i].sum())
    assert _kept_set(dets[off:off + counts[i]]) == _kept_set(srt[keep])


def test_max_size_frame(H, oracle, synth):
    f = synth.eyeblink_frame(1, 1280, 1024, config=3)
    W = synth.filters(5)
    det = H.Detector(W, max_w=1280, max_h=1024, max_batch=1)
    ft = dev(f)
    for l, (a, b) in enumerate(zip(det.features(ft), oracle.frame_features(f))):
        _feat_check(a, b, "1280x1024 level %d" % l)
    for a, b in zip(det.scores(ft), oracle.frame_scores(f, W)):
        assert np.abs(a.cpu().numpy() - b).max() <= SCORE_ATOL


def test_planted_template_top_detection(H, oracle, synth):
    f = synth.single_frame(320, 240)
    feats = oracle.frame_features(f)
    lvl, u, v = 1, 6, 9
    Wt = feats[lvl][u:u + 10, v:v + 10, :].copy()
    Wt = (Wt - Wt.mean())[None].astype(np.float32)
    det = H.Detector(Wt, max_w=320, max_h=240, max_batch=1)
    dets, _ = det.detect([dev(f)])
    top = dets[np.argmax(dets["score"])]
    ok, _ = oracle.detect(f, Wt.astype(np.float64))
    assert (int(top["level"]), int(top["u"]), int(top["v"])) == \
        (int(ok[0]["level"]), int(ok[0]["u"]), int(ok[0]["v"]))
    assert abs(float(top["score"]) - ok[0]["score"]) <= SCORE_ATOL


def test_pinned_output_and_plan_cache(H, synth):
    """Kept boxes written by the device straight into pinned host memory
    equal the staged path; a repeated batch (cached plan) on buffers whose
    contents changed gives the new frames' results."""
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=3)
    frames = [dev(synth.eyeblink_frame(i)) for i in range(4)]
    d1, c1 = det.detect(frames)
    out, keep = H.pinned_dets(4 * 2000)
    d2, c2 = det.detect(frames, out=out)
    assert c1.tolist() == c2.tolist() and np.array_equal(d1, d2)
    d3, c3 = det.detect(frames, out=out)          # cached plans, same frames
    assert c3.tolist() == c1.tolist() and np.array_equal(d3, d1)
    for i, f in enumerate(frames):                 # same buffers, new contents
        f.copy_(dev(synth.eyeblink_frame(50 + i)))
    d4, c4 = det.detect(frames)
    fresh = H.Detector(W, max_w=640, max_h=480, max_batch=3)
    d5, c5 = fresh.detect([f.clone() for f in frames])
    assert c4.tolist() == c5.tolist()
    assert _kept_set(d4) == _kept_set(d5)
