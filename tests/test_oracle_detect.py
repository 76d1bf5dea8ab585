"""Pins of the oracle's correlation, threshold, boxes and NMS (paper Section
4.1.1: 10x10-cell linear filters of 3100 weights, five rotations, strict
threshold, suppression to the best-scoring detection; reading R7/R8)."""
import numpy as np
import pytest

from paper_2006_00816_gb300 import synth


def test_correlate_matches_sliding_window_tensordot(oracle):
    rng = np.random.default_rng(2)
    feat = rng.random((14, 17, 31))
    filt = rng.normal(0, 1, (3, 10, 10, 31))
    got = oracle.correlate(feat, filt)
    win = np.lib.stride_tricks.sliding_window_view(feat, (10, 10), axis=(0, 1))
    # win: [nu][nv][31][10][10]
    exp = np.einsum("uvcab,fabc->fuv", win, filt)
    assert got.shape == (3, 5, 8)
    assert np.allclose(got, exp, rtol=1e-12, atol=1e-12)


def test_correlate_linear_in_filter(oracle):
    rng = np.random.default_rng(9)
    feat = rng.random((12, 12, 31))
    w1, w2 = rng.normal(size=(2, 1, 10, 10, 31))
    s1, s2 = oracle.correlate(feat, w1), oracle.correlate(feat, w2)
    s12 = oracle.correlate(feat, w1 + w2)
    assert np.allclose(s12, s1 + s2, rtol=0, atol=1e-12)


def test_single_window_level(oracle):
    """An 80x80 level holds exactly one window (zero-padded energy)."""
    img = synth.single_frame(80, 80, config=9, axes=(40, 50))
    feats = oracle.frame_features(img)
    assert len(feats) == 1 and feats[0].shape == (10, 10, 31)
    W = synth.filters(2, config=9).astype(np.float64)
    s = oracle.frame_scores(img, W)
    assert s[0].shape == (2, 1, 1)
    assert s[0][1, 0, 0] == pytest.approx(float((W[1] * feats[0]).sum()), rel=1e-12)


def test_planted_template(oracle):
    """Filter = the feature window at (level, u, v): its score there is
    ||f||^2, and by Cauchy-Schwarz the normalised score peaks there."""
    img = synth.single_frame()
    feats = oracle.frame_features(img)
    lvl, u, v = 2, 4, 7
    Wt = feats[lvl][u:u + 10, v:v + 10, :][None].copy()
    s = oracle.frame_scores(img, Wt)[lvl][0]
    assert s[u, v] == pytest.approx(float((Wt ** 2).sum()), rel=1e-12)
    win = np.lib.stride_tricks.sliding_window_view(feats[lvl], (10, 10), axis=(0, 1))
    norms = np.sqrt((win ** 2).sum(axis=(2, 3, 4)))
    norm_score = s / np.maximum(norms, 1e-300)
    assert np.unravel_index(np.argmax(norm_score), norm_score.shape) == (u, v)


def test_constant_frame_no_detections(oracle):
    img = np.full((240, 320), 128, np.uint8)
    W = synth.filters(5)
    dets, ncand = oracle.detect(img, W, threshold=0.0)
    assert ncand == 0 and len(dets) == 0
    # scores are exactly zero; a negative threshold admits every window
    _, ncand = oracle.detect(img, W, threshold=-1e-12)
    assert ncand == 5 * 1407


def test_candidates_are_strictly_above_threshold(oracle):
    img = synth.single_frame()
    W = synth.filters(1, config=1)
    scores = oracle.frame_scores(img, W)
    for t in (0.0, 0.05):
        c = oracle.frame_candidates(img, W, threshold=t)
        assert len(c) == sum(int((s > t).sum()) for s in scores)
        assert (c["score"] > t).all()
    c = oracle.frame_candidates(img, W, skip_levels=2)
    assert (c["level"] >= 2).all()
    assert len(c) == sum(int((s > 0).sum()) for s in scores[2:])


def test_box_mapping(oracle):
    x, y, w, h = oracle.box(640, 480, 533, 400, 3, 5)
    assert w == pytest.approx(80 * 640 / 533, rel=1e-15)
    assert h == pytest.approx(80 * 480 / 400, rel=1e-15)
    assert x == pytest.approx(40 * 640 / 533, rel=1e-15)
    assert y == pytest.approx(24 * 480 / 400, rel=1e-15)


@pytest.mark.parametrize("du,dv", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 1), (1, 2), (3, 0),
                                   (0, 3), (2, 2), (4, 0), (3, 1), (0, 4), (5, 5)])
def test_same_level_suppression_rule(oracle, du, dv):
    """Equal 80x80 boxes offset by (8du, 8dv) have IoU k/(200-k) with
    k = (10-|du|)(10-|dv|), so they suppress iff k > 200/3."""
    a = oracle.box(640, 480, 640, 480, 5, 5)
    b = oracle.box(640, 480, 640, 480, 5 + du, 5 + dv)
    k = (10 - abs(du)) * (10 - abs(dv))
    assert oracle.iou(a, b) == pytest.approx(k / (200 - k), rel=1e-12)
    c = np.zeros(2, oracle.DET_DTYPE)
    for i, (uu, vv, s) in enumerate([(5, 5, 1.0), (5 + du, 5 + dv, 0.5)]):
        c[i]["u"], c[i]["v"], c[i]["score"] = uu, vv, s
        c[i]["x"], c[i]["y"], c[i]["w"], c[i]["h"] = oracle.box(640, 480, 640, 480, uu, vv)
    _, keep = oracle.nms(c, 0.5)
    assert keep[0]
    assert keep[1] == (not (k > 200 / 3))


def _random_cands(oracle, rng, n):
    c = np.zeros(n, oracle.DET_DTYPE)
    c["level"] = rng.integers(0, 3, n)
    c["filter"] = rng.integers(0, 5, n)
    c["u"] = rng.integers(0, 12, n)
    c["v"] = rng.integers(0, 12, n)
    c["score"] = np.round(rng.random(n), 2)      # many exact ties
    sizes = [(640, 480), (533, 400), (444, 333)]
    for i in range(n):
        wl, hl = sizes[c["level"][i]]
        c[i]["x"], c[i]["y"], c[i]["w"], c[i]["h"] = oracle.box(640, 480, wl, hl,
                                                                int(c["u"][i]), int(c["v"][i]))
    return c


def test_nms_fixed_point_characterisation(oracle):
    """Greedy NMS is the unique set K with: c in K  <=>  no member of K
    ranked above c overlaps c by more than the IoU threshold."""
    rng = np.random.default_rng(12)
    c = _random_cands(oracle, rng, 300)
    srt, keep = oracle.nms(c, 0.5)
    # rank order: score desc, then (level, filter, u, v) asc
    keys = [(-r["score"], r["level"], r["filter"], r["u"], r["v"]) for r in srt]
    assert keys == sorted(keys)
    boxes = [(r["x"], r["y"], r["w"], r["h"]) for r in srt]
    for i in range(len(srt)):
        blocked = any(keep[j] and oracle.iou(boxes[i], boxes[j]) > 0.5 for j in range(i))
        assert keep[i] == (not blocked)
    # identical boxes (same level and position, other filter) never both survive
    kept = srt[keep]
    pos = list(zip(kept["level"], kept["u"], kept["v"]))
    assert len(pos) == len(set(pos))


def test_adjacent_levels_interact_two_apart_do_not(oracle):
    """Level boxes differ in size by >= 1.2x per axis per step, so boxes two
    levels apart have IoU <= 1/1.44^2 < 0.5, while adjacent ones can exceed it."""
    sizes = oracle.level_sizes(640, 480)
    best_adj, best_two = 0.0, 0.0
    for l in range(len(sizes) - 1):
        for m, store in ((l + 1, "adj"), (l + 2, "two")):
            if m >= len(sizes):
                continue
            a = oracle.box(640, 480, *sizes[l], 3, 3)
            for u in range(0, 6):
                for v in range(0, 6):
                    b = oracle.box(640, 480, *sizes[m], u, v)
                    r = oracle.iou(a, b)
                    if store == "adj":
                        best_adj = max(best_adj, r)
                    else:
                        best_two = max(best_two, r)
    assert best_adj > 0.5
    assert best_two < 0.5


def test_detect_planted_template_top(oracle):
    img = synth.single_frame()
    feats = oracle.frame_features(img)
    lvl, u, v = 1, 6, 9
    Wt = feats[lvl][u:u + 10, v:v + 10, :][None].copy()
    Wt = Wt - Wt.mean()            # zero-mean template: background scores ~ 0
    dets, _ = oracle.detect(img, Wt, threshold=0.0)
    s = oracle.frame_scores(img, Wt)
    best = max((sc.max(), l) for l, sc in enumerate(s))
    top = dets[0]
    assert top["score"] == pytest.approx(best[0], rel=1e-15)
    assert top["level"] == best[1]


def test_nms_threshold_is_strict(oracle):
    """Boxes (0,0,3,1) and (1,0,3,1): intersection 2, union 4, IoU exactly 0.5
    -> both survive; shifting by a quarter pixel less (IoU > 0.5) suppresses."""
    for shift, both in [(1.0, True), (0.75, False)]:
        c = np.zeros(2, oracle.DET_DTYPE)
        c[0]["score"], c[1]["score"] = 2.0, 1.0
        c[0]["x"], c[0]["w"], c[0]["h"] = 0.0, 3.0, 1.0
        c[1]["x"], c[1]["w"], c[1]["h"] = shift, 3.0, 1.0
        if shift == 1.0:
            assert oracle.iou((0.0, 0.0, 3.0, 1.0), (1.0, 0.0, 3.0, 1.0)) == 0.5
        _, keep = oracle.nms(c, 0.5)
        assert keep.tolist() == [True, both]
