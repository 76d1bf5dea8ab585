"""Oracle pins for the skip-largest-scales / direct-to-size pyramid (Section
5.1: with a face of at least 20 % of the frame the largest scale need not be
scanned; Section 6.6, future work: scale the frame straight to the largest
level that is needed, then continue in 5/6 steps).

The direct step to level s uses the pixel-centre aligned bilinear rule with
the ratio (6/5)^s.  Bilinear interpolation reproduces any function that is
linear in x and in y exactly, so ramps pin the coordinate mapping and the
rounding; s = 1 must reduce to the 5/6 step; constant and offset images pin
the weights summing to one."""
from fractions import Fraction

import numpy as np
import pytest


def _src_coord(x, s):
    return (Fraction(2 * x + 1) * Fraction(6, 5) ** s - 1) / 2


def _round_half_up(q):
    return int((q + Fraction(1, 2)) // 1)


def test_direct_s1_is_the_five_sixths_step(oracle):
    rng = np.random.default_rng(3)
    for (h, w) in [(240, 320), (97, 81), (123, 250)]:
        f = rng.integers(0, 256, (h, w), dtype=np.uint8)
        a = oracle.downscale_direct_u8(f, 1, 5 * w // 6, 5 * h // 6)
        assert np.array_equal(a, oracle.downscale_u8(f))


@pytest.mark.parametrize("s", [2, 3, 4])
def test_direct_ramps_exact(oracle, s):
    h, w = 100, 150                       # x + y stays below 256: no clipping
    sizes = oracle.level_sizes(w, h, min_size=8)
    dw, dh = sizes[s]
    X0 = np.arange(w)[None, :]
    Y0 = np.arange(h)[:, None]
    cases = [(np.broadcast_to(X0 + 20, (h, w)), lambda X, Y: X + 20),
             (np.broadcast_to(Y0 + 7, (h, w)), lambda X, Y: Y + 7),
             (X0 + Y0, lambda X, Y: X + Y)]
    for img, fn in cases:
        assert img.max() <= 255
        got = oracle.downscale_direct_u8(np.ascontiguousarray(img, np.uint8), s, dw, dh)
        for y in range(0, dh, 3):
            for x in range(0, dw, 2):
                want = fn(_src_coord(x, s), _src_coord(y, s))
                assert int(got[y, x]) == _round_half_up(want), (s, x, y)


@pytest.mark.parametrize("s", [2, 3])
def test_direct_constant_and_offset(oracle, s):
    rng = np.random.default_rng(11)
    h, w = 160, 200
    sizes = oracle.level_sizes(w, h, min_size=8)
    dw, dh = sizes[s]
    const = np.full((h, w), 173, np.uint8)
    assert np.all(oracle.downscale_direct_u8(const, s, dw, dh) == 173)
    base = rng.integers(0, 200, (h, w), dtype=np.uint8)
    a = oracle.downscale_direct_u8(base, s, dw, dh).astype(int)
    b = oracle.downscale_direct_u8(base + np.uint8(55), s, dw, dh).astype(int)
    assert np.array_equal(b, a + 55)          # weights sum to exactly one


def test_pyramid_ex_structure(oracle):
    f = np.random.default_rng(5).integers(0, 256, (480, 640), dtype=np.uint8)
    plain = oracle.pyramid_u8(f)
    skip_only = oracle.pyramid_u8(f, skip_levels=3)
    for a, b in zip(plain, skip_only):        # skipping alone changes no pixel
        assert np.array_equal(a, b)
    s = 3
    d = oracle.pyramid_u8(f, skip_levels=s, direct=True)
    assert len(d) == len(plain)
    assert np.array_equal(d[0], f)
    for l in range(1, s):
        assert not d[l].any()                 # not computed
    assert np.array_equal(d[s], oracle.downscale_direct_u8(f, s, *plain[s].shape[::-1]))
    for l in range(s + 1, len(d)):            # then 5/6 steps from level s
        assert np.array_equal(d[l], oracle.downscale_u8(d[l - 1]))
    # s = 1: direct changes nothing
    for a, b in zip(plain, oracle.pyramid_u8(f, skip_levels=1, direct=True)):
        assert np.array_equal(a, b)


def test_direct_candidates_use_the_direct_levels(oracle):
    from paper_2006_00816_gb300 import synth
    f = synth.eyeblink_frame(4)
    W = synth.filters(2, config=9)
    s = 2
    pyr = oracle.pyramid_u8(f, skip_levels=s, direct=True)
    feats = oracle.frame_features(f, skip_levels=s, direct=True)
    for l in range(len(pyr)):
        if 1 <= l < s:
            assert not feats[l].any()
        else:
            ref = oracle.features(oracle.cell_hist(pyr[l].astype(np.float64)))
            assert np.array_equal(feats[l], ref)
    c = oracle.frame_candidates(f, W, skip_levels=s, direct=True)
    assert len(c) > 0 and c["level"].min() >= s
    sc = oracle.frame_scores(f, W, skip_levels=s, direct=True)
    n = sum(int((x > 0).sum()) for l, x in enumerate(sc) if l >= s)
    assert n == len(c)
    k, nc = oracle.detect(f, W, skip_levels=s, direct=True)
    assert nc == len(c) and 0 < len(k) <= len(c)
