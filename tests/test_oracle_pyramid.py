"""Pins of the oracle's pyramid (paper Section 4.1.1: 5/6 steps down to the
80x80 window; readings R1/R2) against closed forms, exact rational brute
force and the paper's own 128x96 -> 107x80 example."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def test_level_sizes_table(oracle):
    # closed form: w' = floor(5w/6), h' = floor(5h/6), keep while min >= 80
    assert oracle.level_sizes(320, 240) == [(320, 240), (266, 200), (221, 166), (184, 138),
                                            (153, 115), (127, 95)]
    l640 = oracle.level_sizes(640, 480)
    assert [w for w, _ in l640] == [640, 533, 444, 370, 308, 256, 213, 177, 147, 122]
    assert [h for _, h in l640] == [480, 400, 333, 277, 230, 191, 159, 132, 110, 91]
    assert len(oracle.level_sizes(1280, 720)) == 12
    assert oracle.level_sizes(1280, 720)[-1] == (170, 95)
    assert len(oracle.level_sizes(1280, 1024)) == 14
    assert oracle.level_sizes(1280, 1024)[-1] == (117, 93)
    assert oracle.level_sizes(128, 128) == [(128, 128), (106, 106), (88, 88)]
    assert oracle.level_sizes(79, 200) == []
    assert oracle.level_sizes(80, 80) == [(80, 80)]
    # pixel and window totals for 640x480
    assert sum(w * h for w, h in l640) == 974_981
    assert sum((w // 8 - 9) * (h // 8 - 9) for w, h in l640) == 9537


def test_paper_face_size_example(oracle):
    """The paper: a face of at least 20 % of a 640x480 frame is 128x96 at the
    largest scale and about 107x80 after one 5/6 step, so the largest scale can
    be skipped.  Map the face through the level-1 size of the 640x480 pyramid."""
    facts = json.load(open(GOLDEN))
    f = facts["min_face_640x480"]
    W, H = f["frame"]
    fw, fh = int(W * f["fraction"]), int(H * f["fraction"])
    assert [fw, fh] == f["level0_face"]
    (w0, h0), (w1, h1) = oracle.level_sizes(W, H)[:2]
    face1 = [round(fw * w1 / w0), round(fh * h1 / h0)]
    assert face1 == f["level1_face"]
    assert min(face1) >= facts["window_px"]["value"]
    assert facts["scale_step"]["num"] == 5 and facts["scale_step"]["den"] == 6


@pytest.mark.parametrize("value", [0, 1, 77, 254, 255])
def test_constant_level_stays_constant(oracle, value):
    img = np.full((97, 131), value, np.uint8)
    for lv in oracle.pyramid_u8(img):
        assert (lv == value).all()


@pytest.mark.parametrize("a,b", [(1, 0), (2, 3), (5, 7)])
def test_horizontal_ramp_exact(oracle, a, b):
    # bilinear resampling of a linear function is exact: a*(12x+1)/10 + b,
    # then rounded half up.  a=5 gives 6x+1+b.
    w, h = 48, 90
    x = np.arange(w)
    img = np.tile((a * x + b).astype(np.uint8), (h, 1))
    out = oracle.downscale_u8(img)
    w2 = 5 * w // 6
    xs = np.arange(w2)
    expect = np.floor(a * (12 * xs + 1) / 10 + b + 0.5).astype(np.int64)
    assert (out.astype(np.int64) == expect[None, :]).all()
    if a == 5:
        assert (out[0].astype(np.int64) == 6 * xs + 1 + b).all()


def test_plane_exact_float_mode(oracle):
    w, h = 90, 84
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    img = 0.75 * x - 1.25 * y + 3.0
    out = oracle.downscale_f64(img)
    y2, x2 = np.mgrid[0:5 * h // 6, 0:5 * w // 6].astype(np.float64)
    expect = 0.75 * (12 * x2 + 1) / 10 - 1.25 * (12 * y2 + 1) / 10 + 3.0
    assert np.allclose(out, expect, rtol=0, atol=1e-12)


def _brute_downscale(img):
    """Exact rational bilinear sample at (x+1/2)*6/5 - 1/2 with round half up,
    written from the continuous-coordinate definition."""
    h, w = img.shape
    out = np.zeros((5 * h // 6, 5 * w // 6), np.int64)
    for yy in range(out.shape[0]):
        sy = (Fraction(2 * yy + 1, 2)) * Fraction(6, 5) - Fraction(1, 2)
        y0 = sy.numerator // sy.denominator
        gy = sy - y0
        for xx in range(out.shape[1]):
            sx = (Fraction(2 * xx + 1, 2)) * Fraction(6, 5) - Fraction(1, 2)
            x0 = sx.numerator // sx.denominator
            gx = sx - x0
            v = ((1 - gx) * (1 - gy) * int(img[y0, x0])
                 + gx * (1 - gy) * int(img[y0, min(x0 + 1, w - 1)])
                 + (1 - gx) * gy * int(img[min(y0 + 1, h - 1), x0])
                 + gx * gy * int(img[min(y0 + 1, h - 1), min(x0 + 1, w - 1)]))
            q = v + Fraction(1, 2)
            out[yy, xx] = q.numerator // q.denominator
    return out


@pytest.mark.parametrize("shape", [(24, 30), (37, 41), (80, 81)])
def test_downscale_brute_force(oracle, shape):
    rng = np.random.default_rng(7 + shape[0])
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    assert (oracle.downscale_u8(img).astype(np.int64) == _brute_downscale(img)).all()


def test_offset_invariance(oracle):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 200, size=(150, 170)).astype(np.uint8)
    p0 = oracle.pyramid_u8(img)
    p1 = oracle.pyramid_u8(img + 40)
    for a, b in zip(p0, p1):
        assert (b.astype(np.int64) - a == 40).all()


def test_float_mode_within_half_of_integer_step(oracle):
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(96, 120)).astype(np.uint8)
    u8 = oracle.downscale_u8(img).astype(np.float64)
    f = oracle.downscale_f64(img.astype(np.float64))
    assert np.abs(u8 - f).max() <= 0.5 + 1e-12
