"""Pins of the oracle's gradient, orientation binning and cell histograms
(paper Section 4.1.1: 18 signed directions, 8x8 cells, each pixel voting into
its four nearest cells; readings R3-R5)."""
import math

import numpy as np
import pytest


def _atan2_bin(dx, dy):
    """Nearest of the 18 centres at 20*b degrees, from the angle itself."""
    if dx == 0 and dy == 0:
        return -1
    if dx == 0:                     # exact tie between two centres: reading R4
        return 4 if dy > 0 else 13
    th = math.degrees(math.atan2(dy, dx)) % 360.0
    return int(math.floor(th / 20.0 + 0.5)) % 18


def test_orientation_exhaustive_integer_gradients(oracle):
    """All 511^2 integer gradients an 8-bit image can produce."""
    L = oracle.lib()
    bad = 0
    for dx in range(-255, 256):
        for dy in range(-255, 256):
            if L.hgo_orientation_bin(float(dx), float(dy)) != _atan2_bin(dx, dy):
                bad += 1
    assert bad == 0


def test_orientation_decision_has_fp32_margin():
    """The largest-|dot| decision for integer gradients never sits within
    single-precision rounding of a tie, except the exact dx == 0 ties: the
    gap between the two best |dot| values is far above fp32 error."""
    d = np.arange(-255, 256, dtype=np.float64)
    DX, DY = np.meshgrid(d, d, indexing="ij")
    k = np.arange(9)
    c, s = np.cos(np.radians(20.0 * k)), np.sin(np.radians(20.0 * k))
    dots = np.abs(DX[..., None] * c + DY[..., None] * s)
    srt = np.sort(dots, axis=-1)
    gap = srt[..., -1] - srt[..., -2]
    nz = (DX != 0)
    # fp32 rounding of |dot| <= 361 (two products and a sum) stays below 5e-5
    assert gap[nz].min() > 2e-4
    c32, s32 = c.astype(np.float32), s.astype(np.float32)
    d32 = np.abs(DX.astype(np.float32)[..., None] * c32 + DY.astype(np.float32)[..., None] * s32)
    assert ((np.argmax(d32, -1) != np.argmax(dots, -1)) & nz).sum() == 0


def test_orientation_special_cases(oracle):
    assert oracle.orientation_bin(0, 0) == -1
    assert oracle.orientation_bin(0, 5) == 4
    assert oracle.orientation_bin(0, -5) == 13
    assert oracle.orientation_bin(3, 0) == 0
    assert oracle.orientation_bin(-3, 0) == 9
    # 45 degrees -> nearest centre 40 (bin 2); 135 -> 140 (bin 7)
    assert oracle.orientation_bin(10, 10) == 2
    assert oracle.orientation_bin(-10, 10) == 7


def _tent(pos, centre):
    return max(0.0, 1.0 - abs(pos - centre) / 8.0)


def _brute_hist(img):
    """Per-cell gather: sum over voting pixels of mag * tent_x * tent_y into
    the pixel's bin, tents centred on the cell centres 8j+4."""
    h, w = img.shape
    cx, cy = w // 8, h // 8
    out = np.zeros((cy, cx, 18))
    xmax, ymax = min(w - 2, 8 * cx - 1), min(h - 2, 8 * cy - 1)
    for y in range(1, ymax + 1):
        for x in range(1, xmax + 1):
            dx = img[y, x + 1] - img[y, x - 1]
            dy = img[y + 1, x] - img[y - 1, x]
            b = _atan2_bin(dx, dy)
            if b < 0:
                continue
            m = math.hypot(dx, dy)
            for i in range(cy):
                ty = _tent(y + 0.5, 8 * i + 4)
                if ty == 0:
                    continue
                for j in range(cx):
                    tx = _tent(x + 0.5, 8 * j + 4)
                    if tx:
                        out[i, j, b] += m * tx * ty
    return out


@pytest.mark.parametrize("shape,integer", [((40, 32), True), ((35, 43), True),
                                           ((24, 40), False)])
def test_hist_brute_force(oracle, shape, integer):
    rng = np.random.default_rng(11 + shape[1])
    if integer:
        img = rng.integers(0, 256, size=shape).astype(np.float64)
    else:
        img = rng.normal(100, 30, size=shape)
    got = oracle.cell_hist(img)
    exp = _brute_hist(img)
    assert got.shape == exp.shape
    assert np.allclose(got, exp, rtol=1e-12, atol=1e-9)


def test_constant_image_zero_hist(oracle):
    assert not oracle.cell_hist(np.full((64, 72), 93.0)).any()


def test_horizontal_ramp_closed_form(oracle):
    """I = a*x: every voting pixel has dx = 2a, dy = 0 -> bin 0, magnitude 2a;
    cell totals are 2a * (sum of x tents) * (sum of y tents); interior cells
    receive 2a * 8 * 8."""
    a = 0.5
    h, w = 72, 96
    img = np.tile(a * np.arange(w, dtype=np.float64), (h, 1))
    got = oracle.cell_hist(img)
    cx, cy = w // 8, h // 8
    xs = range(1, min(w - 2, 8 * cx - 1) + 1)
    ys = range(1, min(h - 2, 8 * cy - 1) + 1)
    sx = np.array([sum(_tent(x + 0.5, 8 * j + 4) for x in xs) for j in range(cx)])
    sy = np.array([sum(_tent(y + 0.5, 8 * i + 4) for y in ys) for i in range(cy)])
    exp = 2 * a * sy[:, None] * sx[None, :]
    assert np.allclose(got[..., 0], exp, rtol=1e-12)
    assert not got[..., 1:].any()
    assert got[3, 4, 0] == pytest.approx(2 * a * 64)


def test_mirror_permutes_bins(oracle):
    """Horizontal flip of a real-valued image (w = 8 cx) maps cell j to
    cx-1-j and bin o to (9 - o) mod 18; dx == 0 never happens for random reals."""
    rng = np.random.default_rng(21)
    img = rng.normal(0, 1, size=(48, 64))
    h0 = oracle.cell_hist(img)
    h1 = oracle.cell_hist(img[:, ::-1].copy())
    perm = [(9 - o) % 18 for o in range(18)]
    assert np.allclose(h1[:, ::-1, :][..., perm], h0, rtol=1e-12, atol=1e-12)
