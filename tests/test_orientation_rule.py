"""The CUDA histogram stage decides each pixel's orientation sector with the
FP32 test |dy| > fl(|dx| tan(b)) for the four sector boundaries b = 10, 30,
50, 70 degrees (Section 4.1.1: one of eighteen signed directions, nearest
centre).  This checks, on the host, that the constants written in the
kernel source make that test agree with the exact rule for every 8-bit
gradient, i.e. that FP32 rounding never moves a vote to another bin, and
that the resulting bin equals the oracle's FP64 bin for all 511^2 integer
gradients."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2006_00816_gb300", "csrc",
                   "hog_stages.cuh")


def _kernel_constants():
    txt = open(SRC).read()
    body = txt[txt.index("orientation_bin_f(int dx, int dy)"):]
    body = body[:body.index("}")]
    vals = [float(v) for v in re.findall(r"fx \* ([0-9.]+)f", body)]
    assert len(vals) == 4, vals
    return np.array(vals, dtype=np.float32)


def _sector_fp32(ax, ay, T):
    fx = ax.astype(np.float32)
    fy = ay.astype(np.float32)
    q = np.zeros(ax.shape, np.int64)
    for t in T:
        q += fy > (fx * t).astype(np.float32)      # one FP32 product, then an exact compare
    return q


def _bin(dx, dy, q):
    right = (dx > 0) | ((dx == 0) & (dy > 0))
    base = np.where(right, 0, 9)
    b = np.where(right == (dy >= 0), base + q, base - q)
    return np.where(b < 0, b + 18, b)


def test_fp32_sector_test_is_exact_on_8bit_gradients():
    T = _kernel_constants()
    assert np.allclose(T, np.tan(np.deg2rad([10, 30, 50, 70])), rtol=1e-7)
    ax, ay = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    q = _sector_fp32(ax, ay, T)
    exact = np.zeros_like(q)
    for deg in (10, 30, 50, 70):
        th = math.radians(deg)
        exact += (ay * math.cos(th) - ax * math.sin(th)) > 0
    assert np.array_equal(q, exact)


def test_fp32_bins_equal_oracle_bins(oracle):
    T = _kernel_constants()
    dx, dy = np.meshgrid(np.arange(-255, 256), np.arange(-255, 256), indexing="ij")
    dx, dy = dx.ravel(), dy.ravel()
    b = _bin(dx, dy, _sector_fp32(np.abs(dx), np.abs(dy), T))
    nz = (dx != 0) | (dy != 0)
    ob = np.array([oracle.orientation_bin(int(x), int(y)) for x, y in zip(dx[nz], dy[nz])])
    assert np.array_equal(b[nz], ob)
