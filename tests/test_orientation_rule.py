"""The CUDA histogram stage decides each pixel's orientation sector with
four saturated FP32 FMAs, sat(2^20 |dy| - 1024 - |dx| T) with T =
fl32(2^20 tan(b)), for the sector boundaries b = 10, 30, 50, 70 degrees
(Section 4.1.1: one of eighteen signed directions, nearest centre).  This
checks, on the host, that the constants written in the kernel source make
each FMA exactly 0 or 1 and equal to the exact test |dy| > |dx| tan(b) for
every 8-bit gradient, i.e. that FP32 rounding never moves a vote to another
bin, and that the resulting bin equals the oracle's FP64 bin for all 511^2
integer gradients."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2006_00816_gb300", "csrc",
                   "hog_stages.cuh")


def _kernel_constants():
    txt = open(SRC).read()
    body = txt[txt.index("orientation_bin_f(float dxf, float dyf)"):]
    body = body[:body.index("\n}")]
    vals = [float(v) for v in re.findall(r"fmaf\(ax, -([0-9.]+)f, y\)", body)]
    assert len(vals) == 4, vals
    assert "fmaf(ay, 1048576.0f, -1024.0f)" in body
    assert "fmaf(dyf, 9.5367431640625e-07f, dxf)" in body and "- 4.5f" in body
    assert "8388608.0f + 9.0f * (float)S" in body and "& 0x7FFFFFu" in body
    return np.array(vals, dtype=np.float32)


def _fma_values(ax, ay, T):
    """fl32(fma(|dx|, -T, 2^20 |dy| - 1024)) for each boundary: the product and
    the difference are exact in FP64 (at most 32 significant bits), so one
    rounding to FP32 is the FMA's."""
    y = ay.astype(np.float64) * 1048576.0 - 1024.0
    return [(y - ax.astype(np.float64) * np.float64(t)).astype(np.float32) for t in T]


def _sector_fp32(ax, ay, T):
    q = np.zeros(ax.shape, np.int64)
    for v in _fma_values(ax, ay, T):
        q += np.clip(v, 0.0, 1.0).astype(np.int64)     # saturate: 0 or 1 (checked below)
    return q


def _bin(dx, dy, q):
    """The kernel's quadrant step: b = 9 + sU (sR (q - 4.5) - 4.5), sR the sign
    of dx + 2^-20 dy (exact here in FP64; its sign is the FP32 FMA's), sU the
    sign of dy, +1 for zero; 18 is bin 0."""
    xs = dx.astype(np.float64) + dy.astype(np.float64) * 2.0 ** -20
    sr = np.where(xs < 0, -1.0, 1.0)
    su = np.where(dy < 0, -1.0, 1.0)
    b = (9.0 + su * (sr * (q - 4.5) - 4.5)).astype(np.int64)
    return np.where(b == 18, 0, b)          # the kernel's partial row 18 is added to bin 0


def test_fma_values_saturate_to_0_or_1():
    T = _kernel_constants()
    assert np.allclose(T / 1048576.0, np.tan(np.deg2rad([10, 30, 50, 70])), rtol=1e-7)
    ax, ay = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    for v in _fma_values(ax, ay, T):
        assert not ((v > 0.0) & (v < 1.0)).any()
        assert v[v > 0].min() > 1000.0 and v[v <= 0].max() <= -1000.0


def test_fma_sector_test_is_exact_on_8bit_gradients():
    T = _kernel_constants()
    ax, ay = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    q = _sector_fp32(ax, ay, T)
    exact = np.zeros_like(q)
    for deg in (10, 30, 50, 70):
        th = math.radians(deg)
        exact += (ay * math.cos(th) - ax * math.sin(th)) > 0
    assert np.array_equal(q, exact)


def test_fma_bins_equal_oracle_bins(oracle):
    T = _kernel_constants()
    dx, dy = np.meshgrid(np.arange(-255, 256), np.arange(-255, 256), indexing="ij")
    dx, dy = dx.ravel(), dy.ravel()
    b = _bin(dx, dy, _sector_fp32(np.abs(dx), np.abs(dy), T))
    nz = (dx != 0) | (dy != 0)
    ob = np.array([oracle.orientation_bin(int(x), int(y)) for x, y in zip(dx[nz], dy[nz])])
    assert np.array_equal(b[nz], ob)
