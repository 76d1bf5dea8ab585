"""Seeded synthetic inputs shaped like the eyeblink-camera workloads.

This module draws inputs only: frames, filter banks, labelled crops and
arrival times.  It contains none of the detector's arithmetic (no pyramid,
gradient, histogram, normalisation, correlation or suppression), so both the
CUDA path and the FP64 oracle can consume what it produces without sharing
method code.

Recipe (the paper's recordings are private 640x480 8-bit grayscale eyeblink
videos, Section 6.1; these arrays stand in for them):

* background: white N(0,1) noise, separable Gaussian blur (sigma 2 px,
  radius 6, reflecting borders), rescaled to standard deviation 25, plus 110;
* a bright filled ellipse (+70) with a 2-px linear soft edge, the "face";
* for the eyeblink stream, a dark band (-60) over the top of the ellipse
  whose lower edge sweeps from the ellipse top to its mid-line and back with
  a 100-frame period (the "eyelid"), and a slowly drifting ellipse centre;
* clip to [0, 255], round half up, store as uint8.

Seeds: ``200600816 + 1_000_000 * config + index`` for frame ``index`` of
workload ``config`` (PCG64).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 200600816

#: Frame sizes (w, h) of the mixed-resolution workload.
MIXED_SIZES = ((320, 240), (640, 480), (1280, 720), (1280, 1024))


def seed_for(config: int, index: int) -> int:
    return BASE_SEED + 1_000_000 * int(config) + int(index)


def _rng(config: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, index)))


def _gauss_taps(sigma: float = 2.0, radius: int = 6) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-0.5 * (t / sigma) ** 2)
    return g / g.sum()


def _blur_axis(a: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    r = len(taps) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    p = np.pad(a, pad, mode="reflect")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for k, wk in enumerate(taps):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(k, k + n)
        out += wk * p[tuple(sl)]
    return out


def smooth_noise(rng: np.random.Generator, h: int, w: int,
                 std: float = 25.0, mean: float = 110.0) -> np.ndarray:
    """Blurred white noise rescaled to the given mean and std (float64)."""
    z = rng.standard_normal((h, w))
    taps = _gauss_taps()
    z = _blur_axis(_blur_axis(z, taps, 0), taps, 1)
    s = z.std()
    if s > 0:
        z = z / s
    return mean + std * z


def ellipse_alpha(h: int, w: int, cx: float, cy: float, ax: float, ay: float,
                  edge: float = 2.0) -> np.ndarray:
    """Coverage in [0,1] of a filled ellipse (semi-axes ax, ay) with a linear
    soft edge ``edge`` pixels wide, evaluated at pixel centres."""
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    r = np.sqrt(((x + 0.5 - cx) / ax) ** 2 + ((y + 0.5 - cy) / ay) ** 2)
    signed = (1.0 - r) * min(ax, ay)          # ~pixels inside the boundary
    return np.clip(signed / edge + 0.5, 0.0, 1.0)


def _to_u8(img: np.ndarray) -> np.ndarray:
    return np.floor(np.clip(img, 0.0, 255.0) + 0.5).astype(np.uint8)


def single_frame(w: int = 320, h: int = 240, config: int = 1, index: int = 0,
                 axes=(80.0, 100.0)) -> np.ndarray:
    """One frame of smoothed noise with one planted bright ellipse whose full
    axes are ``axes`` = (width, height) pixels, centre seeded fully inside."""
    rng = _rng(config, index)
    img = smooth_noise(rng, h, w)
    ax, ay = axes[0] / 2.0, axes[1] / 2.0
    cx = rng.uniform(ax + 2, max(ax + 2, w - ax - 2))
    cy = rng.uniform(ay + 2, max(ay + 2, h - ay - 2))
    img += 70.0 * ellipse_alpha(h, w, cx, cy, ax, ay)
    return _to_u8(img)


def eyeblink_frame(index: int, w: int = 640, h: int = 480, config: int = 2) -> np.ndarray:
    """Frame ``index`` of the seeded eyeblink stream: a face-sized ellipse
    (axes 0.3w x 0.4h, i.e. at least 20 % of the frame) drifting slowly, with
    a dark "eyelid" band sweeping over its upper half every 100 frames."""
    stream = _rng(config, 999_999)                 # stream-level constants
    cx0, cy0 = stream.uniform(0.4, 0.6) * w, stream.uniform(0.4, 0.6) * h
    amp_x, amp_y = stream.uniform(0.02, 0.08) * w, stream.uniform(0.02, 0.06) * h
    per_x, per_y = stream.uniform(300, 700), stream.uniform(300, 700)
    ph_x, ph_y = stream.uniform(0, 2 * np.pi), stream.uniform(0, 2 * np.pi)
    rng = _rng(config, index)
    img = smooth_noise(rng, h, w)
    ax, ay = 0.15 * w, 0.2 * h
    cx = cx0 + amp_x * np.sin(2 * np.pi * index / per_x + ph_x)
    cy = cy0 + amp_y * np.sin(2 * np.pi * index / per_y + ph_y)
    alpha = ellipse_alpha(h, w, cx, cy, ax, ay)
    img += 70.0 * alpha
    top, mid = cy - ay, cy
    phase = 0.5 - 0.5 * np.cos(2 * np.pi * (index % 100) / 100.0)
    lid = top + (mid - top) * phase
    y = np.arange(h, dtype=np.float64)[:, None] + 0.5
    band = np.clip((lid - y) / 2.0 + 0.5, 0.0, 1.0)  # 2-px soft lower edge
    img -= 60.0 * band * alpha
    return _to_u8(img)


def eyeblink_stream(n: int, w: int = 640, h: int = 480, start: int = 0,
                    config: int = 2) -> np.ndarray:
    """``n`` consecutive eyeblink frames as a uint8 array [n, h, w]."""
    return np.stack([eyeblink_frame(start + i, w, h, config) for i in range(n)])


def mixed_sizes(n: int, config: int = 3) -> list:
    """Seeded uniform categorical mix of frame sizes (w, h)."""
    rng = _rng(config, 888_888)
    idx = rng.integers(0, len(MIXED_SIZES), size=n)
    return [MIXED_SIZES[i] for i in idx]


def mixed_frames(n: int, config: int = 3) -> list:
    """``n`` frames of seeded mixed resolution (list of uint8 [h, w])."""
    out = []
    for i, (w, h) in enumerate(mixed_sizes(n, config)):
        out.append(eyeblink_frame(i, w, h, config))
    return out


def filters(n_filters: int = 5, config: int = 2, std: float = 0.01) -> np.ndarray:
    """Filter bank W[f][row][col][channel], shape (F, 10, 10, 31), float32,
    drawn N(0, std^2)."""
    rng = _rng(config, 900_000)
    return (std * rng.standard_normal((n_filters, 10, 10, 31))).astype(np.float32)


def crops(n: int = 64, size: int = 128, config: int = 4):
    """Labelled crops: odd indices carry a planted ellipse (label +1), even
    ones are background (label -1).  Returns (uint8 [n,size,size], float32 [n])."""
    imgs, labels = [], []
    for i in range(n):
        rng = _rng(config, i)
        img = smooth_noise(rng, size, size)
        if i % 2 == 1:
            ax = rng.uniform(0.25, 0.4) * size
            ay = rng.uniform(0.3, 0.45) * size
            cx = rng.uniform(0.4, 0.6) * size
            cy = rng.uniform(0.4, 0.6) * size
            img += 70.0 * ellipse_alpha(size, size, cx, cy, ax, ay)
        imgs.append(_to_u8(img))
        labels.append(1.0 if i % 2 == 1 else -1.0)
    return np.stack(imgs), np.asarray(labels, dtype=np.float32)


def arrivals(n_cameras: int = 8, seconds: float = 10.0, period_ms: float = 2.0,
             jitter_ms: float = 0.2, config: int = 5) -> list:
    """Per-camera arrival times in seconds: a fixed period plus exponential
    jitter (mean ``jitter_ms``)."""
    out = []
    for cam in range(n_cameras):
        rng = _rng(config, cam)
        k = int(seconds * 1000.0 / period_ms)
        t = np.arange(k) * period_ms * 1e-3 + rng.exponential(jitter_ms * 1e-3, size=k)
        out.append(t)
    return out


def serving_cameras():
    """The 8-camera serving mix: four 640x480 and four 1280x1024 streams."""
    return [(640, 480)] * 4 + [(1280, 1024)] * 4


def camera_frame(cam: int, index: int, config: int = 5) -> np.ndarray:
    """Frame ``index`` of camera ``cam`` of the serving mix: an eyeblink
    stream at that camera's resolution, seeded per camera."""
    w, h = serving_cameras()[cam]
    return eyeblink_frame(index, w, h, config=10 * config + cam)
