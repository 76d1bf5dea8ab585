"""FP64 CPU oracle of the HOG detection path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product library never loads it,
and it shares no code with the CUDA path: it wraps ``hog_oracle.c`` (plain C,
double precision, written step by step from the paper's Section 4.1.1) via
ctypes.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force on tiny inputs or facts the
paper states.  The one thing that stays unpinned is the paper's own level
count for 640x480 (it quotes twelve scales; the 5/6 rule down to an 80x80
window gives ten).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hog_oracle.c")
_LIB = os.path.join(_HERE, "libhog_oracle.so")

CELL, WIN, NBIN, NFEAT = 8, 10, 18, 31
EPS, TAU = 1e-4, 0.2


class Det(C.Structure):
    _fields_ = [("level", C.c_int32), ("filter", C.c_int32), ("u", C.c_int32),
                ("v", C.c_int32), ("score", C.c_double), ("x", C.c_double),
                ("y", C.c_double), ("w", C.c_double), ("h", C.c_double)]


DET_DTYPE = np.dtype([("level", "<i4"), ("filter", "<i4"), ("u", "<i4"), ("v", "<i4"),
                      ("score", "<f8"), ("x", "<f8"), ("y", "<f8"), ("w", "<f8"),
                      ("h", "<f8")])


def build(force: bool = False) -> str:
    """Compile hog_oracle.c into a shared library beside it (gcc, -O2,
    -ffp-contract=off for identical results on x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        d, i, sz = C.c_double, C.c_int, C.c_size_t
        u8p, dp, i32p = P(C.c_uint8), P(C.c_double), P(C.c_int32)
        sig = {
            "hgo_level_sizes": (i, [i, i, i, P(C.c_int), P(C.c_int), i]),
            "hgo_downscale_u8": (None, [u8p, i, i, i, u8p, i]),
            "hgo_downscale_f64": (None, [dp, i, i, dp]),
            "hgo_orientation_bin": (i, [d, d]),
            "hgo_cell_hist": (None, [dp, i, i, dp]),
            "hgo_features": (None, [dp, i, i, d, d, dp]),
            "hgo_correlate": (None, [dp, i, i, dp, i, dp]),
            "hgo_iou": (d, [P(Det), P(Det)]),
            "hgo_box": (None, [i, i, i, i, i, i, P(Det)]),
            "hgo_nms": (i, [P(Det), i, d, i32p]),
            "hgo_pyramid_u8": (i, [u8p, i, i, i, i, u8p, sz]),
            "hgo_downscale_direct_u8": (None, [u8p, i, i, i, i, u8p, i, i, i]),
            "hgo_pyramid_u8_ex": (i, [u8p, i, i, i, i, i, i, u8p, sz]),
            "hgo_frame_features_ex": (i, [u8p, i, i, i, i, i, i, d, d, i, dp, sz]),
            "hgo_frame_scores_ex": (i, [u8p, i, i, i, i, i, i, d, d, dp, i, dp, sz]),
            "hgo_frame_candidates_ex": (i, [u8p, i, i, i, i, i, i, d, d, d, dp, i, P(Det), i]),
            "hgo_detect_ex": (i, [u8p, i, i, i, i, i, i, d, d, d, d, dp, i, P(Det), i, i32p]),
            "hgo_in_roi": (i, [i, i, i, i, i, i, i, dp]),
            "hgo_detect_roi": (i, [u8p, i, i, i, i, i, i, d, d, d, d, dp, i, dp, P(Det), i,
                                   i32p]),
            "hgo_pyramid_f64": (i, [dp, i, i, i, dp, sz]),
            "hgo_frame_features": (i, [u8p, i, i, i, i, d, d, i, dp, sz]),
            "hgo_frame_scores": (i, [u8p, i, i, i, i, d, d, dp, i, dp, sz]),
            "hgo_frame_candidates": (i, [u8p, i, i, i, i, i, d, d, d, dp, i, P(Det), i]),
            "hgo_detect": (i, [u8p, i, i, i, i, i, d, d, d, d, dp, i, P(Det), i, i32p]),
            "hgo_detect_many": (i, [u8p, i, sz, i, i, i, i, i, d, d, d, d, dp, i, P(Det), i,
                                    i32p, i]),
            "hgo_hinge_loss": (d, [dp, i, i, i, dp, i, d, d, dp, dp, i32p]),
            "hgo_hinge_backward": (d, [dp, i, i, i, dp, i, d, d, dp, dp, dp]),
            "hgo_forward_signature": (C.c_uint64, [dp, i, i, i, d, d, dp]),
            "hgo_forward_state": (None, [dp, i, i, i, d, d, dp, i32p, i32p, i32p,
                                         P(C.c_int8), u8p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


# --------------------------------------------------------------------------
# thin numpy-facing wrappers


def level_sizes(w, h, min_size=80):
    ws = (C.c_int * 128)()
    hs = (C.c_int * 128)()
    n = lib().hgo_level_sizes(int(w), int(h), int(min_size), ws, hs, 128)
    return [(ws[k], hs[k]) for k in range(min(n, 128))]


def downscale_u8(img):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.zeros((5 * h // 6, 5 * w // 6), np.uint8)
    lib().hgo_downscale_u8(_p(img, C.c_uint8), w, h, w, _p(out, C.c_uint8), out.shape[1])
    return out


def downscale_f64(img):
    img = np.ascontiguousarray(img, dtype=np.float64)
    h, w = img.shape
    out = np.zeros((5 * h // 6, 5 * w // 6), np.float64)
    lib().hgo_downscale_f64(_p(img, C.c_double), w, h, _p(out, C.c_double))
    return out


def orientation_bin(dx, dy):
    return lib().hgo_orientation_bin(float(dx), float(dy))


def cell_hist(img):
    img = np.ascontiguousarray(img, dtype=np.float64)
    h, w = img.shape
    out = np.zeros((h // CELL, w // CELL, NBIN), np.float64)
    lib().hgo_cell_hist(_p(img, C.c_double), w, h, _p(out, C.c_double))
    return out


def features(hist, eps=EPS, tau=TAU):
    hist = np.ascontiguousarray(hist, dtype=np.float64)
    cy, cx, _ = hist.shape
    out = np.zeros((cy, cx, NFEAT), np.float64)
    lib().hgo_features(_p(hist, C.c_double), cx, cy, eps, tau, _p(out, C.c_double))
    return out


def correlate(feat, filt):
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    filt = np.ascontiguousarray(filt, dtype=np.float64)
    cy, cx, _ = feat.shape
    nf = filt.shape[0]
    out = np.zeros((nf, max(cy - WIN + 1, 0), max(cx - WIN + 1, 0)), np.float64)
    lib().hgo_correlate(_p(feat, C.c_double), cx, cy, _p(filt, C.c_double), nf,
                        _p(out, C.c_double))
    return out


def downscale_direct_u8(img, s, dw, dh):
    """Direct-to-size downscale of a level-0 image to (dw, dh) with the ratio
    (6/5)^s (Section 6.6, future work); s = 1 is the 5/6 step."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.zeros((dh, dw), np.uint8)
    lib().hgo_downscale_direct_u8(_p(img, C.c_uint8), w, h, w, int(s), _p(out, C.c_uint8),
                                  dw, dh, dw)
    return out


def pyramid_u8(frame, min_size=80, skip_levels=0, direct=False):
    """List of uint8 levels of the exact-integer pyramid.  direct=True with
    skip_levels = s >= 2: level s straight from level 0, levels 1..s-1 zero."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = frame.shape
    sizes = level_sizes(w, h, min_size)
    cap = sum(a * b for a, b in sizes)
    buf = np.zeros(max(cap, 1), np.uint8)
    lib().hgo_pyramid_u8_ex(_p(frame, C.c_uint8), w, h, w, min_size, int(skip_levels),
                            int(bool(direct)), _p(buf, C.c_uint8), cap)
    out, off = [], 0
    for lw, lh in sizes:
        out.append(buf[off:off + lw * lh].reshape(lh, lw))
        off += lw * lh
    return out


def pyramid_f64(img, min_size=80):
    img = np.ascontiguousarray(img, dtype=np.float64)
    h, w = img.shape
    sizes = level_sizes(w, h, min_size)
    cap = sum(a * b for a, b in sizes)
    buf = np.zeros(max(cap, 1), np.float64)
    lib().hgo_pyramid_f64(_p(img, C.c_double), w, h, min_size, _p(buf, C.c_double), cap)
    out, off = [], 0
    for lw, lh in sizes:
        out.append(buf[off:off + lw * lh].reshape(lh, lw))
        off += lw * lh
    return out


def frame_features(frame, min_size=80, eps=EPS, tau=TAU, float_mode=False, skip_levels=0,
                   direct=False):
    """List of per-level feature maps [cy][cx][31] (float64)."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = frame.shape
    sizes = level_sizes(w, h, min_size)
    cap = sum((a // CELL) * (b // CELL) for a, b in sizes) * NFEAT
    buf = np.zeros(max(cap, 1), np.float64)
    lib().hgo_frame_features_ex(_p(frame, C.c_uint8), w, h, w, min_size, int(skip_levels),
                                int(bool(direct)), eps, tau, int(bool(float_mode)),
                                _p(buf, C.c_double), cap)
    out, off = [], 0
    for lw, lh in sizes:
        n = (lh // CELL) * (lw // CELL) * NFEAT
        out.append(buf[off:off + n].reshape(lh // CELL, lw // CELL, NFEAT))
        off += n
    return out


def frame_scores(frame, filt, min_size=80, eps=EPS, tau=TAU, skip_levels=0, direct=False):
    """List of per-level score maps [F][cy-9][cx-9] (float64)."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    filt = np.ascontiguousarray(filt, dtype=np.float64)
    h, w = frame.shape
    nf = filt.shape[0]
    sizes = level_sizes(w, h, min_size)
    dims = [((b // CELL) - WIN + 1, (a // CELL) - WIN + 1) for a, b in sizes]
    cap = sum(nf * nu * nv for nu, nv in dims)
    buf = np.zeros(max(cap, 1), np.float64)
    lib().hgo_frame_scores_ex(_p(frame, C.c_uint8), w, h, w, min_size, int(skip_levels),
                              int(bool(direct)), eps, tau, _p(filt, C.c_double), nf,
                              _p(buf, C.c_double), cap)
    out, off = [], 0
    for nu, nv in dims:
        out.append(buf[off:off + nf * nu * nv].reshape(nf, nu, nv))
        off += nf * nu * nv
    return out


def frame_candidates(frame, filt, min_size=80, skip_levels=0, eps=EPS, tau=TAU,
                     threshold=0.0, direct=False):
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    filt = np.ascontiguousarray(filt, dtype=np.float64)
    h, w = frame.shape
    nf = filt.shape[0]
    cap = sum(nf * max(b // CELL - WIN + 1, 0) * max(a // CELL - WIN + 1, 0)
              for a, b in level_sizes(w, h, min_size))
    out = np.zeros(max(cap, 1), DET_DTYPE)
    n = lib().hgo_frame_candidates_ex(_p(frame, C.c_uint8), w, h, w, min_size, skip_levels,
                                      int(bool(direct)), eps, tau, threshold,
                                      _p(filt, C.c_double), nf, _p(out, Det), cap)
    return out[:n].copy()


def nms(cands, iou=0.5):
    """Greedy NMS; returns (cands sorted in rank order, keep flags)."""
    c = np.ascontiguousarray(cands, dtype=DET_DTYPE).copy()
    keep = np.zeros(max(len(c), 1), np.int32)
    lib().hgo_nms(_p(c, Det), len(c), iou, _p(keep, C.c_int32))
    return c, keep[:len(c)].astype(bool)


def box(W0, H0, Wl, Hl, u, v):
    d = Det()
    lib().hgo_box(W0, H0, Wl, Hl, u, v, C.byref(d))
    return (d.x, d.y, d.w, d.h)


def iou(a, b):
    da, db = Det(), Det()
    da.x, da.y, da.w, da.h = a
    db.x, db.y, db.w, db.h = b
    return lib().hgo_iou(C.byref(da), C.byref(db))


def detect(frame, filt, min_size=80, skip_levels=0, eps=EPS, tau=TAU, threshold=0.0,
           nms_iou=0.5, direct=False):
    """Kept detections of one frame in rank order, and the candidate count."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    filt = np.ascontiguousarray(filt, dtype=np.float64)
    h, w = frame.shape
    nf = filt.shape[0]
    cap = sum(nf * max(b // CELL - WIN + 1, 0) * max(a // CELL - WIN + 1, 0)
              for a, b in level_sizes(w, h, min_size))
    out = np.zeros(max(cap, 1), DET_DTYPE)
    ncand = C.c_int32(0)
    k = lib().hgo_detect_ex(_p(frame, C.c_uint8), w, h, w, min_size, skip_levels,
                            int(bool(direct)), eps, tau, threshold, nms_iou,
                            _p(filt, C.c_double), nf, _p(out, Det), cap, C.byref(ncand))
    return out[:k].copy(), ncand.value


def in_roi(W0, H0, Wl, Hl, level, u, v, roi):
    """Whether window (u, v) of a level is scanned under roi = (x0, y0, x1,
    y1, lmin, lmax): level in range and the window's frame-pixel centre in
    the half-open box (Section 6.6, future work)."""
    r = np.ascontiguousarray(roi, dtype=np.float64)
    return bool(lib().hgo_in_roi(W0, H0, Wl, Hl, level, u, v, _p(r, C.c_double)))


def detect_roi(frame, filt, roi, min_size=80, skip_levels=0, eps=EPS, tau=TAU, threshold=0.0,
               nms_iou=0.5, direct=False):
    """Kept detections of one frame restricted to roi = (x0, y0, x1, y1,
    lmin, lmax), in rank order, and the restricted candidate count."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    filt = np.ascontiguousarray(filt, dtype=np.float64)
    r = np.ascontiguousarray(roi, dtype=np.float64)
    h, w = frame.shape
    nf = filt.shape[0]
    cap = sum(nf * max(b // CELL - WIN + 1, 0) * max(a // CELL - WIN + 1, 0)
              for a, b in level_sizes(w, h, min_size))
    out = np.zeros(max(cap, 1), DET_DTYPE)
    ncand = C.c_int32(0)
    k = lib().hgo_detect_roi(_p(frame, C.c_uint8), w, h, w, min_size, skip_levels,
                             int(bool(direct)), eps, tau, threshold, nms_iou,
                             _p(filt, C.c_double), nf, _p(r, C.c_double), _p(out, Det), cap,
                             C.byref(ncand))
    return out[:k].copy(), ncand.value


def detect_many(frames, filt, n_threads=1, min_size=80, skip_levels=0, eps=EPS, tau=TAU,
                threshold=0.0, nms_iou=0.5, cap_per_frame=None):
    """All frames of one size [n, h, w]; returns (list of kept arrays, threads used)."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    filt = np.ascontiguousarray(filt, dtype=np.float64)
    n, h, w = frames.shape
    nf = filt.shape[0]
    if cap_per_frame is None:
        cap_per_frame = sum(nf * max(b // CELL - WIN + 1, 0) * max(a // CELL - WIN + 1, 0)
                            for a, b in level_sizes(w, h, min_size))
    out = np.zeros(max(n * cap_per_frame, 1), DET_DTYPE)
    counts = np.zeros(max(n, 1), np.int32)
    used = lib().hgo_detect_many(_p(frames, C.c_uint8), n, h * w, w, h, w, min_size,
                                 skip_levels, eps, tau, threshold, nms_iou,
                                 _p(filt, C.c_double), nf, _p(out, Det), cap_per_frame,
                                 _p(counts, C.c_int32), int(n_threads))
    res = [out[i * cap_per_frame:i * cap_per_frame + min(counts[i], cap_per_frame)].copy()
           for i in range(n)]
    return res, used


# --------------------------------------------------------------------------
# training adjoint (float pyramid, hinge loss on the best window of a filter)


def hinge_loss(imgs, labels, filt, min_size=80, eps=EPS, tau=TAU):
    """(loss, best scores [n], best windows [n, 3] as (level, u, v))."""
    imgs = np.ascontiguousarray(imgs, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.float64)
    filt = np.ascontiguousarray(filt, dtype=np.float64).reshape(10, 10, 31)
    n, h, w = imgs.shape
    sc = np.zeros(n, np.float64)
    win = np.zeros((n, 3), np.int32)
    loss = lib().hgo_hinge_loss(_p(imgs, C.c_double), n, w, h, _p(labels, C.c_double), min_size,
                                eps, tau, _p(filt, C.c_double), _p(sc, C.c_double),
                                _p(win, C.c_int32))
    return loss, sc, win


def hinge_backward(imgs, labels, filt, min_size=80, eps=EPS, tau=TAU, with_image=True):
    """(loss, dW [10,10,31], dI [n,h,w] or None)."""
    imgs = np.ascontiguousarray(imgs, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.float64)
    filt = np.ascontiguousarray(filt, dtype=np.float64).reshape(10, 10, 31)
    n, h, w = imgs.shape
    dW = np.zeros((10, 10, 31), np.float64)
    dI = np.zeros((n, h, w), np.float64) if with_image else None
    loss = lib().hgo_hinge_backward(_p(imgs, C.c_double), n, w, h, _p(labels, C.c_double),
                                    min_size, eps, tau, _p(filt, C.c_double), _p(dW, C.c_double),
                                    _p(dI, C.c_double) if with_image else None)
    return loss, dW, dI


def forward_signature(img, filt, min_size=80, eps=EPS, tau=TAU):
    img = np.ascontiguousarray(img, dtype=np.float64)
    filt = np.ascontiguousarray(filt, dtype=np.float64).reshape(10, 10, 31)
    h, w = img.shape
    return lib().hgo_forward_signature(_p(img, C.c_double), w, h, min_size, eps, tau,
                                       _p(filt, C.c_double))


def forward_state(img, filt, min_size=80, eps=EPS, tau=TAU):
    """Discrete state of the float-mode forward of one crop that the adjoint
    holds fixed: ((level, u, v) of the best window, bins [lh, lw] int8 of
    that level (-1: no vote), trunc [100, 4, 27] uint8 (1: x N_k < tau))."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    filt = np.ascontiguousarray(filt, dtype=np.float64).reshape(10, 10, 31)
    h, w = img.shape
    best = np.zeros(3, np.int32)
    lw, lh = C.c_int32(0), C.c_int32(0)
    bins = np.full(w * h, -1, np.int8)
    trunc = np.zeros((WIN * WIN, 4, NBIN + 9), np.uint8)
    lib().hgo_forward_state(_p(img, C.c_double), w, h, min_size, eps, tau, _p(filt, C.c_double),
                            _p(best, C.c_int32), C.byref(lw), C.byref(lh),
                            bins.ctypes.data_as(C.POINTER(C.c_int8)), _p(trunc, C.c_uint8))
    return (tuple(int(x) for x in best), bins[:lw.value * lh.value].reshape(lh.value, lw.value),
            trunc)
