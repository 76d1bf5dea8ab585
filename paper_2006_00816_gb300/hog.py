"""Python binding of libhog (ctypes; argument marshalling only).

Every step of the detection path runs in the CUDA kernels behind the C ABI of
``include/hog.h``.  PyTorch supplies device memory and the current stream.
If ``libhog.so`` is missing this module raises at import: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhog.so")

HOG_OK, HOG_EINVAL, HOG_ENOMEM, HOG_ECUDA, HOG_ECAPACITY, HOG_ETIMEOUT, HOG_EINTERNAL = (
    0, -1, -2, -3, -4, -5, -6)
HOG_EBUSY = -7
NFEAT, NBIN, CELL, WIN = 31, 18, 8, 10
TRAIN_RP = (WIN + 2) * CELL + CELL   # pixels per side of a crop's adjoint region (hog_backward_state)

if not os.path.exists(LIB_PATH):
    raise ImportError("libhog.so not built (run __graft_entry__.build()): %s" % LIB_PATH)
_lib = C.CDLL(LIB_PATH)


class Params(C.Structure):
    _fields_ = [("cell", C.c_int32), ("win_cells_w", C.c_int32), ("win_cells_h", C.c_int32),
                ("scale_num", C.c_int32), ("scale_den", C.c_int32), ("min_size", C.c_int32),
                ("skip_levels", C.c_int32), ("eps", C.c_float), ("trunc", C.c_float),
                ("threshold", C.c_float), ("nms_iou", C.c_float), ("max_w", C.c_int32),
                ("max_h", C.c_int32), ("max_batch", C.c_int32),
                ("max_dets_per_frame", C.c_int32), ("float_pyramid", C.c_int32),
                ("direct_first", C.c_int32)]


class Frame(C.Structure):
    _fields_ = [("data", C.c_void_p), ("w", C.c_int32), ("h", C.c_int32), ("pitch", C.c_int32)]


class Det(C.Structure):
    _fields_ = [("frame", C.c_int32), ("level", C.c_int32), ("filter", C.c_int32),
                ("u", C.c_int32), ("v", C.c_int32), ("score", C.c_float), ("x", C.c_double),
                ("y", C.c_double), ("w", C.c_double), ("h", C.c_double)]


class Roi(C.Structure):
    """hog_roi: frame-pixel box [x0, x1) x [y0, y1) for window centres and
    the scanned level range [lmin, lmax]."""
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double),
                ("lmin", C.c_int32), ("lmax", C.c_int32)]


def roi_around(det, W: int, H: int, margin: float = 0.5, dlev: int = 1) -> Roi:
    """hog_roi_around: region of interest around one detection record (a
    DET_DTYPE row): its box grown by margin x its size on each side, levels
    within dlev of its level."""
    d = Det(int(det["frame"]), int(det["level"]), int(det["filter"]), int(det["u"]),
            int(det["v"]), float(det["score"]), float(det["x"]), float(det["y"]),
            float(det["w"]), float(det["h"]))
    r = Roi()
    rc = _lib.hog_roi_around(C.byref(d), int(W), int(H), float(margin), int(dlev), C.byref(r))
    if rc:
        raise HogError(rc, "hog_roi_around")
    return r


class ErtParams(C.Structure):
    """hog_ert_params: the landmark stand-in's shape (68 landmarks, cascade
    levels, trees per level, tree depth, sampled pixels per level, seed)."""
    _fields_ = [("landmarks", C.c_int32), ("cascades", C.c_int32), ("trees", C.c_int32),
                ("depth", C.c_int32), ("features", C.c_int32), ("seed", C.c_uint64)]


class StageStat(C.Structure):
    _fields_ = [("ms", C.c_double), ("launches", C.c_int64), ("units", C.c_int64)]


STAGES = ("pyramid", "hist", "feat", "corr", "nms", "fused")


class Level(C.Structure):
    _fields_ = [("w", C.c_int32), ("h", C.c_int32), ("cx", C.c_int32), ("cy", C.c_int32),
                ("offset", C.c_int64)]


SERVER_CLASSES = 4


class ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("max_lanes", C.c_int32), ("queue_cap", C.c_int32),
                ("batched_mode", C.c_int32), ("mem_reserve", C.c_int64),
                ("class_w", C.c_int32 * SERVER_CLASSES), ("class_h", C.c_int32 * SERVER_CLASSES),
                ("class_lanes", C.c_int32 * SERVER_CLASSES)]


class Result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("tag", C.c_int64), ("status", C.c_int32),
                ("count", C.c_int32), ("stored", C.c_int32), ("lane_class", C.c_int32),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("device_ms", C.c_double), ("batch", C.c_int32), ("lane", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "completed", "failed", "rejected", "batches",
                                         "batched_frames", "max_inflight", "lanes", "lane_bytes",
                                         "pending")] + [
        (k, C.c_int64 * SERVER_CLASSES) for k in ("class_lanes", "class_bytes", "class_frames")]


DET_DTYPE = np.dtype([("frame", "<i4"), ("level", "<i4"), ("filter", "<i4"), ("u", "<i4"),
                      ("v", "<i4"), ("score", "<f4"), ("x", "<f8"), ("y", "<f8"), ("w", "<f8"),
                      ("h", "<f8")], align=True)
assert DET_DTYPE.itemsize == C.sizeof(Det) == 56

_P, _vp, _i32 = C.POINTER, C.c_void_p, C.c_int32
_SIGS = {
    "hog_default_params": (None, [_P(Params)]),
    "hog_level_geometry": (C.c_int, [_P(Params), _i32, _i32, _P(Level), _i32, _P(_i32)]),
    "hog_create": (C.c_int, [_P(Params), _vp, _i32, _P(_vp)]),
    "hog_set_filters": (C.c_int, [_vp, _vp, _i32]),
    "hog_destroy": (None, [_vp]),
    "hog_last_error": (C.c_char_p, [_vp]),
    "hog_pyramid": (C.c_int, [_vp, _P(Frame), _vp, C.c_size_t, _P(Level), _i32, _P(_i32), _vp]),
    "hog_features": (C.c_int, [_vp, _P(Frame), _vp, C.c_size_t, _P(Level), _i32, _P(_i32), _vp]),
    "hog_scores": (C.c_int, [_vp, _P(Frame), _vp, C.c_size_t, _P(Level), _i32, _P(_i32), _vp]),
    "hog_detect": (C.c_int, [_vp, _P(Frame), _i32, _vp, _i32, _P(_i32), _vp]),
    "hog_detect_roi": (C.c_int, [_vp, _P(Frame), _P(Roi), _i32, _vp, _i32, _P(_i32), _vp]),
    "hog_default_ert_params": (None, [_P(ErtParams)]),
    "hog_ert_create": (C.c_int, [_P(ErtParams), _P(_vp)]),
    "hog_ert_destroy": (None, [_vp]),
    "hog_ert_fit": (C.c_int, [_vp, _vp, _i32, _i32, _i32, _P(Det), _vp, _vp]),
    "hog_pipeline_run": (C.c_int, [_vp, _vp, _P(Frame), _i32, _i32, _i32, _i32, _vp, _vp, _vp,
                                   _P(C.c_double), _vp]),
    "hog_roi_around": (C.c_int, [_P(Det), _i32, _i32, C.c_double, _i32, _P(Roi)]),
    "hog_detect_host": (C.c_int, [_vp, _P(Frame), _i32, _vp, _i32, _P(_i32), _vp]),
    "hog_detect_batched": (C.c_int, [_vp, _P(Frame), _i32, _vp, _i32, _P(_i32), _vp]),
    "hog_set_batched_mode": (C.c_int, [_vp, _i32]),
    "hog_set_nms_cluster": (C.c_int, [_vp, _i32]),
    "hog_set_corr_engine": (C.c_int, [_vp, _i32]),
    "hog_get_corr_engine": (C.c_int, [_vp, _P(_i32)]),
    "hog_nms_cluster_size": (C.c_int, [_vp, _i32, _i32, _i32, _P(_i32)]),
    "hog_autotune": (C.c_int, [_vp, _P(Frame), _i32, C.c_char_p, _vp]),
    "hog_get_tuning": (C.c_int, [_vp, _P(_i32), _P(_i32)]),
    "hog_debug_waits": (C.c_int, [_vp, C.c_int64, _i32]),
    "hog_features_static": (C.c_int, [_P(Params), _P(Frame), _vp, C.c_size_t, _P(Level), _i32,
                                      _P(_i32), C.c_char_p, C.c_size_t, _vp]),
    "hog_backward": (C.c_int, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _P(C.c_float),
                               _i32, _vp]),
    "hog_backward_state": (C.c_int, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp,
                                     _P(C.c_float), _i32, _vp, _vp, _vp, _vp]),
    "hog_set_profiling": (C.c_int, [_vp, _i32]),
    "hog_stage_stats": (C.c_int, [_vp, _vp, _i32, _i32]),
    "hog_default_server_config": (None, [_P(ServerConfig)]),
    "hog_server_create": (C.c_int, [_P(Params), _vp, _i32, _P(ServerConfig), _P(_vp)]),
    "hog_server_submit": (C.c_int, [_vp, _vp, _i32, _i32, _i32, C.c_int64, _P(C.c_uint64)]),
    "hog_server_poll": (C.c_int, [_vp, _P(Result), _i32, _vp, _i32, _P(_i32), _i32]),
    "hog_server_get_stats": (C.c_int, [_vp, _P(ServerStats)]),
    "hog_server_destroy": (None, [_vp]),
    "hog_server_last_error": (C.c_char_p, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

#: every symbol the header declares (the CPU tests check the library exports them)
EXPORTED = tuple(_SIGS)


class HogError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libhog error %d: %s" % (code, msg))
        self.code = code


def default_params(**kw) -> Params:
    p = Params()
    _lib.hog_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def level_geometry(w: int, h: int, params: Params | None = None):
    p = params or default_params()
    lv = (Level * 64)()
    n = _i32(0)
    rc = _lib.hog_level_geometry(C.byref(p), int(w), int(h), lv, 64, C.byref(n))
    if rc:
        raise HogError(rc, "level geometry")
    return [(lv[i].w, lv[i].h, lv[i].cx, lv[i].cy, lv[i].offset) for i in range(n.value)]


def features_static(frame, params: Params | None = None, stream=None):
    """hog_features_static: features of one device frame (<= 640x480) with no
    device allocation by the library; the output tensor is allocated here by
    the caller side (torch).  Returns (list of [cy, cx, 31] tensors, rc, msg)."""
    import torch
    if not (isinstance(frame, torch.Tensor) and frame.is_cuda):
        raise ValueError("hog_features_static wants a CUDA uint8 tensor [h, w]")
    p = params or default_params()
    fr = _frame_of(frame)
    geo = level_geometry(fr.w, fr.h, p) if fr.w <= 16384 and fr.h <= 16384 else []
    total = sum(g[2] * g[3] * NFEAT for g in geo)
    # the C side works on the current device: make it the frame's
    with torch.cuda.device(frame.device):
        out = torch.empty(max(total, 1), dtype=torch.float32, device=frame.device)
        lv = (Level * 64)()
        n = _i32(0)
        err = C.create_string_buffer(256)
        rc = _lib.hog_features_static(C.byref(p), C.byref(fr), C.c_void_p(out.data_ptr()),
                                      out.numel(), lv, 64, C.byref(n), err, 256, _stream_ptr(stream))
    res = []
    if rc == 0:
        for i in range(n.value):
            k = lv[i].cx * lv[i].cy * NFEAT
            res.append(out[lv[i].offset:lv[i].offset + k].view(lv[i].cy, lv[i].cx, NFEAT))
    return res, rc, err.value.decode()


def pinned_dets(n):
    """A DET_DTYPE numpy array of n entries in pinned host memory (kept alive
    by the returned tensor), for ``Detector.detect(..., out=...)``."""
    import torch
    t = torch.empty(n * DET_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    return t.numpy().view(DET_DTYPE), t


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _frame_of(t) -> Frame:
    """A device uint8 tensor [h, w] (row stride in bytes = pitch)."""
    assert t.dtype.itemsize == 1 and t.dim() == 2 and t.is_cuda
    return Frame(C.c_void_p(t.data_ptr()), int(t.shape[1]), int(t.shape[0]), int(t.stride(0)))


# hog_frame as a numpy record, so that a batch of descriptors is built with
# array operations rather than one ctypes object per frame
FRAME_DTYPE = np.dtype({"names": ["data", "w", "h", "pitch"],
                        "formats": ["<u8", "<i4", "<i4", "<i4"],
                        "offsets": [Frame.data.offset, Frame.w.offset, Frame.h.offset,
                                    Frame.pitch.offset],
                        "itemsize": C.sizeof(Frame)})


def _frame_table(frames, on_device):
    """hog_frame descriptors of a batch of uint8 frames, as a FRAME_DTYPE
    array (at least one entry; the caller passes the true count).  ``frames``
    is a list of [h, w] frames or one [n, h, w] array whose frame i starts at
    base + i * stride 0.  on_device: CUDA tensors (torch); else host numpy
    arrays or host torch tensors (a list entry that is not a row-strided
    uint8 array is copied to one, and the copy is kept alive in the second
    return value)."""
    if on_device:
        import torch
        if isinstance(frames, torch.Tensor):
            t = frames
            if t.dtype != torch.uint8 or t.dim() != 3 or not t.is_cuda or (t.numel() and t.stride(2) != 1):
                raise ValueError("want a CUDA uint8 tensor [n, h, w] with unit column stride")
            n = int(t.shape[0])
            tab = np.zeros(max(n, 1), FRAME_DTYPE)
            tab["data"][:n] = t.data_ptr() + np.arange(n, dtype=np.uint64) * np.uint64(t.stride(0))
            tab["w"][:n], tab["h"][:n], tab["pitch"][:n] = t.shape[2], t.shape[1], t.stride(1)
            return tab, None
        rows = []
        for t in frames:
            if t.dtype != torch.uint8 or t.dim() != 2 or not t.is_cuda:
                raise ValueError("want CUDA uint8 tensors [h, w]")
            rows.append((t.data_ptr(), t.shape[1], t.shape[0], t.stride(0)))
        return np.array(rows or [(0, 0, 0, 0)], FRAME_DTYPE), None
    if not isinstance(frames, (list, tuple, np.ndarray)) and hasattr(frames, "numpy"):
        frames = frames.numpy()        # a host torch tensor: a view, pinned memory stays pinned
    if isinstance(frames, np.ndarray) and frames.ndim == 3:
        a = frames
        if a.dtype != np.uint8 or (a.size and (a.strides[2] != 1 or a.strides[1] < a.shape[2]
                                               or a.strides[0] < 0)):
            a = np.ascontiguousarray(a, dtype=np.uint8)
        n = a.shape[0]
        tab = np.zeros(max(n, 1), FRAME_DTYPE)
        tab["data"][:n] = a.ctypes.data + np.arange(n, dtype=np.uint64) * np.uint64(a.strides[0])
        tab["w"][:n], tab["h"][:n], tab["pitch"][:n] = a.shape[2], a.shape[1], a.strides[1]
        return tab, a
    keep, rows = [], []
    for f in frames:
        if not (isinstance(f, np.ndarray) and f.dtype == np.uint8 and f.ndim == 2
                and f.strides[1] == 1 and f.strides[0] >= f.shape[1]):
            f = np.ascontiguousarray(f, dtype=np.uint8)
        keep.append(f)
        rows.append((f.ctypes.data, f.shape[1], f.shape[0], f.strides[0]))
    return np.array(rows or [(0, 0, 0, 0)], FRAME_DTYPE), keep


def _tab_ptr(tab):
    return tab.ctypes.data_as(_P(Frame))


class Detector:
    """One libhog context (filters on the device, arenas allocated once)."""

    def __init__(self, filters, **params):
        self.params = default_params(**params)
        w = np.ascontiguousarray(np.asarray(filters, dtype=np.float32))
        assert w.ndim == 4 and w.shape[1:] == (10, 10, NFEAT), w.shape
        self.n_filters = w.shape[0]
        h = _vp()
        rc = _lib.hog_create(C.byref(self.params), w.ctypes.data_as(_vp), self.n_filters,
                             C.byref(h))
        if rc:
            raise HogError(rc, _lib.hog_last_error(None).decode())
        self._h = h

    # --------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.hog_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc and rc not in allow:
            raise HogError(rc, _lib.hog_last_error(self._h).decode())
        return rc

    def set_profiling(self, on=True):
        self._check(_lib.hog_set_profiling(self._h, int(bool(on))))

    def stage_stats(self, reset=False):
        """{stage: (gpu_ms, launches, units)} accumulated since the last reset."""
        st = (StageStat * len(STAGES))()
        self._check(_lib.hog_stage_stats(self._h, st, len(STAGES), int(bool(reset))))
        return {n: (st[i].ms, st[i].launches, st[i].units) for i, n in enumerate(STAGES)}

    def backward(self, images, labels, weights, with_image=True, recompute=False, stream=None):
        """hog_backward on device tensors: images float32 [n,h,w], labels
        float32 [n], weights float32 [10,10,31].  Returns (loss, dW, dI)."""
        import torch
        assert images.is_cuda and images.dtype == torch.float32 and images.is_contiguous()
        n, h, w = images.shape
        labels = labels.contiguous()
        weights = weights.contiguous()
        dW = torch.empty((10, 10, NFEAT), dtype=torch.float32, device=images.device)
        dI = torch.empty_like(images) if with_image else None
        loss = C.c_float(0.0)
        self._check(_lib.hog_backward(self._h, C.c_void_p(images.data_ptr()), n, w, h,
                                      C.c_void_p(labels.data_ptr()), C.c_void_p(weights.data_ptr()),
                                      C.c_void_p(dW.data_ptr()),
                                      C.c_void_p(dI.data_ptr()) if dI is not None else None,
                                      C.byref(loss), int(bool(recompute)), _stream_ptr(stream)))
        return loss.value, dW, dI

    def backward_state(self, images, labels, weights, recompute=False, stream=None):
        """hog_backward_state: (loss, dW, dI, best [n, 4] (level, u, v,
        active), bins [n, 104, 104] uint8, trunc [n, 100, 4, 27] uint8) --
        the gradients and the discrete state the adjoint held fixed."""
        import torch
        assert images.is_cuda and images.dtype == torch.float32 and images.is_contiguous()
        n, h, w = images.shape
        labels = labels.contiguous()
        weights = weights.contiguous()
        dev = images.device
        dW = torch.empty((10, 10, NFEAT), dtype=torch.float32, device=dev)
        dI = torch.empty_like(images)
        best = np.zeros((n, 4), np.int32)
        bins = torch.full((n, TRAIN_RP, TRAIN_RP), 255, dtype=torch.uint8, device=dev)
        trunc = torch.zeros((n, WIN * WIN, 4, NBIN + 9), dtype=torch.uint8, device=dev)
        loss = C.c_float(0.0)
        self._check(_lib.hog_backward_state(
            self._h, C.c_void_p(images.data_ptr()), n, w, h, C.c_void_p(labels.data_ptr()),
            C.c_void_p(weights.data_ptr()), C.c_void_p(dW.data_ptr()), C.c_void_p(dI.data_ptr()),
            C.byref(loss), int(bool(recompute)), best.ctypes.data_as(_vp),
            C.c_void_p(bins.data_ptr()), C.c_void_p(trunc.data_ptr()), _stream_ptr(stream)))
        return loss.value, dW, dI, best, bins, trunc

    def set_batched_mode(self, mode):
        """1: persistent fused launch, 0: one launch per stage."""
        self._check(_lib.hog_set_batched_mode(self._h, int(mode)))

    def set_corr_engine(self, engine):
        """Correlation: 0 FP32 CUDA cores, 1 tcgen05 tensor cores (fp16 hi/lo split)."""
        self._check(_lib.hog_set_corr_engine(self._h, int(engine)))

    def corr_engine(self):
        e = _i32(0)
        self._check(_lib.hog_get_corr_engine(self._h, C.byref(e)))
        return e.value

    def set_nms_cluster(self, c):
        """Suppression launch: 1 one CTA per frame, 2/4/8/16 cluster size,
        0 automatic (default)."""
        self._check(_lib.hog_set_nms_cluster(self._h, int(c)))

    def nms_cluster_size(self, n_frames, w, h):
        c = _i32(0)
        self._check(_lib.hog_nms_cluster_size(self._h, int(n_frames), int(w), int(h), C.byref(c)))
        return c.value

    def autotune(self, frames, cache_path=None, stream=None):
        """Run the autotuner on a sample batch of device frames; returns
        (batched_mode, corr_policy)."""
        tab, _ = _frame_table(frames, True)
        path = cache_path.encode() if cache_path else None
        self._check(_lib.hog_autotune(self._h, _tab_ptr(tab), len(frames), path,
                                      _stream_ptr(stream)))
        return self.tuning()

    def tuning(self):
        m, p = _i32(0), _i32(0)
        self._check(_lib.hog_get_tuning(self._h, C.byref(m), C.byref(p)))
        return m.value, p.value

    def debug_waits(self, polls=0, withhold=False):
        """hog_debug_waits: poll budget of the fused launch's dependency
        waits (0 = default) and, with withhold, a wait that is bound to run
        out (the error path's test)."""
        self._check(_lib.hog_debug_waits(self._h, int(polls), int(bool(withhold))))

    def last_error(self):
        return _lib.hog_last_error(self._h).decode()

    def set_filters(self, filters):
        w = np.ascontiguousarray(np.asarray(filters, dtype=np.float32))
        self._check(_lib.hog_set_filters(self._h, w.ctypes.data_as(_vp), w.shape[0]))
        self.n_filters = w.shape[0]

    # --------------------------------------------------------------
    def pyramid(self, frame, stream=None):
        """List of device uint8 tensors, one per level."""
        import torch
        fr = _frame_of(frame)
        geo = level_geometry(fr.w, fr.h, self.params)
        total = sum(g[0] * g[1] for g in geo)
        out = torch.empty(max(total, 1), dtype=torch.uint8, device=frame.device)
        lv = (Level * 64)()
        n = _i32(0)
        self._check(_lib.hog_pyramid(self._h, C.byref(fr), C.c_void_p(out.data_ptr()), out.numel(),
                                     lv, 64, C.byref(n), _stream_ptr(stream)))
        return [out[lv[i].offset:lv[i].offset + lv[i].w * lv[i].h].view(lv[i].h, lv[i].w)
                for i in range(n.value)]

    def features(self, frame, stream=None):
        """List of device float32 tensors [cy, cx, 31], one per level."""
        import torch
        fr = _frame_of(frame)
        geo = level_geometry(fr.w, fr.h, self.params)
        total = sum(g[2] * g[3] * NFEAT for g in geo)
        out = torch.empty(max(total, 1), dtype=torch.float32, device=frame.device)
        lv = (Level * 64)()
        n = _i32(0)
        self._check(_lib.hog_features(self._h, C.byref(fr), C.c_void_p(out.data_ptr()),
                                      out.numel(), lv, 64, C.byref(n), _stream_ptr(stream)))
        res = []
        for i in range(n.value):
            k = lv[i].cx * lv[i].cy * NFEAT
            res.append(out[lv[i].offset:lv[i].offset + k].view(lv[i].cy, lv[i].cx, NFEAT))
        return res

    def scores(self, frame, stream=None):
        """List of device float32 tensors [F, cy-9, cx-9], one per level."""
        import torch
        fr = _frame_of(frame)
        geo = level_geometry(fr.w, fr.h, self.params)
        F = self.n_filters
        dims = [(max(g[3] - 9, 0), max(g[2] - 9, 0)) for g in geo]
        total = sum(F * a * b for a, b in dims)
        out = torch.empty(max(total, 1), dtype=torch.float32, device=frame.device)
        lv = (Level * 64)()
        n = _i32(0)
        self._check(_lib.hog_scores(self._h, C.byref(fr), C.c_void_p(out.data_ptr()), out.numel(),
                                    lv, 64, C.byref(n), _stream_ptr(stream)))
        res = []
        for i in range(n.value):
            nu, nv = dims[i]
            res.append(out[lv[i].offset:lv[i].offset + F * nu * nv].view(F, nu, nv))
        return res

    def _detect_call(self, call, n, det_cap, allow_capacity, out):
        """Shared tail of the detect entry points: the output buffer, the
        call (call(dets_ptr, det_cap, counts_ptr) -> rc) and the kept rows."""
        if out is not None:
            assert out.dtype == DET_DTYPE and out.flags.c_contiguous
            dets = out
            det_cap = len(out) if det_cap is None else min(det_cap, len(out))
        else:
            if det_cap is None:
                det_cap = max(n, 1) * int(self.params.max_dets_per_frame)
            dets = np.empty(max(det_cap, 1), DET_DTYPE)
        counts = np.zeros(max(n, 1), np.int32)
        rc = call(dets.ctypes.data_as(_vp), det_cap, counts.ctypes.data_as(_P(_i32)))
        self._check(rc, allow=(HOG_ECAPACITY,) if allow_capacity else ())
        total = min(int(np.minimum(counts[:n], self.params.max_dets_per_frame).sum()), det_cap)
        if out is not None:
            return dets[:total], counts[:n].copy()
        return dets[:total].copy(), counts[:n].copy()

    def detect(self, frames, det_cap=None, stream=None, allow_capacity=False, out=None,
               batched=False):
        """Detect on device uint8 frames: a list of [h, w] tensors or one
        [n, h, w] tensor.  Returns (dets, counts): dets a numpy structured
        array (DET_DTYPE), counts int32 per frame.  With ``out`` (a DET_DTYPE
        array, e.g. a view of pinned memory, which the device then fills
        directly), dets is a view of ``out``.  ``batched``:
        hog_detect_batched (persistent fused launch, graphs)."""
        fn = _lib.hog_detect_batched if batched else _lib.hog_detect
        n = len(frames)
        tab, _ = _frame_table(frames, True)
        sp = _stream_ptr(stream)
        return self._detect_call(lambda d, cap, c: fn(self._h, _tab_ptr(tab), n, d, cap, c, sp),
                                 n, det_cap, allow_capacity, out)

    def detect_roi(self, frames, rois, det_cap=None, stream=None, allow_capacity=False, out=None):
        """hog_detect_roi: as detect, each frame restricted to its region of
        interest rois[i] = (x0, y0, x1, y1, lmin, lmax) or a Roi."""
        n = len(frames)
        assert len(rois) == n
        tab, _ = _frame_table(frames, True)
        ra = (Roi * max(n, 1))(*[r if isinstance(r, Roi) else Roi(*[float(x) for x in r[:4]],
                                                                     int(r[4]), int(r[5]))
                                 for r in rois])
        sp = _stream_ptr(stream)
        return self._detect_call(
            lambda d, cap, c: _lib.hog_detect_roi(self._h, _tab_ptr(tab), ra, n, d, cap, c, sp),
            n, det_cap, allow_capacity, out)

    def detect_host(self, frames, det_cap=None, stream=None, allow_capacity=False, out=None):
        """Same as detect, from host uint8 frames (a list of [h, w] numpy
        arrays or one [n, h, w] array), copied in the call; frames in pinned
        memory that follow each other move in one copy."""
        n = len(frames)
        tab, keep = _frame_table(frames, False)
        sp = _stream_ptr(stream)
        return self._detect_call(
            lambda d, cap, c: _lib.hog_detect_host(self._h, _tab_ptr(tab), n, d, cap, c, sp),
            n, det_cap, allow_capacity, out)


def default_server_config(classes=None, **kw) -> ServerConfig:
    """hog_server_config with the defaults, fields set from kw; classes: a
    list of (w, h, lanes) lane size classes (at most SERVER_CLASSES)."""
    c = ServerConfig()
    _lib.hog_default_server_config(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    for k, (w, h, n) in enumerate(classes or []):
        c.class_w[k], c.class_h[k], c.class_lanes[k] = int(w), int(h), int(n)
    return c


class Ert:
    """Host landmark stage stand-in (hog_ert): regression-tree cascade with
    seeded parameters, the paper's ERT structure and cost (Section 4.2); its
    landmarks carry no meaning."""

    def __init__(self, **params):
        self.params = ErtParams()
        _lib.hog_default_ert_params(C.byref(self.params))
        for k, v in params.items():
            setattr(self.params, k, v)
        h = _vp()
        rc = _lib.hog_ert_create(C.byref(self.params), C.byref(h))
        if rc:
            raise HogError(rc, "hog_ert_create")
        self._h = h

    def fit(self, img, det):
        """Landmarks [68, 2] and EAR [2] for one host uint8 image and one
        DET_DTYPE record."""
        img = np.ascontiguousarray(img, dtype=np.uint8)
        h, w = img.shape
        d = Det(int(det["frame"]), int(det["level"]), int(det["filter"]), int(det["u"]),
                int(det["v"]), float(det["score"]), float(det["x"]), float(det["y"]),
                float(det["w"]), float(det["h"]))
        lm = np.zeros((68, 2), np.float32)
        ear = np.zeros(2, np.float32)
        rc = _lib.hog_ert_fit(self._h, img.ctypes.data_as(_vp), w, h, w, C.byref(d),
                              lm.ctypes.data_as(_vp), ear.ctypes.data_as(_vp))
        if rc:
            raise HogError(rc, "hog_ert_fit")
        return lm, ear

    def close(self):
        if getattr(self, "_h", None):
            _lib.hog_ert_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pipeline_run(det, ert, frames, batch, n_threads, pipelined, stream=None):
    """hog_pipeline_run on host uint8 frames (numpy arrays; pinned ones
    copy asynchronously).  Returns (landmarks [n, 68, 2], ear [n, 2],
    has_face [n], seconds)."""
    n = len(frames)
    tab, keep = _frame_table(frames, False)
    lm = np.zeros((max(n, 1), 68, 2), np.float32)
    ear = np.zeros((max(n, 1), 2), np.float32)
    face = np.zeros(max(n, 1), np.int32)
    sec = C.c_double(0.0)
    rc = _lib.hog_pipeline_run(det._h, ert._h, _tab_ptr(tab), n, int(batch), int(n_threads), int(pipelined),
                               lm.ctypes.data_as(_vp), ear.ctypes.data_as(_vp),
                               face.ctypes.data_as(_vp), C.byref(sec), _stream_ptr(stream))
    det._check(rc)
    return lm[:n], ear[:n], face[:n], sec.value


class Server:
    """Continuous-batching detection server (hog_server_*): camera threads
    ``submit`` host frames, a native worker batches whatever has arrived onto
    several in-flight lanes, ``poll`` returns finished results with their
    submit-to-result latency."""

    def __init__(self, filters, config: ServerConfig | None = None, **params):
        f = np.ascontiguousarray(filters, dtype=np.float32)
        assert f.ndim == 4 and f.shape[1:] == (WIN, WIN, NFEAT)
        self.params = default_params(**params)
        self.config = config or default_server_config()
        h = _vp()
        rc = _lib.hog_server_create(C.byref(self.params), f.ctypes.data_as(_vp), f.shape[0],
                                    C.byref(self.config), C.byref(h))
        if rc:
            raise HogError(rc, (_lib.hog_server_last_error(None) or b"").decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.hog_server_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, frame, tag=0):
        """Queue one host uint8 frame [h, w]; returns the request id, or None
        when the queue is full (HOG_EBUSY)."""
        f = np.ascontiguousarray(frame, dtype=np.uint8)
        rid = C.c_uint64(0)
        rc = _lib.hog_server_submit(self._h, f.ctypes.data_as(_vp), f.shape[1], f.shape[0],
                                    f.strides[0], int(tag), C.byref(rid))
        if rc == HOG_EBUSY:
            return None
        if rc:
            raise HogError(rc, "submit %dx%d" % (f.shape[1], f.shape[0]))
        return rid.value

    def poll(self, cap=64, det_cap=None, wait_us=0):
        """Up to cap finished results: a list of dicts (id, tag, status, count,
        latency_ms, queue_ms, dets: DET_DTYPE array)."""
        if det_cap is None:
            det_cap = cap * int(self.params.max_dets_per_frame)
        res = (Result * cap)()
        dets = np.empty(max(det_cap, 1), DET_DTYPE)
        n = _i32(0)
        rc = _lib.hog_server_poll(self._h, res, cap, dets.ctypes.data_as(_vp), det_cap, C.byref(n),
                                  int(wait_us))
        if rc:
            raise HogError(rc, "poll")
        out, off = [], 0
        for i in range(n.value):
            r = res[i]
            out.append(dict(id=r.id, tag=r.tag, status=r.status, count=r.count,
                            latency_ms=r.latency_ms, queue_ms=r.queue_ms,
                            device_ms=r.device_ms, batch=r.batch, lane=r.lane,
                            lane_class=r.lane_class, dets=dets[off:off + r.stored].copy()))
            off += r.stored
        return out

    def stats(self):
        st = ServerStats()
        _lib.hog_server_get_stats(self._h, C.byref(st))
        out = {}
        for k, _ in ServerStats._fields_:
            v = getattr(st, k)
            out[k] = list(v) if k.startswith("class_") else v
        return out


def hinge_loss(detector, images, labels, weights, recompute=False):
    """Differentiable hinge loss on the best window score (torch autograd):
    the adjoint is libhog's hand-written hog_backward."""
    return _HingeLoss.apply(images, weights, labels, detector, recompute)


def _make_autograd():
    import torch

    class HingeLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, images, weights, labels, detector, recompute):
            need_dI = bool(ctx.needs_input_grad[0])
            loss, dW, dI = detector.backward(images.detach().float().contiguous(),
                                             labels.detach().float().contiguous(),
                                             weights.detach().float().contiguous(),
                                             with_image=need_dI, recompute=recompute)
            ctx.save_for_backward(dW, dI if dI is not None else dW.new_empty(0))
            ctx.need_dI = need_dI
            return images.new_tensor(loss)

        @staticmethod
        def backward(ctx, grad):
            dW, dI = ctx.saved_tensors
            gI = (grad * dI) if ctx.need_dI else None
            return gI, grad * dW, None, None, None

    return HingeLoss


class _Lazy:
    fn = None

    def apply(self, *a):
        if _Lazy.fn is None:
            _Lazy.fn = _make_autograd()
        return _Lazy.fn.apply(*a)


_HingeLoss = _Lazy()
