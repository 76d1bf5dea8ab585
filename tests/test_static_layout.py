"""Host-side checks of hog_features_static (the no-allocation features entry
point), run without a GPU.

The entry point validates its arguments and lays out its fixed 4 MiB
scratch array and its job table on the host before it touches a device.  So
on a machine without a GPU every legal frame (up to 640x480) must get past
those checks and fail only at the device lookup, with HOG_ECUDA; a frame
whose layout did not fit would return HOG_EINVAL ("scratch too small" or
"job table too small") instead.  Frames beyond the limit get HOG_EINVAL
with a clear message.  With a GPU present the same sweep runs on the device
in test_zz_no_alloc.py, so this file is skipped there.
"""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def H():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: the device sweep covers this")
    except ImportError:
        pass
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog
    return hog


def _call(H, w, h):
    p = H.default_params()
    # a frame pointer the host code never dereferences (no device exists)
    fr = H.Frame(C.c_void_p(4096), int(w), int(h), int(w))
    lv = (H.Level * 64)()
    n = C.c_int32(0)
    err = C.create_string_buffer(256)
    rc = H._lib.hog_features_static(C.byref(p), C.byref(fr), C.c_void_p(4096), 1 << 40, lv, 64,
                                    C.byref(n), err, 256, None)
    return rc, err.value.decode(), n.value


def test_every_legal_size_passes_the_layout_checks(H):
    sizes = [(w, h) for w in range(600, 641) for h in range(470, 481)]
    sizes += [(w, h) for w in range(80, 641, 16) for h in range(80, 481, 16)]
    sizes += [(640, 480), (80, 80)]
    for w, h in sizes:
        rc, msg, n = _call(H, w, h)
        assert rc == H.HOG_ECUDA and "device" in msg, (w, h, rc, msg)
        assert n >= 1


def test_oversize_and_tiny_frames(H):
    for w, h in ((641, 480), (640, 481), (1280, 1024)):
        rc, msg, _ = _call(H, w, h)
        assert rc == H.HOG_EINVAL and "exceeds the static limit 640x480" in msg
    rc, msg, n = _call(H, 79, 300)          # no level: nothing to do, no device needed
    assert rc == 0 and n == 0
