"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/hog.h declares, and its host-only logic (parameter validation, level
geometry) behaves; no GPU compute is called here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hog():
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog as H
    return H


def _declared():
    txt = open(os.path.join(ROOT, "include", "hog.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hog_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(hog):
    names = _declared()
    assert "hog_create" in names and "hog_detect" in names and "hog_destroy" in names
    lib = C.CDLL(hog.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hog.EXPORTED)


def test_default_params(hog):
    p = hog.default_params()
    assert (p.cell, p.win_cells_w, p.win_cells_h, p.scale_num, p.scale_den) == (8, 10, 10, 5, 6)
    assert p.min_size == 80 and p.threshold == 0.0 and abs(p.nms_iou - 0.5) < 1e-7
    assert abs(p.eps - 1e-4) < 1e-9 and abs(p.trunc - 0.2) < 1e-7


def test_level_geometry_matches_oracle(hog, oracle):
    for w, h in [(320, 240), (640, 480), (1280, 720), (1280, 1024), (128, 128), (80, 80),
                 (81, 97), (79, 300)]:
        g = hog.level_geometry(w, h)
        assert [(a, b) for a, b, *_ in g] == oracle.level_sizes(w, h)
        off = 0
        for lw, lh, cx, cy, o in g:
            assert (cx, cy) == (lw // 8, lh // 8)
            assert o == off
            off += cx * cy * 31


@pytest.mark.parametrize("field,value", [("cell", 4), ("win_cells_w", 8), ("scale_num", 3),
                                         ("min_size", 40), ("nms_iou", 0.3), ("max_batch", 0),
                                         ("skip_levels", -1), ("eps", 0.0),
                                         ("max_dets_per_frame", 0)])
def test_create_rejects_bad_params(hog, field, value):
    import numpy as np
    p = hog.default_params(**{field: value})
    w = np.zeros((1, 10, 10, 31), np.float32)
    h = C.c_void_p()
    rc = hog._lib.hog_create(C.byref(p), w.ctypes.data_as(C.c_void_p), 1, C.byref(h))
    assert rc == hog.HOG_EINVAL
    assert not h.value
    assert len(hog._lib.hog_last_error(None)) > 0


def test_create_rejects_bad_filter_count(hog):
    import numpy as np
    p = hog.default_params()
    w = np.zeros((9, 10, 10, 31), np.float32)
    h = C.c_void_p()
    for n in (0, 9):
        rc = hog._lib.hog_create(C.byref(p), w.ctypes.data_as(C.c_void_p), n, C.byref(h))
        assert rc == hog.HOG_EINVAL


def test_null_safety(hog):
    hog._lib.hog_destroy(None)
    assert hog._lib.hog_detect(None, None, 0, None, 0, None, None) == hog.HOG_EINVAL
    assert hog._lib.hog_level_geometry(None, 10, 10, None, 0, None) == hog.HOG_EINVAL


@pytest.mark.parametrize("field,value", [("max_batch", 0), ("max_batch", 1025), ("max_lanes", 0),
                                         ("max_lanes", 17), ("queue_cap", 4),
                                         ("batched_mode", 2), ("mem_reserve", -1)])
def test_server_rejects_bad_config(hog, field, value):
    import numpy as np
    c = hog.default_server_config(**{field: value})
    if field == "queue_cap":
        c.max_batch = 8
    p = hog.default_params()
    w = np.zeros((1, 10, 10, 31), np.float32)
    h = C.c_void_p()
    rc = hog._lib.hog_server_create(C.byref(p), w.ctypes.data_as(C.c_void_p), 1, C.byref(c),
                                    C.byref(h))
    assert rc == hog.HOG_EINVAL and not h.value
    assert field.split("_")[-1] in hog._lib.hog_server_last_error(None).decode()


def test_server_rejects_bad_params_and_nulls(hog):
    import numpy as np
    c = hog.default_server_config()
    assert (c.max_batch, c.max_lanes, c.queue_cap, c.batched_mode) == (8, 3, 64, -1)
    p = hog.default_params(cell=4)
    w = np.zeros((1, 10, 10, 31), np.float32)
    h = C.c_void_p()
    rc = hog._lib.hog_server_create(C.byref(p), w.ctypes.data_as(C.c_void_p), 1, C.byref(c),
                                    C.byref(h))
    assert rc == hog.HOG_EINVAL and not h.value
    assert hog._lib.hog_server_create(C.byref(p), None, 1, None, C.byref(h)) == hog.HOG_EINVAL
    n = C.c_int32(5)
    assert hog._lib.hog_server_submit(None, None, 1, 1, 1, 0, None) == hog.HOG_EINVAL
    assert hog._lib.hog_server_poll(None, None, 0, None, 0, C.byref(n), 0) == hog.HOG_EINVAL
    hog._lib.hog_server_destroy(None)


def test_frame_table_layout_and_forms(hog):
    """The numpy hog_frame table has the C struct's layout, and a list of
    frames and one [n, h, w] array give the same descriptors; arrays that
    are not row-strided uint8 are copied to ones that are."""
    import numpy as np
    assert hog.FRAME_DTYPE.itemsize == C.sizeof(hog.Frame)
    for name, _ in hog.Frame._fields_:
        assert hog.FRAME_DTYPE.fields[name][1] == getattr(hog.Frame, name).offset
    a = np.arange(4 * 6 * 9, dtype=np.uint8).reshape(4, 6, 9)
    t3, _ = hog._frame_table(a, False)
    tl, _ = hog._frame_table(list(a), False)
    assert t3.tolist() == tl.tolist()
    assert t3["data"].tolist() == [a.ctypes.data + i * 54 for i in range(4)]
    assert (t3["w"] == 9).all() and (t3["h"] == 6).all() and (t3["pitch"] == 9).all()
    sub = a[:, 1:5, 2:7]                      # row-strided view: kept as is, pitch 9
    ts, _ = hog._frame_table(sub, False)
    assert ts["data"].tolist() == [a.ctypes.data + i * 54 + 11 for i in range(4)]
    assert (ts["w"] == 5).all() and (ts["h"] == 4).all() and (ts["pitch"] == 9).all()
    for bad in (a[:, ::-1], a[:, :, ::2], a.astype(np.int16), a[::-1]):
        tb, keep = hog._frame_table(bad, False)
        want = np.ascontiguousarray(bad, dtype=np.uint8)
        for i in range(4):                    # descriptors point at a dense copy
            got = np.ctypeslib.as_array(C.cast(int(tb["data"][i]), C.POINTER(C.c_uint8)),
                                        (int(tb["h"][i]), int(tb["pitch"][i])))
            assert np.array_equal(got[:, :int(tb["w"][i])], want[i])
        tlist, keep2 = hog._frame_table(list(bad), False)
        assert (tlist["w"] == tb["w"]).all() and (tlist["pitch"] == tlist["w"]).all()
    t0, _ = hog._frame_table([], False)
    assert len(t0) == 1 and int(t0["data"][0]) == 0
    e, _ = hog._frame_table(np.zeros((0, 4, 4), np.uint8), False)
    assert len(e) == 1


def test_frame_table_host_torch_tensor(hog):
    """A host torch tensor [n, h, w] is taken as a view of its memory (no
    copy), the same descriptors as its numpy view."""
    import numpy as np
    torch = pytest.importorskip("torch")
    t = torch.arange(3 * 5 * 16, dtype=torch.int64).remainder(256).to(torch.uint8).reshape(3, 5, 16)
    tab, _ = hog._frame_table(t, False)
    ref, _ = hog._frame_table(t.numpy(), False)
    assert tab.tolist() == ref.tolist()
    assert int(tab["data"][0]) == t.data_ptr()
    tl, _ = hog._frame_table(list(t), False)   # a list of 2-D tensors
    assert (tl["w"] == 16).all() and (tl["h"] == 5).all()
