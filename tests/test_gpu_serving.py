"""GPU tests of the continuous-batching server (hog_server_*): eight camera
threads (four 640x480, four 1280x1024, plus frames too small for one level)
submit concurrently; every result equals hog_detect_host on that frame
alone, bit for bit; a full queue refuses with HOG_EBUSY and loses nothing it
accepted; closing with requests in flight finishes them."""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog
    return hog


@pytest.fixture(scope="module")
def S():
    from paper_2006_00816_gb300 import synth
    return synth


@pytest.fixture(scope="module")
def streams(S):
    """Per camera: 5 frames, plus one 60x300 frame (0 levels) on camera 0."""
    fr = {c: [S.camera_frame(c, k) for k in range(5)] for c in range(8)}
    fr[0].insert(2, np.full((60, 300), 9, np.uint8))
    return fr


@pytest.fixture(scope="module")
def alone(H, S, streams):
    det = H.Detector(S.filters(5), max_w=1280, max_h=1024, max_batch=1)
    return {(c, k): det.detect_host([f])[0] for c, fs in streams.items() for k, f in enumerate(fs)}


def _drain(srv, want, timeout=60.0):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout:
        for r in srv.poll(cap=16, wait_us=20000):
            got[r["tag"]] = r
    return got


def _tag(c, k):
    return (c << 32) | k


@pytest.mark.parametrize("mode", [0, 1])
def test_concurrent_cameras_equal_alone(H, S, streams, alone, mode):
    cfg = H.default_server_config(max_batch=8, max_lanes=3, queue_cap=64, batched_mode=mode)
    with H.Server(S.filters(5), cfg, max_w=1280, max_h=1024) as srv:
        def camera(c):
            for k, f in enumerate(streams[c]):
                while srv.submit(f, tag=_tag(c, k)) is None:
                    time.sleep(0.001)
                time.sleep(0.002)            # 500 frames/s per camera

        th = [threading.Thread(target=camera, args=(c,)) for c in range(8)]
        for t in th:
            t.start()
        want = sum(len(v) for v in streams.values())
        got = _drain(srv, want)
        for t in th:
            t.join()
        st = srv.stats()
    assert len(got) == want
    for (c, k), ref in alone.items():
        r = got[_tag(c, k)]
        assert r["status"] == 0 and r["count"] == len(ref), (c, k)
        assert r["dets"].tobytes() == ref.tobytes(), (c, k)
        assert r["latency_ms"] >= r["queue_ms"] >= 0.0
    assert st["completed"] == want and st["failed"] == 0 and st["submitted"] == want
    assert st["batched_frames"] == want and 1 <= st["batches"] <= want
    assert 1 <= st["lanes"] <= 3 and st["pending"] == 0


def test_full_queue_refuses_and_keeps_accepted(H, S, streams, alone):
    cfg = H.default_server_config(max_batch=1, max_lanes=1, queue_cap=2)
    big = streams[4]
    accepted, refused = [], 0
    with H.Server(S.filters(5), cfg, max_w=1280, max_h=1024) as srv:
        for k in range(40):
            rid = srv.submit(big[k % 5], tag=k)
            if rid is None:
                refused += 1
            else:
                accepted.append(k)
        got = _drain(srv, len(accepted))
        st = srv.stats()
    assert refused > 0 and st["rejected"] == refused
    assert sorted(got) == accepted
    for k in accepted:
        assert got[k]["dets"].tobytes() == alone[(4, k % 5)].tobytes()


def test_close_with_requests_in_flight(H, S, streams):
    cfg = H.default_server_config(max_batch=4, max_lanes=2, queue_cap=16)
    srv = H.Server(S.filters(5), cfg, max_w=1280, max_h=1024)
    for k in range(16):
        assert srv.submit(streams[k % 8][k % 5], tag=k) is not None
    srv.close()                                   # drains, then stops the worker
    srv.close()


def test_poll_splits_boxes_by_capacity(H, S, streams, alone):
    cfg = H.default_server_config(max_batch=2, max_lanes=1, queue_cap=8)
    with H.Server(S.filters(5), cfg, max_w=1280, max_h=1024) as srv:
        srv.submit(streams[1][0], tag=1)
        srv.submit(streams[5][0], tag=2)
        got = []
        t0 = time.time()
        while len(got) < 2 and time.time() - t0 < 30:
            got += srv.poll(cap=1, det_cap=3, wait_us=20000)
    ref = {1: alone[(1, 0)], 2: alone[(5, 0)]}
    for r in got:
        assert r["count"] == len(ref[r["tag"]])
        n = min(3, r["count"])
        assert len(r["dets"]) == n and r["dets"].tobytes() == ref[r["tag"]][:n].tobytes()
