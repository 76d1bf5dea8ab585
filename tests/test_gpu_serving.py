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


def test_lane_classes_admit_small_frames_while_large_ones_wait(H, S, alone, streams):
    """Lanes sized for the camera mix: two lanes for frames up to 640x480
    and one for 1280x1024.  A burst of large frames queues for the one large
    lane while small frames submitted after them are admitted to the small
    lanes and finish first; no large frame runs on a small lane, the small
    lanes hold less device memory than the large one, and every result is
    the frame's hog_detect result alone."""
    cfg = H.default_server_config(max_batch=1, queue_cap=64, mem_reserve=0,
                                  classes=[(640, 480, 2), (1280, 1024, 1)])
    big = [(c, k) for c in (4, 5, 6, 7) for k in range(3)]      # 1280x1024 cameras
    small = [(c, k) for c in (1, 2, 3) for k in range(4)]       # 640x480 cameras
    with H.Server(S.filters(5), config=cfg, max_w=1280, max_h=1024) as srv:
        st = srv.stats()
        assert st["class_lanes"][:2] == [2, 1] and st["lanes"] == 3
        assert 0 < st["class_bytes"][0] < st["class_bytes"][1]
        order = []
        for c, k in big + small:                 # all large frames first
            assert srv.submit(streams[c][k], tag=_tag(c, k)) is not None
        got = {}
        t0 = time.time()
        while len(got) < len(big) + len(small) and time.time() - t0 < 60:
            for r in srv.poll(cap=16, wait_us=20000):
                got[r["tag"]] = r
                order.append(r["tag"])
        assert len(got) == len(big) + len(small)
        for c, k in big + small:
            r = got[_tag(c, k)]
            assert r["status"] == 0
            assert r["lane_class"] == (1 if (c, k) in big else 0)
            want = alone[(c, k)]
            assert r["count"] == len(want) and r["dets"].tobytes() == want.tobytes()
        # small frames were admitted while large ones waited for their lane
        last_big = max(order.index(_tag(c, k)) for c, k in big)
        first_small = min(order.index(_tag(c, k)) for c, k in small)
        assert first_small < last_big
        st = srv.stats()
        assert st["class_frames"][:2] == [len(small), len(big)]


def test_lane_classes_validation(H, S):
    bad = H.default_server_config(classes=[(640, 480, 2)])     # nothing holds 1280x1024
    with pytest.raises(H.HogError):
        H.Server(S.filters(5), config=bad, max_w=1280, max_h=1024)
    bad = H.default_server_config(classes=[(640, 480, 9), (1280, 1024, 9)])   # 18 lanes
    with pytest.raises(H.HogError):
        H.Server(S.filters(5), config=bad, max_w=1280, max_h=1024)
