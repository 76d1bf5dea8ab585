"""GPU tests of the batched path (hog_detect_batched): the persistent fused
launch and the per-stage launches, each replayed as a CUDA graph, give the
same detections bit for bit as hog_detect, for frames of mixed resolution;
the autotuner only changes speed, never results."""
import json
import os

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
def synth():
    from paper_2006_00816_gb300 import synth as S
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _mixed(S, n):
    return [dev(f) for f in S.mixed_frames(n)]


@pytest.mark.parametrize("mode", [1, 0])
def test_batched_equals_per_stage(H, synth, mode):
    W = synth.filters(5)
    det = H.Detector(W, max_w=1280, max_h=1024, max_batch=6)
    det.set_batched_mode(mode)
    frames = _mixed(synth, 9) + [dev(np.full((90, 100), 7, np.uint8))]
    ref, rc = det.detect(frames)
    for call in range(3):            # eager, graph capture, graph replay
        got, gc = det.detect(frames, batched=True)
        assert gc.tolist() == rc.tolist(), (mode, call)
        assert np.array_equal(got, ref), (mode, call)


def test_batched_640x480_stream(H, synth):
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=32)
    frames = [dev(f) for f in synth.eyeblink_stream(40)]
    ref, rc = det.detect(frames)
    out, keep = H.pinned_dets(40 * 2000)
    for _ in range(3):
        got, gc = det.detect(frames, batched=True, out=out)
        assert gc.tolist() == rc.tolist()
        assert np.array_equal(got, ref)


def test_autotune_keeps_results_and_caches(H, synth, tmp_path):
    W = synth.filters(5)
    det = H.Detector(W, max_w=1280, max_h=1024, max_batch=8)
    frames = _mixed(synth, 8)
    path = str(tmp_path / "tune.json")
    mode, pol = det.autotune(frames, cache_path=path)
    assert mode in (0, 1) and 0 <= pol <= 3
    rec = json.load(open(path))
    assert rec["batched_mode"] == mode and rec["corr_policy"] == pol
    assert len(rec["corr_ms_by_policy"]) == 4
    # the per-frame call under the chosen correlation engine
    ref, rc = det.detect(frames)
    got, gc = det.detect(frames, batched=True)
    assert gc.tolist() == rc.tolist()
    assert np.array_equal(got, ref)       # tile shapes change speed, not arithmetic
    # a fresh context loads the cached choice without measuring
    det2 = H.Detector(W, max_w=1280, max_h=1024, max_batch=8)
    assert det2.autotune(frames, cache_path=path) == (mode, pol)
    os.remove(path)


def test_batch_tensor_and_chunked_host_copies(H, synth):
    """One [n, h, w] tensor gives the same detections as the list of its
    frames, per frame and batched; hog_detect_host, which moves host frames
    in chunks of max_batch / 2 through two staging halves (copies of the
    next chunk overlapping detection of this one), gives the device result
    for a pinned [n, h, w] array (one copy per chunk), for plain numpy
    frames of several sizes and for row-strided views."""
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=4)
    host = synth.eyeblink_stream(11)
    fd = dev(host)
    ref, rc = det.detect([fd[i] for i in range(11)])
    for batched in (False, True):
        got, gc = det.detect(fd, batched=batched)
        assert gc.tolist() == rc.tolist() and np.array_equal(got, ref), batched
    pinned = torch.from_numpy(host).pin_memory().numpy()
    for frames in (pinned, list(pinned), list(host), host):
        got, gc = det.detect_host(frames)
        assert gc.tolist() == rc.tolist() and np.array_equal(got, ref)
    mixed = [host[0], host[1][:300, :500], np.ascontiguousarray(host[2][::2, ::2]),
             host[3][17:400, 33:600], np.full((90, 100), 7, np.uint8), host[4],
             np.zeros((0, 0), np.uint8), pinned[5][:, :320], host[6]]
    want, wc = det.detect([dev(f) for f in mixed])
    for _ in range(2):
        got, gc = det.detect_host(mixed)
        assert gc.tolist() == wc.tolist() and np.array_equal(got, want)
    got, gc = det.detect_host(mixed[:1])                 # one frame: no chunking
    assert gc[0] == wc[0]


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 1])
def test_host_chunks_with_one_suppression(H, synth, mode):
    """hog_detect_host on a group of more than max_batch / 2 frames runs the
    per-frame stages chunk by chunk (each chunk in buffer slots of its own)
    and one suppression launch over the whole group: per-stage and fused
    modes give the device result, on a full group, a group with a ragged
    last chunk, two groups, and with the output capacity cut short."""
    W = synth.filters(5)
    det = H.Detector(W, max_w=640, max_h=480, max_batch=8)
    det.set_batched_mode(mode)
    host = synth.eyeblink_stream(19, start=40)
    pinned = torch.from_numpy(host).pin_memory().numpy()
    fd = dev(host)
    for n in (8, 7, 19):
        ref, rc = det.detect([fd[i] for i in range(n)])
        for _ in range(2):   # the second call replays the cached plans' graphs
            got, gc = det.detect_host(pinned[:n])
            assert gc.tolist() == rc.tolist() and np.array_equal(got, ref), n
            assert (got["frame"] == np.repeat(np.arange(n), rc)).all()
    ref, rc = det.detect([fd[i] for i in range(8)])
    cap = int(rc[:3].sum()) + 5
    part, pc = det.detect_host(pinned[:8], det_cap=cap, allow_capacity=True)
    assert pc.tolist() == rc.tolist() and len(part) == cap
    assert np.array_equal(part, ref[:cap])


@pytest.mark.gpu
def test_host_chunks_mixed_workspace_classes(H, synth):
    """A chunked host group whose frames fall in two suppression workspace
    classes (whole workspace in shared memory, key words alone in shared
    memory), which one back plan launches side by side: equal to the device
    batch and to the per-frame calls."""
    W = synth.filters(5)
    frames = synth.mixed_frames(12)
    sizes = {f.shape for f in frames}
    assert (1024, 1280) in sizes or (720, 1280) in sizes
    assert (480, 640) in sizes or (240, 320) in sizes
    det = H.Detector(W, max_w=1280, max_h=1024, max_batch=8)
    ref, rc = det.detect([dev(f) for f in frames])
    dev_b, dc = det.detect([dev(f) for f in frames], batched=True)
    assert dc.tolist() == rc.tolist() and np.array_equal(dev_b, ref)
    for _ in range(2):
        got, gc = det.detect_host(frames)
        assert gc.tolist() == rc.tolist() and np.array_equal(got, ref)
