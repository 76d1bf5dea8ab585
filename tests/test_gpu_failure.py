"""Failure path of the bounded device waits, tested without a GPU fault.

The persistent fused launch (hog_detect_batched in mode 1) orders its work
items by dependency and lets an item wait, a bounded number of polls, on the
completion counter of the items it reads.  hog_debug_waits makes one such
wait expect a completion that no item gives (host-side injection: the plan's
first dependency target is raised by one) and shortens the poll budget, so
the wait runs out: the launch stops, the call returns HOG_ETIMEOUT, and the
context keeps working once the injection is switched off.
"""
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


def test_withheld_completion_times_out_and_context_recovers(H):
    from paper_2006_00816_gb300 import synth
    W = synth.filters(5)
    frames = torch.from_numpy(synth.eyeblink_stream(12)).cuda()
    det = H.Detector(W, max_w=640, max_h=480, max_batch=12)
    ref, rc = det.detect(frames)
    det.set_batched_mode(1)
    got, gc = det.detect(frames, batched=True)
    assert np.array_equal(gc, rc) and got.tobytes() == ref.tobytes()

    det.debug_waits(polls=2000, withhold=True)
    for call in range(2):                        # eager, then the captured graph
        t0 = time.perf_counter()
        with pytest.raises(H.HogError) as ei:
            det.detect(frames, batched=True)
        assert ei.value.code == H.HOG_ETIMEOUT, call
        assert "bounded device wait" in det.last_error()
        assert time.perf_counter() - t0 < 10.0   # 2000 polls, not 2^24
    torch.cuda.synchronize()                     # the context is still usable

    det.debug_waits(polls=0, withhold=False)
    for call in range(3):                        # eager, capture, replay
        got, gc = det.detect(frames, batched=True)
        assert np.array_equal(gc, rc) and got.tobytes() == ref.tobytes(), call
    got, gc = det.detect(frames)
    assert got.tobytes() == ref.tobytes()
    with pytest.raises(H.HogError):
        det.debug_waits(polls=-1)
    det.close()
