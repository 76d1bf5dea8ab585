"""hog_features_static: the features entry point for callers that cannot
allocate device memory (a hard-deadline frame loop, where cudaMalloc may
block and synchronise the device, or a host application whose own pool owns
all device memory).  Its scratch is a fixed 4 MiB device array inside
libhog, so frames are limited to 640x480.

The test calls it through the C ABI twice in a row on different frames and
compares each result with hog_features (the context-based entry point)
within the feature tolerance of the parity tests; it also checks that an
oversize frame is rejected with a clear message.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FEAT_RTOL, FEAT_FLOOR = 1e-5, 1e-6


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog
    return hog


def test_static_features_match_context_features(H):
    from paper_2006_00816_gb300 import synth
    det = H.Detector(synth.filters(1), max_w=640, max_h=480, max_batch=1)
    # an exact 640x480 frame (the largest legal size), then a ragged one
    frames = [synth.eyeblink_frame(4), synth.single_frame(333, 211, config=13)]
    assert frames[0].shape == (480, 640)
    for f in frames:                       # two calls in a row, different sizes
        ft = torch.from_numpy(f).cuda()
        got, rc, msg = H.features_static(ft)
        assert rc == 0, msg
        ref = det.features(ft)
        assert len(got) == len(ref) > 0
        for g, r in zip(got, ref):
            g = g.cpu().numpy().astype(np.float64)
            r = r.cpu().numpy().astype(np.float64)
            assert g.shape == r.shape
            assert np.all(np.abs(g - r) <= FEAT_RTOL * np.maximum(np.abs(r), FEAT_FLOOR))
    det.close()


def test_static_features_reject_oversize(H):
    big = torch.zeros((481, 640), dtype=torch.uint8, device="cuda")
    _, rc, msg = H.features_static(big)
    assert rc == H.HOG_EINVAL
    assert "exceeds the static limit 640x480" in msg


def test_static_every_legal_size_fits(H):
    """The scratch layout and the job table hold every frame up to the limit:
    a sweep over widths and heights (the exact 640x480 limit included, the
    largest legal frame) returns HOG_OK for each, never the scratch-too-small
    or job-table-too-small error."""
    sizes = [(w, h) for w in range(80, 641, 7) for h in (80, 241, 479, 480)]
    sizes += [(w, h) for h in range(80, 481, 7) for w in (639, 640)]
    sizes += [(640, 480), (640, 479), (639, 480), (80, 80), (81, 80)]
    buf = torch.randint(0, 256, (480, 640), dtype=torch.uint8, device="cuda")
    for w, h in sizes:
        got, rc, msg = H.features_static(buf[:h, :w])
        assert rc == 0, (w, h, msg)
        assert len(got) >= 1
    torch.cuda.synchronize()
