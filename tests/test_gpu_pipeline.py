"""CPU/GPU pipeline (hog_pipeline_run; Sections 5.2 and 5.3, Table 8):
face detection on the GPU overlapped with the host landmark stage.  The
pipelined and the sequential order give the same outputs bit for bit, and
each frame's landmarks are hog_ert_fit on that frame's best detection from
hog_detect."""
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


def test_pipeline_orders_agree_and_match_per_frame(H):
    from paper_2006_00816_gb300 import synth
    frames = [synth.eyeblink_frame(i) for i in range(21)] + [np.full((480, 640), 9, np.uint8)]
    det = H.Detector(synth.filters(5), max_w=640, max_h=480, max_batch=8)
    ert = H.Ert(cascades=4, trees=60, depth=4, features=100, seed=3)
    seq = H.pipeline_run(det, ert, frames, batch=8, n_threads=4, pipelined=0)
    pipe = H.pipeline_run(det, ert, frames, batch=8, n_threads=4, pipelined=1)
    for a, b in zip(seq[:3], pipe[:3]):
        assert np.array_equal(a, b)
    lm, ear, face, _ = pipe
    assert face[-1] == 0 and not lm[-1].any()          # constant frame: no detection
    for i, f in enumerate(frames):
        d, c = det.detect([torch.from_numpy(f).cuda()])
        assert bool(face[i]) == (c[0] > 0)
        if c[0] == 0:
            continue
        best = d[int(np.argmax(d["score"]))]
        ref_lm, ref_ear = ert.fit(f, best)
        assert np.array_equal(lm[i], ref_lm), i
        assert np.array_equal(ear[i], ref_ear), i
    ert.close()
