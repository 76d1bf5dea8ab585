"""Oracle pins for region-of-interest detection (Section 6.6, future work:
scan only the scales and locations near the previous frame's face).  A
window is scanned iff its level is in [lmin, lmax] and its frame-pixel
centre lies in [x0, x1) x [y0, y1).  Checked against an exact rational
evaluation of the centre, against plain detection for an all-covering
region, and for subset relations."""
from fractions import Fraction

import numpy as np
import pytest

BIG = 1e9


def _cands_in(oracle, cands, W, H, roi):
    sizes = oracle.level_sizes(W, H)
    x0, y0, x1, y1, lmin, lmax = (Fraction(r) for r in roi)
    keep = []
    for c in cands:
        l, u, v = int(c["level"]), int(c["u"]), int(c["v"])
        Wl, Hl = sizes[l]
        cx = Fraction(8 * v + 40) * Fraction(W, Wl)
        cy = Fraction(8 * u + 40) * Fraction(H, Hl)
        if lmin <= l <= lmax and x0 <= cx < x1 and y0 <= cy < y1:
            keep.append((l, int(c["filter"]), u, v))
    return sorted(keep)


@pytest.fixture(scope="module")
def case():
    from paper_2006_00816_gb300 import synth
    return synth.eyeblink_frame(6), synth.filters(3, config=8)


def test_roi_all_covering_equals_plain(oracle, case):
    f, W = case
    a, na = oracle.detect(f, W)
    b, nb = oracle.detect_roi(f, W, (-BIG, -BIG, BIG, BIG, 0, 99))
    assert na == nb and a.tobytes() == b.tobytes()


def test_roi_empty(oracle, case):
    f, W = case
    k, n = oracle.detect_roi(f, W, (300.5, 200.5, 300.5, 400.0, 0, 99))
    assert n == 0 and len(k) == 0
    k, n = oracle.detect_roi(f, W, (-BIG, -BIG, BIG, BIG, 5, 4))
    assert n == 0 and len(k) == 0


@pytest.mark.parametrize("roi", [(150.3, 90.7, 470.1, 390.9, 1, 4),
                                 (0.0, 0.0, 320.0, 480.0, 0, 9),
                                 (333.3, 17.9, 640.0, 301.1, 3, 3)])
def test_roi_candidates_match_exact_centres(oracle, case, roi):
    f, W = case
    allc = oracle.frame_candidates(f, W)
    want = _cands_in(oracle, allc, 640, 480, roi)
    # the restricted candidate count, and the kept boxes, come from that set
    k, n = oracle.detect_roi(f, W, roi)
    assert n == len(want)
    kept = sorted((int(r["level"]), int(r["filter"]), int(r["u"]), int(r["v"])) for r in k)
    assert set(kept) <= set(want)
    # greedy NMS over exactly that set gives the kept boxes
    sel = np.array([(int(c["level"]), int(c["filter"]), int(c["u"]), int(c["v"])) in set(want)
                    for c in allc])
    srt, keep = oracle.nms(allc[sel], 0.5)
    assert sorted((int(r["level"]), int(r["filter"]), int(r["u"]), int(r["v"]))
                  for r in srt[keep]) == kept


def test_roi_subset(oracle, case):
    f, W = case
    big = (100.0, 50.0, 560.0, 430.0, 0, 9)
    small = (200.0, 120.0, 450.0, 360.0, 1, 6)
    allc = oracle.frame_candidates(f, W)
    assert set(_cands_in(oracle, allc, 640, 480, small)) <= set(_cands_in(oracle, allc, 640, 480, big))
    assert oracle.in_roi(640, 480, 640, 480, 0, 0, 0, (40.0, 40.0, 41.0, 41.0, 0, 0))
    assert not oracle.in_roi(640, 480, 640, 480, 0, 0, 0, (40.5, 40.0, 41.0, 41.0, 0, 0))
