"""Pins of the oracle's energy, block normalisation, truncation and the 31
features (paper Section 4.1.1: energy sum_{n<9}(h_n+h_{n+9})^2 over the cell
and its eight neighbours; 18 signed + 9 unsigned + 4 energy features;
reading R6: eps 1e-4, tau 0.2, texture weight 0.2357)."""
import json
import math
import os

import numpy as np
import pytest

EPS, TAU, TW = 1e-4, 0.2, 0.2357
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def test_feature_dimension_matches_paper(oracle):
    facts = json.load(open(GOLDEN))
    assert oracle.NFEAT == facts["feature_dim"]["value"] == sum(facts["feature_dim"]["parts"])
    assert oracle.NBIN == facts["n_orientations"]["value"]
    assert oracle.CELL == facts["cell_px"]["value"]
    assert oracle.WIN * oracle.WIN * oracle.NFEAT == facts["filter_weights"]["value"]
    f = oracle.features(np.zeros((3, 3, 18)))
    assert f.shape == (3, 3, 31)


def test_constant_image_zero_features(oracle):
    img = np.full((120, 96), 201, np.uint8)
    for f in oracle.frame_features(img):
        assert not f.any()


def _ramp_hist(a, h=96, w=128):
    img = np.tile(a * np.arange(w, dtype=np.float64), (h, 1))
    return img


@pytest.mark.parametrize("a,clipped", [(0.5, True), (1e-5, False)])
def test_uniform_gradient_closed_form(oracle, a, clipped):
    """Interior cells of a horizontal ramp hold h0 = 2a*64 in bin 0 only, with
    identical neighbours, so S_k = 4 h0^2 and N_k = 1/sqrt(4 h0^2 + eps)."""
    img = _ramp_hist(a)
    hist = oracle.cell_hist(img)
    f = oracle.features(hist)
    h0 = 2 * a * 64
    n = 1.0 / math.sqrt(4 * h0 * h0 + EPS)
    r = min(h0 * n, TAU)
    assert clipped == (h0 * n > TAU)
    for i, j in [(3, 4), (5, 7), (6, 9)]:
        cell = f[i, j]
        assert cell[0] == pytest.approx(0.5 * 4 * r, rel=1e-12)
        assert cell[18] == pytest.approx(0.5 * 4 * r, rel=1e-12)
        for k in range(4):
            assert cell[27 + k] == pytest.approx(TW * r, rel=1e-12)
        others = [o for o in range(27) if o not in (0, 18)]
        assert not cell[others].any()


def test_block_neighbourhoods(oracle):
    """A 3x3 cell grid whose cells each hold a distinct value in bin 0 only.
    Without clipping, f[27+k] of the centre = TW * h_c * N_k, so N_k exposes
    which 2x2 block enters S_k: k=0 up-left, 1 up-right, 2 down-left,
    3 down-right."""
    vals = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]]) * 2e-4
    hist = np.zeros((3, 3, 18))
    hist[..., 0] = vals
    f = oracle.features(hist)
    E = vals ** 2
    blocks = {0: [(0, 0), (0, 1), (1, 0), (1, 1)], 1: [(0, 1), (0, 2), (1, 1), (1, 2)],
              2: [(1, 0), (1, 1), (2, 0), (2, 1)], 3: [(1, 1), (1, 2), (2, 1), (2, 2)]}
    hc = vals[1, 1]
    for k, cells in blocks.items():
        S = sum(E[c] for c in cells)
        N = 1.0 / math.sqrt(S + EPS)
        assert hc * N < TAU
        assert f[1, 1, 27 + k] == pytest.approx(TW * hc * N, rel=1e-12)
    # a corner cell sees zero energy outside the grid
    N00 = [1 / math.sqrt(E[0, 0] + EPS),
           1 / math.sqrt(E[0, 0] + E[0, 1] + EPS),
           1 / math.sqrt(E[0, 0] + E[1, 0] + EPS),
           1 / math.sqrt(E[0, 0] + E[0, 1] + E[1, 0] + E[1, 1] + EPS)]
    for k in range(4):
        assert f[0, 0, 27 + k] == pytest.approx(TW * vals[0, 0] * N00[k], rel=1e-12)


def test_energy_uses_opposite_bin_pairs(oracle):
    """E pairs bin n with n+9 (sum then square): h_2 = h_11 = x gives E = 4x^2,
    whereas h_2 = h_12 = x gives E = 2x^2."""
    x = 1e-3
    for pair, E in [((2, 11), 4 * x * x), ((2, 12), 2 * x * x)]:
        hist = np.zeros((1, 1, 18))
        hist[0, 0, list(pair)] = x
        f = oracle.features(hist)
        N = 1.0 / math.sqrt(E + EPS)
        assert f[0, 0, 27] == pytest.approx(TW * 2 * x * N, rel=1e-12)


def test_truncation_bounds_on_frames(oracle):
    from paper_2006_00816_gb300 import synth
    img = synth.single_frame()
    feats = oracle.frame_features(img)
    for f in feats:
        assert (f >= 0).all()
        assert f[..., :27].max() <= 0.4 + 1e-15
        assert f[..., 27:].max() <= TW * 18 * TAU + 1e-15
    # the unnormalised products h*N stay below 1 (S_k >= E >= (h_o+h_o+9)^2)
    lv = oracle.pyramid_u8(img)[1].astype(np.float64)
    hist = oracle.cell_hist(lv)
    E = ((hist[..., :9] + hist[..., 9:]) ** 2).sum(-1)
    assert ((hist[..., :9] + hist[..., 9:]) ** 2 <= E[..., None] + 1e-9).all()


def test_mirror_permutes_features(oracle):
    rng = np.random.default_rng(8)
    img = rng.normal(0, 1, size=(64, 80))
    f0 = oracle.features(oracle.cell_hist(img))
    f1 = oracle.features(oracle.cell_hist(img[:, ::-1].copy()))[:, ::-1, :]
    perm = ([(9 - o) % 18 for o in range(18)] + [18 + (9 - o) % 9 for o in range(9)]
            + [28, 27, 30, 29])
    assert np.allclose(f1[..., perm], f0, rtol=1e-12, atol=1e-14)


def test_offset_invariance_features(oracle):
    rng = np.random.default_rng(4)
    img = rng.integers(0, 180, size=(100, 120)).astype(np.uint8)
    a = oracle.frame_features(img)
    b = oracle.frame_features(img + 60)
    for x, y in zip(a, b):
        assert (x == y).all()
