"""Pins of the oracle's training adjoint (hinge loss on the best window
score of one filter, float pyramid) against FP64 central finite differences
of the oracle's own forward pass (eps 1e-3, relative tolerance 1e-3),
skipping perturbations that change a discrete state (orientation bins,
argmax window, truncation set)."""
import numpy as np
import pytest

from paper_2006_00816_gb300 import synth


@pytest.fixture(scope="module")
def batch(oracle):
    """Four 128x128 crops (three levels).  The filter is a zero-mean copy of
    crop 1's level-1 features (plus noise), so the best window of that crop
    lies on a downscaled level and the pyramid adjoint is exercised."""
    imgs, labels = synth.crops(4, size=128, config=41)
    feats = oracle.frame_features(imgs[1], float_mode=True)
    W = feats[1][1:11, 1:11, :].copy()
    W = (W - W.mean()) + 0.01 * synth.filters(1, config=41)[0]
    return imgs.astype(np.float64), labels.astype(np.float64), W.astype(np.float64)


def test_fixture_reaches_a_downscaled_level(oracle, batch):
    imgs, labels, W = batch
    _, _, win = oracle.hinge_loss(imgs, labels, W)
    assert (win[:, 0] >= 1).any()


def _loss_one(oracle, img, y, W, n):
    loss, _, _ = oracle.hinge_loss(img[None], np.array([y]), W)
    return loss / n            # crop's share of the batch-mean loss


def test_loss_definition(oracle, batch):
    imgs, labels, W = batch
    loss, s, win = oracle.hinge_loss(imgs, labels, W)
    assert loss == pytest.approx(np.mean(np.maximum(0.0, 1.0 - labels * s)), rel=1e-14)
    # best score equals the max over the oracle's float-mode score maps
    for i in range(len(imgs)):
        feats = oracle.frame_features(imgs[i].astype(np.uint8), float_mode=True)
        best = max(oracle.correlate(f, W[None])[0].max() for f in feats)
        assert s[i] == pytest.approx(best, rel=1e-12)


def test_dW_matches_finite_differences(oracle, batch):
    imgs, labels, W = batch
    loss, dW, _ = oracle.hinge_backward(imgs, labels, W, with_image=False)
    rng = np.random.default_rng(5)
    eps = 1e-3
    for _ in range(40):
        a, b, c = rng.integers(0, 10), rng.integers(0, 10), rng.integers(0, 31)
        Wp, Wm = W.copy(), W.copy()
        Wp[a, b, c] += eps
        Wm[a, b, c] -= eps
        _, sp, wp = oracle.hinge_loss(imgs, labels, Wp)
        _, sm, wm = oracle.hinge_loss(imgs, labels, Wm)
        if not np.array_equal(wp, wm):
            continue                          # argmax changed: not differentiable here
        fd = (oracle.hinge_loss(imgs, labels, Wp)[0] - oracle.hinge_loss(imgs, labels, Wm)[0]) / (2 * eps)
        assert fd == pytest.approx(dW[a, b, c], rel=1e-6, abs=1e-12)


def test_dI_matches_finite_differences(oracle, batch):
    imgs, labels, W = batch
    n = len(imgs)
    loss, dW, dI = oracle.hinge_backward(imgs, labels, W)
    eps = 1e-3
    gmax = np.abs(dI).max()
    assert gmax > 0
    rng = np.random.default_rng(9)
    checked = 0
    for i in range(n):
        sig0 = oracle.forward_signature(imgs[i], W)
        nz = np.argwhere(np.abs(dI[i]) > 1e-3 * gmax)
        picks = nz[rng.choice(len(nz), size=min(25, len(nz)), replace=False)] if len(nz) else []
        for (y, x) in picks:
            p, m = imgs[i].copy(), imgs[i].copy()
            p[y, x] += eps
            m[y, x] -= eps
            if (oracle.forward_signature(p, W) != sig0 or
                    oracle.forward_signature(m, W) != sig0):
                continue
            fd = (_loss_one(oracle, p, labels[i], W, n) - _loss_one(oracle, m, labels[i], W, n)) / (2 * eps)
            g = dI[i, y, x]
            assert abs(fd - g) <= 1e-3 * abs(g) + 1e-6 * gmax, (i, y, x, fd, g)
            checked += 1
    assert checked >= 40


def test_inactive_crop_has_zero_gradient(oracle, batch):
    imgs, labels, W = batch
    _, s, _ = oracle.hinge_loss(imgs, labels, W)
    # labels scaled so that every margin y*s >= 2 > 1 -> inactive -> zero gradients
    loss, dW, dI = oracle.hinge_backward(imgs, np.sign(s) * np.maximum(1.0, 2.0 / np.abs(s)), W)
    assert loss == 0.0 and not dW.any() and not dI.any()


def _fnv(values):
    """The 64-bit FNV-style mix the oracle's forward signature applies to
    each value in turn (x as int64, reinterpreted as uint64)."""
    h = 1469598103934665603
    for x in values:
        h ^= int(x) & 0xFFFFFFFFFFFFFFFF
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _atan2_bin(dx, dy):
    """Nearest of the 18 signed centres 20 b degrees by atan2 (reading R4;
    dx == 0 ties: 4 for dy > 0, 13 for dy < 0; -1 for a zero gradient)."""
    if dx == 0 and dy == 0:
        return -1
    if dx == 0:
        return 4 if dy > 0 else 13
    ang = np.degrees(np.arctan2(dy, dx)) % 360.0
    return int(np.floor(ang / 20.0 + 0.5)) % 18


def test_forward_state_is_the_signature_state(oracle, batch):
    """forward_state returns, as arrays, exactly what forward_signature
    hashes (best window, every bin of its level, the window's truncation
    tests); its bins follow the atan2 rule on the FP64 float pyramid, and the
    truncation tests match a direct evaluation of the normalisers."""
    imgs, labels, W = batch
    for i in range(len(imgs)):
        (l, u, v), bins, trunc = oracle.forward_state(imgs[i], W)
        _, _, win = oracle.hinge_loss(imgs[i:i + 1], labels[i:i + 1], W)
        assert (l, u, v) == tuple(win[0])
        want = _fnv([l, u, v] + bins[1:-1, 1:-1].ravel().tolist() + trunc.ravel().tolist())
        assert want == oracle.forward_signature(imgs[i], W)
        lvl = oracle.pyramid_f64(imgs[i])[l]
        rng = np.random.default_rng(i)
        for y, x in zip(rng.integers(1, lvl.shape[0] - 1, 300), rng.integers(1, lvl.shape[1] - 1, 300)):
            dx = lvl[y, x + 1] - lvl[y, x - 1]
            dy = lvl[y + 1, x] - lvl[y - 1, x]
            assert bins[y, x] == _atan2_bin(dx, dy)
        hist = oracle.cell_hist(lvl)
        cy, cx = hist.shape[:2]
        E = ((hist[..., :9] + hist[..., 9:]) ** 2).sum(-1)
        Ep = np.pad(E, 1)
        for a, b, k in [(0, 0, 0), (4, 7, 3), (9, 9, 1), (5, 2, 2)]:
            ci, cj = u + a, v + b
            ddx, ddy = [(-1, -1), (1, -1), (-1, 1), (1, 1)][k]
            S = Ep[ci + 1, cj + 1] + Ep[ci + 1, cj + 1 + ddx] + Ep[ci + 1 + ddy, cj + 1] + \
                Ep[ci + 1 + ddy, cj + 1 + ddx]
            N = 1.0 / np.sqrt(S + oracle.EPS)
            hc = hist[ci, cj]
            direct = np.concatenate([hc * N < oracle.TAU, (hc[:9] + hc[9:]) * N < oracle.TAU])
            assert np.array_equal(trunc[a * 10 + b, k], direct.astype(np.uint8))
