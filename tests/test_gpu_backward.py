"""GPU tests of the hand-written adjoint (hog_backward): hinge loss on the
best window score of one filter over 64 seeded 128x128 crops (half with a
planted ellipse, labels +1/-1).

Bars: loss and best scores against the FP64 oracle; dW and dI against the
oracle's FP64 adjoint to 1e-3 relative (floor 1e-6 of the largest
magnitude); dI against FP64 central finite differences of the oracle's
forward (eps 1e-3, 1e-3 relative), skipping perturbations that change a
discrete state (bins, best window, truncation set); recompute modes and
repeated calls bit-identical; torch autograd equal to the raw call."""
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
def data(oracle):
    from paper_2006_00816_gb300 import synth
    imgs, labels = synth.crops(64, size=128, config=4)
    # filter: a zero-mean level-1 template of one crop plus N(0, 0.01) noise,
    # so best windows fall on several levels
    feats = oracle.frame_features(imgs[3], float_mode=True)
    W = feats[1][1:11, 1:11, :].copy()
    W = ((W - W.mean()) + synth.filters(1, config=4)[0]).astype(np.float32)
    return imgs.astype(np.float32), labels.astype(np.float32), W


def _close(g, o, rtol=1e-3):
    scale = np.abs(o).max()
    return np.abs(g - o) <= rtol * np.abs(o) + 1e-6 * scale


def test_backward_matches_oracle_adjoint(H, oracle, data):
    imgs, labels, W = data
    det = H.Detector(W[None], max_w=128, max_h=128, max_batch=1)
    ti, tl, tw = (torch.from_numpy(x).cuda() for x in (imgs, labels, W))
    loss, dW, dI = det.backward(ti, tl, tw)
    oloss, osc, owin = oracle.hinge_loss(imgs, labels, W)
    assert loss == pytest.approx(oloss, rel=1e-5, abs=1e-6)
    assert (owin[:, 0] >= 1).any() and (owin[:, 0] == 0).any()
    ol, odW, odI = oracle.hinge_backward(imgs, labels, W)
    g = dW.cpu().numpy().astype(np.float64)
    assert _close(g, odW).all(), np.abs(g - odW).max()
    gi = dI.cpu().numpy().astype(np.float64)
    ok = _close(gi, odI)
    assert ok.mean() > 0.9999, (1 - ok.mean(), np.abs(gi - odI).max(), np.abs(odI).max())
    assert np.linalg.norm(gi - odI) <= 1e-3 * np.linalg.norm(odI)


def test_backward_matches_finite_differences(H, oracle, data):
    imgs, labels, W = data
    n = 16
    imgs, labels = imgs[:n], labels[:n]
    det = H.Detector(W[None], max_w=128, max_h=128, max_batch=1)
    _, _, dI = det.backward(*(torch.from_numpy(x).cuda() for x in (imgs, labels, W)))
    dI = dI.cpu().numpy().astype(np.float64)
    gmax = np.abs(dI).max()
    rng = np.random.default_rng(3)
    eps, checked = 1e-3, 0
    Wd = W.astype(np.float64)
    for i in range(n):
        sig0 = oracle.forward_signature(imgs[i], Wd)
        nz = np.argwhere(np.abs(dI[i]) > 1e-2 * gmax)
        if not len(nz):
            continue
        for (y, x) in nz[rng.choice(len(nz), size=min(6, len(nz)), replace=False)]:
            p = imgs[i].astype(np.float64).copy()
            m = p.copy()
            p[y, x] += eps
            m[y, x] -= eps
            if oracle.forward_signature(p, Wd) != sig0 or oracle.forward_signature(m, Wd) != sig0:
                continue
            lp = oracle.hinge_loss(p[None], labels[i:i + 1], Wd)[0] / n
            lm = oracle.hinge_loss(m[None], labels[i:i + 1], Wd)[0] / n
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - dI[i, y, x]) <= 1e-3 * abs(fd) + 1e-6 * gmax, (i, y, x, fd, dI[i, y, x])
            checked += 1
    assert checked >= 20


def test_recompute_and_repeat_identical(H, data):
    imgs, labels, W = data
    det = H.Detector(W[None], max_w=128, max_h=128, max_batch=1)
    args = [torch.from_numpy(x).cuda() for x in (imgs, labels, W)]
    l0, w0, i0 = det.backward(*args)
    l1, w1, i1 = det.backward(*args, recompute=True)
    l2, w2, i2 = det.backward(*args)
    assert l0 == l1 == l2
    assert torch.equal(w0, w1) and torch.equal(w0, w2)
    assert torch.equal(i0, i1) and torch.equal(i0, i2)


def test_inactive_crops_have_zero_gradient(H, data):
    imgs, labels, W = data
    det = H.Detector(W[None], max_w=128, max_h=128, max_batch=1)
    ti, tw = torch.from_numpy(imgs[:8]).cuda(), torch.from_numpy(W).cuda()
    _, _, _ = det.backward(ti, torch.ones(8, device="cuda"), tw)
    # labels that make every margin at least 2: loss 0, zero gradients
    import oracle as O
    _, s, _ = O.hinge_loss(imgs[:8], np.ones(8), W)
    y = (np.sign(s) * np.maximum(1.0, 2.0 / np.maximum(np.abs(s), 1e-12))).astype(np.float32)
    loss, dW, dI = det.backward(ti, torch.from_numpy(y).cuda(), tw)
    assert loss == 0.0 and not dW.any() and not dI.any()


def test_autograd_function(H, data):
    imgs, labels, W = data
    det = H.Detector(W[None], max_w=128, max_h=128, max_batch=1)
    ti = torch.from_numpy(imgs[:8]).cuda().requires_grad_(True)
    tw = torch.from_numpy(W).cuda().requires_grad_(True)
    tl = torch.from_numpy(labels[:8]).cuda()
    loss = H.hinge_loss(det, ti, tl, tw)
    (2.0 * loss).backward()
    l, dW, dI = det.backward(ti.detach(), tl, tw.detach())
    assert loss.item() == pytest.approx(l)
    assert torch.allclose(tw.grad, 2.0 * dW) and torch.allclose(ti.grad, 2.0 * dI)
