"""Host landmark stage stand-in (hog_ert, Sections 4.2 and 5.2): the paper's
ensemble-of-regression-trees structure with seeded parameters (no trained
model exists here).  Checked against an independent numpy implementation
that regenerates the parameters from the same published counter-based
generator (splitmix64) and walks the same cascade; determinism; the eye
aspect ratio of the mean shape."""
import numpy as np
import pytest

M64 = (1 << 64) - 1


class SplitMix64:
    """Steele, Lea and Flood's SplitMix64 (as published by Vigna)."""

    def __init__(self, seed):
        self.s = seed & M64

    def next(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & M64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def uniform(self):
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, n):
        return int(self.uniform() * n)


def _model(L, T, K, D, P, seed):
    r = SplitMix64(seed)
    mean = np.zeros((L, 2), np.float32)
    for l in range(L):
        mean[l, 0] = np.float32(0.15 + 0.7 * r.uniform())
        mean[l, 1] = np.float32(0.15 + 0.7 * r.uniform())
    px = np.float32([-1.0, -0.5, 0.5, 1.0, 0.5, -0.5])
    py = np.float32([0.0, -1.0, -1.0, 0.0, 1.0, 1.0])
    for e, first in ((0, 36), (1, 42)):
        cx = np.float32(0.3 if e == 0 else 0.7)
        for k in range(6):
            mean[first + k, 0] = cx + np.float32(0.08) * px[k]
            mean[first + k, 1] = np.float32(0.38) + np.float32(0.024) * py[k]
    anchor = np.zeros(T * P, np.int64)
    offset = np.zeros((T * P, 2), np.float32)
    for i in range(T * P):
        anchor[i] = r.below(L)
        offset[i, 0] = np.float32(0.2 * r.uniform() - 0.1)
        offset[i, 1] = np.float32(0.2 * r.uniform() - 0.1)
    nodes, leaves = (1 << D) - 1, 1 << D
    split = np.zeros((T * K * nodes, 2), np.int64)
    thresh = np.zeros(T * K * nodes, np.float32)
    for i in range(T * K * nodes):
        split[i, 0] = r.below(P)
        split[i, 1] = r.below(P)
        thresh[i] = np.float32(60.0 * r.uniform() - 30.0)
    leaf = np.array([np.float32(0.001 * r.uniform() - 0.0005)
                     for _ in range(T * K * leaves * L * 2)], np.float32)
    return mean, anchor.reshape(T, P), offset.reshape(T, P, 2), \
        split.reshape(T, K, nodes, 2), thresh.reshape(T, K, nodes), \
        leaf.reshape(T, K, leaves, L, 2)


def _lround(x):
    x = float(x)
    return int(np.floor(abs(x) + 0.5)) * (1 if x >= 0 else -1)


def _fit(model, img, box, D):
    mean, anchor, offset, split, thresh, leaf = model
    h, w = img.shape
    bx, by, bw, bh = (np.float32(v) for v in box)
    s = np.empty_like(mean)
    s[:, 0] = bx + bw * mean[:, 0]
    s[:, 1] = by + bh * mean[:, 1]
    T, K, nodes = thresh.shape
    for t in range(T):
        x = s[anchor[t], 0] + bw * offset[t, :, 0]
        y = s[anchor[t], 1] + bh * offset[t, :, 1]
        xi = np.array([min(max(_lround(v), 0), w - 1) for v in x])
        yi = np.array([min(max(_lround(v), 0), h - 1) for v in y])
        pv = img[yi, xi].astype(np.float32)
        for k in range(K):
            n = 0
            for _ in range(D):
                a, b = split[t, k, n]
                n = 2 * n + 1 + (1 if np.float32(pv[a] - pv[b]) > thresh[t, k, n] else 0)
            inc = leaf[t, k, n - nodes]
            s[:, 0] = s[:, 0] + bw * inc[:, 0]
            s[:, 1] = s[:, 1] + bh * inc[:, 1]
    return s


def _ear(s, first):
    def d(a, b):
        dx = np.float32(s[first + a, 0] - s[first + b, 0])
        dy = np.float32(s[first + a, 1] - s[first + b, 1])
        return np.float32(np.sqrt(np.float32(dx * dx + dy * dy)))
    return np.float32((d(1, 5) + d(2, 4)) / (np.float32(2.0) * d(0, 3)))


@pytest.fixture(scope="module")
def hog():
    from paper_2006_00816_gb300 import _build
    _build.build()
    from paper_2006_00816_gb300 import hog as H
    return H


def _det(H, x, y, w, h):
    d = np.zeros(1, H.DET_DTYPE)[0]
    d["x"], d["y"], d["w"], d["h"] = x, y, w, h
    return d


@pytest.mark.parametrize("seed", [1, 77])
def test_fit_matches_independent_walk(hog, seed):
    L, T, K, D, P = 68, 3, 20, 3, 50
    ert = hog.Ert(cascades=T, trees=K, depth=D, features=P, seed=seed)
    model = _model(L, T, K, D, P, seed)
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, (120, 160), dtype=np.uint8)
    for box in [(20.5, 10.25, 80.0, 80.0), (100.0, 60.0, 96.5, 96.5), (-5.0, -3.0, 50.0, 50.0)]:
        lm, ear = ert.fit(img, _det(hog, *box))
        ref = _fit(model, img, box, D)
        assert np.array_equal(lm, ref), box
        assert ear[0] == _ear(ref, 36) and ear[1] == _ear(ref, 42)
    ert.close()


def test_determinism_and_mean_shape_ear(hog):
    img = np.random.default_rng(3).integers(0, 256, (480, 640), dtype=np.uint8)
    box = _det(hog, 200.0, 150.0, 160.0, 160.0)
    a = hog.Ert(seed=5)
    b = hog.Ert(seed=5)
    c = hog.Ert(seed=6)
    la, ea = a.fit(img, box)
    lb, eb = b.fit(img, box)
    lc, _ = c.fit(img, box)
    assert np.array_equal(la, lb) and np.array_equal(ea, eb)
    assert not np.array_equal(la, lc)
    # the mean shape's eyes have EAR 0.3: a constant image splits alike every
    # time, so the cascade moves all landmarks by the same leaf sums; the
    # eyes stay hexagons near their mean proportions
    flat = np.full((480, 640), 90, np.uint8)
    one = hog.Ert(cascades=1, trees=1, depth=1, features=2, seed=9)
    _, e = one.fit(flat, box)
    assert abs(e[0] - 0.3) < 0.02 and abs(e[1] - 0.3) < 0.02
    for m in (a, b, c, one):
        m.close()


def test_invalid_params(hog):
    with pytest.raises(hog.HogError):
        hog.Ert(landmarks=5)
    with pytest.raises(hog.HogError):
        hog.Ert(depth=0)
