"""Pins of the oracle's RoI-extraction stages (no GPU): saliency closed
forms, normalisation, the quantile cut against a brute-force sort, and the
morphology against scipy.ndimage plus algebraic identities."""
import numpy as np
import pytest
import scipy.ndimage as ndi


def test_saliency_constant_flow(orc):
    d = np.stack([np.full((9, 7), 3.0), np.full((9, 7), 4.0)])
    S = orc.saliency(d, 0.7)
    assert np.allclose(S, 0.7 * 5.0)
    Sh = orc.normalise(S)
    assert np.all(Sh == 0.0)
    m, _ = orc.threshold(Sh, 0.2)
    assert m.sum() == 0


def test_saliency_ramp(orc):
    """|d| = a*x: interior central difference gives gradient a, the
    replicated border gives a/2."""
    h, w, a = 6, 10, 0.5
    xs = np.tile(np.arange(w, dtype=np.float64), (h, 1))
    d = np.stack([a * xs, np.zeros((h, w))])
    S = orc.saliency(d, 0.7)
    g = np.full((h, w), a)
    g[:, 0] = g[:, -1] = a / 2
    assert np.allclose(S, 0.7 * a * xs + 0.3 * g, atol=1e-12)


def test_saliency_direction_invariance(orc):
    """Saliency depends on |d| only: rotating every vector leaves it unchanged."""
    rng = np.random.default_rng(0)
    d = rng.normal(size=(2, 12, 15))
    ang = 0.83
    r = np.stack([np.cos(ang) * d[0] - np.sin(ang) * d[1], np.sin(ang) * d[0] + np.cos(ang) * d[1]])
    assert np.allclose(orc.saliency(d, 0.7), orc.saliency(r, 0.7), atol=1e-12)


def test_normalise(orc):
    rng = np.random.default_rng(1)
    S = rng.random(500) * 7 + 2
    Sh = orc.normalise(S)
    assert Sh.min() == 0.0 and Sh.max() == 1.0
    o = np.argsort(S)
    assert np.all(np.diff(Sh[o]) >= 0)


@pytest.mark.parametrize("n,q", [(1000, 0.2), (4096, 0.1), (777, 0.5), (10, 0.05)])
def test_threshold_brute_force(orc, n, q):
    rng = np.random.default_rng(n)
    v = rng.random(n)
    m, t = orc.threshold(v, q)
    k = int(np.floor(np.float64(np.float32(q)) * n))
    srt = np.sort(v)[::-1]
    assert t == srt[k]
    assert m.sum() == k  # no ties among random doubles
    assert np.array_equal(m.astype(bool), v > srt[k])


def test_threshold_ties_and_empty(orc):
    v = np.array([0.9, 0.5, 0.5, 0.5, 0.1, 0.0, 0.0, 0.0, 0.0, 0.0])
    m, t = orc.threshold(v, 0.3)  # k = 3 -> t = 0.5, only 0.9 exceeds it
    assert t == 0.5 and m.tolist() == [1] + [0] * 9
    m, _ = orc.threshold(v, 0.05)  # k = 0 -> empty
    assert m.sum() == 0


def test_threshold_f32_brute_force(orc):
    rng = np.random.default_rng(7)
    v = rng.random(3000).astype(np.float32)
    v[::7] = v[3]  # plenty of exact ties
    m, t = orc.threshold_f32(v, 0.2)
    k = int(np.floor(np.float64(np.float32(0.2)) * v.size))
    srt = np.sort(v)[::-1]
    assert t == srt[k]
    assert np.array_equal(m.astype(bool), v > srt[k])


def _sq(r):
    return np.ones((2 * r + 1, 2 * r + 1), bool)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_erode_dilate_match_scipy(orc, r):
    rng = np.random.default_rng(r)
    m = (rng.random((37, 29)) < 0.6).astype(np.uint8)
    e = orc.erode(m, r)
    d = orc.dilate(m, r)
    # Out-of-image pixels ignored: erosion pads with 1, dilation with 0.
    assert np.array_equal(e.astype(bool), ndi.binary_erosion(m, _sq(r), border_value=1))
    assert np.array_equal(d.astype(bool), ndi.binary_dilation(m, _sq(r), border_value=0))
    # Duality: erosion of X is the complement of the dilation of the complement.
    assert np.array_equal(e, 1 - orc.dilate(1 - m, r))


def test_open_close_identities(orc):
    rng = np.random.default_rng(11)
    m = (ndi.gaussian_filter(rng.random((40, 44)), 2) > 0.5).astype(np.uint8)
    m[rng.random(m.shape) < 0.03] ^= 1  # specks and holes
    op = orc.dilate(orc.erode(m, 1), 1)
    assert np.array_equal(orc.dilate(orc.erode(op, 1), 1), op)  # opening is idempotent
    cl = orc.erode(orc.dilate(m, 2), 2)
    assert np.array_equal(orc.erode(orc.dilate(cl, 2), 2), cl)  # closing is idempotent
    assert np.all(op <= m) and np.all(cl >= m)  # anti-extensive / extensive
    out = orc.morph(m, 1, 2)
    ref = ndi.binary_erosion(ndi.binary_dilation(
        ndi.binary_dilation(ndi.binary_erosion(m, _sq(1), border_value=1), _sq(1), border_value=0),
        _sq(2), border_value=0), _sq(2), border_value=1)
    assert np.array_equal(out.astype(bool), ref)
