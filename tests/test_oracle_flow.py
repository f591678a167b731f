"""Pins of the oracle's front end and flow (no GPU).

Each test checks the oracle against something other than itself: library
routines (scipy.ndimage, numpy.linalg.lstsq), closed forms of the
polynomial-expansion model, and the known motion of synthetic patterns.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

from synth import translated_pattern


def test_units(orc):
    raw8 = np.array([0, 1, 128, 255], np.uint8)
    assert np.allclose(orc.units(raw8, 8), [0, 1, 128, 255], atol=1e-12)
    raw12 = np.array([0, 4095, 2048], np.uint16)
    assert np.allclose(orc.units(raw12, 12), [0, 255.0, 2048 * 255 / 4095], atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 16), (17, 23), (5, 9), (64, 48)])
def test_pyr_down_matches_scipy(orc, shape):
    rng = np.random.default_rng(1)
    img = rng.normal(size=shape) * 50 + 100
    b = np.array([1, 4, 6, 4, 1]) / 16.0
    ref = ndi.correlate1d(ndi.correlate1d(img, b, axis=0, mode="nearest"), b, axis=1, mode="nearest")[::2, ::2]
    out = orc.pyr_down(img)
    assert out.shape == ((shape[0] + 1) // 2, (shape[1] + 1) // 2)
    assert np.max(np.abs(out - ref)) < 1e-10


def test_pyr_down_constant(orc):
    out = orc.pyr_down(np.full((13, 10), 7.25))
    assert np.all(out == 7.25)


def _quadratic(h, w, A, b, c):
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    return A[0, 0] * xs ** 2 + 2 * A[0, 1] * xs * ys + A[1, 1] * ys ** 2 + b[0] * xs + b[1] * ys + c


@pytest.mark.parametrize("n_half,sigma", [(2, 1.1), (3, 1.5)])
def test_expansion_of_quadratic_is_exact(orc, n_half, sigma):
    rng = np.random.default_rng(2)
    h, w = 20, 22
    for _ in range(3):
        S = rng.normal(size=(2, 2))
        A = 0.5 * (S + S.T)
        b = rng.normal(size=2) * 3
        f = _quadratic(h, w, A, b, rng.normal())
        F = orc.poly_expand(f, n_half, sigma)
        ys, xs = np.mgrid[n_half:h - n_half, n_half:w - n_half]
        # Local model at x0: f(x0 + y) = y^T A y + (b + 2 A x0)^T y + const
        assert np.allclose(F[0, n_half:h - n_half, n_half:w - n_half], A[0, 0], atol=1e-9)
        assert np.allclose(F[1, n_half:h - n_half, n_half:w - n_half], A[0, 1], atol=1e-9)
        assert np.allclose(F[2, n_half:h - n_half, n_half:w - n_half], A[1, 1], atol=1e-9)
        bx = b[0] + 2 * (A[0, 0] * xs + A[0, 1] * ys)
        by = b[1] + 2 * (A[0, 1] * xs + A[1, 1] * ys)
        assert np.allclose(F[3, n_half:h - n_half, n_half:w - n_half], bx, atol=1e-8)
        assert np.allclose(F[4, n_half:h - n_half, n_half:w - n_half], by, atol=1e-8)


def test_expansion_matches_weighted_lstsq_including_borders(orc):
    """Weighted least squares solved by numpy.linalg.lstsq on the replicated
    neighbourhood, at interior and border pixels of a random image."""
    rng = np.random.default_rng(3)
    h, w, n, sigma = 11, 13, 2, 1.1
    img = rng.normal(size=(h, w)) * 30
    F = orc.poly_expand(img, n, sigma)
    offs = [(u, v) for v in range(-n, n + 1) for u in range(-n, n + 1)]
    Bm = np.array([[1, u, v, u * u, v * v, u * v] for u, v in offs], np.float64)
    sw = np.sqrt(np.array([np.exp(-(u * u + v * v) / (2 * sigma ** 2)) for u, v in offs]))
    for (y, x) in [(0, 0), (0, 7), (5, 6), (10, 12), (1, 12), (7, 1)]:
        f = np.array([img[min(max(y + v, 0), h - 1), min(max(x + u, 0), w - 1)] for u, v in offs])
        r = np.linalg.lstsq(Bm * sw[:, None], f * sw, rcond=None)[0]
        want = [r[3], r[5] / 2, r[4], r[1], r[2]]
        assert np.allclose(F[:, y, x], want, atol=1e-9)


def test_identical_frames_give_zero_flow(orc):
    rng = np.random.default_rng(4)
    img = ndi.gaussian_filter(rng.normal(size=(48, 40)) * 40 + 80, 1.5)
    d = orc.flow(img, img, levels=3)
    assert np.all(d == 0.0)


@pytest.mark.parametrize("iters", [1, 3])
def test_flow_of_shifted_quadratic_is_exact(orc, iters):
    """f2(x) = f1(x - u) for a quadratic f1: then A2 = A1 and
    b2 = b1 - 2 A1 u, so one level with lambda = 0 gives d = u exactly at
    pixels whose expansion, gather and window stay inside the image."""
    h, w, n, r = 48, 50, 2, 7
    A = np.array([[0.4, 0.15], [0.15, 0.25]])
    b = np.array([1.0, -2.0])
    u = np.array([0.6, -0.35])
    f1 = _quadratic(h, w, A, b, 5.0)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    X, Y = xs - u[0], ys - u[1]
    f2 = A[0, 0] * X ** 2 + 2 * A[0, 1] * X * Y + A[1, 1] * Y ** 2 + b[0] * X + b[1] * Y + 5.0
    F1 = orc.poly_expand(f1, n, 1.1)
    F2 = orc.poly_expand(f2, n, 1.1)
    d = orc.flow_iterate(F1, F2, np.zeros((2, h, w)), iters, r, 0.0)
    m = n + r + 2 * iters
    assert np.allclose(d[0, m:h - m, m:w - m], u[0], atol=1e-9)
    assert np.allclose(d[1, m:h - m, m:w - m], u[1], atol=1e-9)


@pytest.mark.parametrize("shift", [(0.3, -0.7), (2.0, 1.0), (-1.4, 0.9)])
def test_translation_of_smooth_pattern_is_recovered(orc, shift):
    """Frame t-1 holds the pattern, frame t the pattern moved by `shift`.
    With f1 = frame t and f2 = frame t-1 the estimated displacement is
    -shift (f2(x) = f1(x + shift)).  Checked where the pattern has
    structure, away from the border."""
    h, w = 96, 96
    prev, cur = translated_pattern(h, w, shift, n_blobs=8, sigma=4.0, seed=5)
    d = orc.flow(cur.numpy(), prev.numpy(), levels=3)
    gy, gx = np.gradient(cur.numpy())
    sel = (np.hypot(gx, gy) > 2.0)
    sel[:12] = sel[-12:] = False
    sel[:, :12] = sel[:, -12:] = False
    assert sel.sum() > 500
    err = np.hypot(d[0][sel] + shift[0], d[1][sel] + shift[1])
    assert np.median(err) < 0.02
    assert np.percentile(err, 95) < 0.05


def test_flow_upsample_closed_forms(orc):
    wc, hc = 6, 5
    const = np.stack([np.full((hc, wc), 0.75), np.full((hc, wc), -1.5)])
    up = orc.flow_upsample(const, 12, 10)
    assert np.allclose(up[0], 1.5) and np.allclose(up[1], -3.0)
    ys, xs = np.mgrid[0:hc, 0:wc].astype(np.float64)
    lin = np.stack([0.5 * xs + 0.25 * ys, -xs])
    up = orc.flow_upsample(lin, 2 * wc - 1, 2 * hc - 1)
    Y, X = np.mgrid[0:2 * hc - 1, 0:2 * wc - 1].astype(np.float64)
    assert np.allclose(up[0], 2 * (0.25 * X + 0.125 * Y), atol=1e-12)
    assert np.allclose(up[1], -X, atol=1e-12)
