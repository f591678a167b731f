"""Pins of the oracle's JPEG2000 front end (no GPU): lifting DWTs against
the published FIR filter banks (tests/golden), perfect reconstruction,
closed forms, the quantisation step table against the published synthesis
filters, the wavelet-domain RoI mask against brute-force support sets, and
the RoI up-shift."""
import numpy as np
import pytest

from tests._taps import fir_analysis_1d, fir_analysis_2d, load_taps, wsym

T97 = load_taps("cdf97_analysis_taps.txt")
T53 = load_taps("legall53_analysis_taps.txt")
S97 = load_taps("cdf97_synthesis_taps.txt")


@pytest.mark.parametrize("n", [2, 3, 8, 9, 31, 64])
def test_dwt97_1d_matches_fir(orc, n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) * 500
    assert np.max(np.abs(orc.dwt1d(x, 97) - fir_analysis_1d(x, T97))) < 1e-9 * 500


@pytest.mark.parametrize("n", [2, 3, 8, 9, 31, 64])
def test_dwt53_1d_within_rounding_of_fir(orc, n):
    """H = x_odd - floor(mean of neighbours) differs from the linear high-pass
    by < 1/2; L adds floor((H + H' + 2)/4), within 1 of the linear low-pass."""
    rng = np.random.default_rng(n)
    x = rng.integers(-2048, 2048, size=n)
    y = orc.dwt1d(x, 53)
    assert np.max(np.abs(y - fir_analysis_1d(x, T53))) <= 1.0


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_perfect_reconstruction_1d(orc, n):
    rng = np.random.default_rng(100 + n)
    x = rng.integers(-5000, 5000, size=n)
    assert np.array_equal(orc.dwt1d(orc.dwt1d(x, 53), 53, inverse=True), x)
    xf = rng.normal(size=n) * 300
    assert np.max(np.abs(orc.dwt1d(orc.dwt1d(xf, 97), 97, inverse=True) - xf)) < 1e-9


@pytest.mark.parametrize("shape,levels", [((16, 16), 3), ((32, 24), 3), ((13, 21), 2), ((64, 64), 5)])
def test_perfect_reconstruction_2d(orc, shape, levels):
    rng = np.random.default_rng(shape[0] * 7 + levels)
    x = rng.integers(-2048, 2048, size=shape)
    assert np.array_equal(orc.dwt2d(orc.dwt2d(x, 53, levels), 53, levels, inverse=True), x)
    xf = x.astype(np.float64)
    r = orc.dwt2d(orc.dwt2d(xf, 97, levels), 97, levels, inverse=True)
    assert np.max(np.abs(r - xf)) < 1e-8


@pytest.mark.parametrize("shape,levels", [((16, 16), 1), ((16, 24), 3), ((15, 10), 2)])
def test_dwt97_2d_matches_fir_mallat(orc, shape, levels):
    rng = np.random.default_rng(9)
    x = rng.normal(size=shape) * 200
    assert np.max(np.abs(orc.dwt2d(x, 97, levels) - fir_analysis_2d(x, T97, levels))) < 1e-8


def test_dwt53_2d_one_level_within_rounding(orc):
    """One 2-D level: vertical integer pass within 1 of linear; the
    horizontal pass maps that error through filters of L1 gain <= 2, plus
    its own rounding of 1: within 3 overall."""
    rng = np.random.default_rng(10)
    x = rng.integers(-2048, 2048, size=(20, 18))
    assert np.max(np.abs(orc.dwt2d(x, 53, 1) - fir_analysis_2d(x, T53, 1))) <= 3.0


def test_constant_and_nyquist_closed_forms(orc):
    c = 37
    y = orc.dwt2d(np.full((16, 16), c), 53, 3)
    assert y[0, 0] == c and np.count_nonzero(y) == 4  # LL3 (2x2) = c, all else 0
    y = orc.dwt2d(np.full((16, 16), c, np.float64), 97, 3)
    assert np.allclose(y[:2, :2], c, atol=1e-9)
    y[:2, :2] = 0
    assert np.max(np.abs(y)) < 1e-9
    a = 3.0
    alt = a * (-1.0) ** np.arange(32)
    y = orc.dwt1d(alt, 97)
    assert np.max(np.abs(y[:16])) < 1e-9                       # low band vanishes at Nyquist
    assert np.allclose(np.abs(y[16:]), 2 * a, atol=1e-9)       # high band gain 2


def test_dc_shift(orc):
    raw = np.array([[0, 2048, 4095]], np.uint16)
    assert orc.dc_shift(raw, 12).tolist() == [[-2048, 0, 2047]]
    raw8 = np.array([0, 128, 255], np.uint8)
    assert orc.dc_shift(raw8, 8).tolist() == [-128, 0, 127]


def test_subband_index_positions(orc):
    w = h = 32
    L = 3
    assert orc.subband_index(20, 3, w, h, L) == 0      # HL1: right half, top half
    assert orc.subband_index(3, 20, w, h, L) == 1      # LH1
    assert orc.subband_index(20, 20, w, h, L) == 2     # HH1
    assert orc.subband_index(10, 2, w, h, L) == 3      # HL2 (x in [8,16))
    assert orc.subband_index(5, 5, w, h, L) == 8       # HH3 (x, y in [4,8))
    assert orc.subband_index(3, 3, w, h, L) == 9       # LL3
    assert orc.subband_index(0, 4, w, h, L) == 7       # LH3


def _basis_norms_1d(levels):
    g0, g1 = S97["lowpass"], S97["highpass"]

    def up(s):
        o = np.zeros(2 * s.size - 1)
        o[::2] = s
        return o

    low = [g0]
    high = [g1]
    for _ in range(1, levels):
        low.append(np.convolve(g0, up(low[-1])))
        high.append(np.convolve(g0, up(high[-1])))
    return [np.sum(v ** 2) for v in low], [np.sum(v ** 2) for v in high]


@pytest.mark.parametrize("levels,bd", [(5, 12), (3, 8)])
def test_delta_table_against_published_synthesis_filters(orc, levels, bd):
    G, delta, eps, mu = orc.delta_table(levels, bd, 1.0)
    nl, nh = _basis_norms_1d(levels)
    for l in range(1, levels + 1):
        want = [nh[l - 1] * nl[l - 1], nl[l - 1] * nh[l - 1], nh[l - 1] * nh[l - 1]]  # HL, LH, HH
        for o in range(3):
            assert abs(G[3 * (l - 1) + o] / want[o] - 1) < 1e-9
    assert abs(G[3 * levels] / (nl[levels - 1] ** 2) - 1) < 1e-9
    for b in range(3 * levels + 1):
        o = 3 if b == 3 * levels else b % 3
        R = bd + (0 if o == 3 else (2 if o == 2 else 1))
        rep = 2.0 ** (R - eps[b]) * (1 + mu[b] / 2048.0)
        assert 0 <= eps[b] <= 31 and 0 <= mu[b] <= 2047
        assert np.float32(rep) == delta[b]
        assert abs(rep * np.sqrt(G[b]) - 1.0) <= 2.0 ** -12


def test_quantise_bounds_and_sign(orc):
    rng = np.random.default_rng(3)
    h = w = 32
    L = 3
    y = (rng.normal(size=(h, w)) * 40).astype(np.float32)
    _, delta, _, _ = orc.delta_table(L, 12, 1.0)
    q = orc.quantise_f32(y, L, delta)
    dl = np.array([[delta[orc.subband_index(x, r, w, h, L)] for x in range(w)] for r in range(h)], np.float64)
    a = np.abs(y.astype(np.float64))
    qa = np.abs(q).astype(np.float64)
    assert np.all(qa * dl <= a * (1 + 1e-6)) and np.all(a < (qa + 1) * dl * (1 + 1e-6))
    assert np.all((q == 0) | (np.sign(q) == np.sign(y)))
    q64 = orc.quantise_f64(y.astype(np.float64), L, delta)
    assert np.max(np.abs(q64 - q)) <= 1


def _impulse_support_97(orc, h, w, levels, pos):
    c = np.zeros((h, w))
    c[pos] = 1.0
    return np.abs(orc.dwt2d(c, 97, levels, inverse=True)) > 1e-13


def _idwt53_linear_1d(v):
    """Linear (rounding-free) 5/3 synthesis, written from the lifting
    equations, for support sets only."""
    n = v.size
    if n < 2:
        return v.copy()
    nl = (n + 1) // 2
    x = np.empty(n)
    x[0::2] = v[:nl]
    x[1::2] = v[nl:]
    for i in range(0, n, 2):
        x[i] -= (x[wsym(i - 1, n)] + x[wsym(i + 1, n)]) / 4
    for i in range(1, n, 2):
        x[i] += (x[wsym(i - 1, n)] + x[wsym(i + 1, n)]) / 2
    return x


def _impulse_support_53(h, w, levels, pos):
    c = np.zeros((h, w))
    c[pos] = 1.0
    cws, chs = [w], [h]
    for _ in range(levels):
        cws.append((cws[-1] + 1) // 2)
        chs.append((chs[-1] + 1) // 2)
    for l in range(levels - 1, -1, -1):
        cw, ch = cws[l], chs[l]
        for y in range(ch):
            c[y, :cw] = _idwt53_linear_1d(c[y, :cw])
        for x in range(cw):
            c[:ch, x] = _idwt53_linear_1d(c[:ch, x])
    return np.abs(c) > 1e-13


@pytest.mark.parametrize("wavelet", [53, 97])
@pytest.mark.parametrize("shape,levels", [((16, 16), 1), ((16, 16), 2), ((24, 20), 3), ((32, 32), 3)])
def test_wavelet_mask_equals_brute_force_support(orc, wavelet, shape, levels):
    rng = np.random.default_rng(shape[0] + levels + wavelet)
    h, w = shape
    pix = np.zeros(shape, np.uint8)
    for _ in range(3):
        y, x = rng.integers(0, h), rng.integers(0, w)
        pix[y:y + 2, x:x + 3] = 1
    cm = orc.wavelet_mask(pix, levels, wavelet)
    for y in range(h):
        for x in range(w):
            sup = (_impulse_support_97(orc, h, w, levels, (y, x)) if wavelet == 97
                   else _impulse_support_53(h, w, levels, (y, x)))
            assert cm[y, x] == int(np.any(sup & (pix == 1))), (y, x)


def test_non_roi_coefficients_do_not_touch_roi_pixels(orc):
    rng = np.random.default_rng(5)
    h, w, L = 32, 32, 3
    pix = np.zeros((h, w), np.uint8)
    pix[8:15, 10:20] = 1
    pix[25:27, 2:5] = 1
    x = rng.normal(size=(h, w)) * 100
    y = orc.dwt2d(x, 97, L)
    cm = orc.wavelet_mask(pix, L, 97)
    r = orc.dwt2d(np.where(cm == 1, y, 0.0), 97, L, inverse=True)
    assert np.max(np.abs(r - x)[pix == 1]) < 1e-9


def test_roi_shift(orc):
    rng = np.random.default_rng(6)
    q = rng.integers(-3000, 3000, size=(8, 8)).astype(np.int32)
    cm = (rng.random((8, 8)) < 0.5).astype(np.uint8)
    s = 5
    out = orc.roi_shift(q, cm, s)
    assert np.array_equal(out[cm == 0], q[cm == 0])
    assert np.array_equal(np.sign(out), np.sign(q))
    assert np.array_equal(np.abs(out[cm == 1]) >> s, np.abs(q[cm == 1]))
    assert np.array_equal(out[cm == 1], q[cm == 1] * (1 << s))
    assert np.array_equal(orc.roi_shift(q, cm, 0), q)
