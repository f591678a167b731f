"""The 9/7 quantiser's quotient, formed without a division.

The dead-zone quantiser decides q = floor(RN(|y| / delta_b)), RN being the
float32 round-to-nearest quotient (the decision is taken in single
precision on both sides).  The DWT kernel forms RN(|y| / delta) from the
correctly rounded reciprocal rd = RN(1 / delta) by one residual
correction (Markstein 1990): q0 = RN(|y| rd), e = RN(|y| - q0 delta) (a
fused multiply-add, exact), q1 = RN(q0 + e rd) (a fused multiply-add).

These tests emulate that sequence with exact rational arithmetic and
float32 rounding written out here, and check q1 against the exactly rounded
quotient for every step of the quantisation tables the library uses, on
random magnitudes and on magnitudes placed next to integer multiples of the
step, where floor(RN(.)) would flip if the quotient were off by an ulp.
"""
from fractions import Fraction
import numpy as np
import pytest

from oracle import oracle as orc


def rn32(x: Fraction) -> Fraction:
    """x rounded to the nearest float32 (ties to even); normal range only."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    p, q = abs(x.numerator), x.denominator
    e = p.bit_length() - q.bit_length()  # 2^(e-1) < p/q < 2^(e+1)
    if (p << max(0, -e)) < (q << max(0, e)):
        e -= 1                           # now 2^e <= p/q < 2^(e+1)
    assert -126 <= e <= 127, "outside the float32 normal range"
    k = 23 - e                           # p/q * 2^k in [2^23, 2^24)
    num, den = (p << k, q) if k >= 0 else (p, q << -k)
    n, r = divmod(num, den)
    if 2 * r > den or (2 * r == den and n % 2 == 1):
        n += 1
    return s * Fraction(n) / (Fraction(2) ** k)


def markstein(a: Fraction, d: Fraction, rd: Fraction) -> Fraction:
    q0 = rn32(a * rd)
    e = rn32(a - q0 * d)
    return rn32(q0 + e * rd)


def _floor(x: Fraction) -> int:
    return x.numerator // x.denominator


def _tables():
    for levels, bits in ((5, 12), (3, 8), (4, 16), (6, 12)):
        _, delta, _, _ = orc.delta_table(levels, bits, 1.0)
        yield from sorted(set(float(v) for v in delta))


def test_residual_is_exact_and_quotient_correctly_rounded():
    rng = np.random.default_rng(97)
    steps = list(_tables())
    assert len(steps) >= 8
    checked = 0
    for dv in steps:
        d = Fraction(dv)
        rd = Fraction(float(np.float32(1.0) / np.float32(dv)))  # IEEE float32 division
        assert rd == rn32(1 / d)
        # random magnitudes over 30 binades
        mags = np.float32(2.0) ** rng.uniform(-10, 20, 80).astype(np.float32)
        mags = mags * rng.uniform(1, 2, 80).astype(np.float32)
        # magnitudes next to k * delta (the floor's decision boundaries)
        ks = rng.integers(1, int(min(2 ** 22, 2 ** 20 / dv)) + 2, 40)
        near = []
        for k in ks:
            c = np.float32(k * dv)
            for off in range(-3, 4):
                v = c
                for _ in range(abs(off)):
                    v = np.nextafter(v, np.float32(np.inf if off > 0 else -np.inf), dtype=np.float32)
                near.append(v)
        for v in list(mags) + near:
            a = Fraction(float(v))
            if a == 0:
                continue
            q0 = rn32(a * rd)
            assert rn32(a - q0 * d) == a - q0 * d  # the fused residual is exact
            exact = rn32(a / d)
            got = markstein(a, d, rd)
            assert got == exact, (dv, float(v), float(got), float(exact))
            assert _floor(got) == _floor(exact)
            checked += 1
    assert checked > 10000


def test_rn32_matches_numpy_float32_rounding():
    """The float32 rounding used above agrees with numpy's on random
    doubles (a check of the emulation, not of the kernel)."""
    rng = np.random.default_rng(3)
    for x in rng.uniform(-1e6, 1e6, 2000):
        assert float(rn32(Fraction(float(x)))) == float(np.float32(x))


def test_quotient_feeds_the_oracle_quantiser_decision():
    """On a random float32 plane, floor(markstein(|y|)) with the sign of y
    equals the oracle's single-precision quantiser, band by band."""
    levels = 3
    _, delta, _, _ = orc.delta_table(levels, 12, 1.0)
    rng = np.random.default_rng(11)
    n = 32
    y = (rng.standard_normal((n, n)) * 300).astype(np.float32)
    q = orc.quantise_f32(y, levels, delta)
    # band of each coefficient in the Mallat layout
    band = np.empty((n, n), np.int64)
    for yy in range(n):
        for xx in range(n):
            lv, b = levels, 3 * levels
            for l in range(1, levels + 1):
                h = n >> l
                if yy >= h or xx >= h:
                    lv = l
                    b = 3 * (l - 1) + (0 if yy < h else (1 if xx < h else 2))
                    break
            band[yy, xx] = b
    for yy in range(n):
        for xx in range(n):
            dv = float(delta[band[yy, xx]])
            rd = Fraction(float(np.float32(1.0) / np.float32(dv)))
            a = Fraction(abs(float(y[yy, xx])))
            m = _floor(markstein(a, Fraction(dv), rd)) if a else 0
            expect = -m if y[yy, xx] < 0 else m
            assert q[yy, xx] == expect, (yy, xx)
