"""Pins of the oracle's registration (§Optical flow extraction: each frame
registered to its predecessor by phase correlation against global
translational drift).

Against ground truth the generator fixes (a smooth pattern translated by a
known shift, with noise): the integer shift exactly and the sub-pixel shift
within 0.3 px; invariants: identical frames give 0, swapping the frames
negates the shift, a level-l estimate scales by 2^l; and the registered
flow of a pure drift is the uniform residual left by the drift estimate."""
import numpy as np
import pytest

from synth.frames import translated_pattern


def _pair(shift, seed, h=128, w=160, noise=2.0):
    a, b = translated_pattern(h, w, shift, n_blobs=8, seed=seed)
    rng = np.random.default_rng(seed + 100)
    return a.numpy() + rng.normal(0, noise, (h, w)), b.numpy() + rng.normal(0, noise, (h, w))


@pytest.mark.parametrize("shift", [(5, -3), (2, 1), (-7, 0), (1, -1), (12, 9), (-11, 8), (0, 0)])
@pytest.mark.parametrize("size", [(128, 160), (96, 128), (128, 128)])
def test_integer_shifts_are_found(orc, shift, size):
    a, b = _pair(shift, seed=sum(shift) + size[1], h=size[0], w=size[1])
    s = orc.phase_correlate(a, b)
    assert (round(s[0]), round(s[1])) == shift
    assert abs(s[0] - shift[0]) <= 0.4 and abs(s[1] - shift[1]) <= 0.4


@pytest.mark.parametrize("shift", [(5.3, -3.6), (2.5, 1.2), (-7.1, 0.4), (0.2, -0.3), (12.7, 9.9)])
def test_subpixel_shifts_within_0_4_px(orc, shift):
    for seed in range(3):
        a, b = _pair(shift, seed)
        s = orc.phase_correlate(a, b)
        assert abs(s[0] - shift[0]) <= 0.4 and abs(s[1] - shift[1]) <= 0.4


def test_identical_frames_and_swapped_frames(orc):
    a, b = _pair((4, -6), seed=7)
    assert orc.phase_correlate(a, a) == (0.0, 0.0)
    s, t = orc.phase_correlate(a, b), orc.phase_correlate(b, a)
    assert (round(s[0]), round(s[1])) == (4, -6) and (round(t[0]), round(t[1])) == (-4, 6)


def test_level_estimate_scales_by_two_to_the_level(orc):
    a, b = _pair((8, -12), seed=3, h=256, w=256, noise=1.0)
    sx, sy = orc.register(a, b, 2)
    assert abs(sx - 8) <= 4 * 0.4 and abs(sy + 12) <= 4 * 0.4


def test_flow_reg_with_zero_drift_is_flow(orc):
    a, b = _pair((1, 1), seed=5, h=64, w=64)
    d0 = orc.flow(b, a, 3)
    d1 = orc.flow_reg(b, a, 3, 2, 1.1, 3, 7, 1e-3, (0.0, 0.0))
    assert np.array_equal(d0, d1)


def test_registered_flow_of_an_exact_drift_is_zero(orc):
    """An integer drift known exactly: the registered predecessor is the
    current frame away from the border, so no motion is left there, in
    textured and flat regions alike."""
    a, b = _pair((6, -4), seed=11, h=128, w=128, noise=0.0)
    d = orc.flow_reg(b, a, 3, 2, 1.1, 3, 7, 1e-3, (6.0, -4.0))
    assert np.abs(d[:, 24:-24, 24:-24]).max() < 1e-6
    d_unreg = orc.flow(b, a, 3)
    assert np.abs(d_unreg[:, 24:-24, 24:-24]).max() > 1.0
