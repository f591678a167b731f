"""Pins of the oracle's optional denoising (§Optical flow extraction: median
filtering, then bilateral filtering, of the flow input; Table 1 "Denoise").

Each check comes from outside the oracle's own formula: the 3x3 median
against scipy's median filter, the bilateral filter against its closed
forms (a constant image is fixed; with an infinite range sigma it is the
normalised Gaussian blur, checked against scipy's correlation; with a
vanishing range sigma it is the identity; a step much higher than the range
sigma is preserved exactly), and salt noise removed by the median step."""
import numpy as np
import pytest

ndimage = pytest.importorskip("scipy.ndimage")


def _gauss_kernel(rb, sigma_s):
    u = np.arange(-rb, rb + 1, dtype=np.float64)
    g = np.exp(-u * u / (2.0 * sigma_s * sigma_s))
    k = np.outer(g, g)
    return k / k.sum()


@pytest.mark.parametrize("h,w", [(1, 7), (9, 1), (16, 16), (23, 37)])
def test_median3_matches_scipy_median_filter(orc, h, w):
    rng = np.random.default_rng(h * 100 + w)
    img = rng.integers(0, 256, size=(h, w)).astype(np.float64)
    ref = ndimage.median_filter(img, size=3, mode="nearest")
    assert np.array_equal(orc.median3(img), ref)


def test_bilateral_keeps_a_constant_image(orc):
    img = np.full((12, 17), 93.25)
    assert np.allclose(orc.bilateral(img, 2, 2.0, 20.0), img, rtol=0, atol=1e-12)


@pytest.mark.parametrize("rb,sigma_s", [(1, 0.8), (2, 2.0), (3, 1.5)])
def test_bilateral_with_infinite_range_sigma_is_the_gaussian_blur(orc, rb, sigma_s):
    rng = np.random.default_rng(rb)
    img = rng.uniform(0, 255, size=(20, 26))
    ref = ndimage.correlate(img, _gauss_kernel(rb, sigma_s), mode="nearest")
    assert np.allclose(orc.bilateral(img, rb, sigma_s, 1e12), ref, rtol=0, atol=1e-9)


def test_bilateral_with_vanishing_range_sigma_is_the_identity(orc):
    rng = np.random.default_rng(3)
    img = rng.permutation(30 * 30).reshape(30, 30).astype(np.float64)  # neighbours differ by >= 1
    assert np.allclose(orc.bilateral(img, 2, 2.0, 1e-3), img, rtol=0, atol=1e-12)


def test_bilateral_preserves_a_high_step(orc):
    img = np.zeros((16, 24))
    img[:, 11:] = 200.0  # exp(-200^2 / (2 * 20^2)) ~ 2e-22
    assert np.allclose(orc.bilateral(img, 2, 2.0, 20.0), img, rtol=0, atol=1e-12)


def test_denoise_removes_salt_noise(orc):
    img = np.full((15, 15), 40.0)
    img[7, 7] = 255.0
    img[2, 12] = 0.0
    assert np.allclose(orc.denoise(img, 2, 2.0, 20.0), 40.0, rtol=0, atol=1e-12)


def test_frame_with_denoise_differs_only_in_the_flow_input(orc):
    """The JPEG2000 front end codes the raw frame whether or not the flow
    input is denoised; the flow itself changes."""
    from synth import pair_u8
    prev, cur = pair_u8(seed=77, h=64, w=64, n_blobs=3)
    p0 = orc.Params()
    p1 = orc.Params()
    p1.denoise = 1
    a = orc.frame(prev.numpy(), cur.numpy(), 8, p0)
    b = orc.frame(prev.numpy(), cur.numpy(), 8, p1)
    assert np.array_equal(a["y"], b["y"])
    assert not np.array_equal(a["flow"], b["flow"])
    assert np.allclose(b["denoised"], orc.denoise(orc.units(cur.numpy(), 8), 2, 2.0, 20.0))
