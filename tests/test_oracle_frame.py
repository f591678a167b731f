"""Whole-frame pins of the oracle pipeline (no GPU)."""
import numpy as np

from synth import pair_u8


def test_identical_frames_give_empty_mask_and_plain_coefficients(orc):
    prev, _ = pair_u8(seed=21, h=64, w=64, n_blobs=4)
    raw = prev.numpy()
    p = orc.Params(pyr_levels=3, dwt_levels=3, wavelet=53)
    out = orc.frame(raw, raw, 8, p)
    assert np.all(out["flow"] == 0.0)
    assert out["mask0"].sum() == 0 and out["mask"].sum() == 0
    assert np.array_equal(out["coeffs"], orc.dwt2d(orc.dc_shift(raw, 8), 53, 3))


def test_first_frame_has_empty_mask(orc):
    _, cur = pair_u8(seed=22, h=32, w=32, n_blobs=2)
    out = orc.frame(None, cur.numpy(), 8, orc.Params(pyr_levels=2, dwt_levels=2, wavelet=97))
    assert out["mask"].sum() == 0
    assert "flow" not in out


def test_moving_blobs_are_covered(orc):
    """256x256 8-bit pair with 12 moving blobs: the mask keeps at most the top
    q fraction before morphology, and it covers the blobs that moved."""
    prev, cur = pair_u8(seed=1001)
    p = orc.Params(pyr_levels=3, dwt_levels=3, wavelet=53, roi_q=0.2)
    out = orc.frame(prev.numpy(), cur.numpy(), 8, p)
    n = 256 * 256
    assert out["mask0"].sum() <= int(np.floor(np.float64(np.float32(0.2)) * n))
    diff = np.abs(cur.numpy().astype(int) - prev.numpy().astype(int)) > 60  # clearly moving edges
    assert diff.sum() > 100
    assert out["mask"][diff].mean() > 0.9
    # coefficients: RoI ones are the plain DWT shifted by s
    plain = orc.dwt2d(orc.dc_shift(cur.numpy(), 8), 53, 3)
    cm = out["cmask"] == 1
    assert np.array_equal(out["coeffs"][~cm], plain[~cm])
    assert np.array_equal(out["coeffs"][cm], plain[cm] * 32)
