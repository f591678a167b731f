"""Removal of small connected components of the RoI mask (§Region of
Interest extraction) on the GPU, through the C ABI, against the oracle.

Stagewise: given the GPU's own cut (mask0), the oracle's opening/closing
followed by its flood-fill component filter must give the GPU's final mask
bit for bit, and the 5/3 coefficients must be those of that mask.  Cases
cover many small components (a low RoI threshold), components spanning
every tile of the frame (a high threshold), ragged frame sizes and a full
2048^2 frame of the batched workload."""
import numpy as np
import pytest

from synth import pair_u8, sequence_u16
from tests._gpu import F, oracle_params, run_stream, u16

pytestmark = pytest.mark.gpu


def _check(orc, frames, bd, **cfg):
    g = run_stream(frames, bd, **cfg)[1]
    p = oracle_params(orc, **cfg)
    morph = orc.morph(g["mask0"], p.r_open, p.r_close)
    ref = orc.remove_small(morph, cfg["min_area"])
    assert np.array_equal(g["mask"], ref)
    cm = orc.wavelet_mask(g["mask"], p.dwt_levels, p.wavelet)
    if p.wavelet == 53:
        y = orc.dwt2d(orc.dc_shift(frames[1], bd), 53, p.dwt_levels)
        assert np.array_equal(g["coeffs"], orc.roi_shift(y, cm, p.scale_shift))
    return int(morph.sum()), int(ref.sum())


@pytest.mark.parametrize("q,min_area", [(0.02, 40), (0.2, 150), (0.9, 400), (0.5, 5000)],
                         ids=["q002_a40", "q02_a150", "q09_a400", "q05_a5000"])
def test_component_filter_parity(orc, q, min_area):
    seq = u16(sequence_u16(6100 + int(q * 100), 2, 512, 384, 40))
    before, after = _check(orc, [seq[0], seq[1]], 12, roi_q=q, min_area=min_area, pyr_levels=4, dwt_levels=4)
    assert after <= before


@pytest.mark.parametrize("h,w", [(72, 40), (48, 64), (16, 16), (200, 264)])
def test_component_filter_ragged_sizes(orc, h, w):
    a, b = pair_u8(seed=6200 + h + w, h=h, w=w, n_blobs=4)
    levels = dict(pyr_levels=2, dwt_levels=3) if min(h, w) > 16 else dict(pyr_levels=2, dwt_levels=1)
    _check(orc, [a.numpy(), b.numpy()], 8, roi_q=0.3, min_area=25, **levels)


def test_component_filter_full_size_2048(orc):
    seq = u16(sequence_u16(3000, 2, 2048, 2048, 200))
    before, after = _check(orc, [seq[0], seq[1]], 12, pyr_levels=5, dwt_levels=5, min_area=500)
    assert 0 < after < before


def test_component_filter_config_is_validated():
    with pytest.raises(F.FlowRoIError) as ei:
        F.Context(min_area=-1)
    assert ei.value.code == F.EINVAL
    with pytest.raises(F.FlowRoIError) as ei:
        F.Context(min_area=(1 << 20) + 1)
    assert ei.value.code == F.EINVAL
