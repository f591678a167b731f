"""Optional denoising of the flow input (§Optical flow extraction: median,
then bilateral filtering; Table 1 "Denoise") on the GPU, through the C ABI,
against the oracle.

Tolerance of the denoised image, 2e-3 in 8-bit units: the median is exact
(integer samples), and the bilateral weights are powers of two from the
hardware's approximate exp2 (relative error ~2^-22 on exponents of at most
~20 for weights that matter, i.e. ~3e-6), times the spread |I(q) - out| of
those neighbours (a few range sigmas, ~60), plus the float sums of 49 terms
of at most 255 (~7e-4) and the fast division (~6e-5).

Stagewise, like the other parity tests: the flow is checked against the
oracle's flow from the GPU's own denoised frames, then the whole frame
against the oracle with denoising."""
import numpy as np
import pytest

from synth import pair_u8, sequence_u16
from tests._gpu import F, fetch, oracle_params, u16

pytestmark = pytest.mark.gpu

DEN_TOL = 2e-3
FLOW_TOL = 1e-3


def _run(frames, bd, **cfg):
    h, w = frames[0].shape
    outs = []
    with F.Context(flags=F.MANUAL | F.KEEP_INTERMEDIATES, **cfg) as ctx:
        for i, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 3, fr, i, bd)
            F.flowroi_flush(ctx.h, 120000)
            g = fetch(ctx.h, 3, i, h, w, True, cfg.get("wavelet", 53))
            g["den"] = np.empty((h, w), np.float32)
            F.flowroi_get_intermediate(ctx.h, 3, i, F.I_DENOISED, g["den"], 60000)
            outs.append(g)
    return outs


@pytest.mark.parametrize("case", [
    dict(h=256, w=256, u16=False, den_radius=2),
    dict(h=192, w=320, u16=True, den_radius=1, den_sigma_s=1.0, den_sigma_r=40.0),
    dict(h=72, w=40, u16=False, den_radius=3, den_sigma_s=3.0, den_sigma_r=10.0),
    dict(h=16, w=16, u16=True, den_radius=2),
], ids=["256_u8_r2", "192x320_u16_r1", "72x40_u8_r3", "16_u16_r2"])
def test_denoise_parity(orc, case):
    case = dict(case)
    h, w, is16 = case.pop("h"), case.pop("w"), case.pop("u16")
    if is16:
        seq = u16(sequence_u16(5100 + h, 2, h, w, max(2, h * w // 4000)))
        frames, bd = [seq[0], seq[1]], 12
    else:
        a, b = pair_u8(seed=5200 + h, h=h, w=w, n_blobs=max(2, h * w // 6000))
        frames, bd = [a.numpy(), b.numpy()], 8
    levels = dict(pyr_levels=2, dwt_levels=1) if min(h, w) < 32 else dict(pyr_levels=3, dwt_levels=3)
    cfg = dict(denoise=1, **case, **levels)
    g0, g1 = _run(frames, bd, **cfg)
    p = oracle_params(orc, **cfg)
    # the denoise kernel against the oracle, on both frames
    for fr, g in ((frames[0], g0), (frames[1], g1)):
        ref = orc.denoise(orc.units(fr, bd), p.den_radius, p.den_sigma_s, p.den_sigma_r)
        err = np.abs(g["den"] - ref).max()
        assert err <= DEN_TOL, f"denoised image error {err}"
    # the flow from the GPU's own denoised frames
    d = orc.flow(g1["den"].astype(np.float64), g0["den"].astype(np.float64), p.pyr_levels, p.poly_n_half,
                 p.poly_sigma, p.iters, p.win_r, p.lam)
    ferr = np.abs(g1["flow"].transpose(2, 0, 1) - d).max()
    assert ferr <= FLOW_TOL, f"flow error {ferr}"
    # the JPEG2000 front end still codes the raw frame (5/3: bit-exact)
    cm = orc.wavelet_mask(g1["mask"], p.dwt_levels, p.wavelet)
    y = orc.dwt2d(orc.dc_shift(frames[1], bd), 53, p.dwt_levels)
    assert np.array_equal(g1["coeffs"], orc.roi_shift(y, cm, p.scale_shift))


def test_denoise_changes_the_mask_only_through_the_flow(orc):
    a, b = pair_u8(seed=5300, h=128, w=128, n_blobs=4)
    frames = [a.numpy(), b.numpy()]
    on = _run(frames, 8, denoise=1)[1]
    with F.Context(flags=F.MANUAL | F.KEEP_INTERMEDIATES) as ctx:
        for i, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 3, fr, i, 8)
        F.flowroi_flush(ctx.h, 60000)
        off = fetch(ctx.h, 3, 1, 128, 128)
        with pytest.raises(F.FlowRoIError) as ei:  # no denoised image when denoising is off
            F.flowroi_get_intermediate(ctx.h, 3, 1, F.I_DENOISED, np.empty((128, 128), np.float32), 1000)
        assert ei.value.code == F.EINVAL
    assert not np.array_equal(on["flow"], off["flow"])
    # with the same mask the coefficients would agree: the DWT input is the raw frame
    assert on["coeffs"].shape == off["coeffs"].shape


def test_denoise_config_is_validated():
    for bad in (dict(denoise=2), dict(denoise=1, den_radius=0), dict(denoise=1, den_radius=4),
                dict(denoise=1, den_sigma_s=0.0), dict(denoise=1, den_sigma_r=-1.0)):
        with pytest.raises(F.FlowRoIError) as ei:
            F.Context(**bad)
        assert ei.value.code == F.EINVAL
