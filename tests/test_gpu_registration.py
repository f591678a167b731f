"""Registration to the predecessor by phase correlation (§Optical flow
extraction) on the GPU, through the C ABI, against the oracle.

Frames: a pair of the synthetic sequence (local motion) cropped from larger
frames at offsets that add a known global drift.  Stagewise: the GPU's
drift against the oracle's phase correlation of the same level images
(float FFT against float64: the integer peak equal, the sub-pixel vertex
within 1e-2 level pixels); the GPU's flow against the oracle's flow of the
pair registered by the GPU's own drift (1e-3 px); the drift against the
known one; and a pair without drift stays close to the unregistered flow."""
import numpy as np
import pytest

from synth import sequence_u16
from tests._gpu import F, fetch, oracle_params, u16

pytestmark = pytest.mark.gpu

FLOW_TOL = 1e-3


def _drift_pair(seed, h, w, s, pad=24, local=True):
    """prev = frame 0, cur = frame 1 (local motion) or frame 0 again, each
    cropped so that the content of cur is moved by s: cur(x) = frame(x - s)."""
    big = u16(sequence_u16(seed, 2, h + 2 * pad, w + 2 * pad, max(4, h * w // 3000)))
    sx, sy = s
    prev = np.ascontiguousarray(big[0][pad:pad + h, pad:pad + w])
    src = big[1] if local else big[0]
    cur = np.ascontiguousarray(src[pad - sy:pad - sy + h, pad - sx:pad - sx + w])
    return prev, cur


def _run(frames, bd, **cfg):
    h, w = frames[0].shape
    with F.Context(flags=F.MANUAL | F.KEEP_INTERMEDIATES, **cfg) as ctx:
        outs = []
        for t, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 2, fr, t, bd)
            F.flowroi_flush(ctx.h, 120000)
            g = fetch(ctx.h, 2, t, h, w)
            if cfg.get("register_frames"):
                g["drift"] = np.empty(2, np.float32)
                F.flowroi_get_intermediate(ctx.h, 2, t, F.I_DRIFT, g["drift"], 60000)
            outs.append(g)
    return outs


@pytest.mark.parametrize("h,w,s,level", [(256, 256, (6, -4), 1), (192, 320, (-8, 12), 2), (128, 128, (0, 0), 1)],
                         ids=["256_s6m4_l1", "192x320_sm8p12_l2", "128_s0_l1"])
def test_registration_parity(orc, h, w, s, level):
    prev, cur = _drift_pair(8000 + h, h, w, s)
    cfg = dict(register_frames=1, reg_level=level, pyr_levels=4, dwt_levels=3)
    g0, g1 = _run([prev, cur], 12, **cfg)
    assert np.all(g0["drift"] == 0.0)  # a first frame has no predecessor
    p = oracle_params(orc, **cfg)
    I0, I1 = orc.units(prev, 12), orc.units(cur, 12)
    ref = np.array(orc.register(I0, I1, level))
    assert np.abs(g1["drift"] - ref).max() <= 1e-2 * (1 << level), (g1["drift"], ref)
    d = orc.flow_reg(I1, I0, p.pyr_levels, p.poly_n_half, p.poly_sigma, p.iters, p.win_r, p.lam,
                     g1["drift"].astype(np.float64))
    ferr = np.abs(g1["flow"].transpose(2, 0, 1) - d).max()
    assert ferr <= FLOW_TOL, f"flow error {ferr}"
    # the rest of the path runs on that flow: saliency, cut, morphology as usual
    Sh = orc.normalise(orc.saliency(g1["flow"].transpose(2, 0, 1).astype(np.float64), p.sal_weight))
    assert np.abs(g1["shat"] - Sh).max() <= 1e-5
    m0, t = orc.threshold_f32(g1["shat"], p.roi_q)
    assert g1["thr"][0] == t and np.array_equal(m0, g1["mask0"])


@pytest.mark.parametrize("s,level", [((6, -4), 1), ((8, -12), 2), ((-3, 9), 1)])
def test_registration_finds_a_pure_drift(orc, s, level):
    prev, cur = _drift_pair(8200 + level, 256, 256, s, local=False)
    g1 = _run([prev, cur], 12, register_frames=1, reg_level=level, pyr_levels=4, dwt_levels=3)[1]
    assert np.abs(g1["drift"] - np.array(s)).max() <= 0.4 * (1 << level)


def test_registration_removes_the_drift_from_the_flow(orc):
    prev, cur = _drift_pair(8100, 256, 256, (7, 5), local=False)
    base = dict(pyr_levels=4, dwt_levels=3)
    reg = _run([prev, cur], 12, register_frames=1, reg_level=1, **base)[1]
    unreg = _run([prev, cur], 12, **base)[1]
    inner = (slice(32, -32), slice(32, -32))
    # the content only drifts: unregistered, its structures show motion of
    # about |s| = 8.6 px; registered, next to none is left
    big_unreg = (np.linalg.norm(unreg["flow"][inner], axis=-1) > 3.0).mean()
    big_reg = (np.linalg.norm(reg["flow"][inner], axis=-1) > 3.0).mean()
    assert big_unreg > 0.02 and big_reg < 0.1 * big_unreg, (big_unreg, big_reg)


def test_registration_config_and_sizes_are_validated():
    for bad in (dict(register_frames=2), dict(register_frames=1, reg_level=0),
                dict(register_frames=1, reg_level=3, pyr_levels=3)):
        with pytest.raises(F.FlowRoIError) as ei:
            F.Context(**bad)
        assert ei.value.code == F.EINVAL
    with F.Context(flags=F.MANUAL, register_frames=1, reg_level=1, pyr_levels=2, dwt_levels=1) as ctx:
        big = np.zeros((16, 4096), np.uint8)  # level 1 is 2048 wide: above the 1024 FFT size
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_submit_frame(ctx.h, 1, big, 0, 8)
        assert ei.value.code == F.EINVAL
