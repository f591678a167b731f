"""GPU path vs oracle, element by element, through the C ABI.

Acceptance (stage by stage, each GPU stage checked on the same input as
the oracle stage; where single precision decides an integer, the oracle
decides in single precision on the GPU's own values):
  - flow (float32) vs the float64 oracle: max abs error <= FLOW_TOL px;
  - normalised saliency from the GPU's flow: abs error <= SAL_TOL;
  - quantile cut on the GPU's own S^: threshold and mask0 bit-exact;
  - opening/closing of the GPU's own mask0: bit-exact;
  - end to end, mask0 differs from the oracle's only where the oracle's
    S^ lies within 1e-4 of its threshold;
  - 5/3 coefficients (DC shift, DWT, wavelet mask, RoI shift) given the
    GPU's mask: bit-exact;
  - 9/7 float coefficients vs float64: abs error <= 64 * D * 2^(B-1) * 2^-24.
    The rounding error of a float32 lifting step is half an ulp of its
    operands, which are bounded by a few times the DC-shifted sample range
    2^(B-1), not by the (often small) output coefficient; a coefficient of
    level l passes 2 x 5 rounded steps per level (4 lifting steps and the
    scaling, columns and rows) of every level up to l, and the lifting
    constants amplify earlier errors by less than 2 per step.  64 ulps of
    2^(B-1) per level bounds the sum.  Quantised + shifted coefficients
    from the GPU's own float coefficients: bit-exact.
"""
import numpy as np
import pytest
import torch

from synth import pair_u8, sequence_u16
from tests._gpu import F, fetch, oracle_params, run_stream, u16

pytestmark = pytest.mark.gpu

FLOW_TOL = 1e-3
SAL_TOL = 1e-5
QBAND = 1e-4


def _stagewise(orc, prev, cur, bd, g, **cfg):
    p = oracle_params(orc, **cfg)
    o = orc.frame(prev, cur, bd, p)
    h, w = cur.shape
    d = g["flow"].transpose(2, 0, 1).astype(np.float64)
    ferr = np.abs(d - o["flow"]).max()
    assert ferr <= FLOW_TOL, f"flow max abs error {ferr}"
    Sh = orc.normalise(orc.saliency(d, p.sal_weight))
    serr = np.abs(g["shat"] - Sh).max()
    assert serr <= SAL_TOL, f"saliency error {serr}"
    m0, t = orc.threshold_f32(g["shat"], p.roi_q)
    assert g["thr"][0] == t
    assert np.array_equal(m0, g["mask0"])
    assert np.array_equal(orc.morph(g["mask0"], p.r_open, p.r_close), g["mask"])
    diff = g["mask0"] != o["mask0"]
    if diff.any():
        assert np.abs(o["Sh"][diff] - o["t"]).max() <= QBAND
    cm = orc.wavelet_mask(g["mask"], p.dwt_levels, p.wavelet)
    if p.wavelet == 53:
        y = orc.dwt2d(orc.dc_shift(cur, bd), 53, p.dwt_levels)
        assert np.array_equal(g["coeffs"], orc.roi_shift(y, cm, p.scale_shift))
    else:
        y = orc.dwt2d(orc.dc_shift(cur, bd).astype(np.float64), 97, p.dwt_levels)
        tol = 64 * p.dwt_levels * 2.0 ** (bd - 1) * 2.0 ** -24
        yerr = np.abs(g["yf"] - y).max()
        assert yerr <= tol, f"9/7 error {yerr} > {tol}"
        _, delta, _, _ = orc.delta_table(p.dwt_levels, bd, p.delta_base)
        q = orc.quantise_f32(g["yf"], p.dwt_levels, delta)
        assert np.array_equal(g["coeffs"], orc.roi_shift(q, cm, p.scale_shift))
    iou = (g["mask"] & o["mask"]).sum() / max(1, (g["mask"] | o["mask"]).sum())
    return dict(flow_err=ferr, sal_err=serr, mask0_diff=int(diff.sum()), iou=iou)


def test_identical_frames_give_zero_flow_and_empty_mask(orc):
    prev, _ = pair_u8(seed=5, h=64, w=64, n_blobs=3)
    a = prev.numpy()
    g0, g1 = run_stream([a, a], 8)
    assert np.all(g1["flow"] == 0.0)
    assert g1["mask0"].sum() == 0 and g1["mask"].sum() == 0
    plain = orc.dwt2d(orc.dc_shift(a, 8), 53, 3)
    assert np.array_equal(g1["coeffs"], plain) and np.array_equal(g0["coeffs"], plain)
    assert g0["mask"].sum() == 0 and np.isinf(g0["thr"][0])


def test_pair_256_u8_53(orc):
    prev, cur = pair_u8(seed=1001)
    g = run_stream([prev.numpy(), cur.numpy()], 8)[1]
    r = _stagewise(orc, prev.numpy(), cur.numpy(), 8, g)
    assert r["iou"] > 0.98


@pytest.mark.parametrize("h,w", [(48, 64), (80, 48), (16, 16), (72, 40)])
def test_ragged_sizes(orc, h, w):
    prev, cur = pair_u8(seed=h * 1000 + w, h=h, w=w, n_blobs=2)
    levels = dict(pyr_levels=2, dwt_levels=3) if h > 16 else dict(pyr_levels=2, dwt_levels=1)
    g = run_stream([prev.numpy(), cur.numpy()], 8, **levels)[1]
    _stagewise(orc, prev.numpy(), cur.numpy(), 8, g, **levels)


@pytest.mark.parametrize("h,w,wav", [(16, 16, 97), (16, 16, 53), (72, 40, 97), (48, 64, 53), (200, 264, 97)])
def test_ragged_sizes_u16(orc, h, w, wav):
    """12-bit frames of ragged and tiny sizes: the staged 16-bit tile loads
    of the expansion and of DWT level 1 at image borders (symmetric
    extension of rows and columns, the mask clipped), including frames
    narrower than a DWT tile's apron."""
    seq = u16(sequence_u16(5000 + h * 7 + w, 2, h, w, 3))
    levels = dict(pyr_levels=2, dwt_levels=3, wavelet=wav) if h > 16 else dict(pyr_levels=2, dwt_levels=2, wavelet=wav)
    g = run_stream([seq[0], seq[1]], 12, **levels)[1]
    _stagewise(orc, seq[0], seq[1], 12, g, **levels)


@pytest.mark.parametrize("cfg", [
    dict(win_r=2),
    dict(win_r=10, poly_n_half=3, poly_sigma=1.5),
    dict(win_r=5, r_open=0, r_close=4, iters=1),
    dict(win_r=9, r_open=2, r_close=0, roi_q=0.05, pyr_levels=4),
], ids=["win5", "win21_poly7", "win11_close4_iter1", "win19_open2_q005"])
def test_method_settings(orc, cfg):
    """Other window sizes (each a separately compiled box-sum kernel with its
    own plane-ring depth), the 7-tap expansion, one iteration and other
    morphology radii, against the oracle with the same settings."""
    prev, cur = pair_u8(seed=4100 + cfg["win_r"], h=192, w=256, n_blobs=8)
    g = run_stream([prev.numpy(), cur.numpy()], 8, **cfg)[1]
    _stagewise(orc, prev.numpy(), cur.numpy(), 8, g, **cfg)


def test_sequence_1024_u16_53_resident_state(orc):
    """Three frames of one 12-bit stream: frames 1 and 2 reuse the resident
    expansion of their predecessor."""
    seq = u16(sequence_u16(2000, 3, 1024, 1024, 80))
    cfg = dict(pyr_levels=4, dwt_levels=5)
    gs = run_stream([seq[0], seq[1], seq[2]], 12, **cfg)
    for t in (1, 2):
        _stagewise(orc, seq[t - 1], seq[t], 12, gs[t], **cfg)


def test_pair_512_u16_97(orc):
    seq = u16(sequence_u16(3001, 2, 512, 512, 30))
    cfg = dict(pyr_levels=5, dwt_levels=5, wavelet=97)
    g = run_stream([seq[0], seq[1]], 12, **cfg)[1]
    _stagewise(orc, seq[0], seq[1], 12, g, **cfg)


def test_full_size_2048_u16_97(orc):
    """Frame geometry and settings of the 16 x 2048^2 batched workload
    (5-level pyramid, 9/7 DWT 5 levels), one stream through the captured
    graph path, one pair checked against the oracle at full size (the full
    16-frame batch is checked against frames run alone in
    test_batch_invariance_16x2048)."""
    seq = u16(sequence_u16(3000, 2, 2048, 2048, 200))
    cfg = dict(pyr_levels=5, dwt_levels=5, wavelet=97)
    g = run_stream([seq[0], seq[1]], 12, **cfg)[1]
    _stagewise(orc, seq[0], seq[1], 12, g, **cfg)


@pytest.mark.parametrize("win_r", [7, 2, 10])
def test_fp16_storage_epe_and_iou(orc, win_r):
    """fp16 storage (the window kernel's separate fp32 sums areas, whose
    ring depth depends on the window radius) against the FP64 oracle."""
    seq = u16(sequence_u16(3002, 2, 512, 512, 30))
    cfg = dict(pyr_levels=5, dwt_levels=5, wavelet=97, win_r=win_r)
    g = run_stream([seq[0], seq[1]], 12, precision=F.FP16, **cfg)[1]
    o = orc.frame(seq[0], seq[1], 12, oracle_params(orc, **cfg))
    d = g["flow"].transpose(2, 0, 1)
    epe = np.hypot(d[0] - o["flow"][0], d[1] - o["flow"][1]).mean()
    iou = (g["mask"] & o["mask"]).sum() / max(1, (g["mask"] | o["mask"]).sum())
    assert epe < 0.05 and iou > 0.9, (epe, iou)
    # integer paths stay exact given the GPU's own mask
    p = oracle_params(orc, **cfg)
    assert np.array_equal(orc.morph(g["mask0"], p.r_open, p.r_close), g["mask"])


@pytest.mark.parametrize("prec,win_r", [("fp32", 2), ("fp32", 5), ("fp32", 10), ("fp16", 10)])
def test_window_ring_several_tiles_per_block(orc, prec, win_r):
    """Window radii whose plane rings differ in depth (in fp32, how many of
    a tile's planes are column-summed at the end of the previous tile's
    iteration: all five at r = 2, four at r = 5, two at r = 10), on a
    2048 x 1024 pair: 512 level-0 tiles of 64 x 64, so every persistent
    block takes several tiles in turn and runs the hand-over between them."""
    seq = u16(sequence_u16(3100 + win_r, 2, 1024, 2048, 100))
    cfg = dict(pyr_levels=3, dwt_levels=3, wavelet=97, win_r=win_r)
    if prec == "fp32":
        g = run_stream([seq[0], seq[1]], 12, **cfg)[1]
        _stagewise(orc, seq[0], seq[1], 12, g, **cfg)
        return
    g = run_stream([seq[0], seq[1]], 12, precision=F.FP16, **cfg)[1]
    o = orc.frame(seq[0], seq[1], 12, oracle_params(orc, **cfg))
    d = g["flow"].transpose(2, 0, 1)
    epe = np.hypot(d[0] - o["flow"][0], d[1] - o["flow"][1]).mean()
    iou = (g["mask"] & o["mask"]).sum() / max(1, (g["mask"] | o["mask"]).sum())
    assert epe < 0.05 and iou > 0.9, (epe, iou)


def test_device_pointer_io_matches_host_io():
    prev, cur = pair_u8(seed=77, h=128, w=128, n_blobs=5)
    host = run_stream([prev.numpy(), cur.numpy()], 8, keep=False)[1]
    with F.Context(flags=F.MANUAL) as ctx:
        for i, fr in enumerate((prev, cur)):
            F.flowroi_submit_frame(ctx.h, 3, fr.cuda().contiguous(), i, 8)
            F.flowroi_flush(ctx.h, 60000)
        m = torch.empty((128, 128), dtype=torch.uint8, device="cuda")
        c = torch.empty((128, 128), dtype=torch.int32, device="cuda")
        F.flowroi_get_mask(ctx.h, 3, 1, m)
        F.flowroi_get_coeffs(ctx.h, 3, 1, c)
    assert np.array_equal(m.cpu().numpy(), host["mask"])
    assert np.array_equal(c.cpu().numpy(), host["coeffs"])


def test_fp16_storage_2048_epe_and_iou_vs_fp64(orc):
    """fp16 storage of pyramid, expansion fields and G, h (float arithmetic,
    float 2x2 solve) on a full-size 2048x2048 pair: flow EPE and mask IoU
    against the float64 oracle, beside the float32 storage path."""
    seq = u16(sequence_u16(3000, 2, 2048, 2048, 200))
    cfg = dict(pyr_levels=5, dwt_levels=5, wavelet=97)
    o = orc.frame(seq[0], seq[1], 12, oracle_params(orc, **cfg))
    res = {}
    for name, prec in (("fp32", F.FP32), ("fp16", F.FP16)):
        g = run_stream([seq[0], seq[1]], 12, precision=prec, **cfg)[1]
        d = g["flow"].transpose(2, 0, 1).astype(np.float64)
        epe = float(np.hypot(d[0] - o["flow"][0], d[1] - o["flow"][1]).mean())
        mx = float(np.abs(d - o["flow"]).max())
        iou = float((g["mask"] & o["mask"]).sum() / max(1, (g["mask"] | o["mask"]).sum()))
        res[name] = (epe, mx, iou)
    print(f"\n2048^2 pair vs float64 oracle: fp32 EPE {res['fp32'][0]:.3e} max {res['fp32'][1]:.3e} IoU {res['fp32'][2]:.5f}; "
          f"fp16 EPE {res['fp16'][0]:.3e} max {res['fp16'][1]:.3e} IoU {res['fp16'][2]:.5f}")
    assert res["fp32"][1] <= FLOW_TOL
    assert res["fp16"][0] < 0.05 and res["fp16"][2] > 0.9


def test_batch_invariance_16x2048():
    """The headline batch: 16 streams of 2048^2 12-bit frames (the bench
    workload's first two frames per stream), each frame index one batch of
    16 through the captured graph; streams 0, 7 and 15 are bit-identical to
    the same streams run alone."""
    S = 16
    seqs = [sequence_u16(3000 + s, 2, 2048, 2048, 200, device="cuda") for s in range(S)]
    cfg = dict(pyr_levels=5, dwt_levels=5, wavelet=97)
    got = {}
    with F.Context(flags=F.MANUAL, **cfg) as ctx:
        for t in range(2):
            for s in range(S):
                F.flowroi_submit_frame(ctx.h, s, seqs[s][t], t, 12)
            assert F.flowroi_step(ctx.h) == S
            F.flowroi_flush(ctx.h, 120000)
        for s in (0, 7, 15):
            got[s] = fetch(ctx.h, s, 1, 2048, 2048, keep=False, wavelet=97)
    for s in (0, 7, 15):
        alone = run_stream([u16(seqs[s][0].cpu()), u16(seqs[s][1].cpu())], 12, keep=False, **cfg)[1]
        assert np.array_equal(got[s]["mask"], alone["mask"]), s
        assert np.array_equal(got[s]["coeffs"], alone["coeffs"]), s
        assert got[s]["mask"].sum() > 0
