"""Helpers of the GPU tests: run frames through the C ABI and read back
every output.  (Uses only the ctypes binding of the CUDA library.)"""
import numpy as np

from paper_2511_14419_gb300 import flowroi as F


def u16(a):
    """int16 tensor/array holding 12-bit samples -> uint16 numpy view."""
    a = a.numpy() if hasattr(a, "numpy") else a
    return np.ascontiguousarray(a).view(np.uint16) if a.dtype == np.int16 else np.ascontiguousarray(a)


def fetch(ctx, sid, idx, h, w, keep=True, wavelet=53, timeout_ms=60000):
    out = {"mask": np.empty((h, w), np.uint8), "coeffs": np.empty((h, w), np.int32)}
    F.flowroi_get_mask(ctx, sid, idx, out["mask"], timeout_ms)
    F.flowroi_get_coeffs(ctx, sid, idx, out["coeffs"], timeout_ms)
    if keep:
        out["flow"] = np.empty((h, w, 2), np.float32)
        out["shat"] = np.empty((h, w), np.float32)
        out["mask0"] = np.empty((h, w), np.uint8)
        out["thr"] = np.empty(1, np.float32)
        F.flowroi_get_intermediate(ctx, sid, idx, F.I_FLOW, out["flow"], timeout_ms)
        F.flowroi_get_intermediate(ctx, sid, idx, F.I_SALIENCY, out["shat"], timeout_ms)
        F.flowroi_get_intermediate(ctx, sid, idx, F.I_MASK0, out["mask0"], timeout_ms)
        F.flowroi_get_intermediate(ctx, sid, idx, F.I_THRESHOLD, out["thr"], timeout_ms)
        if wavelet == 97:
            out["yf"] = np.empty((h, w), np.float32)
            F.flowroi_get_intermediate(ctx, sid, idx, F.I_COEFF_F32, out["yf"], timeout_ms)
    return out


def run_stream(frames, bit_depth, keep=True, plain=False, **cfg):
    """Submit `frames` (list of (H, W) arrays) as one stream, one frame per
    batch, and return the outputs of every frame."""
    flags = (F.KEEP_INTERMEDIATES if keep else 0) | F.MANUAL | (F.PLAIN if plain else 0)
    outs = []
    with F.Context(flags=flags, **cfg) as ctx:
        for i, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 7, fr, i, bit_depth)
            F.flowroi_flush(ctx.h, 120000)
            h, w = fr.shape
            outs.append(fetch(ctx.h, 7, i, h, w, keep, cfg.get("wavelet", 53)))
    return outs


def oracle_params(orc, **cfg):
    p = orc.Params()
    p.pyr_levels = cfg.get("pyr_levels", 3)
    p.dwt_levels = cfg.get("dwt_levels", 3)
    p.wavelet = cfg.get("wavelet", 53)
    p.iters = cfg.get("iters", 3)
    p.win_r = cfg.get("win_r", 7)
    p.poly_n_half = cfg.get("poly_n_half", 2)
    p.poly_sigma = cfg.get("poly_sigma", 1.1)
    p.roi_q = cfg.get("roi_q", 0.2)
    p.scale_shift = cfg.get("scale_shift", 5)
    p.r_open = cfg.get("r_open", 1)
    p.r_close = cfg.get("r_close", 2)
    p.sal_weight = cfg.get("sal_weight", 0.7)
    p.denoise = cfg.get("denoise", 0)
    p.den_radius = cfg.get("den_radius", 2)
    p.den_sigma_s = cfg.get("den_sigma_s", 2.0)
    p.den_sigma_r = cfg.get("den_sigma_r", 20.0)
    return p
