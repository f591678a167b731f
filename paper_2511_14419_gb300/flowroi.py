"""ctypes binding of the FlowRoI C ABI (include/flowroi.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, converts numpy arrays / torch tensors to plain pointers
(with the matching on-device flag) and turns a negative status into a
``FlowRoIError``.  All computation happens in the CUDA library; if it is not
built, importing this module fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

from ._build import LIB

OK = 0
EINVAL, ENOSTREAM, EBUSY, ENOMEM, ETIMEDOUT, EDEVICE, EGONE, ENOTKEPT, ERANGE = -1, -2, -3, -4, -5, -6, -7, -8, -9
U8, U16 = 1, 2
W53, W97 = 53, 97
FP32, FP16 = 32, 16
KEEP_INTERMEDIATES, PLAIN, MANUAL = 0x1, 0x2, 0x4
TEST_EXPIRE_TMA, TEST_EXPIRE_LOOP = 0x100, 0x200
CS_CONTAINER, CS_J2C = 0, 1
I_FLOW, I_SALIENCY, I_MASK0, I_COEFF_F32, I_THRESHOLD, I_DENOISED, I_DRIFT = 1, 2, 3, 4, 5, 6, 7

EXPORTS = [
    "flowroi_abi_version", "flowroi_default_config", "flowroi_create", "flowroi_submit_frame", "flowroi_submit_frames",
    "flowroi_step", "flowroi_get_mask", "flowroi_get_coeffs", "flowroi_get_results", "flowroi_get_intermediate",
    "flowroi_flush", "flowroi_end_stream", "flowroi_get_stats", "flowroi_destroy",
    "flowroi_last_error", "flowroi_quant_steps", "flowroi_compute_stream", "flowroi_set_profiling",
    "flowroi_get_kernel_times", "flowroi_dwt_roi_noalloc", "flowroi_reset_stats",
    "flowroi_encode_codestreams", "flowroi_codestream_bound", "flowroi_get_codestream",
    "flowroi_tiles_check", "flowroi_set_tiles", "flowroi_get_tiles", "flowroi_autotune", "flowroi_route",
]


class FlowRoIError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class flowroi_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("roi_q", ctypes.c_float), ("scale_shift", ctypes.c_int32),
        ("wavelet", ctypes.c_int32), ("dwt_levels", ctypes.c_int32), ("pyr_levels", ctypes.c_int32),
        ("iters", ctypes.c_int32), ("win_r", ctypes.c_int32), ("poly_n_half", ctypes.c_int32),
        ("poly_sigma", ctypes.c_float), ("lambda_", ctypes.c_float), ("sal_weight", ctypes.c_float),
        ("r_open", ctypes.c_int32), ("r_close", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("delta_base", ctypes.c_float), ("max_batch_frames", ctypes.c_int32), ("result_ring", ctypes.c_int32),
        ("flags", ctypes.c_uint32), ("device", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64),
        ("denoise", ctypes.c_int32), ("den_radius", ctypes.c_int32), ("den_sigma_s", ctypes.c_float),
        ("den_sigma_r", ctypes.c_float), ("min_area", ctypes.c_int32), ("adjacent", ctypes.c_int32),
        ("register_frames", ctypes.c_int32), ("reg_level", ctypes.c_int32), ("codestream_bpp", ctypes.c_float),
        ("codestream_format", ctypes.c_int32), ("tile_table", ctypes.c_char_p),
        ("codestream_reset", ctypes.c_int32),
    ]


class flowroi_frame(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("pitch_bytes", ctypes.c_int32), ("dtype", ctypes.c_int32), ("bit_depth", ctypes.c_int32),
        ("frame_idx", ctypes.c_int64), ("data", ctypes.c_void_p), ("data_on_device", ctypes.c_int32),
    ]


class flowroi_cs_job(ctypes.Structure):
    _fields_ = [("coeffs", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("wavelet", ctypes.c_int32), ("shift", ctypes.c_int32),
                ("bit_depth", ctypes.c_int32), ("budget_bytes", ctypes.c_int64), ("out", ctypes.c_void_p),
                ("out_cap", ctypes.c_uint64), ("out_len", ctypes.c_uint64), ("format", ctypes.c_int32),
                ("reset", ctypes.c_int32)]


class flowroi_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("level", ctypes.c_int32), ("iter", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class flowroi_stats(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("frames_submitted", ctypes.c_int64), ("frames_done", ctypes.c_int64),
        ("batches", ctypes.c_int64), ("streams_admitted", ctypes.c_int64), ("admissions_refused", ctypes.c_int64),
        ("bytes_admitted", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64), ("lat_p50_ms", ctypes.c_double),
        ("lat_p99_ms", ctypes.c_double), ("lat_mean_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB)
        P, I, I64, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
        sigs = {
            "flowroi_abi_version": (I, []),
            "flowroi_default_config": (None, [ctypes.POINTER(flowroi_config)]),
            "flowroi_create": (I, [ctypes.POINTER(flowroi_config), ctypes.POINTER(P)]),
            "flowroi_submit_frame": (I, [P, I64, ctypes.POINTER(flowroi_frame)]),
            "flowroi_submit_frames": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(flowroi_frame),
                                          ctypes.POINTER(I)]),
            "flowroi_step": (I, [P]),
            "flowroi_get_mask": (I, [P, I64, I64, P, I, I]),
            "flowroi_get_coeffs": (I, [P, I64, I64, P, I, I]),
            "flowroi_get_results": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(P),
                                        ctypes.POINTER(P), I, I, ctypes.POINTER(I)]),
            "flowroi_get_intermediate": (I, [P, I64, I64, I, P, I, I]),
            "flowroi_flush": (I, [P, I]),
            "flowroi_end_stream": (I, [P, I64]),
            "flowroi_get_stats": (I, [P, ctypes.POINTER(flowroi_stats)]),
            "flowroi_destroy": (None, [P]),
            "flowroi_last_error": (ctypes.c_char_p, [P]),
            "flowroi_quant_steps": (I, [I, I, ctypes.c_float, P, P, P, P]),
            "flowroi_compute_stream": (I, [P, ctypes.POINTER(P)]),
            "flowroi_set_profiling": (I, [P, I]),
            "flowroi_get_kernel_times": (I, [P, ctypes.POINTER(flowroi_kernel_time), I]),
            "flowroi_dwt_roi_noalloc": (I, [P, I, I, I, I, I, P, I, I, I, P, P, P]),
            "flowroi_reset_stats": (I, [P]),
            "flowroi_encode_codestreams": (I, [P, I, ctypes.POINTER(flowroi_cs_job), I]),
            "flowroi_codestream_bound": (ctypes.c_uint64, [I, I, I]),
            "flowroi_route": (ctypes.c_uint32, [I64, ctypes.c_uint32]),
            "flowroi_get_codestream": (I, [P, I64, I64, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), I, I]),
            "flowroi_tiles_check": (I, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_uint64]),
            "flowroi_set_tiles": (I, [P, ctypes.c_char_p]),
            "flowroi_get_tiles": (I, [P, ctypes.c_char_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
            "flowroi_autotune": (I, [ctypes.POINTER(flowroi_config), I, ctypes.POINTER(I), ctypes.POINTER(I), I, I,
                                     ctypes.c_char_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        del U32
        _lib = L
    return _lib


def _check(rc: int, ctx=None) -> int:
    if rc < 0:
        raise FlowRoIError(rc, lib().flowroi_last_error(ctx).decode(errors="replace"))
    return rc


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (must be contiguous)."""
    if hasattr(a, "data_ptr"):  # torch.Tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, 0


# ------------------------------------------------------------ entry points --

def flowroi_abi_version() -> int:
    return lib().flowroi_abi_version()


def flowroi_default_config(**overrides) -> flowroi_config:
    cfg = flowroi_config()
    lib().flowroi_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "tile_table" and isinstance(v, str):
            v = v.encode()
        setattr(cfg, "lambda_" if k == "lam" else k, v)
    return cfg


def flowroi_create(cfg: flowroi_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().flowroi_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def flowroi_submit_frame(ctx, stream_id: int, data, frame_idx: int, bit_depth: int, pitch_bytes: int = 0) -> int:
    """`data`: (H, W) uint8 or uint16 samples (int16 with the same bit
    pattern also accepted), numpy (host) or torch (host or CUDA)."""
    h, w = int(data.shape[0]), int(data.shape[1])
    esz = data.itemsize if hasattr(data, "itemsize") else data.element_size()
    p, dev = _ptr(data)
    f = flowroi_frame(ctypes.sizeof(flowroi_frame), w, h, pitch_bytes, U8 if esz == 1 else U16, bit_depth,
                      frame_idx, p, dev)
    return _check(lib().flowroi_submit_frame(ctx, stream_id, ctypes.byref(f)), ctx)


def _frame(data, frame_idx: int, bit_depth: int, pitch_bytes: int = 0) -> "flowroi_frame":
    h, w = int(data.shape[0]), int(data.shape[1])
    esz = data.itemsize if hasattr(data, "itemsize") else data.element_size()
    p, dev = _ptr(data)
    return flowroi_frame(ctypes.sizeof(flowroi_frame), w, h, pitch_bytes, U8 if esz == 1 else U16, bit_depth,
                         frame_idx, p, dev)


def flowroi_submit_frames(ctx, items) -> tuple:
    """`items`: sequence of (stream_id, data, frame_idx, bit_depth).
    Returns (accepted, status): frames [0, accepted) were submitted; when
    accepted < len(items), status is the refusal code of the next one."""
    n = len(items)
    ids = (ctypes.c_int64 * max(n, 1))(*[int(it[0]) for it in items])
    frs = (flowroi_frame * max(n, 1))(*[_frame(it[1], it[2], it[3]) for it in items])
    st = ctypes.c_int(0)
    k = lib().flowroi_submit_frames(ctx, n, ids, frs, ctypes.byref(st))
    if k < 0:
        _check(k, ctx)
    return k, st.value


def flowroi_step(ctx) -> int:
    return _check(lib().flowroi_step(ctx), ctx)


def flowroi_get_mask(ctx, stream_id: int, frame_idx: int, out, timeout_ms: int = -1) -> int:
    p, dev = _ptr(out)
    return _check(lib().flowroi_get_mask(ctx, stream_id, frame_idx, p, dev, timeout_ms), ctx)


def flowroi_get_coeffs(ctx, stream_id: int, frame_idx: int, out, timeout_ms: int = -1) -> int:
    p, dev = _ptr(out)
    return _check(lib().flowroi_get_coeffs(ctx, stream_id, frame_idx, p, dev, timeout_ms), ctx)


def flowroi_get_results(ctx, items, timeout_ms: int = -1) -> list:
    """Masks and coefficients of several frames in one call (see the C
    header): items = [(stream_id, frame_idx, mask_out, coeffs_out)], each
    output a contiguous array or tensor, or None to skip it; all outputs on
    the host or all on the device.  Returns the per-frame status codes;
    raises FlowRoIError with the first failing frame's code."""
    n = len(items)
    ids = (ctypes.c_int64 * max(n, 1))(*[int(it[0]) for it in items])
    fis = (ctypes.c_int64 * max(n, 1))(*[int(it[1]) for it in items])
    mp = (ctypes.c_void_p * max(n, 1))()
    cp = (ctypes.c_void_p * max(n, 1))()
    dev = None
    for k, (_, _, m, c) in enumerate(items):
        for arr, dst in ((m, mp), (c, cp)):
            if arr is None:
                continue
            p, d = _ptr(arr)
            if dev is None:
                dev = d
            elif d != dev:
                raise ValueError("outputs must all be on the host or all on the device")
            dst[k] = p
    st = (ctypes.c_int * max(n, 1))()
    _check(lib().flowroi_get_results(ctx, n, ids, fis, mp, cp, int(dev or 0), timeout_ms, st), ctx)
    return list(st)[:n]


def flowroi_get_intermediate(ctx, stream_id: int, frame_idx: int, which: int, out, timeout_ms: int = -1) -> int:
    p, dev = _ptr(out)
    return _check(lib().flowroi_get_intermediate(ctx, stream_id, frame_idx, which, p, dev, timeout_ms), ctx)


def flowroi_flush(ctx, timeout_ms: int = -1) -> int:
    return _check(lib().flowroi_flush(ctx, timeout_ms), ctx)


def flowroi_end_stream(ctx, stream_id: int) -> int:
    return _check(lib().flowroi_end_stream(ctx, stream_id), ctx)


def flowroi_get_stats(ctx) -> dict:
    s = flowroi_stats()
    s.struct_size = ctypes.sizeof(flowroi_stats)
    _check(lib().flowroi_get_stats(ctx, ctypes.byref(s)), ctx)
    return {name: getattr(s, name) for name, _ in flowroi_stats._fields_ if name != "struct_size"}


def flowroi_reset_stats(ctx) -> int:
    return _check(lib().flowroi_reset_stats(ctx), ctx)


def flowroi_destroy(ctx) -> None:
    lib().flowroi_destroy(ctx)


def flowroi_last_error(ctx=None) -> str:
    return lib().flowroi_last_error(ctx).decode(errors="replace")


def flowroi_quant_steps(levels: int, bit_depth: int, delta_base: float = 1.0):
    """(delta float32[3L+1], eps int32, mu int32, gain float64) as numpy arrays."""
    import numpy as np
    nb = 3 * levels + 1
    d = np.empty(nb, np.float32)
    e = np.empty(nb, np.int32)
    m = np.empty(nb, np.int32)
    g = np.empty(nb, np.float64)
    _check(lib().flowroi_quant_steps(levels, bit_depth, delta_base, d.ctypes.data, e.ctypes.data, m.ctypes.data,
                                     g.ctypes.data))
    return d, e, m, g


def flowroi_compute_stream(ctx) -> int:
    """The context's compute stream handle (cudaStream_t as an int)."""
    h = ctypes.c_void_p()
    _check(lib().flowroi_compute_stream(ctx, ctypes.byref(h)), ctx)
    return h.value or 0


def flowroi_set_profiling(ctx, on: int) -> int:
    return _check(lib().flowroi_set_profiling(ctx, on), ctx)


def flowroi_get_kernel_times(ctx, cap: int = 256) -> list:
    arr = (flowroi_kernel_time * cap)()
    n = _check(lib().flowroi_get_kernel_times(ctx, arr, cap), ctx)
    return [dict(name=arr[i].name.decode(), level=arr[i].level, iter=arr[i].iter, launches=arr[i].launches,
                 total_ms=arr[i].total_ms) for i in range(n)]


def flowroi_dwt_roi_noalloc(raw, bit_depth: int, mask, wavelet: int, levels: int, scale_shift: int, delta,
                            coeffs, stream: int = 0, pitch_bytes: int = 0) -> int:
    """JPEG2000 front end of one frame with no allocation (see the C header).
    raw: CUDA tensor (H, W) of 1- or 2-byte samples, contiguous or with
    padded rows (unit column stride; its row stride gives the pitch unless
    pitch_bytes is passed); mask: uint8 or bool CUDA tensor (H, W); coeffs:
    int32 CUDA tensor (H, W); delta: host float32 array of 3*levels+1 steps,
    or None (5/3); stream: cudaStream_t handle as an int (0 = default).
    Every shape, dtype and size is checked here before the library is
    called: a smaller mask or coefficient buffer would otherwise be read or
    written past its end on the device."""
    import torch
    if raw.dim() != 2 or mask.dim() != 2 or coeffs.dim() != 2:
        raise ValueError("raw, mask and coeffs must be 2-D (H, W) tensors")
    if not (raw.is_cuda and mask.is_cuda and coeffs.is_cuda):
        raise ValueError("raw, mask and coeffs must be device tensors")
    h, w = int(raw.shape[0]), int(raw.shape[1])
    esz = raw.element_size()
    if esz not in (1, 2) or raw.is_floating_point():
        raise ValueError("raw must hold 1- or 2-byte integer samples")
    if tuple(mask.shape) != (h, w) or tuple(coeffs.shape) != (h, w):
        raise ValueError(f"mask {tuple(mask.shape)} and coeffs {tuple(coeffs.shape)} must both be {(h, w)}")
    if mask.dtype not in (torch.uint8, torch.bool):
        raise ValueError("mask must be uint8 (or bool)")
    if coeffs.dtype != torch.int32:
        raise ValueError("coeffs must be int32")
    mp_, _ = _ptr(mask)
    cp, _ = _ptr(coeffs)
    if raw.is_contiguous():
        rp = raw.data_ptr()
    else:
        if raw.stride(1) != 1 or raw.stride(0) < w:
            raise ValueError("raw must have unit column stride and rows at least W samples apart")
        rp = raw.data_ptr()
        if not pitch_bytes:
            pitch_bytes = raw.stride(0) * esz
    if pitch_bytes and pitch_bytes < w * esz:
        raise ValueError("pitch_bytes smaller than a row")
    dp = None
    if delta is not None:
        import numpy as np
        delta = np.ascontiguousarray(delta, dtype=np.float32)
        if delta.size < 3 * levels + 1:
            raise ValueError(f"delta needs 3*levels+1 = {3 * levels + 1} steps")
        dp = delta.ctypes.data
    rc = lib().flowroi_dwt_roi_noalloc(rp, w, h, pitch_bytes, U8 if esz == 1 else U16, bit_depth, mp_, wavelet, levels,
                                       scale_shift, dp, cp, stream or None)
    if rc < 0:
        raise FlowRoIError(rc, "flowroi_dwt_roi_noalloc rejected the request" if rc == EINVAL else "CUDA error")
    return rc


def flowroi_get_codestream(ctx, stream_id: int, frame_idx: int, out, timeout_ms: int = -1) -> int:
    """Copies a frame's container (config.codestream_bpp > 0) into out (a
    uint8 numpy array or CUDA tensor; its size is the capacity); returns
    the container's length."""
    p, dev = _ptr(out)
    cap = int(out.numel() * out.element_size()) if hasattr(out, "numel") else int(out.nbytes)
    n = ctypes.c_uint64(0)
    _check(lib().flowroi_get_codestream(ctx, stream_id, frame_idx, p, cap, ctypes.byref(n), dev, timeout_ms), ctx)
    return int(n.value)


def flowroi_codestream_bound(width: int, height: int, levels: int) -> int:
    return int(lib().flowroi_codestream_bound(width, height, levels))


def flowroi_route(stream_id: int, n_devices: int) -> int:
    """Device index of a stream among n_devices (see the C header)."""
    if n_devices < 1:
        raise ValueError("n_devices must be >= 1")
    return int(lib().flowroi_route(int(stream_id), int(n_devices)))


class Router:
    """One context per device, streams routed by flowroi_route: submit and
    fetch calls take a stream id and go to that stream's context.  Only
    dispatch lives here; every call is the C ABI's.  make_context(device)
    builds a device's context (default: Context(device=device, **cfg))."""

    def __init__(self, n_devices: int, make_context=None, **cfg):
        if n_devices < 1:
            raise ValueError("n_devices must be >= 1")
        self.n = n_devices
        self._make = make_context or (lambda d: Context(device=d, **cfg))
        self._ctx = {}

    def device_of(self, stream_id: int) -> int:
        return flowroi_route(stream_id, self.n)

    def context(self, stream_id: int):
        d = self.device_of(stream_id)
        if d not in self._ctx:
            self._ctx[d] = self._make(d)
        return self._ctx[d]

    def submit_frame(self, stream_id: int, frame, frame_idx: int, bit_depth: int) -> int:
        c = self.context(stream_id)
        return flowroi_submit_frame(c.h, stream_id, frame, frame_idx, bit_depth)

    def get_mask(self, stream_id: int, frame_idx: int, out, timeout_ms: int = 60000) -> int:
        c = self.context(stream_id)
        return flowroi_get_mask(c.h, stream_id, frame_idx, out, timeout_ms)

    def flush(self, timeout_ms: int = 60000) -> None:
        for c in self._ctx.values():
            flowroi_flush(c.h, timeout_ms)

    def close(self) -> None:
        for c in self._ctx.values():
            c.close()
        self._ctx = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def flowroi_encode_codestreams(ctx, jobs) -> list:
    """Codes coefficient planes into frame containers or JPEG2000
    codestreams (see the C header).  jobs: dicts with coeffs (int32 (H, W)
    numpy array or CUDA tensor), levels, wavelet, shift, bit_depth, budget
    (pass-data bytes, 0 = every pass), format (CS_CONTAINER or CS_J2C),
    reset (0 or 1: contexts reset at every pass) and out (uint8 numpy array
    or CUDA tensor: the destination, its size the capacity).  All on the
    host or all on the device.  Returns the lengths."""
    arr = (flowroi_cs_job * len(jobs))()
    dev = None
    for i, j in enumerate(jobs):
        cp, cdev = _ptr(j["coeffs"])
        op, odev = _ptr(j["out"])
        if dev is None:
            dev = cdev
        if cdev != dev or odev != dev:
            raise ValueError("coeffs and out must all be on the host or all on the device")
        h, w = int(j["coeffs"].shape[0]), int(j["coeffs"].shape[1])
        nbytes = int(j["out"].numel() * j["out"].element_size()) if hasattr(j["out"], "numel") else int(j["out"].nbytes)
        arr[i] = flowroi_cs_job(cp, w, h, j["levels"], j["wavelet"], j.get("shift", 0), j.get("bit_depth", 12),
                                int(j.get("budget", 0)), op, nbytes, 0, int(j.get("format", CS_CONTAINER)),
                                int(j.get("reset", 0)))
    _check(lib().flowroi_encode_codestreams(ctx, len(jobs), arr, int(dev)), ctx)
    return [int(arr[i].out_len) for i in range(len(jobs))]


def flowroi_tiles_check(json_text: str) -> str:
    """'' when the tile table is valid, else the reason (no device used)."""
    err = ctypes.create_string_buffer(512)
    rc = lib().flowroi_tiles_check(json_text.encode(), err, len(err))
    return "" if rc == OK else (err.value.decode(errors="replace") or "invalid")


def flowroi_set_tiles(ctx, json_text) -> int:
    return _check(lib().flowroi_set_tiles(ctx, json_text.encode() if json_text is not None else None), ctx)


def flowroi_get_tiles(ctx) -> str:
    n = ctypes.c_uint64(0)
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().flowroi_get_tiles(ctx, buf, len(buf), ctypes.byref(n)), ctx)
    return buf.value.decode()


def flowroi_autotune(cfg: flowroi_config, sizes, streams: int, steps: int) -> str:
    """Runs the tile search (see the C header) for frame sizes [(w, h), ...]
    and returns the chosen table as JSON text."""
    ws = (ctypes.c_int * len(sizes))(*[int(w) for w, _ in sizes])
    hs = (ctypes.c_int * len(sizes))(*[int(h) for _, h in sizes])
    n = ctypes.c_uint64(0)
    buf = ctypes.create_string_buffer(1 << 16)
    rc = lib().flowroi_autotune(ctypes.byref(cfg), len(sizes), ws, hs, streams, steps, buf, len(buf), ctypes.byref(n))
    if rc < 0:
        raise FlowRoIError(rc, "flowroi_autotune failed (its reason is on stderr)")
    return buf.value.decode()


class Context:
    """Small owner of a context handle (destroyed on close / exit)."""

    def __init__(self, **cfg):
        self.cfg = flowroi_default_config(**cfg)
        self.h = flowroi_create(self.cfg)

    def close(self):
        if self.h:
            flowroi_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
