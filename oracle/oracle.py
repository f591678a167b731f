"""FlowRoI oracle: numpy front end over the plain FP64 C oracle.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference legs import this module.  It
shares no code with the CUDA library (``paper_2511_14419_gb300``) and never
imports it.

Every function below is a thin ctypes marshaller around one stage of
``flowroi_oracle.c`` (see the comments there for the paper passage each stage
follows); ``frame`` chains them in the paper's order for one frame pair:
§Optical flow extraction -> §Region of Interest extraction -> the JPEG2000
front end of §Implementation details.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flowroi_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "orc_ebcot.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double: no fast-math, no FMA
    contraction, so x86 and Arm builds round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_F = ctypes.c_float


def _declare(L):
    sig = {
        "orc_version": (_I, []),
        "orc_units": (None, [_P, _I, _I, _I64, _P]),
        "orc_pyr_down": (None, [_P, _I, _I, _P]),
        "orc_median3": (None, [_P, _I, _I, _P]),
        "orc_remove_small": (None, [_P, _I, _I, _I]),
        "orc_bilateral": (None, [_P, _I, _I, _I, _D, _D, _P]),
        "orc_denoise": (None, [_P, _I, _I, _I, _D, _D, _P, _P]),
        "orc_poly_projector": (_I, [_I, _D, _P]),
        "orc_poly_expand": (_I, [_P, _I, _I, _I, _D, _P]),
        "orc_flow_upsample": (None, [_P, _I, _I, _I, _I, _P]),
        "orc_flow_iterate": (None, [_P, _P, _I, _I, _P, _I, _I, _D, _P]),
        "orc_flow": (_I, [_P, _P, _I, _I, _I, _I, _D, _I, _I, _D, _P]),
        "orc_flow_reg": (_I, [_P, _P, _I, _I, _I, _I, _D, _I, _I, _D, _D, _D, _P]),
        "orc_saliency": (None, [_P, _I, _I, _D, _P]),
        "orc_normalise": (None, [_P, _I64, _P]),
        "orc_quantile_k": (_I64, [_F, _I64]),
        "orc_threshold": (_D, [_P, _I64, _F, _P]),
        "orc_threshold_f32": (_F, [_P, _I64, _F, _P]),
        "orc_erode": (None, [_P, _I, _I, _I, _P]),
        "orc_dilate": (None, [_P, _I, _I, _I, _P]),
        "orc_morph": (None, [_P, _I, _I, _I, _I, _P]),
        "orc_dwt53_1d": (None, [_P, _I, _P]),
        "orc_idwt53_1d": (None, [_P, _I, _P]),
        "orc_dwt97_1d": (None, [_P, _I, _P]),
        "orc_idwt97_1d": (None, [_P, _I, _P]),
        "orc_dwt53_2d": (None, [_P, _I, _I, _I]),
        "orc_idwt53_2d": (None, [_P, _I, _I, _I]),
        "orc_dwt97_2d": (None, [_P, _I, _I, _I]),
        "orc_idwt97_2d": (None, [_P, _I, _I, _I]),
        "orc_dc_shift": (None, [_P, _I, _I, _I64, _P]),
        "orc_subband_index": (_I, [_I, _I, _I, _I, _I]),
        "orc_delta_table": (_I, [_I, _I, _D, _P, _P, _P, _P]),
        "orc_quantise_f32": (None, [_P, _I, _I, _I, _P, _P]),
        "orc_quantise_f64": (None, [_P, _I, _I, _I, _P, _P]),
        "orc_wavelet_mask": (None, [_P, _I, _I, _I, _I, _P]),
        "orc_roi_shift": (_I, [_P, _P, _I64, _I]),
        "orc_mq_roundtrip": (ctypes.c_long, [_P, _P, ctypes.c_long, _P, _P]),
        "orc_mq_table": (_I, [_P, _P, _P, _P]),
        "orc_context_tables": (None, [_P, _P, _P]),
        "orc_t1_encode": (_I, [_P, _I, _I, _I, _I, _P, ctypes.c_long, _P, _P, _P, _I]),
        "orc_t1_decode": (None, [_P, _P, _I, _I, _I, _I, _I, _I, _P, _I, _I]),
        "orc_hull": (_I, [_I, _P, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _c(a, dtype):
    """Contiguous array of the given dtype (copied only when needed)."""
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- stages --

def units(raw: np.ndarray, bit_depth: int) -> np.ndarray:
    raw = np.ascontiguousarray(raw)
    out = np.empty(raw.shape, np.float64)
    lib().orc_units(_ptr(raw), raw.dtype.itemsize, bit_depth, raw.size, _ptr(out))
    return out


def remove_small(mask: np.ndarray, min_area: int) -> np.ndarray:
    """Mask without its 8-connected components of fewer than min_area pixels."""
    out = np.ascontiguousarray(mask, dtype=np.uint8).copy()
    h, w = out.shape
    lib().orc_remove_small(_ptr(out), w, h, int(min_area))
    return out


def adjacent_merge(own_masks, k: int):
    """§Region of Interest extraction: masks of neighbouring frames
    incorporated (Table 1 "Adjacent factor").  Reading: the RoI mask of
    frame j is the union of the per-frame masks of frames j-k .. j+k that
    exist (the window is cut at both ends of the sequence)."""
    n = len(own_masks)
    out = []
    for j in range(n):
        m = np.zeros_like(own_masks[j])
        for i in range(max(0, j - k), min(n - 1, j + k) + 1):
            m = m | own_masks[i]
        out.append(m)
    return out


def median3(img: np.ndarray) -> np.ndarray:
    """3x3 median, replicate border (§Optical flow extraction, denoising)."""
    img = _c(img, np.float64)
    h, w = img.shape
    out = np.empty_like(img)
    lib().orc_median3(_ptr(img), w, h, _ptr(out))
    return out


def bilateral(img: np.ndarray, rb: int, sigma_s: float, sigma_r: float) -> np.ndarray:
    """Bilateral filter over a (2rb+1)^2 square, replicate border."""
    img = _c(img, np.float64)
    h, w = img.shape
    out = np.empty_like(img)
    lib().orc_bilateral(_ptr(img), w, h, rb, sigma_s, sigma_r, _ptr(out))
    return out


def denoise(img: np.ndarray, rb: int, sigma_s: float, sigma_r: float) -> np.ndarray:
    """Median 3x3, then bilateral (the paper's two-step denoising)."""
    img = _c(img, np.float64)
    h, w = img.shape
    tmp, out = np.empty_like(img), np.empty_like(img)
    lib().orc_denoise(_ptr(img), w, h, rb, sigma_s, sigma_r, _ptr(tmp), _ptr(out))
    return out


def pyr_down(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.float64)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2), np.float64)
    lib().orc_pyr_down(_ptr(img), w, h, _ptr(out))
    return out


def poly_projector(n_half: int, sigma: float) -> np.ndarray:
    m = 2 * n_half + 1
    P = np.empty((6, m * m), np.float64)
    if lib().orc_poly_projector(n_half, sigma, _ptr(P)) != 0:
        raise ValueError("singular Gram matrix")
    return P


def poly_expand(img: np.ndarray, n_half: int, sigma: float) -> np.ndarray:
    """(5, h, w): A11, A12, A22, b1, b2."""
    img = _c(img, np.float64)
    h, w = img.shape
    out = np.empty((5, h, w), np.float64)
    if lib().orc_poly_expand(_ptr(img), w, h, n_half, sigma, _ptr(out)) != 0:
        raise ValueError("singular Gram matrix")
    return out


def flow_upsample(dc: np.ndarray, w: int, h: int) -> np.ndarray:
    dc = _c(dc, np.float64)
    out = np.empty((2, h, w), np.float64)
    lib().orc_flow_upsample(_ptr(dc), dc.shape[2], dc.shape[1], w, h, _ptr(out))
    return out


def flow_iterate(f1, f2, dprior, iters: int, win_r: int, lam: float) -> np.ndarray:
    f1 = _c(f1, np.float64)
    f2 = _c(f2, np.float64)
    dprior = _c(dprior, np.float64)
    _, h, w = f1.shape
    out = np.empty((2, h, w), np.float64)
    lib().orc_flow_iterate(_ptr(f1), _ptr(f2), w, h, _ptr(dprior), iters, win_r, lam, _ptr(out))
    return out


def flow(cur: np.ndarray, prev: np.ndarray, levels: int, n_half: int = 2, sigma: float = 1.1,
         iters: int = 3, win_r: int = 7, lam: float = 1e-3) -> np.ndarray:
    """(2, h, w) flow (dx, dy) on the grid of `cur`; f1 = cur, f2 = prev."""
    cur = _c(cur, np.float64)
    prev = _c(prev, np.float64)
    h, w = cur.shape
    out = np.empty((2, h, w), np.float64)
    if lib().orc_flow(_ptr(cur), _ptr(prev), w, h, levels, n_half, sigma, iters, win_r, lam, _ptr(out)) != 0:
        raise ValueError("bad flow arguments")
    return out


def flow_reg(cur: np.ndarray, prev: np.ndarray, levels: int, n_half: int, sigma: float, iters: int,
             win_r: int, lam: float, drift) -> np.ndarray:
    """flow() against the previous frame registered to the current one by
    the drift s = (sx, sy) (cur(x) ~ prev(x - s)): the flow that is left
    after the drift."""
    cur = _c(cur, np.float64)
    prev = _c(prev, np.float64)
    h, w = cur.shape
    out = np.empty((2, h, w), np.float64)
    if lib().orc_flow_reg(_ptr(cur), _ptr(prev), w, h, levels, n_half, sigma, iters, win_r, lam,
                          float(drift[0]), float(drift[1]), _ptr(out)) != 0:
        raise ValueError("bad flow arguments")
    return out


def _next_pow2(n: int) -> int:
    return 1 << max(0, (int(n) - 1).bit_length())


def phase_correlate(prev_img: np.ndarray, cur_img: np.ndarray):
    """§Optical flow extraction: each frame is registered to its predecessor
    by phase correlation (global translational drift).  Readings: both
    images Hann-windowed (symmetric, over the image size) and zero-padded to
    the next power of two per axis, each after its mean is removed (else
    the window's own, unshifted, spectrum dominates); X = F_cur conj(F_prev),
    R = X / (|X| + 0.01 max|X|) (the normalised cross-power spectrum, with
    frequencies that carry almost no energy kept from dominating through
    their noise); r = real(IFFT(R)); the first
    maximum of r (row-major) gives the integer shift, wrapped to
    (-N/2, N/2]; each axis refined by the vertex of the parabola through r
    at the peak and its two circular neighbours (when that parabola opens
    downwards; clamped to +-0.5).  Returns (sx, sy): the content moved by
    +s from prev to cur, cur(x) ~ prev(x - s)."""
    a = _c(prev_img, np.float64)
    b = _c(cur_img, np.float64)
    h, w = a.shape
    wy = np.hanning(h) if h > 1 else np.ones(1)
    wx = np.hanning(w) if w > 1 else np.ones(1)
    win = np.outer(wy, wx)
    ny, nx = _next_pow2(h), _next_pow2(w)
    A = np.fft.fft2((a - a.mean()) * win, s=(ny, nx))
    B = np.fft.fft2((b - b.mean()) * win, s=(ny, nx))
    X = B * np.conj(A)
    mag = np.abs(X)
    R = X / (mag + 0.01 * mag.max()) if mag.max() > 0 else X
    r = np.real(np.fft.ifft2(R))
    k = int(np.argmax(r))
    ky, kx = divmod(k, nx)

    def sub(c0, cm, cp):
        den = cm - 2.0 * c0 + cp
        if den >= 0.0:
            return 0.0
        return float(np.clip((cm - cp) / (2.0 * den), -0.5, 0.5))

    dx = sub(r[ky, kx], r[ky, (kx - 1) % nx], r[ky, (kx + 1) % nx])
    dy = sub(r[ky, kx], r[(ky - 1) % ny, kx], r[(ky + 1) % ny, kx])
    sx = (kx - nx if kx > nx // 2 else kx) + dx
    sy = (ky - ny if ky > ny // 2 else ky) + dy
    return sx, sy


def register(prev_img: np.ndarray, cur_img: np.ndarray, level: int):
    """Global drift (level-0 pixels) from phase correlation of the level-`level`
    pyramid images of the two flow inputs."""
    a, b = _c(prev_img, np.float64), _c(cur_img, np.float64)
    for _ in range(level):
        a, b = pyr_down(a), pyr_down(b)
    sx, sy = phase_correlate(a, b)
    return sx * (1 << level), sy * (1 << level)


def saliency(d: np.ndarray, alpha: float) -> np.ndarray:
    d = _c(d, np.float64)
    _, h, w = d.shape
    out = np.empty((h, w), np.float64)
    lib().orc_saliency(_ptr(d), w, h, alpha, _ptr(out))
    return out


def normalise(S: np.ndarray) -> np.ndarray:
    S = _c(S, np.float64)
    out = np.empty_like(S)
    lib().orc_normalise(_ptr(S), S.size, _ptr(out))
    return out


def quantile_k(q: float, n: int) -> int:
    return int(lib().orc_quantile_k(q, n))


def threshold(Sh: np.ndarray, q: float):
    """(mask0 uint8, t) on double values."""
    Sh = _c(Sh, np.float64)
    m = np.empty(Sh.shape, np.uint8)
    t = lib().orc_threshold(_ptr(Sh), Sh.size, q, _ptr(m))
    return m, float(t)


def threshold_f32(Sh: np.ndarray, q: float):
    """(mask0 uint8, t) decided on single-precision values."""
    Sh = _c(Sh, np.float32)
    m = np.empty(Sh.shape, np.uint8)
    t = lib().orc_threshold_f32(_ptr(Sh), Sh.size, q, _ptr(m))
    return m, np.float32(t)


def erode(m: np.ndarray, r: int) -> np.ndarray:
    m = _c(m, np.uint8)
    out = np.empty_like(m)
    lib().orc_erode(_ptr(m), m.shape[1], m.shape[0], r, _ptr(out))
    return out


def dilate(m: np.ndarray, r: int) -> np.ndarray:
    m = _c(m, np.uint8)
    out = np.empty_like(m)
    lib().orc_dilate(_ptr(m), m.shape[1], m.shape[0], r, _ptr(out))
    return out


def morph(m: np.ndarray, r_open: int, r_close: int) -> np.ndarray:
    m = _c(m, np.uint8)
    out = np.empty_like(m)
    lib().orc_morph(_ptr(m), m.shape[1], m.shape[0], r_open, r_close, _ptr(out))
    return out


def dwt1d(x: np.ndarray, wavelet: int, inverse: bool = False) -> np.ndarray:
    if wavelet == 53:
        a = _c(x, np.int32).copy()
        tmp = np.empty_like(a)
        (lib().orc_idwt53_1d if inverse else lib().orc_dwt53_1d)(_ptr(a), a.size, _ptr(tmp))
    else:
        a = _c(x, np.float64).copy()
        tmp = np.empty_like(a)
        (lib().orc_idwt97_1d if inverse else lib().orc_dwt97_1d)(_ptr(a), a.size, _ptr(tmp))
    return a


def dwt2d(x: np.ndarray, wavelet: int, levels: int, inverse: bool = False) -> np.ndarray:
    h, w = x.shape
    if wavelet == 53:
        a = _c(x, np.int32).copy()
        (lib().orc_idwt53_2d if inverse else lib().orc_dwt53_2d)(_ptr(a), w, h, levels)
    else:
        a = _c(x, np.float64).copy()
        (lib().orc_idwt97_2d if inverse else lib().orc_dwt97_2d)(_ptr(a), w, h, levels)
    return a


def dc_shift(raw: np.ndarray, bit_depth: int) -> np.ndarray:
    raw = np.ascontiguousarray(raw)
    out = np.empty(raw.shape, np.int32)
    lib().orc_dc_shift(_ptr(raw), raw.dtype.itemsize, bit_depth, raw.size, _ptr(out))
    return out


def subband_index(x: int, y: int, w: int, h: int, levels: int) -> int:
    return int(lib().orc_subband_index(x, y, w, h, levels))


def delta_table(levels: int, bit_depth: int, delta_base: float = 1.0):
    """(G, delta float32, eps, mu), each of length 3*levels+1."""
    nb = 3 * levels + 1
    G = np.empty(nb, np.float64)
    d = np.empty(nb, np.float32)
    e = np.empty(nb, np.int32)
    m = np.empty(nb, np.int32)
    if lib().orc_delta_table(levels, bit_depth, delta_base, _ptr(G), _ptr(d), _ptr(e), _ptr(m)) != 0:
        raise ValueError("quantisation step exponent out of range")
    return G, d, e, m


def quantise_f32(y: np.ndarray, levels: int, delta: np.ndarray) -> np.ndarray:
    y = _c(y, np.float32)
    d = _c(delta, np.float32)
    h, w = y.shape
    q = np.empty((h, w), np.int32)
    lib().orc_quantise_f32(_ptr(y), w, h, levels, _ptr(d), _ptr(q))
    return q


def quantise_f64(y: np.ndarray, levels: int, delta: np.ndarray) -> np.ndarray:
    y = _c(y, np.float64)
    d = _c(delta, np.float32)
    h, w = y.shape
    q = np.empty((h, w), np.int32)
    lib().orc_quantise_f64(_ptr(y), w, h, levels, _ptr(d), _ptr(q))
    return q


def wavelet_mask(pix: np.ndarray, levels: int, wavelet: int) -> np.ndarray:
    pix = _c(pix, np.uint8)
    h, w = pix.shape
    out = np.empty_like(pix)
    lib().orc_wavelet_mask(_ptr(pix), w, h, levels, wavelet, _ptr(out))
    return out


def roi_shift(q: np.ndarray, cmask: np.ndarray, s: int) -> np.ndarray:
    a = _c(q, np.int32).copy()
    m = _c(cmask, np.uint8)
    if lib().orc_roi_shift(_ptr(a), _ptr(m), a.size, s) != 0:
        raise OverflowError("RoI up-shift overflows int32")
    return a


# ------------------------------------------- embedded block coding (f4) --
#
# The JPEG2000 coder downstream of the front end (orc_ebcot.c): tier-1
# coding of 64 x 64 code-blocks, rate control to a byte budget, a frame
# container, and the decoder used for PSNR.

CB = 64
ORI_LL, ORI_HL, ORI_LH, ORI_HH = 0, 1, 2, 3
_MAGIC = b"FRJ2"
_HDR = 32
_ENT = 16


def mq_roundtrip(d: np.ndarray, cx: np.ndarray):
    """MQ-encode decisions d in contexts cx (one terminated codeword) and
    decode them back: (codeword bytes, decoded decisions)."""
    d = _c(d, np.uint8)
    cx = _c(cx, np.uint8)
    code = np.zeros(2 * d.size + 16, np.uint8)
    out = np.empty_like(d)
    n = lib().orc_mq_roundtrip(_ptr(d), _ptr(cx), d.size, _ptr(code), _ptr(out))
    return code[:n].copy(), out


def mq_table():
    """The MQ coder's probability states (JPEG2000 Part 1, Annex C, Table
    C.2) as (qe, next after MPS, next after LPS, switch) int arrays."""
    a = [np.zeros(47, np.int32) for _ in range(4)]
    lib().orc_mq_table(*[_ptr(x) for x in a])
    return tuple(a)


def context_tables():
    """The coding-pass context rules (Annex D, Tables D.1 and D.3): the
    zero-coding label zc[ori, d, v, h] (ori 0 LL, 1 HL, 2 LH, 3 HH; h, v,
    d the significant horizontal, vertical, diagonal neighbours), and the
    sign-coding label and flip bit sc[vc + 1, hc + 1], flip[vc + 1, hc + 1]
    (hc, vc the clipped sign contributions)."""
    zc = np.zeros(4 * 45, np.int32)
    sc = np.zeros(9, np.int32)
    fl = np.zeros(9, np.int32)
    lib().orc_context_tables(_ptr(zc), _ptr(sc), _ptr(fl))
    return zc.reshape(4, 5, 3, 3), sc.reshape(3, 3), fl.reshape(3, 3)


def t1_encode(q: np.ndarray, ori: int, reset: bool = False):
    """Tier-1 coding of one code-block: (planes, pass lengths, pass
    distortion decreases, bytes of all passes back to back).  Every pass is
    terminated; with `reset` the contexts also restart at every pass."""
    q = _c(q, np.int32)
    h, w = q.shape
    cap = 8 * 64 * 64 * 96
    out = np.empty(cap, np.uint8)
    planes = ctypes.c_int(0)
    plen = np.zeros(96, np.int32)
    dist = np.zeros(96, np.float64)
    n = lib().orc_t1_encode(_ptr(q), w, w, h, ori, _ptr(out), cap, ctypes.byref(planes), _ptr(plen), _ptr(dist),
                            int(reset))
    if n == -2:
        raise OverflowError("code-block magnitude of 2^24 or more")
    if n < 0:
        raise OverflowError("code-block output too large")
    return planes.value, plen[:n].copy(), dist[:n].copy(), out[: int(plen[:n].sum())].copy()


def t1_decode(code: np.ndarray, plen: np.ndarray, nkept: int, planes: int, w: int, h: int, ori: int,
              midpoint: bool = True, reset: bool = False) -> np.ndarray:
    code = _c(code, np.uint8)
    plen = _c(plen, np.int32)
    q = np.zeros((h, w), np.int32)
    lib().orc_t1_decode(_ptr(code), _ptr(plen), nkept, planes, w, h, ori, int(midpoint), _ptr(q), w, int(reset))
    return q


def codeblocks(w: int, h: int, levels: int):
    """Code-blocks of a Mallat coefficient plane in codestream order: the
    low-low band, then HL, LH, HH of each level from the coarsest; 64 x 64
    blocks from each band's origin, in raster order.  Yields (band index,
    orientation, x0, y0, width, height); band indices follow the
    quantisation-step table (HL, LH, HH of level l at 3(l-1), +1, +2; low-low
    at 3 levels)."""
    out = []
    bands = [(3 * levels, ORI_LL, 0, 0, w >> levels, h >> levels)]
    for l in range(levels, 0, -1):
        bw, bh = w >> l, h >> l
        bands += [(3 * (l - 1), ORI_HL, bw, 0, bw, bh), (3 * (l - 1) + 1, ORI_LH, 0, bh, bw, bh),
                  (3 * (l - 1) + 2, ORI_HH, bw, bh, bw, bh)]
    for b, ori, bx, by, bw, bh in bands:
        for y in range(0, bh, CB):
            for x in range(0, bw, CB):
                out.append((b, ori, bx + x, by + y, min(CB, bw - x), min(CB, bh - y)))
    return out


def hull(plen: np.ndarray, dist: np.ndarray):
    """Lower convex hull of a code-block's truncation points: (pass counts,
    slopes), slopes strictly decreasing (slope[0] unused)."""
    n = len(plen)
    R = np.zeros(n + 1, np.int64)
    D = np.zeros(n + 1, np.float64)
    for k in range(n):  # cumulative, in pass order
        R[k + 1] = R[k] + int(plen[k])
        D[k + 1] = D[k] + float(dist[k])
    hk = np.zeros(n + 1, np.int32)
    hs = np.zeros(n + 1, np.float64)
    m = lib().orc_hull(n, _ptr(R), _ptr(D), _ptr(hk), _ptr(hs))
    return hk[:m].copy(), hs[:m].copy(), R


def pcrd(blocks, budget: int, iters: int = 64):
    """Rate control: passes kept per code-block so that the kept pass bytes
    fit `budget` (0: keep every pass).  The slope threshold lambda is found
    by `iters` bisection steps on [0, 2 max slope + 1]; a block keeps the
    passes up to its last hull point whose slope is >= lambda."""
    hs = [hull(b["plen"], b["dist"]) for b in blocks]
    full = sum(int(b["plen"].sum()) for b in blocks)
    if budget <= 0 or full <= budget:
        return [len(b["plen"]) for b in blocks]

    def keep(lam):
        ks, tot = [], 0
        for hk, sl, R in hs:
            j = 0
            while j + 1 < len(hk) and sl[j + 1] >= lam:
                j += 1
            ks.append(int(hk[j]))
            tot += int(R[hk[j]])
        return ks, tot

    lo = 0.0
    hi = 2.0 * max([float(sl[1]) for hk, sl, R in hs if len(hk) > 1] + [0.0]) + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if keep(mid)[1] <= budget:
            hi = mid
        else:
            lo = mid
    return keep(hi)[0]


def encode_frame(coeffs: np.ndarray, levels: int, wavelet: int, shift: int, bit_depth: int, budget: int = 0,
                 fmt: str = "container", delta_base: float = 1.0, reset: bool = False):
    """Tier-1 coding of every code-block of a Mallat plane, rate control to
    `budget` bytes of pass data (0: lossless in the passes), and the frame
    container: a 32-byte header, a 16-byte entry per code-block, then per
    code-block the kept passes' 16-bit lengths and bytes; with fmt="j2c" a
    JPEG2000 Part 1 codestream of the same kept passes instead
    (codestream_j2c).  With `reset` every block is coded with its contexts
    reset at every pass (the header's flags word, bit 0; COD's code-block
    style).  Returns (bytes, block records)."""
    import struct
    coeffs = _c(coeffs, np.int32)
    h, w = coeffs.shape
    blocks = []
    for b, ori, x0, y0, cw, ch in codeblocks(w, h, levels):
        planes, plen, dist, code = t1_encode(coeffs[y0:y0 + ch, x0:x0 + cw], ori, reset)
        blocks.append(dict(band=b, ori=ori, x0=x0, y0=y0, w=cw, h=ch, planes=planes, plen=plen, dist=dist,
                           code=code))
    nkeep = pcrd(blocks, budget)
    data, table = [], []
    off = 0
    for blk, k in zip(blocks, nkeep):
        blk["nkeep"] = k
        body = np.asarray(blk["plen"][:k], "<u2").tobytes() + blk["code"][: int(blk["plen"][:k].sum())].tobytes()
        table.append(struct.pack("<IHHBBBBBBH", off, blk["x0"], blk["y0"], blk["w"] - 1, blk["h"] - 1, blk["band"],
                                 blk["planes"], len(blk["plen"]), k, 0))
        data.append(body)
        off += len(body)
    if fmt == "j2c":
        return codestream_j2c(blocks, w, h, levels, wavelet, bit_depth, delta_base, reset), blocks
    hdr = struct.pack("<4sIIIBBBBIII", _MAGIC, 1, w, h, wavelet, levels, shift, bit_depth, len(blocks), off,
                      1 if reset else 0)
    return hdr + b"".join(table) + b"".join(data), blocks


# ------------------------------------------- JPEG2000 Part 1 codestream --
# ISO/IEC 15444-1: Annex A (markers), Annex B (tier-2: packets, tag trees,
# packet headers), Annex E (the quantisation exponents and M_b).  One tile,
# one component, one quality layer, LRCP progression, no precinct
# partition (one precinct per resolution: one packet per resolution),
# 64 x 64 code-blocks, code-block style "termination on each coding pass"
# (byte 0x04; with reset also "reset context probabilities on coding pass
# boundaries", 0x02: the style byte's bits, Annex A.6.1),
# no RGN marker: Part 1 signals only the maximum-shift RoI method, so the
# scaling-based RoI travels in the coefficients themselves (a Part 1
# decoder returns the up-shifted coefficients; undoing the shift needs the
# RoI mask, as the scaling method does).


class _BitWriter:
    """Packet-header bits, most significant first; a byte that follows a
    0xFF byte carries only 7 bits (its MSB is 0), and the header never ends
    on 0xFF (Annex B.10.1)."""

    def __init__(self):
        self.out = bytearray()
        self.cur = 0
        self.n = 0
        self.cap = 8

    def put(self, b: int):
        self.cur = (self.cur << 1) | (b & 1)
        self.n += 1
        if self.n == self.cap:
            self.out.append(self.cur)
            self.cap = 7 if self.cur == 0xFF else 8
            self.cur = 0
            self.n = 0

    def put_bits(self, v: int, nbits: int):
        for i in range(nbits - 1, -1, -1):
            self.put((v >> i) & 1)

    def flush(self) -> bytes:
        if self.n:
            self.out.append(self.cur << (self.cap - self.n))
            self.n = 0
        if self.out and self.out[-1] == 0xFF:
            self.out.append(0)
        return bytes(self.out)


class _TagTree:
    """Tag tree over a nx x ny grid of leaves (Annex B.10.2): every node
    holds the minimum of the leaves below it; a leaf's value is sent as the
    path from the root down, each node's value in excess of its parent's as
    0 bits closed by a 1 bit, and only up to a threshold; what a node has
    already sent is remembered (low bound, known)."""

    def __init__(self, nx: int, ny: int, values):
        self.levels = []
        w, h = nx, ny
        while True:
            self.levels.append((w, h))
            if w == 1 and h == 1:
                break
            w, h = (w + 1) // 2, (h + 1) // 2
        big = 1 << 30
        self.val = [[big] * (lw * lh) for lw, lh in self.levels]
        self.low = [[0] * (lw * lh) for lw, lh in self.levels]
        self.known = [[False] * (lw * lh) for lw, lh in self.levels]
        for y in range(ny):
            for x in range(nx):
                v = values[y * nx + x]
                xx, yy = x, y
                for l, (lw, lh) in enumerate(self.levels):
                    i = yy * lw + xx
                    self.val[l][i] = min(self.val[l][i], v)
                    xx, yy = xx // 2, yy // 2

    def encode(self, bw: _BitWriter, x: int, y: int, threshold: int):
        path = []
        xx, yy = x, y
        for l, (lw, lh) in enumerate(self.levels):
            path.append((l, yy * lw + xx))
            xx, yy = xx // 2, yy // 2
        low = 0
        for l, i in reversed(path):  # root first
            low = max(low, self.low[l][i])
            while low < threshold:
                if low >= self.val[l][i]:
                    if not self.known[l][i]:
                        bw.put(1)
                        self.known[l][i] = True
                    break
                bw.put(0)
                low += 1
            self.low[l][i] = low


def _passes_codeword(bw: _BitWriter, n: int):
    """Number of coding passes included (Annex B.10.6, Table B.4)."""
    if n == 1:
        bw.put(0)
    elif n == 2:
        bw.put_bits(0b10, 2)
    elif n <= 5:
        bw.put_bits(0b1100 | (n - 3), 4)
    elif n <= 36:
        bw.put_bits(0b1111, 4)
        bw.put_bits(n - 6, 5)
    elif n <= 164:
        bw.put_bits(0b111111111, 9)
        bw.put_bits(n - 37, 7)
    else:
        raise ValueError("more than 164 coding passes")


def band_exponents(levels: int, wavelet: int, bit_depth: int, delta_base: float = 1.0):
    """(eps, mu) per band of the quantisation-step table's index: 9/7 the
    steps' JPEG2000 form; 5/3 (no quantisation) eps = bit depth + log2 of
    the band's nominal gain (0 LL, 1 HL and LH, 2 HH), mu = 0."""
    nb = 3 * levels + 1
    if wavelet == 97:
        _, _, e, m = delta_table(levels, bit_depth, delta_base)
        return [int(v) for v in e], [int(v) for v in m]
    eps = [bit_depth + (0 if b == 3 * levels else (1 if b % 3 < 2 else 2)) for b in range(nb)]
    return eps, [0] * nb


def codestream_j2c(blocks, w: int, h: int, levels: int, wavelet: int, bit_depth: int,
                   delta_base: float = 1.0, reset: bool = False) -> bytes:
    """A JPEG2000 Part 1 codestream of one frame from its code-blocks' kept
    passes (encode_frame's block records with 'nkeep').  The guard bits G are
    the fewest (at least 1) for which every block's bit-planes fit the
    band's M_b = G + eps_b - 1 (Annex E.1); more than 7 cannot be signalled."""
    import struct
    eps, mu = band_exponents(levels, wavelet, bit_depth, delta_base)
    need = [blk["planes"] - eps[blk["band"]] + 1 for blk in blocks if blk["planes"] > 0]
    G = max([1] + need)
    if G > 7:
        raise ValueError("coefficient bit-planes beyond what 7 guard bits signal")
    # band order of QCD and of the packets: LL_D, then HL, LH, HH of D .. 1
    order = [3 * levels] + [3 * (l - 1) + o for l in range(levels, 0, -1) for o in range(3)]
    cs = bytearray(b"\xff\x4f")  # SOC
    cs += struct.pack(">HHHIIIIIIIIHBBB", 0xFF51, 41, 0, w, h, 0, 0, w, h, 0, 0, 1, bit_depth - 1, 1, 1)  # SIZ
    style = 0x04 | (0x02 if reset else 0)
    cs += struct.pack(">HHBBHBBBBBB", 0xFF52, 12, 0, 0, 1, 0, levels, 4, 4, style, 1 if wavelet == 53 else 0)  # COD
    if wavelet == 53:
        cs += struct.pack(">HHB", 0xFF5C, 3 + len(order), G << 5) + bytes(eps[b] << 3 for b in order)
    else:
        cs += struct.pack(">HHB", 0xFF5C, 3 + 2 * len(order), (G << 5) | 2)
        cs += b"".join(struct.pack(">H", (eps[b] << 11) | mu[b]) for b in order)
    # packets, one per resolution: LL_D, then (HL, LH, HH) of level D .. 1
    byband = {}
    for blk in blocks:
        byband.setdefault(blk["band"], []).append(blk)
    res = [[3 * levels]] + [[3 * (l - 1), 3 * (l - 1) + 1, 3 * (l - 1) + 2] for l in range(levels, 0, -1)]
    data = bytearray()
    for bands in res:
        bw = _BitWriter()
        body = bytearray()
        if not any(blk["nkeep"] > 0 for b in bands for blk in byband.get(b, [])):
            bw.put(0)  # empty packet
        else:
            bw.put(1)
            for b in bands:
                bl = byband.get(b, [])
                if not bl:
                    continue
                x0s = sorted({blk["x0"] for blk in bl})
                y0s = sorted({blk["y0"] for blk in bl})
                nx, ny = len(x0s), len(y0s)
                Mb = G + eps[b] - 1
                incl = _TagTree(nx, ny, [0 if blk["nkeep"] > 0 else 1 for blk in bl])
                zbp = _TagTree(nx, ny, [Mb - blk["planes"] for blk in bl])
                for j, blk in enumerate(bl):
                    cx, cy = j % nx, j // nx
                    incl.encode(bw, cx, cy, 1)
                    n = blk["nkeep"]
                    if n == 0:
                        continue
                    zbp.encode(bw, cx, cy, 1 << 30)
                    _passes_codeword(bw, n)
                    lens = [int(v) for v in blk["plen"][:n]]
                    need_bits = max(max(1, L.bit_length()) for L in lens)
                    k = max(0, need_bits - 3)  # Lblock starts at 3
                    bw.put_bits((1 << (k + 1)) - 2, k + 1)  # k ones, then a zero
                    for L in lens:  # one codeword segment per pass
                        bw.put_bits(L, 3 + k)
                    body += blk["code"][: sum(lens)].tobytes()
        data += bw.flush() + body
    psot = 12 + 2 + len(data)
    cs += struct.pack(">HHHIBB", 0xFF90, 10, 0, psot, 0, 1) + b"\xff\x93" + data + b"\xff\xd9"
    return bytes(cs)


def decode_frame(stream: bytes, midpoint: bool = True) -> np.ndarray:
    """The Mallat coefficient plane recovered from a frame container (kept
    passes only; unknown low bits at the interval midpoint when
    `midpoint`; the blocks decoded with their contexts reset at every pass
    when the header's flags word has bit 0 set)."""
    import struct
    magic, ver, w, h, wav, levels, shift, bd, nb, nbytes, flags = struct.unpack_from("<4sIIIBBBBIII", stream, 0)
    if magic != _MAGIC or ver != 1 or flags & ~1:
        raise ValueError("not a frame container")
    reset = bool(flags & 1)
    out = np.zeros((h, w), np.int32)
    base = _HDR + nb * _ENT
    oris = {b: o for b, o, *_ in codeblocks(w, h, levels)}
    for i in range(nb):
        off, x0, y0, cw1, ch1, band, planes, npass, k, _ = struct.unpack_from("<IHHBBBBBBH", stream, _HDR + i * _ENT)
        p = base + off
        plen = np.frombuffer(stream, "<u2", k, p).astype(np.int32)
        code = np.frombuffer(stream, np.uint8, int(plen.sum()), p + 2 * k)
        out[y0:y0 + ch1 + 1, x0:x0 + cw1 + 1] = t1_decode(code, plen, k, planes, cw1 + 1, ch1 + 1, oris[band],
                                                          midpoint, reset)
    return out


def unshift_dequantise(q: np.ndarray, cmask: np.ndarray, shift: int, levels: int, wavelet: int, bit_depth: int,
                       delta_base: float = 1.0) -> np.ndarray:
    """Inverse of the RoI up-shift (RoI coefficients, known from the
    wavelet-domain mask, shifted back down) and of the quantiser (9/7: y =
    q delta_b; 5/3: y = q), as the transform's input type."""
    q = _c(q, np.int64)
    m = _c(cmask, np.uint8) != 0
    a = np.abs(q)
    a = np.where(m, a >> shift, a)
    q = np.sign(q) * a
    if wavelet == 53:
        return q.astype(np.int32)
    _, delta, _, _ = delta_table(levels, bit_depth, delta_base)
    h, w = q.shape
    d = np.empty((h, w), np.float64)
    for y in range(h):
        for x in range(w):
            d[y, x] = delta[subband_index(x, y, w, h, levels)]
    return q.astype(np.float64) * d


def reconstruct(y: np.ndarray, levels: int, wavelet: int, bit_depth: int) -> np.ndarray:
    """Inverse DWT, inverse DC shift and clipping to the sample range."""
    x = dwt2d(y, wavelet, levels, inverse=True)
    x = np.rint(np.asarray(x, np.float64)) + 2.0 ** (bit_depth - 1)
    return np.clip(x, 0, 2 ** bit_depth - 1).astype(np.int64)


def psnr(a: np.ndarray, b: np.ndarray, bit_depth: int) -> float:
    e = np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)
    peak = 2.0 ** bit_depth - 1
    return float("inf") if e == 0 else 10.0 * np.log10(peak * peak / e)


# ------------------------------------------------------------- pipeline --

@dataclass
class Params:
    """Method parameters (the paper's Table 1 plus the estimator constants it
    leaves unstated)."""
    pyr_levels: int = 3
    iters: int = 3
    win_r: int = 7
    poly_n_half: int = 2
    poly_sigma: float = 1.1
    lam: float = 1e-3
    sal_weight: float = 0.7
    roi_q: float = 0.2
    r_open: int = 1
    r_close: int = 2
    wavelet: int = 53
    dwt_levels: int = 3
    scale_shift: int = 5
    delta_base: float = 1.0
    min_area: int = 0          # components below this many pixels removed (0: off; reading)
    adjacent: int = 0          # Table 1 "Adjacent factor" k (sequence() merges masks of j-k..j+k)
    register: int = 0          # registration of each frame to its predecessor (phase correlation)
    reg_level: int = 2         # pyramid level the phase correlation runs on (reading)
    denoise: int = 0           # Table 1 "Denoise" (off: a valid setting)
    den_radius: int = 2        # bilateral square radius (reading)
    den_sigma_s: float = 2.0   # bilateral spatial sigma, px (reading)
    den_sigma_r: float = 20.0  # bilateral range sigma, 8-bit units (reading)


def frame(prev_raw, cur_raw, bit_depth: int, p: Params, y_f32=None):
    """Whole hot path for one frame pair (prev_raw = frame t-1 or None).

    Returns a dict: flow (2,h,w) f64, S, Sh (f64), t, mask0, mask (uint8),
    y (DWT coefficients: int32 for 5/3, f64 for 9/7), cmask (wavelet-domain
    mask), q (quantised), coeffs (int32 after the RoI up-shift).  With no
    predecessor the mask is empty (the first frame of a stream has no flow).

    For 9/7, `y_f32` may carry single-precision DWT coefficients computed
    elsewhere: quantisation then decides on those values (same precision as
    a single-precision transform) instead of on the oracle's f64 values.
    """
    h, w = cur_raw.shape
    out = {}
    if prev_raw is not None:
        I1 = units(cur_raw, bit_depth)
        I2 = units(prev_raw, bit_depth)
        if p.denoise:
            I1 = denoise(I1, p.den_radius, p.den_sigma_s, p.den_sigma_r)
            I2 = denoise(I2, p.den_radius, p.den_sigma_s, p.den_sigma_r)
            out["denoised"] = I1
        if p.register:
            # flow of the pair after the predecessor is registered to the
            # current frame by the drift s (cur(x) ~ prev(x - s))
            s = register(I2, I1, p.reg_level)
            d = flow_reg(I1, I2, p.pyr_levels, p.poly_n_half, p.poly_sigma, p.iters, p.win_r, p.lam, s)
            out["drift"] = s
        else:
            d = flow(I1, I2, p.pyr_levels, p.poly_n_half, p.poly_sigma, p.iters, p.win_r, p.lam)
        S = saliency(d, p.sal_weight)
        Sh = normalise(S)
        mask0, t = threshold(Sh, p.roi_q)
        mask = morph(mask0, p.r_open, p.r_close)
        if p.min_area > 1:
            out["mask_morph"] = mask
            mask = remove_small(mask, p.min_area)
        out.update(flow=d, S=S, Sh=Sh, t=t, mask0=mask0)
    else:
        mask = np.zeros((h, w), np.uint8)
    out["mask"] = mask
    x = dc_shift(cur_raw, bit_depth)
    cm = wavelet_mask(mask, p.dwt_levels, p.wavelet)
    if p.wavelet == 53:
        y = dwt2d(x, 53, p.dwt_levels)
        q = y
    else:
        y = dwt2d(x.astype(np.float64), 97, p.dwt_levels)
        _, delta, _, _ = delta_table(p.dwt_levels, bit_depth, p.delta_base)
        q = quantise_f32(y_f32, p.dwt_levels, delta) if y_f32 is not None else quantise_f64(y, p.dwt_levels, delta)
        out["delta"] = delta
    out.update(y=y, cmask=cm, q=q, coeffs=roi_shift(q, cm, p.scale_shift))
    return out


def sequence(raw_frames, bit_depth: int, p: Params):
    """Whole hot path for a finished sequence of frames of one stream: each
    frame's own mask from frame() (flow against its predecessor), then the
    adjacent-factor merge, then the JPEG2000 front end of every frame with
    its merged mask.  Returns a list of dicts (own_mask, mask, coeffs, ...)."""
    outs = [frame(raw_frames[t - 1] if t > 0 else None, raw_frames[t], bit_depth, p) for t in range(len(raw_frames))]
    merged = adjacent_merge([o["mask"] for o in outs], p.adjacent)
    for o, m, raw in zip(outs, merged, raw_frames):
        o["own_mask"] = o["mask"]
        o["mask"] = m
        x = dc_shift(raw, bit_depth)
        cm = wavelet_mask(m, p.dwt_levels, p.wavelet)
        if p.wavelet == 53:
            q = dwt2d(x, 53, p.dwt_levels)
        else:
            y = dwt2d(x.astype(np.float64), 97, p.dwt_levels)
            _, delta, _, _ = delta_table(p.dwt_levels, bit_depth, p.delta_base)
            q = quantise_f64(y, p.dwt_levels, delta)
        o.update(cmask=cm, q=q, coeffs=roi_shift(q, cm, p.scale_shift))
    return outs
