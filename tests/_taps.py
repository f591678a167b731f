"""Reads the published filter taps stored under tests/golden/ and builds
plain FIR filter-bank references from them (independent of the oracle's
lifting code)."""
import os

import numpy as np

_GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_taps(name):
    out = {}
    with open(os.path.join(_GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            half = np.array([float(v) for v in vals])
            out[key] = np.concatenate([half[:0:-1], half])  # full symmetric filter
    return out


def wsym(i, n):
    """Whole-sample symmetric extension index."""
    if n == 1:
        return 0
    p = 2 * (n - 1)
    i %= p
    return i if i <= n - 1 else p - i


def fir_analysis_1d(x, taps):
    """Low band at even centres, high band at odd centres, symmetric
    extension; returns concatenated (low, high)."""
    x = np.asarray(x, np.float64)
    n = x.size
    h0, h1 = taps["lowpass"], taps["highpass"]
    r0, r1 = h0.size // 2, h1.size // 2
    low = [sum(h0[k + r0] * x[wsym(c + k, n)] for k in range(-r0, r0 + 1)) for c in range(0, n, 2)]
    high = [sum(h1[k + r1] * x[wsym(c + k, n)] for k in range(-r1, r1 + 1)) for c in range(1, n, 2)]
    return np.array(low + high)


def fir_analysis_2d(img, taps, levels):
    """Multi-level Mallat transform: per level, columns then rows."""
    a = np.array(img, np.float64)
    h, w = a.shape
    cw, ch = w, h
    for _ in range(levels):
        for x in range(cw):
            a[:ch, x] = fir_analysis_1d(a[:ch, x], taps)
        for y in range(ch):
            a[y, :cw] = fir_analysis_1d(a[y, :cw], taps)
        cw, ch = (cw + 1) // 2, (ch + 1) // 2
    return a
