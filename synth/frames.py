"""Scene rendering for synthetic microscopy frames (see the package docstring)."""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

_PATCH = 48  # side of the square patch each blob is rendered into


@dataclass
class Scene:
    """Blob parameters of one stream (all tensors of length n_blobs)."""
    cx: torch.Tensor
    cy: torch.Tensor
    a: torch.Tensor       # semi-axis along the blob's own x axis
    b: torch.Tensor       # semi-axis along its y axis
    theta: torch.Tensor   # orientation
    peak: torch.Tensor    # plateau value above background
    static: torch.Tensor  # bool: blob never moves


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _u(g, n, lo, hi, device):
    return lo + (hi - lo) * torch.rand(n, generator=g, device=device, dtype=torch.float64)


def make_scene(g: torch.Generator, h: int, w: int, n_blobs: int, axis_range, peak_range,
               static_frac: float, device) -> Scene:
    cx = _u(g, n_blobs, 0.0, w - 1.0, device)
    cy = _u(g, n_blobs, 0.0, h - 1.0, device)
    a = _u(g, n_blobs, *axis_range, device)
    b = _u(g, n_blobs, *axis_range, device)
    theta = _u(g, n_blobs, 0.0, math.pi, device)
    peak = _u(g, n_blobs, *peak_range, device)
    static = torch.rand(n_blobs, generator=g, device=device) < static_frac
    return Scene(cx, cy, a, b, theta, peak, static)


def render(scene: Scene, h: int, w: int, background: float, edge_sigma: float, device) -> torch.Tensor:
    """Noise-free float64 image: background plus every blob's smooth-edged
    ellipse (plateau `peak`, edge profile of a Gaussian-blurred step)."""
    img = torch.full((h * w,), background, dtype=torch.float64, device=device)
    n = scene.cx.numel()
    if n == 0:
        return img.view(h, w)
    half = _PATCH // 2
    off = torch.arange(-half, half, device=device, dtype=torch.float64)
    x0 = torch.floor(scene.cx)
    y0 = torch.floor(scene.cy)
    gx = x0[:, None, None] + off[None, None, :]          # (n, 1, P)
    gy = y0[:, None, None] + off[None, :, None]          # (n, P, 1)
    dx = gx - scene.cx[:, None, None]
    dy = gy - scene.cy[:, None, None]
    c = torch.cos(scene.theta)[:, None, None]
    s = torch.sin(scene.theta)[:, None, None]
    u = (c * dx + s * dy) / scene.a[:, None, None]
    v = (-s * dx + c * dy) / scene.b[:, None, None]
    rho = torch.sqrt(u * u + v * v)
    radius = torch.sqrt(scene.a * scene.b)[:, None, None]
    dist = (1.0 - rho) * radius                            # ~ signed distance to the rim
    prof = 0.5 * torch.erfc(-dist / (math.sqrt(2.0) * edge_sigma))
    val = scene.peak[:, None, None] * prof                 # (n, P, P)
    ix = gx.expand(n, _PATCH, _PATCH)
    iy = gy.expand(n, _PATCH, _PATCH)
    inside = (ix >= 0) & (ix < w) & (iy >= 0) & (iy < h)
    idx = (iy.clamp(0, h - 1) * w + ix.clamp(0, w - 1)).long()
    img.index_put_((idx[inside],), val[inside], accumulate=True)
    return img.view(h, w)


def _move(scene: Scene, g, step_sigma: float, h: int, w: int, device) -> Scene:
    n = scene.cx.numel()
    sx = step_sigma * torch.randn(n, generator=g, device=device, dtype=torch.float64)
    sy = step_sigma * torch.randn(n, generator=g, device=device, dtype=torch.float64)
    sx = torch.where(scene.static, torch.zeros_like(sx), sx)
    sy = torch.where(scene.static, torch.zeros_like(sy), sy)
    cx = _reflect(scene.cx + sx, w - 1.0)
    cy = _reflect(scene.cy + sy, h - 1.0)
    return Scene(cx, cy, scene.a, scene.b, scene.theta, scene.peak, scene.static)


def _reflect(x: torch.Tensor, hi: float) -> torch.Tensor:
    x = torch.where(x < 0, -x, x)
    return torch.where(x > hi, 2 * hi - x, x)


def pair_u8(seed: int, h: int = 256, w: int = 256, n_blobs: int = 12, max_shift: float = 3.0,
            device="cpu"):
    """(prev, cur) uint8 frames: 8-bit background N(20, 3^2), blobs with
    semi-axes U[6,10], plateau U[120,200], edge blur sigma 1.5, each blob
    translated by U[0, max_shift] px in a random direction."""
    device = torch.device(device)
    g = _gen(seed, device)
    sc = make_scene(g, h, w, n_blobs, (6.0, 10.0), (100.0, 180.0), 0.0, device)
    mag = _u(g, n_blobs, 0.0, max_shift, device)
    ang = _u(g, n_blobs, 0.0, 2 * math.pi, device)
    sc2 = Scene(sc.cx + mag * torch.cos(ang), sc.cy + mag * torch.sin(ang), sc.a, sc.b, sc.theta,
                sc.peak, sc.static)
    out = []
    for s in (sc, sc2):
        img = render(s, h, w, 20.0, 1.5, device)
        img = img + 3.0 * torch.randn(h, w, generator=g, device=device, dtype=torch.float64)
        out.append(img.round().clamp(0, 255).to(torch.uint8))
    return out[0], out[1]


def sequence_u16(seed: int, n_frames: int, h: int, w: int, n_blobs: int, static_frac: float = 0.1,
                 step_sigma: float = 1.5, device="cpu", read_noise: float = 10.0) -> torch.Tensor:
    """(n_frames, h, w) int16 tensor holding 12-bit samples (0..4095; the
    bit pattern equals uint16).  Background 200 ADU, blob peaks U[1500,3500]
    ADU above it, semi-axes U[5,12], random walk N(0, step_sigma^2) per axis
    per frame with `static_frac` of blobs fixed, Poisson shot noise plus
    N(0, read_noise^2) read noise."""
    device = torch.device(device)
    g = _gen(seed, device)
    sc = make_scene(g, h, w, n_blobs, (5.0, 12.0), (1500.0, 3500.0), static_frac, device)
    frames = torch.empty((n_frames, h, w), dtype=torch.int16, device=device)
    for t in range(n_frames):
        if t:
            sc = _move(sc, g, step_sigma, h, w, device)
        clean = render(sc, h, w, 200.0, 1.5, device).to(torch.float32)
        noisy = torch.poisson(clean, generator=g) + read_noise * torch.randn(
            h, w, generator=g, device=device, dtype=torch.float32)
        frames[t] = noisy.round().clamp(0, 4095).to(torch.int16)
    return frames


def translated_pattern(h: int, w: int, shift, n_blobs: int = 6, sigma: float = 4.0, seed: int = 0,
                       amplitude: float = 120.0):
    """Two float64 images of a smooth pattern (sum of isotropic Gaussian
    bumps of width `sigma` on a background of 20): the second is the first
    moved by `shift` = (sx, sy) px, i.e. second(x) = first(x - shift).
    Blob centres keep 3*sigma from the border."""
    g = _gen(seed, "cpu")
    m = 3 * sigma + 4
    cx = _u(g, n_blobs, m, w - 1 - m, "cpu")
    cy = _u(g, n_blobs, m, h - 1 - m, "cpu")
    ys, xs = torch.meshgrid(torch.arange(h, dtype=torch.float64), torch.arange(w, dtype=torch.float64),
                            indexing="ij")

    def draw(ox, oy):
        img = torch.full((h, w), 20.0, dtype=torch.float64)
        for i in range(n_blobs):
            img += amplitude * torch.exp(-((xs - cx[i] - ox) ** 2 + (ys - cy[i] - oy) ** 2) / (2 * sigma ** 2))
        return img

    return draw(0.0, 0.0), draw(float(shift[0]), float(shift[1]))
