"""Seeded synthetic microscopy frames (the only module both the CUDA path's
tests/benchmark and the oracle's tests draw inputs from).

It renders frames shaped like ComplexEye recordings of migrating immune
cells: a dim, noisy background with bright, blurred elliptical blobs that
move between frames.  It holds none of the method's arithmetic (no flow,
saliency, thresholding, morphology or wavelet code): only scene rendering and
noise.  Everything is torch, so the same recipe runs on the CPU (tests) and
on a GPU (large benchmark workloads); a seed fixes the scene exactly on a
given device.

Recipes (all sizes in pixels):
  * ``pair_u8``: 8-bit pair, background N(20, 3^2), blobs with semi-axes
    U[6, 10], random orientation, plateau intensity U[120, 200], edges
    blurred with sigma 1.5; each blob moves U[0, 3] px in a random direction.
  * ``sequence_u16``: 12-bit sequence, background 200 ADU, blob peaks
    U[1500, 3500] ADU, semi-axes U[5, 12], random walk with N(0, 1.5^2)
    steps per axis per frame (10% of blobs static), Poisson shot noise plus
    N(0, 10^2) read noise, clipped to [0, 4095].
"""
from .frames import (  # noqa: F401
    Scene,
    make_scene,
    pair_u8,
    render,
    sequence_u16,
    translated_pattern,
)
