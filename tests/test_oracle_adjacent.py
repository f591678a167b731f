"""Pins of the oracle's adjacent-factor merge (§Region of Interest
extraction: RoI masks of neighbouring frames incorporated; Table 1
"Adjacent factor"), by closed forms: k = 0 is the identity; a pixel set in
one frame only appears exactly in the frames within distance k (cut at the
sequence ends); the merge contains every frame's own mask; and the
sequence driver codes every frame with its merged mask."""
import numpy as np


def test_k0_is_the_identity(orc):
    rng = np.random.default_rng(0)
    own = [(rng.random((5, 7)) < 0.3).astype(np.uint8) for _ in range(4)]
    assert all(np.array_equal(a, b) for a, b in zip(orc.adjacent_merge(own, 0), own))


def test_single_pixel_windows(orc):
    n, k = 7, 2
    for src in range(n):
        own = [np.zeros((3, 3), np.uint8) for _ in range(n)]
        own[src][1, 2] = 1
        merged = orc.adjacent_merge(own, k)
        for j in range(n):
            assert merged[j][1, 2] == (1 if abs(j - src) <= k else 0)
            assert merged[j].sum() == merged[j][1, 2]


def test_merge_contains_own_masks_and_is_monotone_in_k(orc):
    rng = np.random.default_rng(1)
    own = [(rng.random((8, 8)) < 0.1).astype(np.uint8) for _ in range(6)]
    m1, m2 = orc.adjacent_merge(own, 1), orc.adjacent_merge(own, 2)
    for o, a, b in zip(own, m1, m2):
        assert np.all(a >= o) and np.all(b >= a)


def test_sequence_codes_each_frame_with_its_merged_mask(orc):
    from synth import pair_u8
    a, b = pair_u8(seed=91, h=64, w=64, n_blobs=3)
    c, _ = pair_u8(seed=92, h=64, w=64, n_blobs=3)
    frames = [a.numpy(), b.numpy(), c.numpy()]
    p = orc.Params()
    p.adjacent = 1
    outs = orc.sequence(frames, 8, p)
    merged = orc.adjacent_merge([o["own_mask"] for o in outs], 1)
    for o, m, raw in zip(outs, merged, frames):
        assert np.array_equal(o["mask"], m)
        cm = orc.wavelet_mask(m, p.dwt_levels, p.wavelet)
        y = orc.dwt2d(orc.dc_shift(raw, 8), 53, p.dwt_levels)
        assert np.array_equal(o["coeffs"], orc.roi_shift(y, cm, p.scale_shift))
