"""Adjacent-factor mask merge (§Region of Interest extraction; Table 1
"Adjacent factor") on the GPU, through the C ABI, against the oracle.

Stagewise: each frame's own mask is the oracle's opening/closing (and
component filter) of the GPU's own cut (mask0); the delivered mask of
frame j must be the oracle's union of those over frames j-k .. j+k (cut at
the ends of the submitted sequence) bit for bit, and the 5/3 coefficients
those of the delivered mask.  Also: a frame's results wait for frame j+k
(or a flush), end_stream finishes the waiting frames, and batching several
streams gives the same results as one stream alone."""
import time

import numpy as np
import pytest

from synth import sequence_u16
from tests._gpu import F, fetch, oracle_params, u16

pytestmark = pytest.mark.gpu


def _frames(seed, n, h=192, w=256):
    return [f for f in u16(sequence_u16(seed, n, h, w, 14))]


def _submit(ctx, sid, fr, t, bd):
    """Submit, waiting while the stream's ring slot is still in use (its
    frame's front end runs k batches later; a flush would finish the
    stream's last frames early, so the tests only wait)."""
    for _ in range(20000):
        try:
            return F.flowroi_submit_frame(ctx, sid, fr, t, bd)
        except F.FlowRoIError as e:
            if e.code != F.EBUSY:
                raise
            time.sleep(0.001)
    raise TimeoutError("ring slot never freed")


def _run(streams, bd, **cfg):
    """streams: {sid: frames}; frames submitted round-robin, one step per
    round, then a flush.  Returns {sid: [outputs per frame]}."""
    out = {}
    with F.Context(flags=F.MANUAL | F.KEEP_INTERMEDIATES, **cfg) as ctx:
        n = max(len(v) for v in streams.values())
        for t in range(n):
            for sid, frs in streams.items():
                if t < len(frs):
                    _submit(ctx.h, sid, frs[t], t, bd)
            F.flowroi_step(ctx.h)
        F.flowroi_flush(ctx.h, 120000)
        for sid, frs in streams.items():
            h, w = frs[0].shape
            out[sid] = [fetch(ctx.h, sid, t, h, w) for t in range(len(frs))]
    return out


def _check(orc, frames, gs, bd, **cfg):
    p = oracle_params(orc, **cfg)
    own = [orc.morph(g["mask0"], p.r_open, p.r_close) for g in gs]
    if cfg.get("min_area", 0) > 1:
        own = [orc.remove_small(m, cfg["min_area"]) for m in own]
    merged = orc.adjacent_merge(own, cfg["adjacent"])
    for t, (g, m, raw) in enumerate(zip(gs, merged, frames)):
        assert np.array_equal(g["mask"], m), f"frame {t}"
        cm = orc.wavelet_mask(m, p.dwt_levels, p.wavelet)
        y = orc.dwt2d(orc.dc_shift(raw, bd), 53, p.dwt_levels)
        assert np.array_equal(g["coeffs"], orc.roi_shift(y, cm, p.scale_shift)), f"frame {t}"
    return merged


@pytest.mark.parametrize("k,n", [(1, 6), (2, 7), (4, 5)])
def test_adjacent_merge_parity(orc, k, n):
    frames = _frames(7000 + k, n)
    cfg = dict(adjacent=k, result_ring=max(2 * k + 2, n), roi_q=0.1)  # every frame's results kept
    gs = _run({5: frames}, 12, **cfg)[5]
    merged = _check(orc, frames, gs, 12, **cfg)
    assert any(m.sum() > g["mask0"].sum() for m, g in zip(merged, gs))  # the merge adds pixels


def test_adjacent_with_component_filter_and_batched_streams(orc):
    a, b = _frames(7100, 5), _frames(7101, 4, 128, 192)
    cfg = dict(adjacent=1, result_ring=5, min_area=30)
    both = _run({1: a, 2: b}, 12, **cfg)
    _check(orc, a, both[1], 12, **cfg)
    _check(orc, b, both[2], 12, **cfg)
    alone = _run({1: a}, 12, **cfg)[1]
    for x, y in zip(alone, both[1]):
        assert np.array_equal(x["mask"], y["mask"]) and np.array_equal(x["coeffs"], y["coeffs"])


def test_results_wait_for_the_next_k_frames_or_a_flush():
    frames = _frames(7200, 4)
    with F.Context(flags=F.MANUAL, adjacent=1, result_ring=4) as ctx:
        for t, fr in enumerate(frames[:3]):
            F.flowroi_submit_frame(ctx.h, 9, fr, t, 12)
            F.flowroi_step(ctx.h)
        m = np.empty(frames[0].shape, np.uint8)
        F.flowroi_get_mask(ctx.h, 9, 1, m, 60000)       # frame 2 is in: frame 1 is complete
        with pytest.raises(F.FlowRoIError) as ei:       # frame 2 waits for frame 3
            F.flowroi_get_mask(ctx.h, 9, 2, m, 200)
        assert ei.value.code == F.ETIMEDOUT
        F.flowroi_flush(ctx.h, 60000)                   # finishes frame 2 with frames 1..2
        F.flowroi_get_mask(ctx.h, 9, 2, m, 1000)
        # a later frame continues the stream after the flush
        F.flowroi_submit_frame(ctx.h, 9, frames[3], 3, 12)
        F.flowroi_flush(ctx.h, 60000)
        F.flowroi_get_mask(ctx.h, 9, 3, m, 1000)
        st = F.flowroi_get_stats(ctx.h)
        assert st["frames_done"] == 4


def test_end_stream_finishes_the_waiting_frames():
    frames = _frames(7300, 3)
    with F.Context(flags=F.MANUAL, adjacent=2, result_ring=6) as ctx:
        for t, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 4, fr, t, 12)
            F.flowroi_step(ctx.h)
        assert F.flowroi_end_stream(ctx.h, 4) == F.OK
        assert F.flowroi_get_stats(ctx.h)["frames_done"] == 3


def test_adjacent_config_is_validated():
    for bad in (dict(adjacent=-1), dict(adjacent=5), dict(adjacent=2, result_ring=5)):
        with pytest.raises(F.FlowRoIError) as ei:
            F.Context(**bad)
        assert ei.value.code == F.EINVAL
