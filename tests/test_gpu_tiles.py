"""Tile shapes change how the kernels cut their work, never what they
compute: the same frames under the built-in shapes and under two other
tables (every tunable of every kernel moved) give bit-identical flow,
saliency, masks and coefficients, and one of them is checked against the
oracle stage by stage.  A mixed-width batch with per-width entries equals
its frames run alone.  The search runs and returns a table that a context
loads."""
import json

import numpy as np
import pytest

from synth import sequence_u16
from tests._gpu import F, fetch, u16
from tests.test_gpu_parity import _stagewise

pytestmark = pytest.mark.gpu


def _table(entries):
    return json.dumps({"format": "flowroi-tiles-1", "entries": entries})


def _all_widths(param, value, storage=32, **extra):
    return [dict(param=param, w=w, storage=storage, value=value, **extra) for w in (256, 512, 1024, 2048, 4096, 8192)]


TABLE_A = _table(
    [e for l in range(1, 6) for e in _all_widths("dwt_seg", 8, level=l)]
    + [dict(param="update_rows", storage=32, value=32)] + _all_widths("saliency_rows", 64)
    + [dict(param="blocks_per_sm", kernel=k, storage=32, value=1) for k in ("expand", "update", "window", "mask", "dwt")]
    + [dict(param="dwt_variant", storage=32, value=6)])
TABLE_B = _table(
    [e for l in range(1, 6) for e in _all_widths("dwt_seg", 64 if l == 1 else 12, level=l)]
    + [dict(param="update_rows", storage=32, value=8)] + _all_widths("saliency_rows", 16)
    + [dict(param="blocks_per_sm", kernel=k, storage=32, value=2) for k in ("expand", "update", "window", "mask", "dwt")]
    + [dict(param="dwt_variant", storage=32, value=5)])


def _run(frames, tiles, bit_depth=12, keep=True, **cfg):
    outs = []
    with F.Context(flags=(F.KEEP_INTERMEDIATES if keep else 0) | F.MANUAL, **cfg) as ctx:
        if tiles is not None:
            F.flowroi_set_tiles(ctx.h, tiles)
        for i, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 3, fr, i, bit_depth)
            F.flowroi_flush(ctx.h, 120000)
            h, w = fr.shape
            outs.append(fetch(ctx.h, 3, i, h, w, keep, cfg.get("wavelet", 53)))
    return outs


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_tile_tables_give_identical_results(orc):
    seq = u16(sequence_u16(3303, 2, 768, 1024, 60))
    cfg = dict(pyr_levels=5, dwt_levels=5, wavelet=97)
    base = _run([seq[0], seq[1]], None, **cfg)[1]
    for t in (TABLE_A, TABLE_B):
        assert F.flowroi_tiles_check(t) == ""
        _same(base, _run([seq[0], seq[1]], t, **cfg)[1])
    _stagewise(orc, seq[0], seq[1], 12, _run([seq[0], seq[1]], TABLE_A, **cfg)[1], **cfg)


def test_tile_table_from_config_file(tmp_path):
    seq = u16(sequence_u16(3304, 2, 256, 512, 20))
    p = tmp_path / "t.json"
    p.write_text(TABLE_B)
    cfg = dict(pyr_levels=4, dwt_levels=4, wavelet=53)
    a = _run([seq[0], seq[1]], None, keep=False, **cfg)[1]
    outs = []
    with F.Context(flags=F.MANUAL, tile_table=str(p), **cfg) as ctx:
        got = json.loads(F.flowroi_get_tiles(ctx.h))
        assert len(got["entries"]) == len(json.loads(TABLE_B)["entries"])
        for i, fr in enumerate((seq[0], seq[1])):
            F.flowroi_submit_frame(ctx.h, 3, fr, i, 12)
            F.flowroi_flush(ctx.h, 60000)
        outs = fetch(ctx.h, 3, 1, 256, 512, False)
    _same(a, outs)


def test_mixed_width_batch_with_per_width_entries():
    """One batch of a 512-wide and a 1024-wide stream, each width class on
    its own DWT and saliency shapes, equals each stream alone."""
    t = _table([dict(param="dwt_seg", w=512, storage=32, level=l, value=8) for l in range(1, 4)]
               + [dict(param="dwt_seg", w=1024, storage=32, level=l, value=48) for l in range(1, 4)]
               + [dict(param="update_rows", storage=32, value=8),
                  dict(param="saliency_rows", w=512, storage=32, value=8), dict(param="saliency_rows", w=1024, storage=32, value=64)])
    s1 = u16(sequence_u16(3305, 2, 256, 512, 20))
    s2 = u16(sequence_u16(3306, 2, 512, 1024, 40))
    cfg = dict(pyr_levels=4, dwt_levels=3, wavelet=97)
    alone1 = _run([s1[0], s1[1]], None, keep=False, **cfg)[1]
    alone2 = _run([s2[0], s2[1]], None, keep=False, **cfg)[1]
    with F.Context(flags=F.MANUAL, **cfg) as ctx:
        F.flowroi_set_tiles(ctx.h, t)
        for i in range(2):
            F.flowroi_submit_frame(ctx.h, 1, s1[i], i, 12)
            F.flowroi_submit_frame(ctx.h, 2, s2[i], i, 12)
            F.flowroi_flush(ctx.h, 60000)
        m1 = fetch(ctx.h, 1, 1, 256, 512, False, 97)
        m2 = fetch(ctx.h, 2, 1, 512, 1024, False, 97)
    _same(alone1, m1)
    _same(alone2, m2)


def test_autotune_returns_a_loadable_table(tmp_path):
    cfg = F.flowroi_default_config(wavelet=53, dwt_levels=3, pyr_levels=3)
    text = F.flowroi_autotune(cfg, [(256, 256)], 2, 1)
    assert F.flowroi_tiles_check(text) == ""
    t = json.loads(text)
    params = {e["param"] for e in t["entries"]}
    assert {"dwt_seg", "update_rows", "saliency_rows", "blocks_per_sm", "dwt_variant"} <= params
    p = tmp_path / "tuned.json"
    p.write_text(text)
    seq = u16(sequence_u16(3307, 2, 256, 256, 10))
    a = _run([seq[0], seq[1]], None, keep=False, wavelet=53, dwt_levels=3, pyr_levels=3)[1]
    with F.Context(flags=F.MANUAL, tile_table=str(p), wavelet=53, dwt_levels=3, pyr_levels=3) as ctx:
        for i in range(2):
            F.flowroi_submit_frame(ctx.h, 3, seq[i], i, 12)
            F.flowroi_flush(ctx.h, 60000)
        b = fetch(ctx.h, 3, 1, 256, 256, False)
    _same(a, b)
