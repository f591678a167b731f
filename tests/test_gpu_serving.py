"""Serving behaviour of the CUDA library through the C ABI: batch
invariance (a frame's results are bit-identical alone, in a mixed batch of
streams of different resolutions, on the plain per-frame path and under the
continuously batching scheduler thread), admission by HBM budget, result
ring eviction, bounded waits and argument errors."""
import threading
import time

import numpy as np
import pytest

from synth import pair_u8, sequence_u16
from tests._gpu import F, fetch, run_stream, u16

pytestmark = pytest.mark.gpu


def _streams():
    """Four streams of different geometry / format (two frames each)."""
    out = []
    for sid, (h, w) in enumerate([(256, 256), (128, 192), (512, 256), (64, 64)]):
        if sid % 2 == 0:
            a, b = pair_u8(seed=900 + sid, h=h, w=w, n_blobs=6)
            out.append((sid, [a.numpy(), b.numpy()], 8))
        else:
            s = u16(sequence_u16(950 + sid, 2, h, w, 12))
            out.append((sid, [s[0], s[1]], 12))
    return out


def _same(a, b):
    for k in ("mask", "coeffs", "flow", "mask0", "shat", "thr"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("wavelet", [53, 97])
def test_batch_invariance_mixed_resolutions(wavelet):
    cfg = dict(pyr_levels=3, dwt_levels=3, wavelet=wavelet)
    alone = {sid: run_stream(frames, bd, **cfg)[1] for sid, frames, bd in _streams()}
    plain = {sid: run_stream(frames, bd, plain=True, **cfg)[1] for sid, frames, bd in _streams()}
    with F.Context(flags=F.MANUAL | F.KEEP_INTERMEDIATES, **cfg) as ctx:
        for t in range(2):
            for sid, frames, bd in _streams():
                F.flowroi_submit_frame(ctx.h, sid, frames[t], t, bd)
            assert F.flowroi_step(ctx.h) == 4  # one batch holds every stream's frame
            F.flowroi_flush(ctx.h, 60000)
        mixed = {sid: fetch(ctx.h, sid, 1, frames[1].shape[0], frames[1].shape[1], wavelet=wavelet)
                 for sid, frames, bd in _streams()}
        st = F.flowroi_get_stats(ctx.h)
        assert st["batches"] == 2 and st["frames_done"] == 8 and st["kernel_launches"] > 0
    for sid in alone:
        _same(alone[sid], mixed[sid])
        _same(alone[sid], plain[sid])


def test_batch_submit_matches_per_frame_submit_and_stops_at_a_refusal():
    cfg = dict(pyr_levels=3, dwt_levels=3, wavelet=53)
    streams = _streams()
    alone = {sid: run_stream(frames, bd, **cfg)[1] for sid, frames, bd in streams}
    with F.Context(flags=F.MANUAL | F.KEEP_INTERMEDIATES, result_ring=2, **cfg) as ctx:
        for t in range(2):
            k, st = F.flowroi_submit_frames(ctx.h, [(sid, frames[t], t, bd) for sid, frames, bd in streams])
            assert (k, st) == (4, F.OK)
            assert F.flowroi_step(ctx.h) == 4
            F.flowroi_flush(ctx.h, 60000)
        for sid, frames, bd in streams:
            _same(alone[sid], fetch(ctx.h, sid, 1, frames[1].shape[0], frames[1].shape[1], wavelet=53))
        # frame 2 of stream 0 and 1 fit; a frame index that does not
        # increase is refused and nothing after it is looked at
        sid0, fr0, bd0 = streams[0]
        sid1, fr1, bd1 = streams[1]
        k, st = F.flowroi_submit_frames(ctx.h, [(sid0, fr0[0], 2, bd0), (sid1, fr1[0], 1, bd1), (sid1, fr1[0], 3, bd1)])
        assert (k, st) == (1, F.EINVAL)
        assert "not after" in F.flowroi_last_error(ctx.h)
        # an empty batch is a no-op; a negative count is an argument error
        assert F.flowroi_submit_frames(ctx.h, []) == (0, F.OK)
        assert F.lib().flowroi_submit_frames(ctx.h, -1, None, None, None) == F.EINVAL


def test_get_results_matches_the_per_frame_getters():
    """flowroi_get_results: the masks and coefficients of several streams'
    frames in one call equal flowroi_get_mask / flowroi_get_coeffs frame by
    frame, into host and into device buffers; a skipped output stays
    untouched; a frame that cannot be read (unknown stream, a frame not
    submitted) gets its own status while the others are still copied."""
    import torch
    cfg = dict(pyr_levels=3, dwt_levels=3, wavelet=97)
    streams = _streams()
    with F.Context(flags=F.MANUAL, **cfg) as ctx:
        for t in range(2):
            F.flowroi_submit_frames(ctx.h, [(sid, frames[t], t, bd) for sid, frames, bd in streams])
            F.flowroi_step(ctx.h)
        F.flowroi_flush(ctx.h, 60000)
        want = {}
        for sid, frames, bd in streams:
            h, w = frames[1].shape
            m, c = np.empty((h, w), np.uint8), np.empty((h, w), np.int32)
            F.flowroi_get_mask(ctx.h, sid, 1, m)
            F.flowroi_get_coeffs(ctx.h, sid, 1, c)
            want[sid] = (m, c)
        outs = {sid: (np.full(frames[1].shape, 7, np.uint8), np.full(frames[1].shape, 7, np.int32))
                for sid, frames, bd in streams}
        st = F.flowroi_get_results(ctx.h, [(sid, 1, outs[sid][0], outs[sid][1]) for sid, _, _ in streams])
        assert st == [F.OK] * len(streams)
        for sid in want:
            assert np.array_equal(outs[sid][0], want[sid][0]) and np.array_equal(outs[sid][1], want[sid][1])
        # device outputs, coefficients only for the first stream
        dev = {sid: (torch.zeros(frames[1].shape, dtype=torch.uint8, device="cuda"),
                     torch.zeros(frames[1].shape, dtype=torch.int32, device="cuda")) for sid, frames, bd in streams}
        items = [(sid, 1, None if sid == 0 else dev[sid][0], dev[sid][1]) for sid, _, _ in streams]
        assert F.flowroi_get_results(ctx.h, items) == [F.OK] * len(streams)
        for sid in want:
            assert np.array_equal(dev[sid][1].cpu().numpy(), want[sid][1])
            if sid == 0:
                assert not dev[sid][0].any()
            else:
                assert np.array_equal(dev[sid][0].cpu().numpy(), want[sid][0])
        # per-frame failures: the readable frames are still copied
        sid1, fr1, _ = streams[1]
        m1 = np.zeros(fr1[1].shape, np.uint8)
        import ctypes
        ids = (ctypes.c_int64 * 3)(999, sid1, sid1)
        fis = (ctypes.c_int64 * 3)(1, 1, 5)
        mp = (ctypes.c_void_p * 3)(None, m1.ctypes.data, None)
        cp = (ctypes.c_void_p * 3)()
        st = (ctypes.c_int * 3)()
        rc = F.lib().flowroi_get_results(ctx.h, 3, ids, fis, mp, cp, 0, 1000, st)
        assert rc == F.ENOSTREAM and list(st) == [F.ENOSTREAM, F.OK, F.ENOSTREAM]
        assert np.array_equal(m1, want[sid1][0])
        assert F.lib().flowroi_get_results(ctx.h, -1, None, None, None, None, 0, 0, None) == F.EINVAL
        assert F.flowroi_get_results(ctx.h, []) == []


def test_scheduler_thread_matches_manual():
    streams = _streams()
    manual = {sid: run_stream(frames, bd, keep=False)[1] for sid, frames, bd in streams}
    with F.Context() as ctx:  # scheduler thread, continuous batching
        for t in range(2):
            for sid, frames, bd in streams:
                F.flowroi_submit_frame(ctx.h, sid, frames[t], t, bd)
        for sid, frames, bd in streams:
            h, w = frames[1].shape
            got = fetch(ctx.h, sid, 1, h, w, keep=False, timeout_ms=60000)
            assert np.array_equal(got["mask"], manual[sid]["mask"])
            assert np.array_equal(got["coeffs"], manual[sid]["coeffs"])
        st = F.flowroi_get_stats(ctx.h)
        assert st["frames_done"] == 8 and st["lat_p99_ms"] >= st["lat_p50_ms"] > 0


def test_admission_by_hbm_budget():
    a, _ = pair_u8(seed=1, h=256, w=256)
    with F.Context(flags=F.MANUAL) as probe:
        F.flowroi_submit_frame(probe.h, 0, a.numpy(), 0, 8)
        one = F.flowroi_get_stats(probe.h)["bytes_admitted"]
    with F.Context(flags=F.MANUAL, hbm_budget_bytes=int(one * 1.5)) as ctx:
        F.flowroi_submit_frame(ctx.h, 1, a.numpy(), 0, 8)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_submit_frame(ctx.h, 2, a.numpy(), 0, 8)
        assert ei.value.code == F.EBUSY
        F.flowroi_flush(ctx.h, 60000)
        F.flowroi_end_stream(ctx.h, 1)
        F.flowroi_submit_frame(ctx.h, 2, a.numpy(), 0, 8)  # admitted once the budget is free
        st = F.flowroi_get_stats(ctx.h)
        assert st["admissions_refused"] == 1 and st["streams_admitted"] == 1


def test_ring_eviction_timeout_and_order_errors():
    frames = [pair_u8(seed=s, h=64, w=64)[0].numpy() for s in range(4)]
    out = np.empty((64, 64), np.uint8)
    with F.Context(flags=F.MANUAL, result_ring=2) as ctx:
        for i in range(3):
            F.flowroi_submit_frame(ctx.h, 5, frames[i], i, 8)
            F.flowroi_flush(ctx.h, 60000)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_mask(ctx.h, 5, 0, out, 1000)
        assert ei.value.code == F.EGONE
        F.flowroi_get_mask(ctx.h, 5, 2, out, 1000)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_submit_frame(ctx.h, 5, frames[3], 2, 8)  # not after frame 2
        assert ei.value.code == F.EINVAL
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_submit_frame(ctx.h, 5, np.zeros((32, 64), np.uint8), 9, 8)  # geometry change
        assert ei.value.code == F.EINVAL
        F.flowroi_submit_frame(ctx.h, 5, frames[3], 10, 8)  # submitted, never stepped
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_mask(ctx.h, 5, 10, out, 50)
        assert ei.value.code == F.ETIMEDOUT
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_mask(ctx.h, 5, 11, out, 50)
        assert ei.value.code == F.ENOSTREAM
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_intermediate(ctx.h, 5, 2, F.I_FLOW, np.empty((64, 64, 2), np.float32), 50)
        assert ei.value.code == F.ENOTKEPT
        F.flowroi_step(ctx.h)
        F.flowroi_get_mask(ctx.h, 5, 10, out, 60000)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_submit_frame(ctx.h, 6, np.zeros((64, 60), np.uint8), 0, 8)  # not a multiple of 8
        assert ei.value.code == F.EINVAL


def test_many_streams_and_frames_in_flight():
    """16 streams x 6 frames under the scheduler thread, results fetched
    while later frames are queued; each matches its stream run alone."""
    seqs = [u16(sequence_u16(4000 + s, 6, 128, 128, 8)) for s in range(16)]
    ref = {s: run_stream([seqs[s][t] for t in range(6)], 12, keep=False) for s in (0, 7, 15)}
    with F.Context(result_ring=8) as ctx:
        for t in range(6):
            for s in range(16):
                F.flowroi_submit_frame(ctx.h, s, seqs[s][t], t, 12)
        for s in (0, 7, 15):
            for t in range(6):
                got = fetch(ctx.h, s, t, 128, 128, keep=False)
                assert np.array_equal(got["mask"], ref[s][t]["mask"])
                assert np.array_equal(got["coeffs"], ref[s][t]["coeffs"])
        F.flowroi_flush(ctx.h, 60000)
        st = F.flowroi_get_stats(ctx.h)
        assert st["frames_done"] == 96 and st["batches"] >= 6


def test_admission_while_batches_are_in_flight():
    """A stream refused for lack of HBM budget (EBUSY) is admitted without a
    flush once another thread ends a stream, while the scheduler thread keeps
    a third stream's batches going; the late stream's results, and the busy
    stream's, equal the same streams run alone."""
    cfg = dict(pyr_levels=4, dwt_levels=4, wavelet=97)
    A = u16(sequence_u16(7001, 3, 512, 512, 20))
    B = u16(sequence_u16(7002, 10, 512, 512, 20))
    C = u16(sequence_u16(7003, 3, 512, 512, 20))
    alone_B = run_stream([B[t] for t in range(10)], 12, keep=False, **cfg)
    alone_C = run_stream([C[t] for t in range(3)], 12, keep=False, **cfg)
    with F.Context(flags=F.MANUAL, **cfg) as probe:
        F.flowroi_submit_frame(probe.h, 0, A[0], 0, 12)
        one = F.flowroi_get_stats(probe.h)["bytes_admitted"]

    def submit_retry(ctx, sid, fr, idx):
        for _ in range(20000):
            try:
                return F.flowroi_submit_frame(ctx.h, sid, fr, idx, 12)
            except F.FlowRoIError as e:
                if e.code != F.EBUSY:
                    raise
                time.sleep(0.0005)
        raise TimeoutError("submission stayed refused")

    with F.Context(hbm_budget_bytes=int(2.5 * one), result_ring=8, **cfg) as ctx:  # scheduler thread
        for t in range(3):
            F.flowroi_submit_frame(ctx.h, 1, A[t], t, 12)
        for t in range(3):
            F.flowroi_submit_frame(ctx.h, 2, B[t], t, 12)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_submit_frame(ctx.h, 3, C[0], 0, 12)
        assert ei.value.code == F.EBUSY
        errs = []

        def ender():
            try:
                fetch(ctx.h, 1, 2, 512, 512, keep=False, wavelet=97)
                for t in range(3, 6):  # more of B's frames queued while A ends
                    submit_retry(ctx, 2, B[t], t)
                F.flowroi_end_stream(ctx.h, 1)
            except Exception as e:  # reported by the main thread
                errs.append(e)

        th = threading.Thread(target=ender)
        th.start()
        submit_retry(ctx, 3, C[0], 0)  # admitted once A's budget is returned; no flush
        for t in range(6, 10):
            submit_retry(ctx, 2, B[t], t)
        for t in (1, 2):
            submit_retry(ctx, 3, C[t], t)
        th.join(60)
        assert not th.is_alive() and not errs, errs
        for t in range(3):
            got = fetch(ctx.h, 3, t, 512, 512, keep=False, wavelet=97, timeout_ms=60000)
            assert np.array_equal(got["mask"], alone_C[t]["mask"]) and np.array_equal(got["coeffs"], alone_C[t]["coeffs"])
        for t in (8, 9):
            got = fetch(ctx.h, 2, t, 512, 512, keep=False, wavelet=97, timeout_ms=60000)
            assert np.array_equal(got["mask"], alone_B[t]["mask"]) and np.array_equal(got["coeffs"], alone_B[t]["coeffs"])
        st = F.flowroi_get_stats(ctx.h)
        assert st["admissions_refused"] >= 1 and st["streams_admitted"] == 2  # B and C (A ended)
