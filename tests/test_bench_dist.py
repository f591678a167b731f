"""Multi-rank aggregation of bench.py on CPU (gloo, world size 2): every
rank runs its own replica; the job time is the slowest rank's and the
throughput counts every rank's frames."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t = bench.max_over_ranks(1.5 + rank, ws, "cpu")  # rank 1 is the slow one
    q.put((rank, t, bench.job_throughput(100, ws, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, thr in out:
        assert t == 2.5
        assert thr == pytest.approx(200 / 2.5)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(16, 1, 2.0) == 8.0
    assert [bench.frame_index(t, 4) for t in range(8)] == [0, 1, 2, 3, 2, 1, 0, 1]


def test_all_cores_oracle_sample_spawns_one_process_per_core():
    """The all-cores CPU baseline: two spawned oracle processes on crops of
    a small synthetic pair; the rate is the sum of the processes' rates,
    scaled to the workload's frame size."""
    import numpy as np

    import bench
    from synth import sequence_u16
    seq = sequence_u16(11, 2, 128, 128, 6, device="cpu")
    fc = [(seq[0].numpy().view(np.uint16), seq[1].numpy().view(np.uint16))]
    wl = dict(h=128, w=128, bit_depth=12, pyr_levels=3, dwt_levels=3, wavelet=97)
    fps, procs, n, el = bench.cpu_sample_parallel(wl, fc, procs=2, budget_s=0.2, crop=64, per_proc=2)
    assert procs == 2 and n >= 2 and el >= 0.2
    # two processes, each at least one 64x64 crop in at most el seconds
    assert fps >= 2 * (64 * 64) / (128 * 128) / el * 0.5
    assert fps > 0


def test_all_cores_oracle_sample_reports_a_failing_process():
    """A worker whose oracle call fails ends the sample with an exception
    (no respawn, no wait for the deadline)."""
    import time

    import numpy as np

    import bench
    fc = [(np.zeros((64, 64), np.uint16), np.zeros((64, 64), np.uint16))]
    wl = dict(h=64, w=64, bit_depth=12, dwt_levels=2, wavelet=53)  # no pyr_levels: KeyError in the workers
    t0 = time.monotonic()
    with pytest.raises(RuntimeError, match="KeyError"):
        bench.cpu_sample_parallel(wl, fc, procs=2, budget_s=0.1, crop=32, per_proc=1)
    assert time.monotonic() - t0 < 60


def _route_worker(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2511_14419_gb300 import flowroi as F
    mine = bench.rank_streams(F.flowroi_route, 16, ws, rank)
    every = [None] * ws
    dist.all_gather_object(every, mine)
    q.put((rank, mine, every))
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_take_disjoint_routed_stream_sets_gloo():
    """Each rank of a 2-rank job serves the 16 streams the library routes to
    it; the ranks agree on the split and no stream is served twice."""
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_route_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2511_14419_gb300 import flowroi as F
    views = {rank: every for rank, _, every in out}
    assert views[0] == views[1]
    sets = views[0]
    assert all(len(s) == 16 for s in sets)
    assert not set(sets[0]) & set(sets[1])
    for r, ids in enumerate(sets):
        assert all(F.flowroi_route(i, ws) == r for i in ids)
