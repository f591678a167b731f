"""Stream -> device routing (flowroi_route, the Router dispatch and the
bench's per-rank stream sets), on the host only.

The routing is a consistent hash, so its defining properties pin it: every
id lands in [0, n); one device takes everything; going from n to n + 1
devices moves an id only to the new device, and about 1/(n + 1) of the ids;
the devices get about equal shares."""
import numpy as np
import pytest

import bench
from paper_2511_14419_gb300 import flowroi as F

IDS = list(range(-200, 20000)) + [2**62, -(2**62), 123456789012345]


def test_range_and_single_device():
    for n in (1, 2, 3, 8, 100):
        d = [F.flowroi_route(i, n) for i in IDS[:3000]]
        assert min(d) >= 0 and max(d) < n
    assert all(F.flowroi_route(i, 1) == 0 for i in IDS)
    assert F.lib().flowroi_route(5, 0) == 2**32 - 1
    with pytest.raises(ValueError):
        F.flowroi_route(5, 0)


def test_deterministic():
    a = [F.flowroi_route(i, 7) for i in IDS]
    b = [F.flowroi_route(i, 7) for i in IDS]
    assert a == b


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 16])
def test_growing_moves_ids_only_to_the_new_device(n):
    before = np.array([F.flowroi_route(i, n) for i in IDS])
    after = np.array([F.flowroi_route(i, n + 1) for i in IDS])
    moved = before != after
    assert np.all(after[moved] == n)
    frac = moved.mean()
    assert abs(frac - 1.0 / (n + 1)) < 0.02, frac


@pytest.mark.parametrize("n", [2, 4, 8])
def test_balanced(n):
    d = np.array([F.flowroi_route(i, n) for i in range(40000)])
    share = np.bincount(d, minlength=n) / d.size
    assert np.all(np.abs(share - 1.0 / n) < 0.02), share


def test_consecutive_ids_are_spread():
    # runs of consecutive stream ids do not pile up on one device
    d = [F.flowroi_route(i, 4) for i in range(64)]
    assert len(set(d[:16])) >= 3


def test_rank_streams_partition():
    ws, S = 4, 16
    sets = [bench.rank_streams(F.flowroi_route, S, ws, r) for r in range(ws)]
    for r, ids in enumerate(sets):
        assert len(ids) == S and ids == sorted(ids)
        assert all(F.flowroi_route(i, ws) == r for i in ids)
    flat = [i for ids in sets for i in ids]
    assert len(set(flat)) == ws * S
    # one rank: the ids 0 .. S-1, as a single-GPU run always used
    assert bench.rank_streams(F.flowroi_route, S, 1, 0) == list(range(S))


class _FakeCtx:
    def __init__(self, d):
        self.d, self.h, self.closed = d, ("ctx", d), False

    def close(self):
        self.closed = True


def test_router_dispatch(monkeypatch):
    calls = []
    monkeypatch.setattr(F, "flowroi_submit_frame", lambda h, sid, *a: calls.append(("submit", h, sid)) or 0)
    monkeypatch.setattr(F, "flowroi_get_mask", lambda h, sid, *a: calls.append(("mask", h, sid)) or 0)
    monkeypatch.setattr(F, "flowroi_flush", lambda h, *a: calls.append(("flush", h)) or 0)
    made = []

    def make(d):
        made.append(d)
        return _FakeCtx(d)

    with F.Router(3, make_context=make) as r:
        for sid in range(12):
            r.submit_frame(sid, None, 0, 12)
            r.get_mask(sid, 0, None)
        r.flush()
        ctxs = list(r._ctx.values())
    for kind, h, *sid in calls:
        if kind != "flush":
            assert h == ("ctx", F.flowroi_route(sid[0], 3))
    assert sorted(made) == sorted(set(made))  # one context per device, made once
    assert sorted({c[1] for c in calls if c[0] == "flush"}) == sorted(("ctx", d) for d in made)
    assert all(c.closed for c in ctxs)
