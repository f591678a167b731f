"""Failure detection of the bounded device waits and loops, driven to
expiry without a fault.

Under FLOWROI_TEST_EXPIRE_TMA the window kernel's producer never issues
one tile's copies, so the consumers' waits for them (and the producer's
waits for slots they never release) run out after 2^12 polls; under
FLOWROI_TEST_EXPIRE_LOOP the component filter's union-find loops give up
after one step.  Either way the kernels return normally, the batch's error
word reaches the host, and the context is poisoned with FLOWROI_EDEVICE and
a message naming the wait; the device itself stays usable and a fresh
context computes the same pair to oracle parity."""
import numpy as np
import pytest
import torch

from synth import pair_u8
from tests._gpu import F, run_stream
from tests.test_gpu_components import _check
from tests.test_gpu_parity import _stagewise

pytestmark = pytest.mark.gpu


def _poisoned_run(flags, **cfg):
    prev, cur = pair_u8(seed=1001)
    with F.Context(flags=F.MANUAL | flags, **cfg) as ctx:
        F.flowroi_submit_frame(ctx.h, 1, prev.numpy(), 0, 8)
        F.flowroi_flush(ctx.h, 60000)  # a first frame has no flow: nothing waits
        F.flowroi_submit_frame(ctx.h, 1, cur.numpy(), 1, 8)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_flush(ctx.h, 60000)
        assert ei.value.code == F.EDEVICE
        out = np.empty((256, 256), np.uint8)
        with pytest.raises(F.FlowRoIError) as e2:
            F.flowroi_get_mask(ctx.h, 1, 1, out, 1000)
        assert e2.value.code == F.EDEVICE
        msg = F.flowroi_last_error(ctx.h)
        with pytest.raises(F.FlowRoIError):  # later submissions are refused too
            F.flowroi_submit_frame(ctx.h, 1, cur.numpy(), 2, 8)
    # the device is still usable
    x = torch.arange(1024, device="cuda", dtype=torch.float32)
    assert float(x.sum().item()) == 1023 * 1024 / 2
    return prev.numpy(), cur.numpy(), msg


def test_tma_wait_runs_out_and_poisons_the_context(orc):
    prev, cur, msg = _poisoned_run(F.TEST_EXPIRE_TMA)
    assert "bounded wait for a TMA copy ran out" in msg, msg
    g = run_stream([prev, cur], 8)[1]  # fresh context, no flag
    _stagewise(orc, prev, cur, 8, g)


def test_union_find_loop_runs_out_and_poisons_the_context(orc):
    prev, cur, msg = _poisoned_run(F.TEST_EXPIRE_LOOP, min_area=20)
    assert "bounded union-find loop ran out" in msg, msg
    # fresh context: the component filter bit-exact against the oracle's
    # flood fill of the GPU's own cut
    _check(orc, [prev, cur], 8, min_area=20, pyr_levels=3, dwt_levels=3)
