"""The stream router on one GPU: streams submitted through flowroi.Router
go to the context of the device flowroi_route names (device 0 when there is
one device), and each stream's masks and coefficients are bit-identical to
a context run directly on that stream alone."""
import numpy as np
import pytest

from synth import pair_u8
from tests._gpu import F, run_stream

pytestmark = pytest.mark.gpu


def test_router_on_one_device_matches_direct_contexts():
    sids = [3, 11, 40, 97]
    pairs = {sid: [f.numpy() for f in pair_u8(seed=500 + sid)] for sid in sids}
    got = {}
    with F.Router(1, flags=F.MANUAL) as r:
        assert all(r.device_of(sid) == 0 for sid in sids)
        for i in range(2):
            for sid in sids:
                r.submit_frame(sid, pairs[sid][i], i, 8)
            r.flush(120000)
        for sid in sids:
            m = np.empty((256, 256), np.uint8)
            c = np.empty((256, 256), np.int32)
            r.get_mask(sid, 1, m, 60000)
            F.flowroi_get_coeffs(r.context(sid).h, sid, 1, c, 60000)
            got[sid] = (m, c)
        assert len(r._ctx) == 1  # one context, on device 0
    for sid in sids:
        want = run_stream(pairs[sid], 8, keep=False)[1]
        assert np.array_equal(got[sid][0], want["mask"])
        assert np.array_equal(got[sid][1], want["coeffs"])
        assert got[sid][0].any()
