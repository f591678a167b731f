"""The allocation-free JPEG2000 front end, flowroi_dwt_roi_noalloc.

Callers that cannot allocate device memory (a fixed device budget, a host
application that owns the device heap, a real-time loop that must not call
cudaMalloc) use this entry point on their own buffers.  Its coefficients
must equal the streaming path's (flowroi_get_coeffs) for the same frame and
RoI mask: both run the same DWT kernel on the same samples with the same
quantisation steps, so the tolerance of the other coefficient tests
applies, bit-exact.  Two calls in a row share the library's fixed array.
"""
import numpy as np
import pytest
import torch

from synth import pair_u8, sequence_u16
from tests._gpu import F, u16

pytestmark = pytest.mark.gpu


def _streaming_path(frames, bit_depth, wavelet, levels):
    """Mask (device tensor) and coefficients (host) of the second frame."""
    h, w = frames[1].shape
    with F.Context(flags=F.MANUAL, wavelet=wavelet, dwt_levels=levels, pyr_levels=3) as ctx:
        for i, fr in enumerate(frames):
            F.flowroi_submit_frame(ctx.h, 1, fr, i, bit_depth)
            F.flowroi_flush(ctx.h, 60000)
        mask = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        F.flowroi_get_mask(ctx.h, 1, 1, mask, 60000)
        coeffs = np.empty((h, w), np.int32)
        F.flowroi_get_coeffs(ctx.h, 1, 1, coeffs, 60000)
    return mask, coeffs


def test_noalloc_matches_streaming_path_on_two_calls():
    # call 1: reversible 5/3, 8-bit 256x256 pair, 3 levels
    prev, cur = pair_u8(seed=4242)
    mask1, ref1 = _streaming_path([prev.numpy(), cur.numpy()], 8, F.W53, 3)
    assert int(mask1.sum()) > 0  # the up-shift is exercised
    out1 = torch.full((256, 256), -7, dtype=torch.int32, device="cuda")
    F.flowroi_dwt_roi_noalloc(cur.cuda(), 8, mask1, F.W53, 3, 5, None, out1)
    torch.cuda.synchronize()
    assert np.array_equal(out1.cpu().numpy(), ref1)

    # call 2, right after and sharing the same fixed array: irreversible
    # 9/7, 12-bit 512x512 pair, 5 levels, quantised
    seq = u16(sequence_u16(4343, 2, 512, 512, 30))
    mask2, ref2 = _streaming_path([seq[0], seq[1]], 12, F.W97, 5)
    assert int(mask2.sum()) > 0
    delta, _, _, _ = F.flowroi_quant_steps(5, 12, 1.0)
    raw2 = torch.from_numpy(seq[1].view(np.int16).copy()).cuda()
    out2 = torch.full((512, 512), -7, dtype=torch.int32, device="cuda")
    F.flowroi_dwt_roi_noalloc(raw2, 12, mask2, F.W97, 5, 5, delta, out2)
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), ref2)


def test_noalloc_allocates_nothing_across_repeated_calls():
    """The entry point's promise: no device allocation.  torch's allocator
    counters stay flat across a run of calls (the library's own cudaMalloc
    calls would not show there, but none exist on this path; the wrapper
    allocates no tensor either), and the result is the same every time."""
    prev, cur = pair_u8(seed=4242)
    mask, ref = _streaming_path([prev.numpy(), cur.numpy()], 8, F.W53, 3)
    raw = cur.cuda()
    out = torch.empty((256, 256), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    a0, r0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(20):
        F.flowroi_dwt_roi_noalloc(raw, 8, mask, F.W53, 3, 5, None, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0 and torch.cuda.memory_reserved() == r0
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("pad", [2, 4])
def test_noalloc_pitched_rows(pad):
    """Rows of a wider 16-bit tensor (row pitch (W + pad) * 2 bytes: 4-byte
    aligned with pad 2, 8-byte aligned with pad 4), bit-exact with the
    streaming path's coefficients of the same frame."""
    seq = u16(sequence_u16(4545 + pad, 2, 256, 512, 20))
    mask, ref = _streaming_path([seq[0], seq[1]], 12, F.W97, 5)
    delta, _, _, _ = F.flowroi_quant_steps(5, 12, 1.0)
    wide = torch.zeros((256, 512 + pad), dtype=torch.int16, device="cuda")
    wide[:, :512] = torch.from_numpy(seq[1].view(np.int16).copy()).cuda()
    out = torch.full((256, 512), -7, dtype=torch.int32, device="cuda")
    F.flowroi_dwt_roi_noalloc(wide[:, :512], 12, mask, F.W97, 5, 5, delta, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_frame_at_the_size_limit():
    """A 2048 x 512 frame (2^20 pixels, the largest the fixed array holds):
    its low-low planes fill the array."""
    seq = u16(sequence_u16(4646, 2, 512, 2048, 40))
    mask, ref = _streaming_path([seq[0], seq[1]], 12, F.W53, 5)
    raw = torch.from_numpy(seq[1].view(np.int16).copy()).cuda()
    out = torch.full((512, 2048), -7, dtype=torch.int32, device="cuda")
    F.flowroi_dwt_roi_noalloc(raw, 12, mask, F.W53, 5, 5, None, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_oversize_and_malformed_requests():
    raw = torch.zeros((2048, 1024), dtype=torch.int16, device="cuda")   # 2^21 pixels > 2^20
    mask = torch.zeros((2048, 1024), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2048, 1024), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FlowRoIError) as ei:
        F.flowroi_dwt_roi_noalloc(raw, 12, mask, F.W53, 3, 5, None, out)
    assert ei.value.code == F.EINVAL
    raw_ok = torch.zeros((64, 40), dtype=torch.int16, device="cuda")   # 40 not a multiple of 2^4
    with pytest.raises(F.FlowRoIError) as ei:
        F.flowroi_dwt_roi_noalloc(raw_ok, 12, torch.zeros((64, 40), dtype=torch.uint8, device="cuda"), F.W53, 4, 5,
                                  None, torch.zeros((64, 40), dtype=torch.int32, device="cuda"))
    assert ei.value.code == F.EINVAL
    with pytest.raises(F.FlowRoIError) as ei:  # 9/7 without quantisation steps
        F.flowroi_dwt_roi_noalloc(raw_ok[:, :32].contiguous(), 12, torch.zeros((64, 32), dtype=torch.uint8, device="cuda"),
                                  F.W97, 3, 5, None, torch.zeros((64, 32), dtype=torch.int32, device="cuda"))
    assert ei.value.code == F.EINVAL
    # malformed buffers are refused before the library is called: a mask or
    # coefficient buffer smaller than the frame, the wrong dtypes, 4-byte samples
    r = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
    m = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    c = torch.zeros((64, 64), dtype=torch.int32, device="cuda")
    for args in ((r, m[:32], c), (r, m, c[:, :32].contiguous()), (r, m, c.to(torch.int16)), (r, m.to(torch.int32), c),
                 (r.to(torch.int32), m, c), (r.float(), m, c)):
        with pytest.raises(ValueError):
            F.flowroi_dwt_roi_noalloc(args[0], 12, args[1], F.W53, 3, 5, None, args[2])
    with pytest.raises(ValueError):  # too few quantisation steps
        F.flowroi_dwt_roi_noalloc(r, 12, m, F.W97, 3, 5, np.ones(5, np.float32), c)
