"""GPU parity of the embedded block coder (flowroi_encode_codestreams)
against the oracle (orc_ebcot.c, oracle.py): the containers are compared
byte for byte.  The coefficient planes are made by the oracle's own front
end (DC shift, DWT, quantisation, wavelet-domain RoI mask, up-shift) from
seeded synthetic 12-bit frames, and the same planes go to both coders.

Every byte is decided by integer arithmetic except the rate control, whose
slopes and bisection are IEEE double operations in the same order on both
sides over the same exact inputs (pass lengths and integer distortion
sums), so the containers must be identical, truncation points included."""
import numpy as np
import pytest
import torch

from oracle import oracle as o
from synth import sequence_u16
from tests._gpu import F
from tests.test_oracle_codestream import _container_blocks, parse

pytestmark = pytest.mark.gpu


def _planes(seed, h, w, levels, wavelet, shift, bd=12, roi_frac=0.3):
    """Oracle coefficient plane of a synthetic frame with a synthetic RoI
    (a centred rectangle covering about roi_frac of the frame)."""
    raw = np.asarray(sequence_u16(seed, 1, h, w, 6)[0]).astype(np.uint16)
    pix = np.zeros((h, w), np.uint8)
    rh, rw = int(h * np.sqrt(roi_frac)), int(w * np.sqrt(roi_frac))
    pix[(h - rh) // 2:(h + rh) // 2, (w - rw) // 2:(w + rw) // 2] = 1
    cm = o.wavelet_mask(pix, levels, wavelet)
    if wavelet == 53:
        q = o.dwt2d(o.dc_shift(raw, bd).astype(np.int64), 53, levels)
    else:
        y = o.dwt2d(o.dc_shift(raw, bd).astype(np.float64), 97, levels)
        _, delta, _, _ = o.delta_table(levels, bd)
        q = o.quantise_f64(y, levels, delta)
    return o.roi_shift(q, cm, shift)


def _gpu(ctx, planes, levels, wavelet, shift, budgets, on_device=False, bd=12, fmt=0, resets=None):
    jobs = []
    for i, (q, b) in enumerate(zip(planes, budgets)):
        h, w = q.shape
        cap = F.flowroi_codestream_bound(w, h, levels)
        r = resets[i] if resets else 0
        if on_device:
            jobs.append(dict(coeffs=torch.from_numpy(q).cuda(), out=torch.zeros(cap, dtype=torch.uint8, device="cuda"),
                             levels=levels, wavelet=wavelet, shift=shift, bit_depth=bd, budget=b, format=fmt, reset=r))
        else:
            jobs.append(dict(coeffs=np.ascontiguousarray(q), out=np.zeros(cap, np.uint8), levels=levels,
                             wavelet=wavelet, shift=shift, bit_depth=bd, budget=b, format=fmt, reset=r))
    lens = F.flowroi_encode_codestreams(ctx, jobs)
    out = []
    for j, n in zip(jobs, lens):
        buf = j["out"].cpu().numpy() if on_device else j["out"]
        out.append(bytes(buf[:n]))
    return out


@pytest.fixture(scope="module")
def ctx():
    with F.Context() as c:
        yield c.h


@pytest.mark.parametrize("h,w,levels", [(256, 256, 3), (200, 264, 3), (16, 16, 2), (192, 320, 4)])
def test_lossless_53_matches_oracle(ctx, h, w, levels):
    q = _planes(h + w, h, w, levels, 53, 5)
    want, _ = o.encode_frame(q, levels, 53, 5, 12, 0)
    got = _gpu(ctx, [q], levels, 53, 5, [0])[0]
    assert got == want


@pytest.mark.parametrize("bpp", [0.25, 1.0, 3.0])
def test_rate_controlled_97_matches_oracle(ctx, bpp):
    h, w, levels = 512, 512, 5
    q = _planes(77, h, w, levels, 97, 5)
    budget = int(bpp * h * w / 8)
    want, blocks = o.encode_frame(q, levels, 97, 5, 12, budget)
    got = _gpu(ctx, [q], levels, 97, 5, [budget])[0]
    assert got == want
    kept = sum(int(b["plen"][:b["nkeep"]].sum()) for b in blocks)
    assert kept <= budget


def test_batch_of_mixed_frames_and_device_pointers(ctx):
    """One call codes frames of different sizes, wavelets are recorded per
    frame; host and device buffers give the same containers."""
    specs = [(128, 192, 3, 53, 0), (256, 256, 4, 97, 20000), (64, 64, 2, 53, 300), (128, 128, 3, 97, 0)]
    planes = [_planes(900 + i, h, w, lv, wav, 5) for i, (h, w, lv, wav, b) in enumerate(specs)]
    for on_device in (False, True):
        for (h, w, lv, wav, b), q in zip(specs, planes):
            got = _gpu(ctx, [q], lv, wav, 5, [b], on_device=on_device)[0]
            want, _ = o.encode_frame(q, lv, wav, 5, 12, b)
            assert got == want
    # the same frames in one call
    same = [(h, w, lv, wav, b) for h, w, lv, wav, b in specs if lv == 3 and wav == 53]
    qs = [q for (h, w, lv, wav, b), q in zip(specs, planes) if lv == 3 and wav == 53]
    got = _gpu(ctx, qs, 3, 53, 5, [b for *_, b in same])
    for q, g, (h, w, lv, wav, b) in zip(qs, got, same):
        assert g == o.encode_frame(q, 3, 53, 5, 12, b)[0]


def test_full_size_2048_97_at_one_bit_per_pixel(ctx):
    """The geometry of the batched workload: 2048^2, 9/7, 5 levels, RoI
    shift 5, 1 bit per pixel of pass data."""
    h = w = 2048
    q = _planes(3000, h, w, 5, 97, 5)
    budget = h * w // 8
    want, _ = o.encode_frame(q, 5, 97, 5, 12, budget)
    got = _gpu(ctx, [q], 5, 97, 5, [budget], on_device=True)[0]
    assert got == want


def test_decoded_container_reconstructs_the_frame(ctx):
    """Lossless 5/3 without RoI shift: the GPU container, decoded and
    inverse-transformed, is the frame (the container is the oracle's, byte
    for byte, so this is the oracle's round trip on the GPU's output)."""
    raw = np.asarray(sequence_u16(4242, 1, 128, 128, 6)[0]).astype(np.uint16)
    q = o.dwt2d(o.dc_shift(raw, 12).astype(np.int64), 53, 3)
    got = _gpu(ctx, [q.astype(np.int32)], 3, 53, 0, [0])[0]
    assert got == o.encode_frame(q, 3, 53, 0, 12, 0)[0]


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_largest_magnitudes_24_planes_match_oracle(ctx, kind):
    """Code-blocks at the largest magnitudes the coder accepts (below 2^24:
    24 bit-planes, 70 passes).  Dense noise makes the most decisions per
    block, so the decision streams and the codeword slots come nearest their
    bounds; sparse spikes among zeros make long run-length stretches in
    every plane.  Lossless and rate-controlled containers byte-identical to
    the oracle's."""
    rng = np.random.default_rng(2424 if kind == "dense" else 2425)
    h = w = 128
    top = (1 << 24) - 1
    if kind == "dense":
        q = rng.integers(-top, top + 1, size=(h, w)).astype(np.int32)
    else:
        q = np.zeros((h, w), np.int32)
        idx = rng.choice(h * w, 300, replace=False)
        q.flat[idx] = rng.integers(-top, top + 1, size=idx.size)
    q[0, 0], q[-1, -1] = top, -top
    assert np.abs(q.astype(np.int64)).max() == top
    for budget in (0, h * w // 4):
        want, _ = o.encode_frame(q, 2, 53, 5, 12, budget)
        got = _gpu(ctx, [q], 2, 53, 5, [budget])[0]
        assert got == want


def test_too_small_output_and_out_of_range_magnitudes(ctx):
    q = _planes(5, 128, 128, 3, 53, 5)
    small = np.zeros(100, np.uint8)
    job = dict(coeffs=q, out=small, levels=3, wavelet=53, shift=5, bit_depth=12, budget=0)
    with pytest.raises(F.FlowRoIError) as ei:
        F.flowroi_encode_codestreams(ctx, [job])
    assert ei.value.code == F.ERANGE
    big = q.copy()
    big[3, 3] = 1 << 24
    cap = F.flowroi_codestream_bound(128, 128, 3)
    job = dict(coeffs=big, out=np.zeros(cap, np.uint8), levels=3, wavelet=53, shift=5, bit_depth=12, budget=0)
    with pytest.raises(F.FlowRoIError) as ei:
        F.flowroi_encode_codestreams(ctx, [job])
    assert ei.value.code == F.ERANGE
    # the context is still usable
    assert _gpu(ctx, [q], 3, 53, 5, [0])[0] == o.encode_frame(q, 3, 53, 5, 12, 0)[0]


@pytest.mark.parametrize("plain,adjacent", [(False, 0), (True, 0), (False, 1)])
def test_stream_path_codestreams_match_the_coder(plain, adjacent):
    """config.codestream_bpp: every frame's container from the stream path
    (coded in the batch's launches, first frames included) equals the coder
    applied to that frame's coefficient plane (whose parity with the oracle
    the tests above establish)."""
    h, w, S, n = 256, 320, 3, 3
    flags = F.MANUAL | (F.PLAIN if plain else 0)
    with F.Context(pyr_levels=3, dwt_levels=3, wavelet=97, codestream_bpp=1.0, flags=flags, adjacent=adjacent) as c:
        seqs = [np.asarray(sequence_u16(700 + s, n, h, w, 8)).astype(np.uint16) for s in range(S)]
        for t in range(n):
            for s in range(S):
                F.flowroi_submit_frame(c.h, s, seqs[s][t], t, 12)
            F.flowroi_step(c.h)
        F.flowroi_flush(c.h, 60000)
        cap = F.flowroi_codestream_bound(w, h, 3)
        for s in range(S):
            for t in range(n):
                coeffs = np.empty((h, w), np.int32)
                F.flowroi_get_coeffs(c.h, s, t, coeffs, 10000)
                out = np.zeros(cap, np.uint8)
                k = F.flowroi_get_codestream(c.h, s, t, out, 10000)
                want = np.zeros(cap, np.uint8)
                m = F.flowroi_encode_codestreams(c.h, [dict(coeffs=coeffs, out=want, levels=3, wavelet=97, shift=5,
                                                            bit_depth=12, budget=h * w // 8)])[0]
                assert k == m and bytes(out[:k]) == bytes(want[:m]), (s, t)
                dev = torch.zeros(cap, dtype=torch.uint8, device="cuda")
                assert F.flowroi_get_codestream(c.h, s, t, dev, 10000) == k
                assert bytes(dev[:k].cpu().numpy()) == bytes(out[:k])
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_codestream(c.h, 0, 1, np.zeros(64, np.uint8), 10000)
        assert ei.value.code == F.ERANGE


def test_stream_path_codestream_off_is_einval():
    with F.Context(pyr_levels=2, dwt_levels=2, flags=F.MANUAL) as c:
        F.flowroi_submit_frame(c.h, 0, np.zeros((64, 64), np.uint16), 0, 12)
        F.flowroi_flush(c.h, 60000)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_codestream(c.h, 0, 0, np.zeros(1024, np.uint8), 10000)
        assert ei.value.code == F.EINVAL


def test_stream_path_out_of_range_coefficients_are_erange():
    """16-bit frames with a 15-bit RoI up-shift give magnitudes of 2^24 and
    more: the frame's container is refused with FLOWROI_ERANGE, its
    coefficients are still delivered, and the context keeps working."""
    h = w = 128
    rng = np.random.default_rng(5)
    with F.Context(pyr_levels=2, dwt_levels=2, wavelet=53, scale_shift=15, codestream_bpp=2.0, flags=F.MANUAL) as c:
        frames = [rng.integers(0, 65536, (h, w)).astype(np.uint16) for _ in range(3)]
        for t, fr in enumerate(frames):
            F.flowroi_submit_frame(c.h, 0, fr, t, 16)
        F.flowroi_flush(c.h, 60000)
        coeffs = np.empty((h, w), np.int32)
        F.flowroi_get_coeffs(c.h, 0, 2, coeffs, 10000)
        mask = np.empty((h, w), np.uint8)
        F.flowroi_get_mask(c.h, 0, 2, mask, 10000)
        assert mask.any() and np.abs(coeffs.astype(np.int64)).max() >= 1 << 24
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_get_codestream(c.h, 0, 2, np.zeros(F.flowroi_codestream_bound(w, h, 2), np.uint8), 10000)
        assert ei.value.code == F.ERANGE
        # the first frame has no RoI, so no shift: its container is there
        assert F.flowroi_get_codestream(c.h, 0, 0, np.zeros(F.flowroi_codestream_bound(w, h, 2), np.uint8), 10000) > 0


# ------------------------------------------------ JPEG2000 codestreams --

@pytest.mark.parametrize("h,w,levels,wavelet,bpp", [(256, 256, 3, 53, 0.0), (200, 264, 3, 97, 1.0),
                                                     (16, 16, 2, 53, 0.0), (512, 512, 5, 97, 0.25),
                                                     (192, 320, 4, 97, 3.0)])
def test_j2c_codestream_matches_oracle(ctx, h, w, levels, wavelet, bpp):
    """format CS_J2C: the GPU's JPEG2000 Part 1 codestream equals the
    oracle's byte for byte, and the independent parser reads back the same
    passes as the container of the same frame."""
    q = _planes(h * 3 + w + levels, h, w, levels, wavelet, 5)
    budget = int(bpp * h * w / 8)
    want, _ = o.encode_frame(q, levels, wavelet, 5, 12, budget, fmt="j2c")
    got = _gpu(ctx, [q], levels, wavelet, 5, [budget], fmt=F.CS_J2C)[0]
    assert got == want
    cont = _gpu(ctx, [q], levels, wavelet, 5, [budget])[0]
    assert parse(got)["blocks"] == _container_blocks(cont)


def test_j2c_full_size_2048_97_at_one_bit_per_pixel(ctx):
    h = w = 2048
    q = _planes(3000, h, w, 5, 97, 5)
    budget = h * w // 8
    want, _ = o.encode_frame(q, 5, 97, 5, 12, budget, fmt="j2c")
    got = _gpu(ctx, [q], 5, 97, 5, [budget], on_device=True, fmt=F.CS_J2C)[0]
    assert got == want


def test_j2c_large_bands_tag_trees_in_global_scratch(ctx):
    """A 6144^2 frame at one level: each band has 48 x 48 code-blocks, whose
    tag trees no longer fit the writer's shared memory, so every band is
    written with its trees in global scratch.  Sparse coefficients keep the
    coding short."""
    h = w = 6144
    rng = np.random.default_rng(6144)
    q = np.zeros((h, w), np.int32)
    idx = rng.choice(h * w, 1500, replace=False)
    q.flat[idx] = rng.integers(-3000, 3001, size=idx.size)
    want, _ = o.encode_frame(q, 1, 53, 5, 12, 0, fmt="j2c")
    got = _gpu(ctx, [q], 1, 53, 5, [0], on_device=True, fmt=F.CS_J2C)[0]
    assert got == want


def test_j2c_in_the_stream_path():
    """config.codestream_format = CS_J2C: each frame's codestream from the
    stream path equals the coder's codestream of that frame's coefficients,
    and it parses."""
    h, w, S, n = 256, 320, 2, 3
    with F.Context(pyr_levels=3, dwt_levels=3, wavelet=97, codestream_bpp=1.0, codestream_format=F.CS_J2C,
                   flags=F.MANUAL) as c:
        seqs = [np.asarray(sequence_u16(710 + s, n, h, w, 8)).astype(np.uint16) for s in range(S)]
        for t in range(n):
            for s in range(S):
                F.flowroi_submit_frame(c.h, s, seqs[s][t], t, 12)
            F.flowroi_step(c.h)
        F.flowroi_flush(c.h, 60000)
        cap = F.flowroi_codestream_bound(w, h, 3)
        for s in range(S):
            for t in range(n):
                coeffs = np.empty((h, w), np.int32)
                F.flowroi_get_coeffs(c.h, s, t, coeffs, 10000)
                out = np.zeros(cap, np.uint8)
                k = F.flowroi_get_codestream(c.h, s, t, out, 10000)
                want, _ = o.encode_frame(coeffs, 3, 97, 5, 12, h * w // 8, fmt="j2c")
                assert bytes(out[:k]) == want, (s, t)
                info = parse(want)
                assert (info["w"], info["h"], info["levels"]) == (w, h, 3)


# ------------------------------- contexts reset at every pass (style 0x02) --

@pytest.mark.parametrize("h,w,levels,wavelet,bpp,fmt", [(256, 256, 3, 53, 0.0, 0), (200, 264, 3, 97, 1.0, 0),
                                                         (512, 512, 5, 97, 0.25, 1), (192, 320, 4, 53, 0.0, 1)])
def test_reset_style_matches_oracle(ctx, h, w, levels, wavelet, bpp, fmt):
    """reset = 1: every pass coded from the initial context states (the
    per-pass MQ state stage instead of the per-block chains), containers
    and codestreams byte for byte the oracle's."""
    q = _planes(h * 5 + w + levels, h, w, levels, wavelet, 5)
    budget = int(bpp * h * w / 8)
    want, _ = o.encode_frame(q, levels, wavelet, 5, 12, budget, fmt="j2c" if fmt else "container", reset=True)
    got = _gpu(ctx, [q], levels, wavelet, 5, [budget], fmt=fmt, resets=[1])[0]
    assert got == want


def test_reset_and_carried_styles_in_one_call(ctx):
    """Frames of both styles in one call: both MQ state stages run, each on
    its own frames, and every container is the oracle's."""
    qs = [_planes(900 + i, 192, 256, 3, 97, 5) for i in range(4)]
    resets = [1, 0, 0, 1]
    budgets = [6000, 6000, 0, 0]
    got = _gpu(ctx, qs, 3, 97, 5, budgets, resets=resets)
    for q, b, r, g in zip(qs, budgets, resets, got):
        assert g == o.encode_frame(q, 3, 97, 5, 12, b, reset=bool(r))[0]


def test_reset_full_size_2048_97_at_one_bit_per_pixel(ctx):
    h = w = 2048
    q = _planes(3001, h, w, 5, 97, 5)
    budget = h * w // 8
    want, _ = o.encode_frame(q, 5, 97, 5, 12, budget, reset=True)
    got = _gpu(ctx, [q], 5, 97, 5, [budget], on_device=True, resets=[1])[0]
    assert got == want


def test_reset_in_the_stream_path():
    """config.codestream_reset = 1 in the stream path (captured launches):
    each frame's container is the oracle's coding of that frame's
    coefficients with the contexts reset at every pass."""
    h, w, S, n = 256, 320, 2, 3
    with F.Context(pyr_levels=3, dwt_levels=3, wavelet=97, codestream_bpp=1.0, codestream_reset=1,
                   flags=F.MANUAL) as c:
        seqs = [np.asarray(sequence_u16(730 + s, n, h, w, 8)).astype(np.uint16) for s in range(S)]
        for t in range(n):
            for s in range(S):
                F.flowroi_submit_frame(c.h, s, seqs[s][t], t, 12)
            F.flowroi_step(c.h)
        F.flowroi_flush(c.h, 60000)
        cap = F.flowroi_codestream_bound(w, h, 3)
        for s in range(S):
            for t in range(n):
                coeffs = np.empty((h, w), np.int32)
                F.flowroi_get_coeffs(c.h, s, t, coeffs, 10000)
                out = np.zeros(cap, np.uint8)
                k = F.flowroi_get_codestream(c.h, s, t, out, 10000)
                want, _ = o.encode_frame(coeffs, 3, 97, 5, 12, h * w // 8, reset=True)
                assert bytes(out[:k]) == want, (s, t)
