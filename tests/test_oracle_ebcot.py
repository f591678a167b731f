"""Pins of the embedded block coder in the oracle (orc_ebcot.c, oracle.py):
the JPEG2000 coder that the paper applies to the RoI-shifted coefficients
(§Implementation details, Table 1), written from the JPEG2000 Part 1
definitions (MQ coder, Annex C; coding passes, Annex D; rate control,
Annex J).

What fixes the oracle here, other than the oracle itself:
  - information theory: an adaptive binary arithmetic coder decodes its own
    output exactly and spends close to the entropy of an i.i.d. source (the
    probability table and its state transitions are what bring it there);
  - invertibility: decoding every pass of a code-block returns the
    coefficients exactly, for every sub-band orientation and block shape;
  - the distortion bookkeeping: after any number of passes, the decoder's
    midpoint reconstruction has exactly the initial error energy minus the
    encoder's reported decreases (an integer identity in doubled units);
  - the reversible chain: 5/3 transform -> code -> container -> decode ->
    inverse transform returns the 12-bit frame bit-exactly;
  - rate control: the kept bytes fit the budget, grow with it, and each
    block's hull is the brute-force upper concave envelope of its
    (bytes, distortion) truncation points.
"""
import struct

import numpy as np
import pytest

from oracle import oracle as o
from synth import sequence_u16

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("seed,p", [(1, 0.02), (2, 0.2), (3, 0.5), (4, 0.9)])
def test_mq_roundtrip(seed, p):
    rng = np.random.default_rng(seed)
    n = 50000
    d = (rng.random(n) < p).astype(np.uint8)
    cx = rng.integers(0, 19, n).astype(np.uint8)
    code, out = o.mq_roundtrip(d, cx)
    assert np.array_equal(out, d)
    assert len(code) > 0


def test_mq_runs_of_one_symbol_cost_almost_nothing():
    n = 100000
    code, out = o.mq_roundtrip(np.zeros(n, np.uint8), np.zeros(n, np.uint8))
    assert np.all(out == 0) and len(code) < 16


@pytest.mark.parametrize("p", [0.01, 0.05, 0.1, 0.3, 0.5])
def test_mq_rate_close_to_entropy(p):
    """An i.i.d. Bernoulli(p) source in one context: the codeword is within
    8% of n H(p) bits (the MQ coder's adaptive estimate is within a few
    per cent of the entropy; a wrong probability table or transition would
    not be)."""
    rng = np.random.default_rng(int(p * 1000))
    n = 200000
    d = (rng.random(n) < p).astype(np.uint8)
    code, out = o.mq_roundtrip(d, np.zeros(n, np.uint8))
    assert np.array_equal(out, d)
    H = -(p * np.log2(p) + (1 - p) * np.log2(1 - p))
    assert 8 * len(code) / n <= 1.08 * H


def _block(rng, h, w, scale, zero_frac):
    q = np.round(rng.standard_normal((h, w)) * scale).astype(np.int64)
    q[rng.random((h, w)) < zero_frac] = 0
    return np.clip(q, -(2 ** 30), 2 ** 30).astype(np.int32)


@pytest.mark.parametrize("ori", [o.ORI_LL, o.ORI_HL, o.ORI_LH, o.ORI_HH])
@pytest.mark.parametrize("h,w,scale,zero_frac", [(64, 64, 40.0, 0.3), (64, 64, 3.0, 0.8), (17, 64, 1e5, 0.0),
                                                 (64, 9, 700.0, 0.5), (1, 1, 5.0, 0.0), (3, 5, 2 ** 20, 0.2), (64, 64, 2 ** 21, 0.1)])
def test_t1_roundtrip_and_pass_count(ori, h, w, scale, zero_frac):
    rng = np.random.default_rng(h * 131 + w * 7 + ori)
    q = _block(rng, h, w, scale, zero_frac)
    planes, plen, dist, code = o.t1_encode(q, ori)
    mx = int(np.abs(q.astype(np.int64)).max())
    assert planes == mx.bit_length()
    assert len(plen) == (3 * planes - 2 if planes else 0)
    assert np.all(plen >= 1) and code.size == plen.sum()
    r = o.t1_decode(code, plen, len(plen), planes, w, h, ori, midpoint=False)
    assert np.array_equal(r, q)


def test_t1_rejects_magnitudes_of_2_to_24():
    q = np.zeros((8, 8), np.int32)
    q[3, 4] = -(2 ** 24)
    with pytest.raises(OverflowError):
        o.t1_encode(q, o.ORI_LL)


def test_t1_all_zero_block_has_no_passes():
    planes, plen, dist, code = o.t1_encode(np.zeros((64, 64), np.int32), o.ORI_HH)
    assert planes == 0 and len(plen) == 0 and code.size == 0


@pytest.mark.parametrize("ori", [o.ORI_LL, o.ORI_HL, o.ORI_LH, o.ORI_HH])
def test_t1_distortion_decreases_match_the_decoder(ori):
    """After k passes the decoder's midpoint reconstruction r has squared
    error sum((2q - 2r)^2) = sum((2q)^2) - (d_1 + ... + d_k), exactly."""
    rng = np.random.default_rng(40 + ori)
    q = _block(rng, 64, 64, 300.0, 0.3)
    planes, plen, dist, code = o.t1_encode(q, ori)
    t = 2 * q.astype(np.int64)
    total = float((t * t).sum())
    cum = np.concatenate([[0.0], np.cumsum(dist)])
    assert cum[-1] == total
    for k in range(len(plen) + 1):
        r = o.t1_decode(code, plen, k, planes, 64, 64, ori, midpoint=True).astype(np.int64)
        e = float(((t - 2 * r) ** 2).sum())
        assert e == total - cum[k], k
    assert np.all(dist >= 0)


@pytest.mark.parametrize("ori", [o.ORI_LL, o.ORI_HL, o.ORI_LH, o.ORI_HH])
@pytest.mark.parametrize("h,w,scale,zero_frac", [(64, 64, 300.0, 0.3), (64, 64, 3.0, 0.8), (17, 40, 2 ** 20, 0.1)])
def test_t1_reset_codes_the_same_decisions(ori, h, w, scale, zero_frac):
    """Resetting the contexts at every pass changes how the MQ coder codes
    each pass's decisions, never which decisions are coded: so the passes'
    distortion decreases are those of the carried-contexts coder, decoding
    the first k passes of either stream gives the same coefficients for
    every k, and the first pass (which starts from the initial states either
    way) is the same codeword.  A later pass that starts from learned states
    gives a different codeword, and a reset stream decoded with carried
    contexts does not come back."""
    rng = np.random.default_rng(h * 17 + w + ori)
    q = _block(rng, h, w, scale, zero_frac)
    planes, plen, dist, code = o.t1_encode(q, ori)
    planes_r, plen_r, dist_r, code_r = o.t1_encode(q, ori, reset=True)
    assert planes_r == planes and len(plen_r) == len(plen)
    assert np.array_equal(dist_r, dist)
    for k in range(len(plen) + 1):
        a = o.t1_decode(code, plen, k, planes, w, h, ori, midpoint=False)
        b = o.t1_decode(code_r, plen_r, k, planes, w, h, ori, midpoint=False, reset=True)
        assert np.array_equal(a, b), k
    assert np.array_equal(b, q)
    assert plen_r[0] == plen[0] and bytes(code_r[:plen[0]]) == bytes(code[:plen[0]])
    ends, ends_r = np.cumsum(plen), np.cumsum(plen_r)
    assert any(bytes(code[ends[k - 1]:ends[k]]) != bytes(code_r[ends_r[k - 1]:ends_r[k]]) for k in range(1, len(plen)))
    wrong = o.t1_decode(code_r, plen_r, len(plen_r), planes, w, h, ori, midpoint=False)
    assert not np.array_equal(wrong, q)


def test_t1_reset_passes_are_independent_codewords():
    """With the contexts reset and every pass terminated, a pass's codeword
    depends only on that pass's decisions: two blocks whose top bit-planes
    differ but whose lower planes (and significance by then) agree give the
    same codewords for the passes of those lower planes.  Block b is block a
    with one already-significant coefficient's top bits changed, which
    changes the decisions of the top passes only (its refinement bits
    there) and, with carried contexts, the states every later pass starts
    from."""
    rng = np.random.default_rng(7)
    a = _block(rng, 64, 64, 200.0, 0.4)
    a[5, 9] = 4000   # 12 planes; planes 0..9 of the others stay below 2^10
    b = a.copy()
    b[5, 9] = 4000 ^ (1 << 10)   # 2976: same top plane (11), bit 10 flipped
    assert int(np.abs(a).max()).bit_length() == int(np.abs(b).max()).bit_length() == 12
    assert int(np.abs(np.delete(a.ravel(), 5 * 64 + 9)).max()) < 1 << 10
    pa, la, _, ca = o.t1_encode(a, o.ORI_HH, reset=True)
    pb, lb, _, cb = o.t1_encode(b, o.ORI_HH, reset=True)
    ea, eb = np.concatenate([[0], np.cumsum(la)]), np.concatenate([[0], np.cumsum(lb)])
    # pass index of plane p's significance pass: 1 + 3 (planes - 2 - p)
    first_same = 1 + 3 * (pa - 2 - 9)
    for k in range(first_same, len(la)):
        assert bytes(ca[ea[k]:ea[k + 1]]) == bytes(cb[eb[k]:eb[k + 1]]), k
    kr = 1 + 3 * (pa - 2 - 10) + 1   # plane 10's refinement pass: one decision, 1 in a, 0 in b
    assert bytes(ca[ea[kr]:ea[kr + 1]]) != bytes(cb[eb[kr]:eb[kr + 1]])
    _, lc, _, cc = o.t1_encode(a, o.ORI_HH)
    _, ld, _, cd = o.t1_encode(b, o.ORI_HH)
    ec, ed = np.concatenate([[0], np.cumsum(lc)]), np.concatenate([[0], np.cumsum(ld)])
    assert any(bytes(cc[ec[k]:ec[k + 1]]) != bytes(cd[ed[k]:ed[k + 1]]) for k in range(first_same, len(lc)))


def _frame(seed, h, w, bd=12):
    return np.asarray(sequence_u16(seed, 1, h, w, 6)[0]).astype(np.uint16)


@pytest.mark.parametrize("h,w,levels", [(256, 256, 3), (192, 320, 4), (64, 64, 2)])
def test_lossless_5_3_frame_roundtrip(h, w, levels):
    """5/3 is reversible: transform, code every pass, parse the container,
    decode, inverse transform, undo the DC shift: the frame comes back
    bit-exactly."""
    bd = 12
    raw = _frame(h * 3 + w, h, w, bd)
    y = o.dwt2d(o.dc_shift(raw, bd).astype(np.int64), 53, levels)
    stream, blocks = o.encode_frame(y, levels, 53, 0, bd, 0)
    r = o.decode_frame(stream, midpoint=False)
    assert np.array_equal(r, y)
    x = o.reconstruct(r, levels, 53, bd)
    assert np.array_equal(x, raw.astype(np.int64))


def test_container_layout():
    bd, levels = 12, 3
    raw = _frame(9, 128, 192, bd)
    y = o.dwt2d(o.dc_shift(raw, bd).astype(np.int64), 53, levels)
    stream, blocks = o.encode_frame(y, levels, 53, 5, bd, 0)
    magic, ver, w, h, wav, lv, sh, b, nb, nbytes, _ = struct.unpack_from("<4sIIIBBBBIII", stream, 0)
    assert (magic, ver, w, h, wav, lv, sh, b) == (b"FRJ2", 1, 192, 128, 53, 3, 5, 12)
    cbs = o.codeblocks(192, 128, levels)
    assert nb == len(cbs) == len(blocks)
    assert len(stream) == 32 + 16 * nb + nbytes
    prev = -1
    for i, (band, ori, x0, y0, cw, ch) in enumerate(cbs):
        off, ex0, ey0, cw1, ch1, eb, planes, npass, k, _ = struct.unpack_from("<IHHBBBBBBH", stream, 32 + 16 * i)
        assert (ex0, ey0, cw1 + 1, ch1 + 1, eb) == (x0, y0, cw, ch, band)
        assert off > prev and k == npass
        prev = off
    # every coefficient belongs to exactly one code-block
    cover = np.zeros((128, 192), np.int32)
    for band, ori, x0, y0, cw, ch in cbs:
        cover[y0:y0 + ch, x0:x0 + cw] += 1
    assert np.all(cover == 1)


def _brute_hull(R, D):
    """Points on the upper concave envelope, by definition: k is on it iff
    no chord between points on either side lies at or above it."""
    n = len(R) - 1
    on = [0]
    for k in range(1, n + 1):
        if D[k] <= max(D[j] for j in range(k)):
            continue
        ok = True
        for a in range(k):
            for b in range(k + 1, n + 1):
                if D[b] <= D[a]:
                    continue
                t = (R[k] - R[a]) / (R[b] - R[a])
                if D[a] + t * (D[b] - D[a]) >= D[k]:
                    ok = False
        if ok:
            on.append(k)
    return on


def test_rate_control_hull_and_budget():
    bd, levels = 12, 3
    raw = _frame(21, 256, 256, bd)
    y = o.dwt2d(o.dc_shift(raw, bd).astype(np.float64), 97, levels)
    _, delta, _, _ = o.delta_table(levels, bd)
    q = o.quantise_f64(y, levels, delta)
    stream, blocks = o.encode_frame(q, levels, 97, 0, bd, 0)
    full = sum(int(b["plen"].sum()) for b in blocks)
    for b in blocks[:40]:
        if len(b["plen"]) == 0:
            continue
        hk, hs, R = o.hull(b["plen"], b["dist"])
        D = np.concatenate([[0.0], np.cumsum(b["dist"])])
        assert list(hk) == _brute_hull(list(R), list(D))
        assert np.all(np.diff(hs[1:]) < 0)
    kept_prev = -1
    for frac in [0.02, 0.05, 0.1, 0.3, 0.6, 1.0]:
        budget = int(frac * full)
        nk = o.pcrd(blocks, budget)
        kept = sum(int(b["plen"][:k].sum()) for b, k in zip(blocks, nk))
        assert kept <= budget
        assert kept >= kept_prev
        kept_prev = kept
    assert o.pcrd(blocks, 0) == [len(b["plen"]) for b in blocks]


def test_lossy_9_7_psnr_grows_with_rate():
    """The quantised 9/7 frame coded at increasing budgets decodes to
    increasing PSNR; every pass kept gives the quantiser's own error."""
    bd, levels = 12, 3
    raw = _frame(33, 256, 256, bd)
    y = o.dwt2d(o.dc_shift(raw, bd).astype(np.float64), 97, levels)
    _, delta, _, _ = o.delta_table(levels, bd)
    q = o.quantise_f64(y, levels, delta)
    zero = np.zeros_like(q, dtype=np.uint8)
    _, blocks = o.encode_frame(q, levels, 97, 0, bd, 0)
    full = sum(int(b["plen"].sum()) for b in blocks)
    ps = []
    for frac in [0.05, 0.15, 0.4, 1.0]:
        stream, _ = o.encode_frame(q, levels, 97, 0, bd, int(frac * full))
        r = o.decode_frame(stream)
        x = o.reconstruct(o.unshift_dequantise(r, zero, 0, levels, 97, bd), levels, 97, bd)
        ps.append(o.psnr(x, raw, bd))
    assert all(b > a for a, b in zip(ps, ps[1:])), ps
    assert ps[-1] > 45.0


def test_roi_upshift_keeps_the_roi_quality_at_low_rates():
    """Scaling-based RoI (§Implementation details, Table 1): with the RoI
    coefficients shifted up by 5 bits, a 0.5 bit-per-pixel codestream
    spends its bytes on the RoI first: the RoI's PSNR is far above the
    background's, and above what the same budget gives the RoI unshifted."""
    bd, levels, s = 12, 3, 5
    h = w = 256
    raw = _frame(57, h, w, bd)
    pix = np.zeros((h, w), np.uint8)
    pix[64:192, 64:192] = 1
    cm = o.wavelet_mask(pix, levels, 97)
    y = o.dwt2d(o.dc_shift(raw, bd).astype(np.float64), 97, levels)
    _, delta, _, _ = o.delta_table(levels, bd)
    q = o.quantise_f64(y, levels, delta)
    budget = int(0.5 * h * w / 8)

    def code(shift):
        qs = o.roi_shift(q, cm, shift) if shift else q
        stream, _ = o.encode_frame(qs, levels, 97, shift, bd, budget)
        r = o.decode_frame(stream)
        return o.reconstruct(o.unshift_dequantise(r, cm, shift, levels, 97, bd), levels, 97, bd)

    x5, x0 = code(s), code(0)
    m = pix.astype(bool)
    roi5, bg5 = o.psnr(x5[m], raw[m], bd), o.psnr(x5[~m], raw[~m], bd)
    roi0 = o.psnr(x0[m], raw[m], bd)
    assert roi5 > bg5 + 6.0, (roi5, bg5)
    assert roi5 > roi0 + 2.0, (roi5, roi0)


def test_mq_table_structure():
    """The probability-state machine of the MQ coder (Annex C, Table C.2)
    has a fixed shape, independent of the exact Qe values: two fast-attack
    MPS chains (states 0-5 and 6-13) that join a steady chain (14-45, ending
    in a self-loop), the MPS sense exchanged by an LPS only in the three
    states whose estimate is 1/2 (0, 6, 14), an MPS always lowering the LPS
    estimate Qe along a chain, an LPS never lowering it, and state 46 the
    fixed uniform state that nothing enters.  A typo in a transition or an
    out-of-order Qe breaks one of these even where the coder still decodes
    its own output."""
    qe, nmps, nlps, sw = o.mq_table()
    assert len(qe) == 47
    assert set(np.flatnonzero(sw)) == {0, 6, 14}
    assert all(qe[i] == 0x5601 for i in (0, 6, 14, 46)) and qe.max() == 0x5601 and qe.min() > 0
    # the uniform state
    assert nmps[46] == 46 and nlps[46] == 46
    assert 46 not in set(nmps[:46]) | set(nlps[:46])
    # MPS chains
    for i in range(46):
        if i in (5, 13):
            assert nmps[i] >= 14  # a fast-attack chain ends in the steady chain
        elif i == 45:
            assert nmps[i] == 45
        else:
            assert nmps[i] == i + 1
        if i != 45:
            assert qe[nmps[i]] < qe[i], i
    # LPS transitions
    for i in range(46):
        if sw[i]:
            assert nlps[i] in (i, i + 1)
        else:
            assert qe[nlps[i]] > qe[i], i
        if i >= 6:
            assert 14 <= nlps[i] <= 45 or (i < 14 and nlps[i] == 6)  # never back to a fast-attack chain
        else:
            assert nlps[i] >= 1
    assert all(nlps[i] >= 6 for i in range(1, 6))


def test_context_rules_structure():
    """Zero coding (Table D.1): labels 0..8, label 0 exactly for an
    insignificant neighbourhood, every label used, the label never falling
    when a neighbour becomes significant, HL the LH rule with horizontal
    and vertical swapped, LL the same rule as LH, and HH driven by the
    diagonals first.  Sign coding (Table D.3): labels 9..13, label 9 and no
    flip for no contribution, and negating both contributions keeps the
    label and flips the predicted sign."""
    zc, sc, fl = o.context_tables()
    for ori in range(4):
        t = zc[ori]  # [d, v, h]
        assert t.min() == 0 and t.max() == 8 and set(t.ravel()) == set(range(9))
        assert (t == 0).sum() == 1 and t[0, 0, 0] == 0
        assert (np.diff(t, axis=0) >= 0).all() and (np.diff(t, axis=1) >= 0).all() and (np.diff(t, axis=2) >= 0).all()
    assert (zc[0] == zc[2]).all()
    assert (zc[1] == zc[2].transpose(0, 2, 1)).all()
    assert not (zc[1] == zc[2]).all()
    # HH: the diagonal count dominates (one more diagonal outranks any h + v
    # once d >= 1), LH: two horizontal neighbours give the top label
    assert zc[3][3:].min() == 8 and zc[3][2].max() == 7 and (zc[2][:, :, 2] == 8).all()
    assert set(sc.ravel()) == set(range(9, 14)) and sc[1, 1] == 9 and fl[1, 1] == 0
    for v in range(3):
        for h in range(3):
            if (h, v) != (1, 1):
                assert sc[v, h] == sc[2 - v, 2 - h] and fl[v, h] != fl[2 - v, 2 - h]
