"""The oracle's JPEG2000 Part 1 codestream (oracle.codestream_j2c) against a
parser written here from the decoding side of the standard (ISO/IEC
15444-1 Annex A markers, Annex B packets: tag trees, number of coding
passes, Lblock and segment lengths, bit unstuffing): every code-block's
bit-plane count, kept passes, pass lengths and bytes read back from the
codestream equal those of the frame container built from the same passes,
and a lossless 5/3 frame decodes back bit-exactly.  The primitives are
pinned separately: Table B.4's codewords, the stuffed bit after 0xFF,
tag trees round-tripped on random grids."""
import struct

import numpy as np
import pytest

from oracle import oracle as O


class BitReader:
    """Packet-header bits, MSB first, skipping the stuffed MSB of a byte
    that follows 0xFF (Annex B.10.1)."""

    def __init__(self, buf: bytes, pos: int):
        self.buf, self.pos = buf, pos
        self.byte, self.left, self.prev = 0, 0, 0

    def bit(self) -> int:
        if self.left == 0:
            self.prev = self.byte if self.pos > 0 else 0
            self.byte = self.buf[self.pos]
            self.pos += 1
            self.left = 7 if self.prev == 0xFF else 8
        self.left -= 1
        return (self.byte >> self.left) & 1

    def bits(self, n: int) -> int:
        v = 0
        for _ in range(n):
            v = (v << 1) | self.bit()
        return v

    def end(self) -> int:
        """Offset of the first byte after the header (the header never ends
        on 0xFF: a byte after a final 0xFF belongs to the header)."""
        return self.pos + (1 if self.byte == 0xFF and self.pos > 0 else 0)


class TagTreeDecoder:
    def __init__(self, nx: int, ny: int):
        self.levels = []
        w, h = nx, ny
        while True:
            self.levels.append((w, h))
            if w == 1 and h == 1:
                break
            w, h = (w + 1) // 2, (h + 1) // 2
        self.low = [[0] * (w * h) for w, h in self.levels]
        self.val = [[None] * (w * h) for w, h in self.levels]

    def decode(self, br: BitReader, x: int, y: int, threshold: int):
        """The leaf's value if it is below `threshold`, else None."""
        path = []
        for lw, lh in self.levels:
            path.append(y * lw + x)
            x, y = x // 2, y // 2
        low = 0
        for l in range(len(self.levels) - 1, -1, -1):
            i = path[l]
            low = max(low, self.low[l][i])
            if self.val[l][i] is None:
                while low < threshold:
                    if br.bit():
                        self.val[l][i] = low
                        break
                    low += 1
            self.low[l][i] = low
        v = self.val[0][path[0]]
        return v if v is not None and v < threshold else None


def num_passes(br: BitReader) -> int:
    if br.bit() == 0:
        return 1
    if br.bit() == 0:
        return 2
    v = br.bits(2)
    if v < 3:
        return 3 + v
    v = br.bits(5)
    if v < 31:
        return 6 + v
    return 37 + br.bits(7)


def parse(cs: bytes, levels_expected=None):
    """Markers and packets -> dict(w, h, levels, wavelet, bit_depth, guard,
    eps, mu, blocks: {(band, x0, y0): (planes, [pass lengths], bytes)})."""
    assert cs[:2] == b"\xff\x4f"
    p = 2
    info = {}
    while True:
        m, L = struct.unpack_from(">HH", cs, p)
        seg = cs[p + 4:p + 2 + L]
        if m == 0xFF51:
            _, w, h, xo, yo, tw, th, txo, tyo, nc, ss, xr, yr = struct.unpack(">HIIIIIIIIHBBB", seg)
            assert (xo, yo, txo, tyo, nc, xr, yr) == (0, 0, 0, 0, 1, 1, 1) and (tw, th) == (w, h) and L == 41
            info.update(w=w, h=h, bit_depth=(ss & 0x7F) + 1)
        elif m == 0xFF52:
            scod, prog, nl, mct, D, xcb, ycb, style, tr = struct.unpack(">BBHBBBBBB", seg)
            assert (scod, prog, nl, mct, xcb, ycb, L) == (0, 0, 1, 0, 4, 4, 12)
            # code-block style byte: termination on each coding pass (0x04),
            # optionally with the contexts reset on pass boundaries (0x02)
            assert style in (0x04, 0x06)
            info.update(levels=D, wavelet=53 if tr == 1 else 97, style=style)
        elif m == 0xFF5C:
            sq = seg[0]
            info["guard"] = sq >> 5
            nb = 3 * info["levels"] + 1
            if sq & 0x1F == 0:
                assert L == 3 + nb
                info["eps"] = [b >> 3 for b in seg[1:1 + nb]]
                info["mu"] = [0] * nb
            else:
                assert sq & 0x1F == 2 and L == 3 + 2 * nb
                vals = struct.unpack(">" + "H" * nb, seg[1:1 + 2 * nb])
                info["eps"] = [v >> 11 for v in vals]
                info["mu"] = [v & 0x7FF for v in vals]
        elif m == 0xFF90:
            isot, psot, tp, tn = struct.unpack(">HIBB", seg)
            assert (L, isot, tp, tn) == (10, 0, 0, 1)
            sot_at = p
            p += 2 + L
            break
        else:
            raise AssertionError(f"unexpected marker {m:04x}")
        p += 2 + L
    assert cs[p:p + 2] == b"\xff\x93"
    p += 2
    assert sot_at + psot == len(cs) - 2 and cs[-2:] == b"\xff\xd9"
    D, w, h = info["levels"], info["w"], info["h"]
    # band order of QCD: LL_D, HL_D, LH_D, HH_D, ..., HL_1, LH_1, HH_1 -> table index
    order = [3 * D] + [3 * (l - 1) + o for l in range(D, 0, -1) for o in range(3)]
    eps = {b: info["eps"][i] for i, b in enumerate(order)}
    blocks = {}
    bands_of_res = [[(3 * D, 0, 0, w >> D, h >> D)]]
    for l in range(D, 0, -1):
        bw, bh = w >> l, h >> l
        bands_of_res.append([(3 * (l - 1), bw, 0, bw, bh), (3 * (l - 1) + 1, 0, bh, bw, bh),
                             (3 * (l - 1) + 2, bw, bh, bw, bh)])
    for bands in bands_of_res:
        br = BitReader(cs, p)
        got = []
        if br.bit():
            for b, bx, by, bw, bh in bands:
                if bw == 0 or bh == 0:
                    continue
                nx, ny = (bw + 63) // 64, (bh + 63) // 64
                incl, zbp = TagTreeDecoder(nx, ny), TagTreeDecoder(nx, ny)
                Mb = info["guard"] + eps[b] - 1
                for cy in range(ny):
                    for cx in range(nx):
                        if incl.decode(br, cx, cy, 1) is None:
                            continue
                        z = zbp.decode(br, cx, cy, 1 << 30)
                        n = num_passes(br)
                        k = 0
                        while br.bit():
                            k += 1
                        lens = [br.bits(3 + k) for _ in range(n)]
                        got.append(((b, bx + 64 * cx, by + 64 * cy), Mb - z, lens))
        p = br.end()
        for key, planes, lens in got:
            nbytes = sum(lens)
            blocks[key] = (planes, lens, cs[p:p + nbytes])
            p += nbytes
    assert p == len(cs) - 2
    info["blocks"] = blocks
    return info


def _container_blocks(stream: bytes):
    _, _, w, h, wav, levels, shift, bd, nb, _, _ = struct.unpack_from("<4sIIIBBBBIII", stream, 0)
    out = {}
    base = 32 + 16 * nb
    for i in range(nb):
        off, x0, y0, _, _, band, planes, _, k, _ = struct.unpack_from("<IHHBBBBBBH", stream, 32 + 16 * i)
        lens = list(np.frombuffer(stream, "<u2", k, base + off).astype(int))
        code = stream[base + off + 2 * k: base + off + 2 * k + sum(lens)]
        if k:
            out[(band, x0, y0)] = (planes, lens, code)
    return out


def _frame(seed, h, w, scale):
    rng = np.random.default_rng(seed)
    q = np.rint(rng.laplace(0, scale, (h, w))).astype(np.int32)
    q[: h // 3, : w // 4] <<= 5  # an up-shifted region
    return q


@pytest.mark.parametrize("h,w,levels,wavelet,budget", [
    (192, 320, 3, 53, 0), (256, 256, 4, 97, 9000), (128, 192, 2, 97, 0), (64, 64, 1, 53, 200)])
def test_codestream_carries_the_containers_passes(h, w, levels, wavelet, budget):
    q = _frame(h + w + levels, h, w, 6.0)
    cont, _ = O.encode_frame(q, levels, wavelet, 5, 12, budget)
    cs, blocks = O.encode_frame(q, levels, wavelet, 5, 12, budget, fmt="j2c")
    info = parse(cs)
    assert (info["w"], info["h"], info["levels"], info["wavelet"], info["bit_depth"]) == (w, h, levels, wavelet, 12)
    eps, mu = O.band_exponents(levels, wavelet, 12)
    order = [3 * levels] + [3 * (l - 1) + o for l in range(levels, 0, -1) for o in range(3)]
    assert info["eps"] == [eps[b] for b in order] and info["mu"] == [mu[b] for b in order]
    # every block's planes fit M_b with the fewest guard bits
    G = info["guard"]
    assert all(blk["planes"] <= G + eps[blk["band"]] - 1 for blk in blocks)
    assert G == 1 or any(blk["planes"] == G + eps[blk["band"]] - 1 for blk in blocks)
    assert info["blocks"] == _container_blocks(cont)


def test_lossless_53_frame_decodes_back_from_the_codestream():
    q = _frame(7, 192, 256, 10.0)
    cs, _ = O.encode_frame(q, 3, 53, 5, 12, 0, fmt="j2c")
    info = parse(cs)
    # rebuild a container from the parsed passes and decode it
    cont, _ = O.encode_frame(q, 3, 53, 5, 12, 0)
    assert info["blocks"] == _container_blocks(cont)
    assert np.array_equal(O.decode_frame(cont), q)


@pytest.mark.parametrize("wavelet,budget", [(53, 0), (97, 6000)])
def test_reset_style_codestream_and_container(wavelet, budget):
    """Contexts reset at every pass: the container's flags word is 1 and
    COD's code-block style byte 0x06; the codestream carries the container's
    passes, the container decodes back (lossless 5/3), and the same frame
    without the reset has flags 0, style 0x04 and the same pass counts kept
    when every pass is kept."""
    q = _frame(11 + wavelet, 192, 256, 8.0)
    cont, blocks = O.encode_frame(q, 3, wavelet, 5, 12, budget, reset=True)
    cs, _ = O.encode_frame(q, 3, wavelet, 5, 12, budget, fmt="j2c", reset=True)
    assert struct.unpack_from("<I", cont, 28)[0] == 1
    info = parse(cs)
    assert info["style"] == 0x06
    assert info["blocks"] == _container_blocks(cont)
    cont0, blocks0 = O.encode_frame(q, 3, wavelet, 5, 12, budget)
    cs0, _ = O.encode_frame(q, 3, wavelet, 5, 12, budget, fmt="j2c")
    assert struct.unpack_from("<I", cont0, 28)[0] == 0 and parse(cs0)["style"] == 0x04
    if budget == 0:
        assert [b["nkeep"] for b in blocks] == [b["nkeep"] for b in blocks0]
        assert np.array_equal(O.decode_frame(cont), q)


def test_all_zero_frame_gives_empty_packets():
    cs, _ = O.encode_frame(np.zeros((64, 64), np.int32), 2, 53, 5, 8, 0, fmt="j2c")
    info = parse(cs)
    assert info["blocks"] == {}
    # SOC SIZ COD QCD SOT SOD, three one-byte empty packets, EOC
    assert cs[-5:] == b"\x00\x00\x00\xff\xd9"


def test_pass_count_codewords_match_table_b4():
    cases = {1: "0", 2: "10", 3: "1100", 4: "1101", 5: "1110", 6: "111100000", 7: "111100001",
             36: "111111110", 37: "1111111110000000", 38: "1111111110000001", 164: "1111111111111111"}
    for n, bits in cases.items():
        bw = O._BitWriter()
        O._passes_codeword(bw, n)
        got = bw.flush() + b"\x00\x00"
        br = BitReader(got, 0)  # the codeword's bits, stuffing removed
        assert "".join(str(br.bit()) for _ in bits) == bits, n
        assert num_passes(BitReader(got, 0)) == n


def test_bit_stuffing_after_ff():
    bw = O._BitWriter()
    bw.put_bits(0xFF, 8)
    bw.put_bits(0b1111111, 7)  # the next byte holds 7 bits, MSB 0
    bw.put_bits(1, 1)
    out = bw.flush()
    assert out == b"\xff\x7f\x80"
    bw = O._BitWriter()
    bw.put_bits(0xFF, 8)  # a header ending on 0xFF gets one more (zero) byte
    assert bw.flush() == b"\xff\x00"
    br = BitReader(b"\xff\x7f\x80", 0)
    assert br.bits(8) == 0xFF and br.bits(7) == 0x7F and br.bit() == 1


def test_tag_trees_round_trip_on_random_grids():
    rng = np.random.default_rng(5)
    for nx, ny in [(1, 1), (3, 1), (1, 5), (5, 3), (7, 6), (16, 16)]:
        vals = rng.integers(0, 6, nx * ny).tolist()
        for thr in (1, 3, 1 << 30):
            tt = O._TagTree(nx, ny, vals)
            bw = O._BitWriter()
            for j in range(nx * ny):
                tt.encode(bw, j % nx, j // nx, thr)
            br = BitReader(bw.flush() + b"\x00" * 4, 0)
            dec = TagTreeDecoder(nx, ny)
            for j in range(nx * ny):
                v = dec.decode(br, j % nx, j // nx, thr)
                assert v == (vals[j] if vals[j] < thr else None), (nx, ny, thr, j)
