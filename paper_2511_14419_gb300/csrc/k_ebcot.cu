// Embedded block coding of the RoI-shifted coefficient planes: the
// JPEG2000 coder that the paper applies to the front end's output
// (§Implementation details, Table 1: RoI coefficients scaled up, then the
// codestream cut to the target compression rate).  Written from the
// JPEG2000 Part 1 definitions (ISO/IEC 15444-1):
//   - MQ arithmetic coder (Annex C), every coding pass terminated, so each
//     pass is a byte segment and a truncation point;
//   - bit-plane coding passes of 64 x 64 code-blocks anchored at each
//     sub-band's origin (Annex D): stripes of four rows, significance
//     propagation, magnitude refinement, cleanup with run-length mode,
//     zero-coding contexts by orientation, sign contexts with the flip bit;
//   - per pass, the decrease of the squared error of the midpoint
//     reconstruction in doubled units (an exact int64 sum, so the warp can
//     add the terms in any order), on the quantised, RoI-shifted
//     coefficients with unit band weights;
//   - rate control (Annex J): each code-block's lower convex hull of
//     (bytes, distortion decrease), the slope threshold found by 64
//     bisection steps on [0, 2 max slope + 1] so that the kept bytes fit
//     the frame's budget;
//   - the frame as this library's container (32-byte header, a 16-byte
//     entry per code-block, then per code-block the kept passes' 16-bit
//     lengths and bytes) or as a JPEG2000 Part 1 codestream (Annex A
//     markers, Annex B packets with tag trees).
//
// Tier-1 coding runs as five kernels, so that no long sequential chain
// waits on another:
//   - k_t1, context modelling, one warp per code-block.  Which samples each
//     pass codes, in which context, and with which decision depends only on
//     the coefficients and the passes before, not on the arithmetic coder,
//     so the warp forms all of a block's (context, decision) pairs in
//     coding order and writes them out, pass by pass.  Lane l holds the
//     block's columns 2l and 2l + 1 as 64-bit column words of every state
//     (significance, sign, refined, visited, the plane's bit, the plane's
//     new significances); a stripe's contexts come from six-row windows of
//     the lane's and its neighbours' columns (shuffles).  The significance
//     pass's chain (a sample turning significant makes the next ones in the
//     scan candidates) is solved per stripe by rounds across the lanes; the
//     cleanup pass's new significances are known at once.  The same warp
//     builds each bit-plane and adds up the distortion decreases.
//   - k_t1_mq, two threads per code-block: the MQ coder's interval
//     register and context states over the block's decisions (the one
//     chain that runs through all passes; the refinement passes' contexts
//     and the others' form two independent chains), recording each pass's
//     starting context states and a byte bound for its codeword;
//     With the contexts reset at every pass (code-block style 0x02, an
//     option) no state runs from pass to pass, and k_t1_mq_pass, one thread
//     per (code-block, pass), takes this stage instead;
//   - k_t1_slots, one warp per code-block: the codewords' slot offsets;
//   - k_t1_mqc, one thread per pass: each pass, a terminated codeword of
//     its own, coded from its starting context states (the initial ones
//     with reset) into its slot;
//   - k_t1_pack, one warp per code-block: the codewords moved to be back to
//     back.
// Then k_pcrd (rate control, one CTA per frame), and the output: k_cs_copy
// (container bodies) or k_j2c (codestream markers and packet headers, one
// warp per frame) and k_j2c_copy (codestream bodies).

#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

// MQ probability estimation table (Annex C, Table C.2): Qe, next index
// after an MPS, after an LPS, and whether an LPS exchanges the MPS; packed
// into one word per state for the coder (Qe bits 0-15, next-after-MPS
// 16-21, next-after-LPS 22-27, exchange bit 28).
struct MqRow {
    uint16_t qe;
    uint8_t nmps, nlps, sw;
};
constexpr MqRow kMqRows[47] = {
    {0x5601, 1, 1, 1},   {0x3401, 2, 6, 0},   {0x1801, 3, 9, 0},   {0x0AC1, 4, 12, 0},  {0x0521, 5, 29, 0},
    {0x0221, 38, 33, 0}, {0x5601, 7, 6, 1},   {0x5401, 8, 14, 0},  {0x4801, 9, 14, 0},  {0x3801, 10, 14, 0},
    {0x3001, 11, 17, 0}, {0x2401, 12, 18, 0}, {0x1C01, 13, 20, 0}, {0x1601, 29, 21, 0}, {0x5601, 15, 14, 1},
    {0x5401, 16, 14, 0}, {0x5101, 17, 15, 0}, {0x4801, 18, 16, 0}, {0x3801, 19, 17, 0}, {0x3401, 20, 18, 0},
    {0x3001, 21, 19, 0}, {0x2801, 22, 19, 0}, {0x2401, 23, 20, 0}, {0x2201, 24, 21, 0}, {0x1C01, 25, 22, 0},
    {0x1801, 26, 23, 0}, {0x1601, 27, 24, 0}, {0x1401, 28, 25, 0}, {0x1201, 29, 26, 0}, {0x1101, 30, 27, 0},
    {0x0AC1, 31, 28, 0}, {0x09C1, 32, 29, 0}, {0x08A1, 33, 30, 0}, {0x0521, 34, 31, 0}, {0x0441, 35, 32, 0},
    {0x02A1, 36, 33, 0}, {0x0221, 37, 34, 0}, {0x0141, 38, 35, 0}, {0x0111, 39, 36, 0}, {0x0085, 40, 37, 0},
    {0x0049, 41, 38, 0}, {0x0025, 42, 39, 0}, {0x0015, 43, 40, 0}, {0x0009, 44, 41, 0}, {0x0005, 45, 42, 0},
    {0x0001, 45, 43, 0}, {0x5601, 46, 46, 0},
};
struct MqTable {
    uint32_t w[47];
    constexpr MqTable() : w{}
    {
        for (int i = 0; i < 47; i++)
            w[i] = kMqRows[i].qe | ((uint32_t)kMqRows[i].nmps << 16) | ((uint32_t)kMqRows[i].nlps << 22) |
                   ((uint32_t)kMqRows[i].sw << 28);
    }
};
__constant__ MqTable kMq = MqTable();

constexpr int kCtxRL = 17, kCtxUni = 18, kNctx = 19;

// Zero-coding context (Table D.1) from the significant horizontal (h),
// vertical (v) and diagonal (d) neighbours; orientation 0 LL, 1 HL
// (horizontally high-pass), 2 LH, 3 HH.
__host__ __device__ constexpr int zc_rule(int ori, int h, int v, int d)
{
    if (ori == 1) {
        const int t = h;
        h = v;
        v = t;
    }
    if (ori != 3) {
        if (h == 2) return 8;
        if (h == 1) return v >= 1 ? 7 : (d >= 1 ? 6 : 5);
        if (v == 2) return 4;
        if (v == 1) return 3;
        return d >= 2 ? 2 : (d == 1 ? 1 : 0);
    }
    const int hv = h + v;
    if (d >= 3) return 8;
    if (d == 2) return hv >= 1 ? 7 : 6;
    if (d == 1) return hv >= 2 ? 5 : (hv == 1 ? 4 : 3);
    return hv >= 2 ? 2 : (hv == 1 ? 1 : 0);
}

// Sign-coding context and flip (Table D.3) by (H + 1) + 3 (V + 1), H and V
// the clipped horizontal and vertical sign contributions; four bits an
// entry: the context minus 9 (bits 0-2) and the flip (bit 3).
constexpr uint64_t sc_packed()
{
    constexpr int ctx[9] = {13, 10, 11, 12, 9, 12, 11, 10, 13};
    constexpr int flip[9] = {1, 1, 0, 1, 0, 0, 1, 0, 0};
    uint64_t v = 0;
    for (int i = 0; i < 9; i++) v |= (uint64_t)((ctx[i] - 9) | (flip[i] << 3)) << (4 * i);
    return v;
}
constexpr uint64_t kScPacked = sc_packed();

constexpr unsigned kFull = 0xffffffffu;
constexpr int kT1Warps = 8;     // code-blocks (one a warp) per CTA of the modelling kernel
constexpr int kMqThreads = 64;  // code-blocks (one a thread) per CTA of the MQ kernel

// Doubled-unit reconstruction once planes >= p are known (0 while m >> p
// == 0); below 2^26 for magnitudes below 2^24.
__device__ __forceinline__ int recon2(uint32_t m, int p)
{
    const uint32_t hi = m >> p;
    return hi == 0 ? 0 : (int)(2u * (hi << p) + (p > 0 ? (1u << p) : 0u));
}
// Decrease of the squared doubled-unit error when the reconstruction moves
// from planes >= pb (pb > 31: nothing known yet) to planes >= pa; both
// errors are below 2^26 in magnitude, so each square is one widening
// product and the difference is exact.
__device__ __forceinline__ long long derr(uint32_t m, int pb, int pa)
{
    const int t = 2 * (int)m;
    const int eb = t - (pb > 31 ? 0 : recon2(m, pb));
    const int ea = t - recon2(m, pa);
    return (long long)eb * eb - (long long)ea * ea;
}

// MQ encoder of one thread (Annex C, software conventions; the byte at BP
// is held in b until BP moves on).
struct Mqe {
    uint32_t a, c, b;
    int ct, bp;
    uint8_t *out;
    int cap;
    bool over;

    __device__ __forceinline__ void init(uint8_t *o, int capacity)
    {
        a = 0x8000;
        c = 0;
        b = 0;
        ct = 12;
        bp = -1;
        out = o;
        cap = capacity;
        over = false;
    }
    __device__ __forceinline__ void emit()
    {
        if (bp >= 0) {
            if (bp < cap) out[bp] = (uint8_t)b;
            else over = true;
        }
    }
    __device__ __forceinline__ void byteout()
    {
        if (b == 0xFF) {
            emit();
            bp++;
            b = c >> 20;
            c &= 0xFFFFF;
            ct = 7;
        } else if (c < 0x8000000) {
            emit();
            bp++;
            b = c >> 19;
            c &= 0x7FFFF;
            ct = 8;
        } else {
            b++;
            if (b == 0xFF) {
                c &= 0x7FFFFFF;
                emit();
                bp++;
                b = c >> 20;
                c &= 0xFFFFF;
                ct = 7;
            } else {
                emit();
                bp++;
                b = (c >> 19) & 0xFFu;  // the carry (bit 27) went into the byte before
                c &= 0x7FFFF;
                ct = 8;
            }
        }
    }
    // Doubles A (and C) until A >= 0x8000, handing out a byte whenever CT
    // reaches zero: the one-bit-at-a-time loop of the definition, taken in
    // runs of min(remaining shifts, CT) bits (1 <= A < 0x8000 here).
    __device__ __forceinline__ void renorm()
    {
        int n = __clz(a) - 16;
        while (n > 0) {
            const int k = n < ct ? n : ct;
            a <<= k;
            c <<= k;
            ct -= k;
            n -= k;
            if (ct == 0) byteout();
        }
    }
    // One decision d in the context whose word (the state's table row |
    // MPS << 31) is cw; tab: the table rows by state index.  The coded
    // sub-interval is picked by selects: the upper one (A - Qe, C + Qe)
    // when the decision is the MPS and no conditional exchange applies, or
    // it is the LPS and one does; else the lower one (Qe).  A renormalises
    // exactly when it falls below 0x8000 (never for an MPS that leaves it
    // there), and the shift stays within CT, with no byte handed out, for
    // most decisions, so the threads of a warp (coding different passes)
    // branch apart only at a byte-out.
    __device__ __forceinline__ void encode(uint32_t &cw, const uint32_t *tab, uint32_t d)
    {
        const uint32_t w = cw, qe = w & 0xFFFFu, mps = w >> 31;
        const uint32_t a1 = a - qe;
        const bool is_mps = d == mps;
        const bool up = is_mps != (a1 < qe);
        a = up ? a1 : qe;
        c += up ? qe : 0u;
        const int n = __clz(a) - 16;
        if (n > 0) {
            cw = is_mps ? (tab[(w >> 16) & 63u] | (mps << 31)) : (tab[(w >> 22) & 63u] | ((mps ^ ((w >> 28) & 1u)) << 31));
            if (n < ct) {
                a <<= n;
                c <<= n;
                ct -= n;
            } else {
                renorm();
            }
        }
    }
    // Terminates the codeword; returns its length in bytes.
    __device__ __forceinline__ int flush()
    {
        const uint32_t tempc = c + a;
        c |= 0xFFFF;
        if (c >= tempc) c -= 0x8000;
        c <<= ct;
        byteout();
        c <<= ct;
        byteout();
        if (b != 0xFF) {
            emit();
            bp++;
        }
        return bp;
    }
};

// ---------------------------------------------------------------------------
// Context modelling by column words.  Lane l of a block's warp holds the
// block's columns x = 2l and 2l + 1 as 64-bit words (bit y = row y) of each
// state: significance, sign, refined, visited in this plane's significance
// pass, the current plane's magnitude bit, and this plane's new
// significances by pass (for the distortion).  A stripe (rows y0 .. y0 + 3)
// is modelled from windows of six rows (y0 - 1 .. y0 + 4) by four columns
// (2l - 1 .. 2l + 2): byte j of a window holds column 2l - 1 + j, bit R of
// that byte row y0 - 1 + R.  The lane's own columns are bytes 1 and 2.

// Rows y0 - 1 .. y0 + 4 of a column word (rows outside the block are 0).
__device__ __forceinline__ uint32_t rows6(uint64_t c, int y0)
{
    return (uint32_t)(y0 == 0 ? (c << 1) : (c >> (y0 - 1))) & 0x3Fu;
}
// Rows y0 .. y0 + 3.
__device__ __forceinline__ uint32_t rows4(uint64_t c, int y0) { return (uint32_t)(c >> y0) & 0xFu; }

// A stripe window from the lane's two column values (c0: column 2l) and
// its neighbours' (columns 2l - 1 and 2l + 2 do not exist at the edges).
__device__ __forceinline__ uint32_t window(uint32_t c0, uint32_t c1, int lane)
{
    const uint32_t own = c0 | (c1 << 8);
    const uint32_t l = __shfl_up_sync(kFull, own, 1) >> 8;
    const uint32_t r = __shfl_down_sync(kFull, own, 1) & 0xFFu;
    return (lane == 0 ? 0u : l) | (own << 8) | (lane == 31 ? 0u : r << 24);
}

// Stripe rows (bits 0-3) of own column j (1 or 2) with at least one of
// the eight neighbours set in window B.
__device__ __forceinline__ uint32_t any_nb(uint32_t B, int j)
{
    const uint32_t D = B | (B << 1) | (B >> 1);  // each column dilated along y
    const uint32_t c = B >> (8 * j);
    return (((D >> (8 * (j - 1))) | (D >> (8 * (j + 1))) | (c << 1) | (c >> 1)) >> 1) & 0xFu;
}

// Sign-coding decision ((context << 1) | bit) of the sample at window row R
// of own column j whose sign is neg; N: the sign window.
__device__ __forceinline__ uint32_t sign_symbol(uint32_t A, uint32_t B, uint32_t N, int j, int R, uint32_t neg)
{
    const int l = 8 * (j - 1) + R, m = 8 * j + R, r = 8 * (j + 1) + R;
    auto ct = [N](uint32_t W, int k) -> int { return ((W >> k) & 1u) ? (((N >> k) & 1u) ? -1 : 1) : 0; };
    int h = ct(A, l) + ct(B, r), v = ct(A, m - 1) + ct(B, m + 1);
    h = h < -1 ? -1 : (h > 1 ? 1 : h);
    v = v < -1 ? -1 : (v > 1 ? 1 : v);
    const uint32_t e = (uint32_t)(kScPacked >> (4 * ((h + 1) + 3 * (v + 1)))) & 0xFu;
    return ((9u + (e & 7u)) << 1) | (neg ^ (e >> 3));
}

// Exclusive prefix sum of v over the warp; total: the sum over all lanes.
__device__ __forceinline__ int warp_excl(int v, int lane, int &total)
{
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    total = __shfl_sync(kFull, incl, 31);
    return incl - v;
}

// Decisions of one own column (j) of a stripe, in scan order: the coded
// rows c (zero coding, then the sign where the sample turns significant,
// rows n); with rl, run-length mode first (the run decision, and where a
// sample of the column turns significant, its row in two uniform
// decisions and its sign; the rows below it then coded one by one).
struct StripeCtx {
    uint32_t A, B, N;
    int y0;
    const uint8_t *zc;
};
__device__ __forceinline__ int col_count(uint32_t c, uint32_t n, bool rl)
{
    if (!rl) return __popc(c) + __popc(n);
    if (!n) return 1;
    const uint32_t below = (0xEu << (__ffs(n) - 1)) & 0xFu;
    return 4 + __popc(c & below) + __popc(n & below);
}
// Zero-coding indices (h | v << 2 | d << 4: significant horizontal,
// vertical and diagonal neighbours) of the four stripe rows of own column j
// at once, one byte per row, when the samples before a sample in scan order
// (the column to the left, the rows above) are seen in A and the ones after
// it in B: each neighbour's row bits are spread to the rows' bytes by a
// multiply (bit i to bit 8i; no two terms meet), then counted bytewise (at
// most 2 + 8 + 64, so no carries).
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return (x * 0x00204081u) & 0x01010101u; }
__device__ __forceinline__ uint32_t zc_word(uint32_t A, uint32_t B, int j)
{
    const uint32_t L = (A >> (8 * (j - 1))) & 0x3Fu, Ca = (A >> (8 * j)) & 0x3Fu, Cb = (B >> (8 * j)) & 0x3Fu,
                   R = (B >> (8 * (j + 1))) & 0x3Fu;
    const uint32_t h = spread4((L >> 1) & 0xFu) + spread4((R >> 1) & 0xFu);
    const uint32_t v = spread4(Ca & 0xFu) + spread4((Cb >> 2) & 0xFu);
    const uint32_t d = spread4(L & 0xFu) + spread4((L >> 2) & 0xFu) + spread4(R & 0xFu) + spread4((R >> 2) & 0xFu);
    return h + 4u * v + 16u * d;
}
__device__ __forceinline__ void col_emit(uint8_t *&o, const StripeCtx &S, int j, uint32_t c, uint32_t n, bool rl,
                                         uint64_t ng)
{
    uint32_t rest = c;
    if (rl) {
        *o++ = (uint8_t)((kCtxRL << 1) | (n != 0 ? 1 : 0));
        if (!n) return;
        const int r = __ffs(n) - 1;
        *o++ = (uint8_t)((kCtxUni << 1) | (r >> 1));
        *o++ = (uint8_t)((kCtxUni << 1) | (r & 1));
        *o++ = (uint8_t)sign_symbol(S.A, S.B, S.N, j, r + 1, (uint32_t)(ng >> (S.y0 + r)) & 1u);
        rest = c & (0xEu << r) & 0xFu;
    }
    if (!rest) return;
    const uint32_t zw = zc_word(S.A, S.B, j);
    for (uint32_t m = rest; m; m &= m - 1) {
        const int r = __ffs(m) - 1;
        const uint32_t nb = (n >> r) & 1u;
        *o++ = (uint8_t)((S.zc[(zw >> (8 * r)) & 0x7Fu] << 1) | nb);
        if (nb) *o++ = (uint8_t)sign_symbol(S.A, S.B, S.N, j, r + 1, (uint32_t)(ng >> (S.y0 + r)) & 1u);
    }
}

// The block state of a lane (its two columns).
struct Cols {
    uint64_t sig[2], neg[2], ref[2], vis[2], bm[2], nsp[2], ncu[2];
};

__device__ __forceinline__ uint32_t dil4(uint32_t p) { return (p | (p << 1) | (p >> 1)) & 0xFu; }
// Seeds s spread down the column through the rows of u.
__device__ __forceinline__ uint32_t fill_down(uint32_t s, uint32_t u)
{
    s |= (s << 1) & u;
    s |= (s << 1) & u;
    s |= (s << 1) & u;
    return s;
}

// Significance propagation over stripe y0: writes the stripe's decisions
// at out (room bytes left) and returns their number.  A sample is coded
// when it is insignificant and has a significant neighbour at its turn, so
// a sample turning significant makes later ones in the scan (the next
// column, the rows below) candidates: the warp finds the new significances
// of each column from those of the column before it (ex: the rows and
// columns that exist), iterating until no lane's left column changes
// (one lane more is settled per round, so at most 33 rounds).
__device__ __forceinline__ int t1_spp(Cols &s, int y0, uint32_t ex0, uint32_t ex1, int lane, const uint8_t *zc,
                                      uint8_t *out, int room, bool &ovf)
{
    const uint32_t B = window(rows6(s.sig[0], y0), rows6(s.sig[1], y0), lane);
    const uint32_t f0 = ~(B >> 9) & ex0, f1 = ~(B >> 17) & ex1;  // insignificant samples
    const uint32_t b0 = any_nb(B, 1) & f0, b1 = any_nb(B, 2) & f1;
    if (!__any_sync(kFull, (b0 | b1) != 0u)) return 0;
    const uint32_t u0 = rows4(s.bm[0], y0) & f0, u1 = rows4(s.bm[1], y0) & f1;
    uint32_t pin = 0, t0 = 0, t1 = 0, n0 = 0, n1 = 0;
    for (int it = 0; it <= 32; it++) {
        t0 = b0 | (dil4(pin) & f0);
        n0 = fill_down(t0 & u0, u0);
        t1 = b1 | (dil4(n0) & f1);
        n1 = fill_down(t1 & u1, u1);
        uint32_t pn = __shfl_up_sync(kFull, n1, 1);
        if (lane == 0) pn = 0;
        const bool moved = pn != pin;
        pin = pn;
        if (!__any_sync(kFull, moved)) break;
    }
    const uint32_t c0 = (t0 | (n0 << 1)) & f0, c1 = (t1 | (n1 << 1)) & f1;
    StripeCtx S;
    S.B = B;
    S.A = B | (pin << 1) | (n0 << 9) | (n1 << 17);
    S.N = __any_sync(kFull, (n0 | n1) != 0u) ? window(rows6(s.neg[0], y0), rows6(s.neg[1], y0), lane) : 0u;
    S.y0 = y0;
    S.zc = zc;
    int total;
    const int at = warp_excl(col_count(c0, n0, false) + col_count(c1, n1, false), lane, total);
    if (total > room) {
        ovf = true;
    } else {
        uint8_t *o = out + at;
        col_emit(o, S, 1, c0, n0, false, s.neg[0]);
        col_emit(o, S, 2, c1, n1, false, s.neg[1]);
    }
    s.sig[0] |= (uint64_t)n0 << y0;
    s.sig[1] |= (uint64_t)n1 << y0;
    s.nsp[0] |= (uint64_t)n0 << y0;
    s.nsp[1] |= (uint64_t)n1 << y0;
    s.vis[0] |= (uint64_t)c0 << y0;
    s.vis[1] |= (uint64_t)c1 << y0;
    return total;
}

// Magnitude refinement over stripe y0: the samples significant before this
// plane; context 16 after their first refinement, else 15 or 14 by whether
// any neighbour is significant.
__device__ __forceinline__ int t1_mrp(Cols &s, int y0, int lane, uint8_t *out, int room, bool &ovf)
{
    const uint32_t B = window(rows6(s.sig[0], y0), rows6(s.sig[1], y0), lane);
    const uint32_t m0 = (B >> 9) & ~rows4(s.vis[0], y0) & 0xFu, m1 = (B >> 17) & ~rows4(s.vis[1], y0) & 0xFu;
    if (!__any_sync(kFull, (m0 | m1) != 0u)) return 0;
    int total;
    const int at = warp_excl(__popc(m0) + __popc(m1), lane, total);
    if (total > room) {
        ovf = true;
    } else {
        uint8_t *o = out + at;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const uint32_t a = any_nb(B, c + 1), rf = rows4(s.ref[c], y0), v = rows4(s.bm[c], y0);
            for (uint32_t m = c ? m1 : m0; m; m &= m - 1) {
                const int r = __ffs(m) - 1;
                const uint32_t ctx = ((rf >> r) & 1u) ? 16u : (((a >> r) & 1u) ? 15u : 14u);
                *o++ = (uint8_t)((ctx << 1) | ((v >> r) & 1u));
            }
        }
    }
    s.ref[0] |= (uint64_t)m0 << y0;
    s.ref[1] |= (uint64_t)m1 << y0;
    return total;
}

// Cleanup over stripe y0: every sample neither significant nor visited is
// coded, so the new significances are known at once; a full column of
// such samples whose neighbourhood is insignificant at its turn is coded
// in run-length mode.
__device__ __forceinline__ int t1_cup(Cols &s, int y0, uint32_t ex0, uint32_t ex1, int lane, const uint8_t *zc,
                                      uint8_t *out, int room, bool &ovf)
{
    const uint32_t B = window(rows6(s.sig[0], y0), rows6(s.sig[1], y0), lane);
    const uint32_t c0 = ~(B >> 9) & ~rows4(s.vis[0], y0) & ex0, c1 = ~(B >> 17) & ~rows4(s.vis[1], y0) & ex1;
    if (!__any_sync(kFull, (c0 | c1) != 0u)) return 0;
    const uint32_t n0 = c0 & rows4(s.bm[0], y0), n1 = c1 & rows4(s.bm[1], y0);
    uint32_t pl = __shfl_up_sync(kFull, n1, 1);
    if (lane == 0) pl = 0;
    StripeCtx S;
    S.B = B;
    S.A = B | (pl << 1) | (n0 << 9) | (n1 << 17);
    S.N = __any_sync(kFull, (n0 | n1) != 0u) ? window(rows6(s.neg[0], y0), rows6(s.neg[1], y0), lane) : 0u;
    S.y0 = y0;
    S.zc = zc;
    // run-length mode: four uncoded samples (a full stripe) and no
    // significant neighbour (the left column as it stands, the own and the
    // right column as before this pass)
    const bool rl0 = c0 == 0xFu && (S.A & 0x3Fu) == 0u && ((B >> 8) & 0x3Fu) == 0u && ((B >> 16) & 0x3Fu) == 0u;
    const bool rl1 = c1 == 0xFu && ((S.A >> 8) & 0x3Fu) == 0u && ((B >> 16) & 0x3Fu) == 0u && ((B >> 24) & 0x3Fu) == 0u;
    int total;
    const int at = warp_excl(col_count(c0, n0, rl0) + col_count(c1, n1, rl1), lane, total);
    if (total > room) {
        ovf = true;
    } else {
        uint8_t *o = out + at;
        col_emit(o, S, 1, c0, n0, rl0, s.neg[0]);
        col_emit(o, S, 2, c1, n1, rl1, s.neg[1]);
    }
    s.sig[0] |= (uint64_t)n0 << y0;
    s.sig[1] |= (uint64_t)n1 << y0;
    s.ncu[0] |= (uint64_t)n0 << y0;
    s.ncu[1] |= (uint64_t)n1 << y0;
    return total;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Geometry of code-block j of a frame (codestream order: low-low band,
// then HL, LH, HH of each level from the coarsest; raster order within a
// band).  Band index as in the quantisation-step table.
__device__ void cb_geometry(int j, int W, int H, int D, int &band, int &ori, int &x0, int &y0, int &cw, int &ch)
{
    for (int k = 0; k <= 3 * D; k++) {
        int l, o, bx, by;
        if (k == 0) {
            l = D;
            o = 0;
        } else {
            l = D - (k - 1) / 3;
            o = 1 + (k - 1) % 3;
        }
        const int bw = W >> l, bh = H >> l;
        bx = (o == 1 || o == 3) ? bw : 0;
        by = (o == 2 || o == 3) ? bh : 0;
        const int nx = (bw + kCb - 1) / kCb, ny = (bh + kCb - 1) / kCb;
        if (j < nx * ny) {
            const int cy = j / nx, cx = j - cy * nx;
            band = o == 0 ? 3 * D : 3 * (l - 1) + (o - 1);
            ori = o;
            x0 = bx + cx * kCb;
            y0 = by + cy * kCb;
            cw = min(kCb, bw - cx * kCb);
            ch = min(kCb, bh - cy * kCb);
            return;
        }
        j -= nx * ny;
    }
    band = ori = x0 = y0 = cw = ch = 0;
}

}  // namespace

// Tier-1 context modelling: one warp per code-block of the job (taken
// dynamically: their costs differ by orders of magnitude).  Writes the
// block's decisions pass by pass (sym, nsym), its plane count and pass
// count (info 0, 1; info 3 = 2 for magnitudes of 2^24 or more) and the
// passes' distortion decreases.
__global__ void __launch_bounds__(32 * kT1Warps) k_t1(const CsJob *__restrict__ job)
{
    __shared__ uint8_t s_zc[4][128];  // zero-coding context by orientation and zero-coding index
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 4 * 128; i += blockDim.x) {
        const int o = i >> 7, b = i & 127;
        // counts beyond their range (h, v > 2, d > 4) never occur
        s_zc[o][b] = (uint8_t)zc_rule(o, min(b & 3, 2), min((b >> 2) & 3, 2), min(b >> 4, 4));
    }
    __syncthreads();
    for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(job->next, 1);
    g = __shfl_sync(kFull, g, 0);
    if (g >= job->ncb) break;
    // frame of the code-block (frames' code-block ranges are consecutive)
    int f = 0;
    while (f + 1 < job->nframes && job->frames[f + 1].cb0 <= g) f++;
    const CsFrame &F = job->frames[f];
    const int jb = g - F.cb0;
    int band, ori, x0, y0b, cw, ch;
    cb_geometry(jb, F.w, F.h, F.levels, band, ori, x0, y0b, cw, ch);
    const int32_t *coef = F.coef + (size_t)y0b * F.w + x0;
    int32_t *info = F.info + (size_t)jb * kCbInfo;
    double *dist = F.dist + (size_t)jb * kMaxPasses;
    int32_t *nsym = F.nsym + (size_t)jb * kMaxPasses;
    uint8_t *const sym = F.sym + (size_t)jb * kSymCap;
    const uint8_t *zc = s_zc[ori];
    const bool has0 = 2 * lane < cw, has1 = 2 * lane + 1 < cw;
    const int32_t *col = coef + 2 * lane;

    Cols s;
#pragma unroll
    for (int c = 0; c < 2; c++) s.sig[c] = s.neg[c] = s.ref[c] = s.vis[c] = s.bm[c] = s.nsp[c] = s.ncu[c] = 0;
    uint32_t mx = 0;
    for (int y = 0; y < ch; y++) {
        const int32_t v0 = has0 ? __ldg(col + (size_t)y * F.w) : 0, v1 = has1 ? __ldg(col + (size_t)y * F.w + 1) : 0;
        mx |= (uint32_t)(v0 < 0 ? -(long long)v0 : v0) | (uint32_t)(v1 < 0 ? -(long long)v1 : v1);
        s.neg[0] |= (uint64_t)(v0 < 0) << y;
        s.neg[1] |= (uint64_t)(v1 < 0) << y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx |= __shfl_xor_sync(kFull, mx, o);
    const int planes = 32 - __clz(mx);
    if (lane == 0) {
        info[0] = planes;
        info[1] = 0;
        info[3] = 0;
    }
    if (planes == 0) continue;
    if (planes > kMaxPlanes) {
        if (lane == 0) {
            info[3] = 2;
            if (job->err) atomicExch(job->err, kErrCbRange);
        }
        continue;
    }
    int k = 0, pos = 0;
    bool ovf = false;
    // plane p's sweep also settles the distortion of plane p + 1's passes
    for (int p = planes - 1; p >= -1; p--) {
        long long dsp = 0, dmr = 0, dcu = 0;
        const int q = p + 1;  // plane whose passes are settled
        uint64_t before[2];   // significant before plane q
#pragma unroll
        for (int c = 0; c < 2; c++) {
            before[c] = s.sig[c] & ~(s.nsp[c] | s.ncu[c]);
            s.bm[c] = 0;
        }
        // rows in two halves of 32, so that the row bits are 32-bit shifts
        for (int ya = 0; ya < ch; ya += 32) {
            const int yb = min(ch, ya + 32);
            uint32_t e1[2], e2[2], e3[2], bw[2] = {0u, 0u};
#pragma unroll
            for (int c = 0; c < 2; c++) {
                e1[c] = (uint32_t)(s.nsp[c] >> ya);
                e2[c] = (uint32_t)(before[c] >> ya);
                e3[c] = (uint32_t)(s.ncu[c] >> ya);
            }
            for (int y = ya; y < yb; y++) {
                const int b = y - ya;
                const int32_t v0 = has0 ? __ldg(col + (size_t)y * F.w) : 0,
                              v1 = has1 ? __ldg(col + (size_t)y * F.w + 1) : 0;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const int32_t v = c ? v1 : v0;
                    const uint32_t m = v < 0 ? (uint32_t)(-(long long)v) : (uint32_t)v;
                    if (p >= 0) bw[c] |= ((m >> p) & 1u) << b;
                    const uint32_t a1 = (e1[c] >> b) & 1u, a2 = (e2[c] >> b) & 1u, a3 = (e3[c] >> b) & 1u;
                    if (a1 | a2 | a3) {  // this plane's passes coded the sample: one event each
                        const long long d = derr(m, a2 ? q + 1 : 32, q);
                        if (a1) dsp += d;
                        else if (a2) dmr += d;
                        else dcu += d;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 2; c++) s.bm[c] |= (uint64_t)bw[c] << ya;
        }
        dsp = warp_sum_ll(dsp);
        dmr = warp_sum_ll(dmr);
        dcu = warp_sum_ll(dcu);
        if (lane == 0 && q < planes) {
            // passes of plane q: cleanup only at the top plane
            if (q == planes - 1) {
                dist[0] = (double)dcu;
            } else {
                const int base = 1 + 3 * (planes - 2 - q);
                dist[base] = (double)dsp;
                dist[base + 1] = (double)dmr;
                dist[base + 2] = (double)dcu;
            }
        }
        if (p < 0) break;
#pragma unroll
        for (int c = 0; c < 2; c++) s.vis[c] = s.nsp[c] = s.ncu[c] = 0;
        for (int type = (p == planes - 1 ? 2 : 0); type <= 2; type++, k++) {
            int n = 0;  // decisions of this pass
            for (int y0 = 0; y0 < ch; y0 += 4) {
                const uint32_t rr = ch - y0 >= 4 ? 0xFu : ((1u << (ch - y0)) - 1u);
                const uint32_t ex0 = has0 ? rr : 0u, ex1 = has1 ? rr : 0u;
                uint8_t *const out = sym + pos + n;
                const int room = kSymCap - pos - n;
                if (type == 0) n += t1_spp(s, y0, ex0, ex1, lane, zc, out, room, ovf);
                else if (type == 1) n += t1_mrp(s, y0, lane, out, room, ovf);
                else n += t1_cup(s, y0, ex0, ex1, lane, zc, out, room, ovf);
            }
            if (lane == 0) {
                nsym[k] = n;
                // passes coded apart take their first decision from here
                if (F.reset) F.ptab[(size_t)jb * kMaxPasses + k].x = pos;
            }
            pos = (pos + n + 15) & ~15;  // the next pass starts 16-byte aligned
        }
    }
    if (lane == 0) {
        info[1] = k;
        if (ovf) {
            info[3] = 1;
            if (job->err) atomicExch(job->err, kErrCbRange);
        }
    }
    }
}

// Reads a code-block's decisions in order from 16-byte pieces, the next
// piece loaded ahead (decision streams start 16-byte aligned and hold
// kSymCap bytes).
struct DecReader {
    const uint4 *p;
    uint4 cur, nxt;
    int i;
    __device__ __forceinline__ void start(const uint8_t *sym, int at)
    {
        p = reinterpret_cast<const uint4 *>(sym);
        i = at;
        const int pc = at >> 4;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        cur = pc * 16 < kSymCap ? __ldg(p + pc) : z;  // at == kSymCap: an empty pass at the end
        nxt = (pc + 1) * 16 < kSymCap ? __ldg(p + pc + 1) : z;
    }
    __device__ __forceinline__ uint32_t next()
    {
        const int ws = (i >> 2) & 3;
        const uint32_t w = ws == 0 ? cur.x : (ws == 1 ? cur.y : (ws == 2 ? cur.z : cur.w));
        const uint32_t d = (w >> ((i & 3) * 8)) & 0xFFu;
        i++;
        if ((i & 15) == 0) {
            cur = nxt;
            if (i + 16 < kSymCap) nxt = __ldg(p + (i >> 4) + 1);
        }
        return d;
    }
};

__device__ __forceinline__ void mq_init_contexts(uint32_t (*cx)[kMqThreads], int t, const uint32_t *tab)
{
    for (int c = 0; c < kNctx; c++) cx[c][t] = tab[c == 0 ? 4 : (c == kCtxRL ? 3 : (c == kCtxUni ? 46 : 0))];
}

__device__ __forceinline__ int cb_frame(const CsJob *job, int g)
{
    int f = 0;
    while (f + 1 < job->nframes && job->frames[f + 1].cb0 <= g) f++;
    return f;
}

// One decision d of the MQ coder's interval register a and context states
// (Annex C), without the code register: a context's state moves on only
// at a renormalisation, and that depends on the interval alone.  w: the
// context word of d (the state's table row | MPS << 31), returned as that
// of the next decision d2 (loaded ahead; forwarded when it is the same
// context); S counts the renormalisation shifts.  Branch-free: both next
// states are looked up before the renormalisation is known.
__device__ __forceinline__ void mq_state_step(uint32_t d, uint32_t d2, uint32_t (*cx)[kMqThreads], int t,
                                              const uint32_t *tab, uint32_t &w, uint32_t &a, int &S)
{
    const uint32_t c1 = (d >> 1) & 31u, c2 = (d2 >> 1) & 31u;
    const uint32_t w2 = cx[c2][t];  // stale when c2 == c1: forwarded below
    const uint32_t qe = w & 0xFFFFu, mps = w >> 31;
    const uint32_t tm = tab[(w >> 16) & 63u], tl = tab[(w >> 22) & 63u];
    const uint32_t a1 = a - qe;
    const bool is_mps = (d & 1u) == mps;
    const bool xchg = a1 < qe;
    const uint32_t a2 = is_mps != xchg ? a1 : qe;  // a1 when the MPS leaves a >= 0x8000
    const int sh = __clz(a2) - 16;                 // 0 exactly then
    a = a2 << sh;
    S += sh;
    const uint32_t wr = is_mps ? (tm | (mps << 31)) : (tl | ((mps ^ ((w >> 28) & 1u)) << 31));
    const uint32_t wn = sh > 0 ? wr : w;
    cx[c1][t] = wn;
    w = c2 == c1 ? wn : w2;
}

// The same for the refinement passes' chain, whose three contexts (14-16)
// stay in registers (w3), so that no context word goes through shared
// memory.
__device__ __forceinline__ void mq_state_step_mr(uint32_t d, uint32_t (&w3)[3], const uint32_t *tab, uint32_t &a,
                                                 int &S)
{
    const uint32_t c = ((d >> 1) - 14u) & 3u;  // 0, 1, 2 (3 never occurs)
    const uint32_t w = c == 0 ? w3[0] : (c == 1 ? w3[1] : w3[2]);
    const uint32_t qe = w & 0xFFFFu, mps = w >> 31;
    const uint32_t tm = tab[(w >> 16) & 63u], tl = tab[(w >> 22) & 63u];
    const uint32_t a1 = a - qe;
    const bool is_mps = (d & 1u) == mps;
    const bool xchg = a1 < qe;
    const uint32_t a2 = is_mps != xchg ? a1 : qe;
    const int sh = __clz(a2) - 16;
    a = a2 << sh;
    S += sh;
    const uint32_t wr = is_mps ? (tm | (mps << 31)) : (tl | ((mps ^ ((w >> 28) & 1u)) << 31));
    const uint32_t wn = sh > 0 ? wr : w;
    w3[0] = c == 0 ? wn : w3[0];
    w3[1] = c == 1 ? wn : w3[1];
    w3[2] = c == 2 ? wn : w3[2];
}

__device__ __forceinline__ uint32_t piece_byte(const uint4 &v, int q)
{
    const uint32_t x = q < 4 ? v.x : (q < 8 ? v.y : (q < 12 ? v.z : v.w));
    return (x >> ((q & 3) * 8)) & 0xFFu;
}

// Renormalisation shifts S of one pass's n decisions (sym 16-byte aligned,
// read 16 at a time with the next 16 loaded ahead) from a fresh interval
// and the context states in s_cx[.][t], which it leaves at their end
// states; mrp: a refinement pass, whose three contexts (14-16) stay in
// registers on the way.
__device__ __forceinline__ int pass_shifts(const uint8_t *sym, int n, bool mrp, uint32_t (*s_cx)[kMqThreads], int t,
                                           const uint32_t *s_tab)
{
    uint32_t a = 0x8000;
    int S = 0;
    if (n <= 0) return 0;
    const uint4 *pp = reinterpret_cast<const uint4 *>(sym);
    const int npc = (n + 15) >> 4;
    uint4 cur = __ldg(pp);
    if (mrp) {
        uint32_t w3[3] = {s_cx[14][t], s_cx[15][t], s_cx[16][t]};
        for (int b = 0; b < npc; b++) {
            const uint4 nx = b + 1 < npc ? __ldg(pp + b + 1) : make_uint4(0u, 0u, 0u, 0u);
            const int rem = n - 16 * b;
            if (rem >= 16) {
#pragma unroll
                for (int q = 0; q < 16; q++) mq_state_step_mr(piece_byte(cur, q), w3, s_tab, a, S);
            } else {
                for (int q = 0; q < rem; q++) mq_state_step_mr(piece_byte(cur, q), w3, s_tab, a, S);
            }
            cur = nx;
        }
        s_cx[14][t] = w3[0];
        s_cx[15][t] = w3[1];
        s_cx[16][t] = w3[2];
    } else {
        uint32_t w = s_cx[(cur.x >> 1) & 31u][t];
        for (int b = 0; b < npc; b++) {
            const uint4 nx = b + 1 < npc ? __ldg(pp + b + 1) : make_uint4(0u, 0u, 0u, 0u);
            const int rem = n - 16 * b;
            if (rem > 16) {
#pragma unroll
                for (int q = 0; q < 16; q++)
                    mq_state_step(piece_byte(cur, q), q < 15 ? piece_byte(cur, q + 1) : (nx.x & 0xFFu), s_cx, t, s_tab,
                                  w, a, S);
            } else {
                for (int q = 0; q < rem; q++)
                    mq_state_step(piece_byte(cur, q), q + 1 < rem ? piece_byte(cur, q + 1) : 0u, s_cx, t, s_tab, w, a,
                                  S);
            }
            cur = nx;
        }
    }
    return S;
}

// MQ coding, first stage: the interval register and context states over a
// code-block's decisions, recording each pass's starting context states
// and the slot its codeword is given: floor(S / 7) + 3 bytes for S
// renormalisation shifts (the first byte leaves after 12 shifts, each
// later one after 7 or 8, and the termination adds two).  The refinement
// passes use contexts 14-16 only and the other passes never do, and every
// pass starts a fresh interval, so a block is two independent chains: one
// thread takes the refinement passes, another the significance and
// cleanup passes.  Blocks whose contexts reset at every pass are left to
// k_t1_mq_pass.
__global__ void __launch_bounds__(kMqThreads) k_t1_mq(const CsJob *__restrict__ job)
{
    __shared__ uint32_t s_cx[32][kMqThreads];  // the contexts of each thread's code-block
    __shared__ uint32_t s_tab[64];             // the probability table rows
    const int t = threadIdx.x;
    for (int i = t; i < 64; i += blockDim.x) s_tab[i] = i < 47 ? kMq.w[i] : 0u;
    __syncthreads();
    for (;;) {
        const int u = atomicAdd(job->next + 1, 1);
        if (u >= 2 * job->ncb) break;
        // the refinement chains first, then the others, so that a warp's
        // threads run one kind of chain
        const bool mrp = u < job->ncb;  // this thread's chain: the refinement passes
        const int g = mrp ? u : u - job->ncb;
        const CsFrame &F = job->frames[cb_frame(job, g)];
        if (F.reset) continue;
        const int jb = g - F.cb0;
        int32_t *info = F.info + (size_t)jb * kCbInfo;
        const int np = info[1];
        if (info[3] != 0 || np <= 0) continue;
        const int32_t *nsym = F.nsym + (size_t)jb * kMaxPasses;
        int4 *ptab = F.ptab + (size_t)jb * kMaxPasses;
        uint32_t *mqs = F.mqs + (size_t)jb * kMaxPasses * kMqWords;
        const uint8_t *sym = F.sym + (size_t)jb * kSymCap;
        mq_init_contexts(s_cx, t, s_tab);
        int pos = 0;
        for (int k = 0; k < np; k++) {
            const int n = nsym[k];
            if (n < 0 || n > kSymCap - pos) {  // never: the model bounds its decisions
                info[3] = 1;
                break;
            }
            const int s0 = pos;
            pos = (pos + n + 15) & ~15;
            if ((k % 3 == 2) != mrp) continue;  // the other chain's pass
            for (int c = 0; c < kNctx; c++) mqs[k * kMqWords + c] = s_cx[c][t];
            const int S = pass_shifts(sym + s0, n, mrp, s_cx, t, s_tab);
            ptab[k] = make_int4(s0, 0, S / 7 + 3, 0);
        }
    }
}

// The same stage for code-blocks whose contexts reset at every pass: each
// pass starts from the initial context states and a fresh interval, so
// its slot bound is a short chain of its own.  One thread per (code-block,
// pass), items ordered like k_t1_mqc's (by bit-plane and pass type, then
// code-block), so that a warp's threads run like passes of neighbouring
// blocks; each pass's first decision was recorded by k_t1.
__global__ void __launch_bounds__(kMqThreads) k_t1_mq_pass(const CsJob *__restrict__ job)
{
    __shared__ uint32_t s_cx[32][kMqThreads];
    __shared__ uint32_t s_tab[64];
    const int t = threadIdx.x;
    for (int i = t; i < 64; i += blockDim.x) s_tab[i] = i < 47 ? kMq.w[i] : 0u;
    __syncthreads();
    const int items = job->ncb * 3 * kMaxPlanes;
    for (;;) {
        const int u = atomicAdd(job->next + 3, 1);
        if (u >= items) break;
        const int kk = u / job->ncb, g = u - kk * job->ncb;
        const int pl = kk / 3, type = kk - 3 * pl;  // type 0 significance, 1 refinement, 2 cleanup
        const CsFrame &F = job->frames[cb_frame(job, g)];
        if (!F.reset) continue;
        const int jb = g - F.cb0;
        int32_t *info = F.info + (size_t)jb * kCbInfo;
        const int planes = info[0];
        if (info[3] != 0 || info[1] <= 0 || pl >= planes || (pl == planes - 1 && type != 2)) continue;
        const int k = pl == planes - 1 ? 0 : 1 + 3 * (planes - 2 - pl) + type;
        if (k >= info[1]) continue;
        int4 *pt = F.ptab + (size_t)jb * kMaxPasses + k;
        const int s0 = pt->x, n = F.nsym[(size_t)jb * kMaxPasses + k];
        if (s0 < 0 || (s0 & 15) != 0 || n < 0 || n > kSymCap - s0) {
            info[3] = 1;  // never: the model bounds its decisions and aligns each pass
            continue;
        }
        mq_init_contexts(s_cx, t, s_tab);
        const int S = pass_shifts(F.sym + (size_t)jb * kSymCap + s0, n, type == 1, s_cx, t, s_tab);
        pt->z = S / 7 + 3;
    }
}

// Slot offsets of each code-block's pass codewords (one warp per block):
// the passes' slots back to back; a block whose slots exceed kCbRegion
// needs more than kCbBytes (see kCbRegion) and gets info 3 = 1.
__global__ void __launch_bounds__(256) k_t1_slots(const CsJob *__restrict__ job)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = w0; g < job->ncb; g += nw) {
        const CsFrame &F = job->frames[cb_frame(job, g)];
        const int jb = g - F.cb0;
        int32_t *info = F.info + (size_t)jb * kCbInfo;
        const int np = info[1];
        if (info[3] != 0 || np <= 0) continue;
        int4 *ptab = F.ptab + (size_t)jb * kMaxPasses;
        int base = 0;
        for (int k0 = 0; k0 < np; k0 += 32) {
            const int k = k0 + lane;
            const int z = k < np ? ptab[k].z : 0;
            int total;
            const int at = warp_excl(z, lane, total);
            if (k < np) ptab[k].y = base + at;
            base += total;
        }
        if (base > kCbRegion && lane == 0) {
            info[3] = 1;
            if (job->err) atomicExch(job->err, kErrCbRange);
        }
    }
}

// MQ coding, second stage: one thread per (code-block, pass), taken
// dynamically: every pass is a terminated codeword of its own, so with its
// starting context states it is coded apart from the others, into its
// slot.
__global__ void __launch_bounds__(kMqThreads) k_t1_mqc(const CsJob *__restrict__ job)
{
    __shared__ uint32_t s_cx[32][kMqThreads];
    __shared__ uint32_t s_tab[64];
    const int t = threadIdx.x;
    for (int i = t; i < 64; i += blockDim.x) s_tab[i] = i < 47 ? kMq.w[i] : 0u;
    __syncthreads();
    const int items = job->ncb * 3 * kMaxPlanes;
    for (;;) {
        const int u = atomicAdd(job->next + 2, 1);
        if (u >= items) break;
        // items ordered by (bit-plane counted from 0, pass type), then
        // code-block: a warp's threads take the same kind of pass on the
        // same plane of neighbouring code-blocks, of similar lengths
        const int kk = u / job->ncb, g = u - kk * job->ncb;
        const int pl = kk / 3, type = kk - 3 * pl;  // type 0 significance, 1 refinement, 2 cleanup
        const CsFrame &F = job->frames[cb_frame(job, g)];
        const int jb = g - F.cb0;
        int32_t *info = F.info + (size_t)jb * kCbInfo;
        const int planes = info[0];
        if (info[3] != 0 || info[1] <= 0 || pl >= planes || (pl == planes - 1 && type != 2)) continue;
        // pass index: the top plane has its cleanup pass only
        const int k = pl == planes - 1 ? 0 : 1 + 3 * (planes - 2 - pl) + type;
        if (k >= info[1]) continue;
        const int4 pt = F.ptab[(size_t)jb * kMaxPasses + k];
        const int n = F.nsym[(size_t)jb * kMaxPasses + k];
        if (pt.x < 0 || n < 0 || n > kSymCap - pt.x || pt.y < 0 || pt.z < 0 || pt.z > kCbRegion - pt.y) {
            info[3] = 1;  // never: the first stage and the slot offsets bound these
            continue;
        }
        if (F.reset) {
            mq_init_contexts(s_cx, t, s_tab);
        } else {
            const uint32_t *mqs = F.mqs + ((size_t)jb * kMaxPasses + k) * kMqWords;
            for (int c = 0; c < kNctx; c++) s_cx[c][t] = mqs[c];
        }
        DecReader rd;
        rd.start(F.sym + (size_t)jb * kSymCap, pt.x);
        Mqe e;
        e.init(F.cbytes + (size_t)jb * kCbRegion + pt.y, pt.z);
        for (int j = 0; j < n; j++) {
            const uint32_t d = rd.next();
            e.encode(s_cx[(d >> 1) & 31u][t], s_tab, d & 1u);
        }
        const int len = e.flush();
        F.plen[(size_t)jb * kMaxPasses + k] = len;
        if (e.over) {  // never: the slot bounds the codeword
            info[3] = 1;
            if (job->err) atomicExch(job->err, kErrCbRange);
        }
    }
}

// Moves each code-block's pass codewords from their slots to be back to
// back from the start of its region (one warp per code-block; a block
// whose passes exceed kCbBytes gets info 3 = 1).  Slots only move down
// and each 256-byte piece is read whole before it is written, so the move
// is in place.
__global__ void __launch_bounds__(256) k_t1_pack(const CsJob *__restrict__ job)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = w0; g < job->ncb; g += nw) {
        const CsFrame &F = job->frames[cb_frame(job, g)];
        const int jb = g - F.cb0;
        int32_t *info = F.info + (size_t)jb * kCbInfo;
        const int np = info[1];
        if (info[3] != 0 || np <= 0) continue;
        const int32_t *plen = F.plen + (size_t)jb * kMaxPasses;
        const int4 *ptab = F.ptab + (size_t)jb * kMaxPasses;
        uint8_t *const region = F.cbytes + (size_t)jb * kCbRegion;
        int total = 0;
        for (int k = lane; k < np; k += 32) total += plen[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(kFull, total, o);
        if (total > job->cbcap) {
            if (lane == 0) {
                info[3] = 1;
                if (job->err) atomicExch(job->err, kErrCbRange);
            }
            continue;
        }
        int dst = 0;
        for (int k = 0; k < np; k++) {
            const int len = plen[k], src = ptab[k].y;
            if (src != dst)
                for (int o = 0; o < len; o += 256) {
                    uint8_t v[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int at = o + q * 32 + lane;
                        v[q] = at < len ? region[src + at] : (uint8_t)0;
                    }
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int at = o + q * 32 + lane;
                        if (at < len) region[dst + at] = v[q];
                    }
                    __syncwarp();
                }
            dst += len;
        }
    }
}

// Rate control and container header / table: one CTA per frame
// (grid-stride over the job's frames).
__global__ void __launch_bounds__(1024) k_pcrd(const CsJob *__restrict__ job)
{
    __shared__ long long s_ll[32];
    __shared__ double s_d[32];
    __shared__ long long s_scan[1024];
    for (int fi = blockIdx.x; fi < job->nframes; fi += gridDim.x) {
    const CsFrame &F = job->frames[fi];
    const int n = F.ncb, tid = threadIdx.x, nt = blockDim.x;
    auto bsum = [&](long long v) {
        v = warp_sum_ll(v);
        __syncthreads();
        if ((tid & 31) == 0) s_ll[tid >> 5] = v;
        __syncthreads();
        long long t = 0;
        for (int i = 0; i < (nt + 31) / 32; i++) t += s_ll[i];
        return t;
    };
    auto bmax = [&](double v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        __syncthreads();
        if ((tid & 31) == 0) s_d[tid >> 5] = v;
        __syncthreads();
        double t = 0.0;
        for (int i = 0; i < (nt + 31) / 32; i++) t = fmax(t, s_d[i]);
        return t;
    };

    // hulls (lower convex hull of the cumulative (bytes, distortion) points)
    long long full = 0, bad = 0;
    double smax = 0.0;
    for (int j = tid; j < n; j += nt) {
        const int g = j;
        const int np = F.info[(size_t)g * kCbInfo + 1];
        if (F.info[(size_t)g * kCbInfo + 3] != 0) bad = 1;
        const int32_t *pl = F.plen + (size_t)g * kMaxPasses;
        const double *di = F.dist + (size_t)g * kMaxPasses;
        int32_t *hk = F.hk + (size_t)g * (kMaxPasses + 1);
        double *hs = F.hs + (size_t)g * (kMaxPasses + 1);
        long long R[kMaxPasses + 1];
        double Dc[kMaxPasses + 1];
        R[0] = 0;
        Dc[0] = 0.0;
        for (int k = 0; k < np; k++) {
            R[k + 1] = R[k] + pl[k];
            Dc[k + 1] = Dc[k] + di[k];
        }
        // hull point i: its pass count in bits 0-7 and the bytes of those
        // passes above (below 2^23: a block over kCbBytes is bad anyway)
        auto pack = [&](int k) { return k | (int)(min(R[k], (long long)((1 << 23) - 1)) << 8); };
        int m = 1;
        hk[0] = 0;
        hs[0] = 0.0;
        for (int k = 1; k <= np; k++) {
            if (!(Dc[k] > Dc[hk[m - 1] & 0xFF])) continue;
            for (;;) {
                const int a = hk[m - 1] & 0xFF;
                const double sl = (Dc[k] - Dc[a]) / (double)(R[k] - R[a]);
                if (m >= 2 && sl >= hs[m - 1]) {
                    m--;
                    continue;
                }
                hk[m] = pack(k);
                hs[m] = sl;
                m++;
                break;
            }
        }
        F.info[(size_t)g * kCbInfo + 4] = m;
        full += R[np];
        if (m > 1) smax = fmax(smax, hs[1]);
    }
    full = bsum(full);
    smax = bmax(smax);
    bad = bsum(bad);

    // The last hull point whose slope is at least lam: the slopes fall
    // strictly along the hull, so a binary search makes the same
    // comparisons' decision as a scan from the start.
    auto kept = [&](int g, double lam, long long *bytes) {
        const int m = F.info[(size_t)g * kCbInfo + 4];
        const int32_t *hk = F.hk + (size_t)g * (kMaxPasses + 1);
        const double *hs = F.hs + (size_t)g * (kMaxPasses + 1);
        int a = 0, z = m - 1;  // hs[1..a] >= lam, hs[z+1..] < lam
        while (a < z) {
            const int mid = (a + z + 1) >> 1;
            if (hs[mid] >= lam) a = mid;
            else z = mid - 1;
        }
        const int h = hk[a];
        *bytes = h >> 8;
        return h & 0xFF;
    };
    const bool all = F.budget <= 0 || full <= F.budget;
    double lo = 0.0, hi = 2.0 * smax + 1.0;
    if (!all) {
        for (int it = 0; it < 64; it++) {
            const double mid = 0.5 * (lo + hi);
            long long tot = 0;
            for (int j = tid; j < n; j += nt) {
                long long b;
                kept(j, mid, &b);
                tot += b;
            }
            tot = bsum(tot);
            if (tot <= F.budget) hi = mid;
            else lo = mid;
        }
    }
    // kept passes and data sizes; offsets by a two-level scan over
    // contiguous chunks of code-blocks
    const int chunk = (n + nt - 1) / nt, j0 = min(n, tid * chunk), j1 = min(n, j0 + chunk);
    long long mine = 0;
    for (int j = j0; j < j1; j++) {
        const int g = j;
        long long b;
        const int nk = all ? F.info[(size_t)g * kCbInfo + 1] : kept(g, hi, &b);
        if (all) {
            b = 0;
            for (int k = 0; k < nk; k++) b += F.plen[(size_t)g * kMaxPasses + k];
        }
        F.info[(size_t)g * kCbInfo + 2] = nk;
        F.info[(size_t)g * kCbInfo + 5] = (int32_t)(2 * nk + b);
        mine += 2 * nk + b;
    }
    // exclusive scan of the per-thread sums
    __syncthreads();
    s_scan[tid] = mine;
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        const long long v = tid >= d ? s_scan[tid - d] : 0;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    long long off = s_scan[tid] - mine;
    const long long data = s_scan[nt - 1];
    const long long total = kCsHeader + (long long)kCsEntry * n + data;
    const bool container = F.format == 0;  // else k_j2c writes the frame
    const bool fits = container && total <= F.cap && bad == 0;
    for (int j = j0; j < j1; j++) {
        const int g = j;
        F.info[(size_t)g * kCbInfo + 6] = (int32_t)off;
        if (fits) {
            int band, ori, x0, y0, cw, ch;
            cb_geometry(j, F.w, F.h, F.levels, band, ori, x0, y0, cw, ch);
            uint8_t *en = F.out + kCsHeader + (size_t)kCsEntry * j;
            const uint32_t o32 = (uint32_t)off;
            en[0] = o32 & 0xFF;
            en[1] = (o32 >> 8) & 0xFF;
            en[2] = (o32 >> 16) & 0xFF;
            en[3] = o32 >> 24;
            en[4] = x0 & 0xFF;
            en[5] = x0 >> 8;
            en[6] = y0 & 0xFF;
            en[7] = y0 >> 8;
            en[8] = (uint8_t)(cw - 1);
            en[9] = (uint8_t)(ch - 1);
            en[10] = (uint8_t)band;
            en[11] = (uint8_t)F.info[(size_t)g * kCbInfo + 0];
            en[12] = (uint8_t)F.info[(size_t)g * kCbInfo + 1];
            en[13] = (uint8_t)F.info[(size_t)g * kCbInfo + 2];
            en[14] = 0;
            en[15] = 0;
        }
        off += F.info[(size_t)g * kCbInfo + 5];
    }
    if (tid == 0 && container) {
        if (fits) {
            uint8_t *hd = F.out;
            auto put32 = [&](int at, uint32_t v) {
                hd[at] = v & 0xFF;
                hd[at + 1] = (v >> 8) & 0xFF;
                hd[at + 2] = (v >> 16) & 0xFF;
                hd[at + 3] = v >> 24;
            };
            hd[0] = 'F';
            hd[1] = 'R';
            hd[2] = 'J';
            hd[3] = '2';
            put32(4, 1u);
            put32(8, (uint32_t)F.w);
            put32(12, (uint32_t)F.h);
            hd[16] = (uint8_t)F.wavelet;
            hd[17] = (uint8_t)F.levels;
            hd[18] = (uint8_t)F.shift;
            hd[19] = (uint8_t)F.bit_depth;
            put32(20, (uint32_t)n);
            put32(24, (uint32_t)data);
            put32(28, F.reset ? 1u : 0u);  // flags: bit 0, contexts reset at every pass
            *F.flen = total;
        } else {
            // did not fit (the length it needs), or a code-block out of range (-1)
            *F.flen = bad ? -1 : -total;
            if (job->err) atomicExch(job->err, kErrCbRange);
        }
    }
    __syncthreads();
    }
}

// Container data: one warp per code-block copies its kept passes' lengths
// and bytes (grid-stride).
__global__ void __launch_bounds__(256) k_cs_copy(const CsJob *__restrict__ job)
{
    const int lane = threadIdx.x & 31;
    for (int g = blockIdx.x * 8 + (threadIdx.x >> 5); g < job->ncb; g += gridDim.x * 8) {
        int f = 0;
        while (f + 1 < job->nframes && job->frames[f + 1].cb0 <= g) f++;
        const CsFrame &F = job->frames[f];
        if (F.format != 0 || *F.flen < 0) continue;
        const int j = g - F.cb0;
        const int32_t *info = F.info + (size_t)j * kCbInfo;
        const int nk = info[2];
        uint8_t *dst = F.out + kCsHeader + (size_t)kCsEntry * F.ncb + info[6];
        const int32_t *pl = F.plen + (size_t)j * kMaxPasses;
        for (int k = lane; k < nk; k += 32) {
            dst[2 * k] = pl[k] & 0xFF;
            dst[2 * k + 1] = (pl[k] >> 8) & 0xFF;
        }
        int nbytes = 0;
        for (int k = 0; k < nk; k++) nbytes += pl[k];
        const uint8_t *src = F.cbytes + (size_t)j * kCbRegion;
        for (int i = lane; i < nbytes; i += 32) dst[2 * nk + i] = src[i];
    }
}

// ---------------------------------------------------------------------------
// JPEG2000 Part 1 codestream of a frame (CsFrame::format 1) from its
// code-blocks' kept passes (ISO/IEC 15444-1 Annex A markers, Annex B
// packets): SOC, SIZ, COD, QCD, one tile-part (SOT, SOD) holding one packet
// per resolution (one layer, LRCP, no precinct partition), EOC.  A packet
// header codes, per band and code-block in raster order, its inclusion and
// its missing most significant bit-planes with two tag trees, the number of
// passes (Table B.4), the Lblock increment and one length per pass (every
// pass is a terminated codeword segment); a byte after 0xFF carries 7 bits
// and a header never ends on 0xFF.  No RGN marker: Part 1 signals only the
// maximum-shift RoI, so the scaling-based up-shift stays in the data.  The
// guard bits are the fewest (at least 1) that make every block's bit-planes
// fit M_b = G + eps_b - 1; more than 7 cannot be signalled (length -1).

namespace {

// Packet-header bits of lane 0, written straight into the output.
struct HdrBits {
    uint8_t *out;
    long long cap, pos;
    uint64_t acc;  // bits not yet emitted (the low `nacc` bits, first bit highest)
    uint32_t last;
    int nacc, room, nbytes;
    bool over;
    __device__ __forceinline__ void init(uint8_t *o, long long c, long long p)
    {
        out = o;
        cap = c;
        pos = p;
        acc = 0;
        last = 0;
        nacc = nbytes = 0;
        room = 8;
        over = false;
    }
    __device__ __forceinline__ void emit(uint32_t b)
    {
        if (pos < cap) out[pos] = (uint8_t)b;
        else over = true;
        pos++;
        nbytes++;
        last = b;
    }
    // Appends the k (<= 32) low bits of v, first bit highest; every byte
    // holds 8 bits, or 7 after a 0xFF byte (bit stuffing).
    __device__ __forceinline__ void put_bits(uint32_t v, int k)
    {
        acc = (acc << k) | (uint64_t)(k == 32 ? v : (v & ((1u << k) - 1u)));
        nacc += k;
        while (nacc >= room) {
            const uint32_t b = (uint32_t)(acc >> (nacc - room)) & ((1u << room) - 1u);
            nacc -= room;
            emit(b);
            room = b == 0xFF ? 7 : 8;
        }
    }
    __device__ __forceinline__ void put(int b) { put_bits((uint32_t)(b & 1), 1); }
    __device__ __forceinline__ void flush()
    {
        if (nacc) {
            emit((uint32_t)(acc & ((1u << nacc) - 1u)) << (room - nacc));
            nacc = 0;
        }
        if (nbytes && last == 0xFF) emit(0);
    }
};

constexpr int kJ2cSmemInts = 12 * 1024;  // k_j2c's tag trees in shared memory: up to 3072 nodes a tree

// A tag tree over nx x ny leaves (in shared memory, or global scratch for
// large bands): per node its value (the least leaf below it) and its
// state (low bound, bit 31: known).  The level loops run over a fixed
// maximum, so the per-level geometry stays in registers.
constexpr int kTTMax = 16;  // levels: bands up to 2^15 code-blocks a side
struct TagTree {
    int *val, *st;
    int nlev, nn, lw[kTTMax], lh[kTTMax], off[kTTMax];
    // node layout of an nx x ny tree (every lane computes the same)
    __device__ __forceinline__ void layout(int *mem, int nx, int ny)
    {
        int w = nx, h = ny, o = 0;
        bool done = false;
        nlev = kTTMax;
#pragma unroll
        for (int l = 0; l < kTTMax; l++) {
            lw[l] = w;
            lh[l] = h;
            off[l] = o;
            if (!done) {
                o += w * h;
                if (w == 1 && h == 1) {
                    nlev = l + 1;
                    done = true;
                }
            }
            w = (w + 1) >> 1;
            h = (h + 1) >> 1;
        }
        nn = o;
        val = mem;
        st = mem + o;
    }
    __device__ __forceinline__ int nodes() const { return nn; }
    // By the warp: leaf q (x = q % nx, y = q / nx) takes leaf(q), each node
    // above the least of its children, every state cleared.
    template <class Leaf>
    __device__ __forceinline__ void build(int lane, Leaf leaf)
    {
        for (int i = lane; i < nn; i += 32) st[i] = 0;
        for (int q = lane; q < lw[0] * lh[0]; q += 32) val[q] = leaf(q);
#pragma unroll
        for (int l = 1; l < kTTMax; l++) {
            if (l >= nlev) break;
            __syncwarp();
            const int w = lw[l], h = lh[l], pw = lw[l - 1], ph = lh[l - 1], po = off[l - 1], o = off[l];
            for (int q = lane; q < w * h; q += 32) {
                const int x = q % w, y = q / w;
                int v = 0x3fffffff;
                for (int dy = 0; dy < 2; dy++)
                    for (int dx = 0; dx < 2; dx++) {
                        const int cx = 2 * x + dx, cy = 2 * y + dy;
                        if (cx < pw && cy < ph) v = min(v, val[po + cy * pw + cx]);
                    }
                val[o + q] = v;
            }
        }
        __syncwarp();
    }
    template <class Bits>
    __device__ __forceinline__ void encode(Bits &bw, int x, int y, int threshold)
    {
        int low = 0;
#pragma unroll
        for (int l = kTTMax - 1; l >= 0; l--) {
            if (l >= nlev) continue;
            const int i = off[l] + (y >> l) * lw[l] + (x >> l);
            bool known = st[i] < 0;
            const int nl = st[i] & 0x7fffffff;
            if (low < nl) low = nl;
            while (low < threshold) {
                if (low >= val[i]) {
                    if (!known) {
                        bw.put(1);
                        known = true;
                    }
                    break;
                }
                bw.put(0);
                low++;
            }
            st[i] = low | (known ? (int)0x80000000 : 0);
        }
    }
};

// Header bits without stuffing, into 32-bit words (first bit highest):
// a code-block's bits after its tag-tree bits (pass count, Lblock
// increment, segment lengths), or a band's whole header bits, formed apart
// and later appended through HdrBits, which stuffs.
struct RawBits {
    uint32_t *w;
    uint64_t acc;
    int nacc, n;  // pending bits, bits so far
    __device__ __forceinline__ void init(uint32_t *words)
    {
        w = words;
        acc = 0;
        nacc = n = 0;
    }
    __device__ __forceinline__ void put_bits(uint32_t v, int k)
    {
        acc = (acc << k) | (uint64_t)(k == 32 ? v : (v & ((1u << k) - 1u)));
        nacc += k;
        n += k;
        if (nacc >= 32) {
            w[(n - nacc) >> 5] = (uint32_t)(acc >> (nacc - 32));
            nacc -= 32;
        }
    }
    __device__ __forceinline__ void put(int b) { put_bits((uint32_t)(b & 1), 1); }
    __device__ __forceinline__ void finish()
    {
        if (nacc) w[(n - nacc) >> 5] = (uint32_t)(acc << (32 - nacc));
    }
};

template <class Bits>
__device__ __forceinline__ void passes_codeword(Bits &bw, int n)
{
    if (n == 1) bw.put(0);
    else if (n == 2) bw.put_bits(2u, 2);
    else if (n <= 5) bw.put_bits(12u | (uint32_t)(n - 3), 4);
    else if (n <= 36) {
        bw.put_bits(15u, 4);
        bw.put_bits((uint32_t)(n - 6), 5);
    } else {
        bw.put_bits(511u, 9);
        bw.put_bits((uint32_t)(n - 37), 7);
    }
}

__device__ __forceinline__ int bit_length(uint32_t v) { return v ? 32 - __clz(v) : 0; }

}  // namespace

// One warp per frame (grid-stride over the job's frames with format 1).
__global__ void __launch_bounds__(32) k_j2c(const CsJob *__restrict__ job)
{
    const int lane = threadIdx.x;
    for (int fi = blockIdx.x; fi < job->nframes; fi += gridDim.x) {
        const CsFrame &F = job->frames[fi];
        if (F.format != 1) continue;
        const int n = F.ncb, D = F.levels, W = F.w, H = F.h;
        uint8_t *const out = F.out;
        const long long cap = F.cap;
        // guard bits, and code-blocks out of the coder's range
        int need = 1, bad = 0;
        for (int j = lane; j < n; j += 32) {
            const int32_t *in = F.info + (size_t)j * kCbInfo;
            if (in[3] != 0) bad = 1;
            if (in[0] > 0) {
                int band, ori, x0, y0, cw, ch;
                cb_geometry(j, W, H, D, band, ori, x0, y0, cw, ch);
                need = max(need, in[0] - (int)F.eps[band] + 1);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            need = max(need, __shfl_xor_sync(0xffffffffu, need, o));
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (bad || need > 7) {
            if (lane == 0) {
                *F.flen = -1;
                if (job->err) atomicExch(job->err, kErrCbRange);
            }
            continue;
        }
        const int G = need;
        long long pos = 0, sot = 0;
        bool over = false;
        if (lane == 0) {
            auto b8 = [&](uint32_t v) {
                if (pos < cap) out[pos] = (uint8_t)v;
                else over = true;
                pos++;
            };
            auto b16 = [&](uint32_t v) { b8(v >> 8); b8(v & 0xFF); };
            auto b32 = [&](uint32_t v) { b16(v >> 16); b16(v & 0xFFFF); };
            b16(0xFF4F);                                      // SOC
            b16(0xFF51); b16(41); b16(0);                     // SIZ: Lsiz, Rsiz
            b32((uint32_t)W); b32((uint32_t)H); b32(0); b32(0);  // image size, offset
            b32((uint32_t)W); b32((uint32_t)H); b32(0); b32(0);  // one tile
            b16(1); b8((uint32_t)(F.bit_depth - 1)); b8(1); b8(1);  // one unsigned component
            b16(0xFF52); b16(12); b8(0); b8(0); b16(1); b8(0);  // COD: LRCP, one layer, no MCT
            b8((uint32_t)D); b8(4); b8(4); b8(F.reset ? 0x06 : 0x04); b8(F.wavelet == 53 ? 1 : 0);
            const int nb = 3 * D + 1;
            b16(0xFF5C);                                      // QCD
            if (F.wavelet == 53) {
                b16((uint32_t)(3 + nb));
                b8((uint32_t)G << 5);
                b8((uint32_t)F.eps[3 * D] << 3);
                for (int l = D; l >= 1; l--)
                    for (int o = 0; o < 3; o++) b8((uint32_t)F.eps[3 * (l - 1) + o] << 3);
            } else {
                b16((uint32_t)(3 + 2 * nb));
                b8(((uint32_t)G << 5) | 2u);
                b16(((uint32_t)F.eps[3 * D] << 11) | F.mu[3 * D]);
                for (int l = D; l >= 1; l--)
                    for (int o = 0; o < 3; o++) {
                        const int b = 3 * (l - 1) + o;
                        b16(((uint32_t)F.eps[b] << 11) | F.mu[b]);
                    }
            }
            sot = pos;
            b16(0xFF90); b16(10); b16(0); b32(0); b8(0); b8(1);  // SOT (Psot filled below)
            b16(0xFF93);                                      // SOD
        }
        pos = __shfl_sync(0xffffffffu, pos, 0);
        // every included block's header bits after its tag-tree bits, by the
        // lanes (into the block's hull-slope scratch, free once rate control
        // is done): word 0 the bit count, then the bits
        for (int j = lane; j < n; j += 32) {
            const int32_t *in = F.info + (size_t)j * kCbInfo;
            uint32_t *tw = reinterpret_cast<uint32_t *>(F.hs + (size_t)j * (kMaxPasses + 1));
            const int nk = in[2];
            RawBits tb;
            tb.init(tw + 1);
            if (nk > 0) {
                passes_codeword(tb, nk);
                const int32_t *pl = F.plen + (size_t)j * kMaxPasses;
                int nbits = 1;
                for (int t = 0; t < nk; t++) nbits = max(nbits, bit_length((uint32_t)pl[t]));
                const int inc = max(0, nbits - 3);  // Lblock starts at 3
                for (int t = 0; t < inc; t++) tb.put(1);
                tb.put(0);
                for (int t = 0; t < nk; t++) tb.put_bits((uint32_t)pl[t], 3 + inc);
                tb.finish();
            }
            tw[0] = (uint32_t)tb.n;
        }
        __syncwarp();
        // packets: resolution 0 holds the low-low band, resolution r the
        // HL, LH, HH bands of level D - r + 1; their code-blocks follow one
        // another in the frame's code-block order
        extern __shared__ int j2c_smem[];
        // Each band's header bits (its packet's part after the `any` bit),
        // coded by one lane per band into its code-blocks' hull scratch
        // (free once rate control is done), when every band's tag trees fit
        // in shared memory; lane 0 then only appends them, stuffing.
        const int NU = 1 + 3 * D;  // bands: the low-low band, then HL, LH, HH from the coarsest level
        auto unit = [&](int u, int &nx, int &ny, int &jb, int &band) {
            int jj = 0;
            for (int r = 0; r <= D; r++) {
                const int nb = r == 0 ? 1 : 3, l = r == 0 ? D : D - r + 1;
                const int ux = ((W >> l) + kCb - 1) / kCb, uy = ((H >> l) + kCb - 1) / kCb;
                const int u0 = r == 0 ? 0 : 1 + 3 * (r - 1);
                if (u < u0 + nb) {
                    const int k = u - u0;
                    nx = ux;
                    ny = uy;
                    jb = jj + k * ux * uy;
                    band = r == 0 ? 3 * D : 3 * (l - 1) + k;
                    return;
                }
                jj += nb * ux * uy;
            }
        };
        int need_smem = NU;
        for (int u = 0; u < NU; u++) {
            int ux, uy, ujb, ub;
            unit(u, ux, uy, ujb, ub);
            TagTree tt;
            tt.layout(j2c_smem, ux, uy);
            need_smem += 4 * tt.nodes();
        }
        const bool par = need_smem <= kJ2cSmemInts;
        int *const ubits = j2c_smem;
        auto ubuf = [&](int jb) { return reinterpret_cast<uint32_t *>(F.hk + (size_t)jb * (kMaxPasses + 1)); };
        if (par) {
            int toff = NU;
            for (int u = 0; u < NU; u++) {
                int ux, uy, ujb, ub;
                unit(u, ux, uy, ujb, ub);
                const int Mb = G + (int)F.eps[ub] - 1;
                TagTree incl, zbp;
                incl.layout(j2c_smem + toff, ux, uy);
                zbp.layout(j2c_smem + toff + 2 * incl.nodes(), ux, uy);
                incl.build(lane, [&](int q) { return F.info[(size_t)(ujb + q) * kCbInfo + 2] > 0 ? 0 : 1; });
                zbp.build(lane, [&](int q) { return Mb - F.info[(size_t)(ujb + q) * kCbInfo + 0]; });
                toff += 4 * incl.nodes();
            }
            if (lane < NU) {
                int ux, uy, ujb, ub;
                unit(lane, ux, uy, ujb, ub);
                int to = NU;
                for (int u = 0; u < lane; u++) {
                    int vx, vy, vjb, vb;
                    unit(u, vx, vy, vjb, vb);
                    TagTree tt;
                    tt.layout(j2c_smem, vx, vy);
                    to += 4 * tt.nodes();
                }
                TagTree incl, zbp;
                incl.layout(j2c_smem + to, ux, uy);
                zbp.layout(j2c_smem + to + 2 * incl.nodes(), ux, uy);
                RawBits raw;
                raw.init(ubuf(ujb));
                auto tail = [&](int q) {
                    return reinterpret_cast<const uint32_t *>(F.hs + (size_t)(ujb + q) * (kMaxPasses + 1));
                };
                // the next block's tail count and first two words loaded ahead
                const int per_u = ux * uy;
                uint32_t nbq = tail(0)[0], w0 = tail(0)[1], w1 = tail(0)[2];
                for (int q = 0; q < per_u; q++) {
                    uint32_t nbn = 0, w0n = 0, w1n = 0;
                    if (q + 1 < per_u) {
                        const uint32_t *tn = tail(q + 1);
                        nbn = tn[0];
                        w0n = tn[1];
                        w1n = tn[2];
                    }
                    const int cx = q % ux, cy = q / ux;
                    incl.encode(raw, cx, cy, 1);
                    const int nb = (int)nbq;
                    if (nb > 0) {  // included
                        zbp.encode(raw, cx, cy, 0x3fffffff);
                        const uint32_t *tw = tail(q);
                        for (int i = 0; i < nb; i += 32) {
                            const int kk = min(32, nb - i);
                            const uint32_t word = i == 0 ? w0 : (i == 32 ? w1 : tw[1 + (i >> 5)]);
                            raw.put_bits(word >> (32 - kk), kk);
                        }
                    }
                    nbq = nbn;
                    w0 = w0n;
                    w1 = w1n;
                }
                raw.finish();
                ubits[lane] = raw.n;
            }
            __syncwarp();
        }
        int j0 = 0;
        for (int r = 0; r <= D; r++) {
            const int nbands = r == 0 ? 1 : 3, l = r == 0 ? D : D - r + 1;
            const int bw = W >> l, bh = H >> l;
            const int nx = (bw + kCb - 1) / kCb, ny = (bh + kCb - 1) / kCb, per = nx * ny;
            const int j1 = j0 + nbands * per;
            int any = 0;
            for (int j = j0 + lane; j < j1; j += 32) any |= F.info[(size_t)j * kCbInfo + 2] > 0;
            any = __any_sync(0xffffffffu, any);
            HdrBits bits;
            if (lane == 0) {
                bits.init(out, cap, pos);
                bits.put(any ? 1 : 0);
            }
            if (any && par) {
                if (lane == 0)
                    for (int k = 0; k < nbands; k++) {
                        const int u = r == 0 ? 0 : 1 + 3 * (r - 1) + k;
                        const uint32_t *rw = ubuf(j0 + k * per);
                        const int nb = ubits[u];
                        for (int i = 0; i < nb; i += 32) {
                            const int kk = min(32, nb - i);
                            bits.put_bits(rw[i >> 5] >> (32 - kk), kk);
                        }
                    }
            } else if (any) {
                for (int k = 0; k < nbands; k++) {
                    const int band = r == 0 ? 3 * D : 3 * (l - 1) + k;
                    const int Mb = G + (int)F.eps[band] - 1;
                    const int jb = j0 + k * per;
                    // the band's two tag trees: in shared memory when they fit
                    TagTree incl, zbp;
                    incl.layout(j2c_smem, nx, ny);
                    int *mem = 4 * incl.nodes() <= kJ2cSmemInts ? j2c_smem : F.hk;
                    incl.layout(mem, nx, ny);
                    zbp.layout(mem + 2 * incl.nodes(), nx, ny);
                    incl.build(lane, [&](int q) { return F.info[(size_t)(jb + q) * kCbInfo + 2] > 0 ? 0 : 1; });
                    zbp.build(lane, [&](int q) { return Mb - F.info[(size_t)(jb + q) * kCbInfo + 0]; });
                    if (lane == 0) {
                        auto tail = [&](int q) {
                            return reinterpret_cast<const uint32_t *>(F.hs + (size_t)(jb + q) * (kMaxPasses + 1));
                        };
                        // the next block's tail count and first two words loaded ahead
                        uint32_t nbq = tail(0)[0], w0 = tail(0)[1], w1 = tail(0)[2];
                        for (int q = 0; q < per; q++) {
                            uint32_t nbn = 0, w0n = 0, w1n = 0;
                            if (q + 1 < per) {
                                const uint32_t *tn = tail(q + 1);
                                nbn = tn[0];
                                w0n = tn[1];
                                w1n = tn[2];
                            }
                            const int cx = q % nx, cy = q / nx;
                            incl.encode(bits, cx, cy, 1);
                            const int nb = (int)nbq;
                            if (nb > 0) {  // included
                                zbp.encode(bits, cx, cy, 0x3fffffff);
                                const uint32_t *tw = tail(q);
                                for (int i = 0; i < nb; i += 32) {
                                    const int kk = min(32, nb - i);
                                    const uint32_t word = i == 0 ? w0 : (i == 32 ? w1 : tw[1 + (i >> 5)]);
                                    bits.put_bits(word >> (32 - kk), kk);
                                }
                            }
                            nbq = nbn;
                            w0 = w0n;
                            w1 = w1n;
                        }
                    }
                    __syncwarp();
                }
            }
            if (lane == 0) {
                bits.flush();
                pos = bits.pos;
                over = over || bits.over;
            }
            pos = __shfl_sync(0xffffffffu, pos, 0);
            // bodies: the included blocks' kept pass bytes, in header order;
            // their offsets here, the copies by k_j2c_copy
            for (int jc = j0; jc < j1; jc += 32) {
                const int j = jc + lane;
                int nbytes = 0;
                int32_t *in = F.info + (size_t)j * kCbInfo;
                if (j < j1 && in[2] > 0) nbytes = in[5] - 2 * in[2];
                int total;
                const int at = warp_excl(nbytes, lane, total);
                if (j < j1) in[7] = (int32_t)(pos + at);
                pos += total;
            }
            j0 = j1;
        }
        if (lane == 0) {
            if (pos + 2 <= cap) {
                out[pos] = 0xFF;
                out[pos + 1] = 0xD9;  // EOC
            }
            pos += 2;
            over = over || pos > cap;
            if (!over) {
                const uint32_t psot = (uint32_t)(pos - 2 - sot);
                out[sot + 6] = (uint8_t)(psot >> 24);
                out[sot + 7] = (uint8_t)(psot >> 16);
                out[sot + 8] = (uint8_t)(psot >> 8);
                out[sot + 9] = (uint8_t)psot;
                *F.flen = pos;
            } else {
                *F.flen = -pos;  // the length it needs
                if (job->err) atomicExch(job->err, kErrCbRange);
            }
        }
        __syncwarp();
    }
}

// Copies the included code-blocks' kept pass bytes into their frames'
// JPEG2000 codestreams at the offsets k_j2c placed them (one warp per
// code-block); frames whose codestream did not fit are left alone.
__global__ void __launch_bounds__(256) k_j2c_copy(const CsJob *__restrict__ job)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = w0; g < job->ncb; g += nw) {
        const CsFrame &F = job->frames[cb_frame(job, g)];
        if (F.format != 1 || *F.flen <= 0) continue;
        const int jb = g - F.cb0;
        const int32_t *in = F.info + (size_t)jb * kCbInfo;
        const int nk = in[2];
        if (nk <= 0) continue;
        const int nbytes = in[5] - 2 * nk;
        const uint8_t *src = F.cbytes + (size_t)jb * kCbRegion;
        uint8_t *dst = F.out + in[7];
#pragma unroll 4
        for (int i = lane; i < nbytes; i += 32) dst[i] = src[i];
    }
}

int ebcot_codeblocks(int w, int h, int levels)
{
    int n = 0;
    for (int k = 0; k <= 3 * levels; k++) {
        const int l = k == 0 ? levels : levels - (k - 1) / 3;
        const int bw = w >> l, bh = h >> l;
        n += ((bw + kCb - 1) / kCb) * ((bh + kCb - 1) / kCb);
    }
    return n;
}

void launch_ebcot(const CsJob *job_dev, int nframes, int ncb, bool chains, bool passes, cudaStream_t s)
{
    const long long items = (long long)ncb * 3 * kMaxPlanes;
    k_t1<<<std::max(1, (ncb + kT1Warps - 1) / kT1Warps), 32 * kT1Warps, 0, s>>>(job_dev);
    if (chains) k_t1_mq<<<std::max(1, (2 * ncb + kMqThreads - 1) / kMqThreads), kMqThreads, 0, s>>>(job_dev);
    if (passes)
        k_t1_mq_pass<<<(int)std::min<long long>(4096, (items + kMqThreads - 1) / kMqThreads), kMqThreads, 0, s>>>(job_dev);
    k_t1_slots<<<std::max(1, std::min(1024, (ncb + 7) / 8)), 256, 0, s>>>(job_dev);
    k_t1_mqc<<<(int)std::min<long long>(4096, (items + kMqThreads - 1) / kMqThreads), kMqThreads, 0, s>>>(job_dev);
    k_t1_pack<<<std::max(1, std::min(1024, (ncb + 7) / 8)), 256, 0, s>>>(job_dev);
    k_pcrd<<<std::max(1, nframes), 1024, 0, s>>>(job_dev);
    k_cs_copy<<<std::max(1, (ncb + 7) / 8), 256, 0, s>>>(job_dev);
    k_j2c<<<std::max(1, nframes), 32, kJ2cSmemInts * sizeof(int), s>>>(job_dev);
    k_j2c_copy<<<std::max(1, std::min(1024, (ncb + 7) / 8)), 256, 0, s>>>(job_dev);
}

void launch_ebcot_persistent(const CsJob *job_dev, int grid_t1, int grid_mq, int grid_copy, bool reset, cudaStream_t s)
{
    k_t1<<<grid_t1, 32 * kT1Warps, 0, s>>>(job_dev);
    if (reset) k_t1_mq_pass<<<4 * grid_mq, kMqThreads, 0, s>>>(job_dev);
    else k_t1_mq<<<grid_mq, kMqThreads, 0, s>>>(job_dev);
    k_t1_slots<<<grid_copy, 256, 0, s>>>(job_dev);
    k_t1_mqc<<<4 * grid_mq, kMqThreads, 0, s>>>(job_dev);
    k_t1_pack<<<grid_copy, 256, 0, s>>>(job_dev);
    k_pcrd<<<kMaxBatch, 1024, 0, s>>>(job_dev);
    k_cs_copy<<<grid_copy, 256, 0, s>>>(job_dev);
    k_j2c<<<kMaxBatch, 32, kJ2cSmemInts * sizeof(int), s>>>(job_dev);
    k_j2c_copy<<<grid_copy, 256, 0, s>>>(job_dev);
}

int occupancy_t1()
{
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t1, 32 * kT1Warps, 0);
    return b;
}

}  // namespace flowroi
