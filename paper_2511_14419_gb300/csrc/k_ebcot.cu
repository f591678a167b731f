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
//   - a frame container: 32-byte header, a 16-byte entry per code-block,
//     then per code-block the kept passes' 16-bit lengths and bytes.
//
// One warp per code-block.  The block's coder state (a 16-bit word per
// coefficient with a one-sample border: neighbour significance counts,
// significance, refinement, visited, sign, the plane's coding event) and
// the current bit-plane as 64-bit row masks live in shared memory.  The
// warp builds each bit-plane from the coefficient plane (coalesced) and,
// in the same sweep, adds up the distortion decreases of the previous
// plane's passes from the events the passes recorded.  The passes go
// stripe by stripe:
//   - magnitude refinement: its members, contexts and decisions depend only
//     on state fixed before the pass, so the whole warp forms the stripe's
//     (context, bit) symbols in scan order into a shared-memory queue and
//     lane 0 only runs the MQ coder over it;
//   - significance propagation and cleanup: the warp forms the stripe's
//     candidate columns by ballot; lane 0 walks them in order and codes
//     their samples (sequential by definition: a sample that becomes
//     significant changes its neighbours' contexts; in the significance
//     pass it makes the next column a candidate).
// The MQ coder keeps each context's probability-table row and MPS in one
// shared-memory word and renormalises by count-leading-zeros.
#include <mutex>

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


// Sign-coding context (Table D.3) and flip bit by (H + 1) + 3 (V + 1),
// H and V the clipped horizontal and vertical sign contributions: bits 0-4
// the context, bit 7 the flip.
__constant__ uint8_t kSc[9] = {13 | 0x80, 10 | 0x80, 11, 12 | 0x80, 9, 12, 11 | 0x80, 10, 13};

// State word of a coefficient.
constexpr uint16_t kNbMask = 0x7F;  // h (bits 0-1), v (2-3), d (4-6) significant-neighbour counts
constexpr uint16_t kSig = 1u << 7, kRef = 1u << 8, kVis = 1u << 9, kNeg = 1u << 10;
constexpr int kEvShift = 11;        // bits 11-12: this plane's event (1 SPP, 2 MRP, 3 cleanup)
constexpr uint16_t kEvMask = 3u << kEvShift;

// Column-major state words: (x, y) at (x + 1) * kColS + y + kRowOff, so a
// stripe's four rows of a column are one aligned 64-bit word; x and y run
// over the block plus a one-sample border.
constexpr int kColS = 72, kRowOff = 4;
constexpr int kT1Warps = 7;  // code-blocks per CTA (three CTAs per SM by shared memory)

struct T1Warp {
    uint16_t st[(kCb + 2) * kColS];
    uint32_t cxw[kNctx + 1];  // MQ contexts: the state's table row (kMq word) | MPS << 31
    uint64_t bm[kCb];         // bit p of the magnitudes, one row per word (bit x)
    uint8_t mq[4 * kCb];      // a stripe's refinement symbols: (context - 14) << 1 | bit
};

__device__ __forceinline__ int contrib(uint16_t w) { return (w & kSig) ? ((w & kNeg) ? -1 : 1) : 0; }

// Doubled-unit reconstruction once planes >= p are known (0 while m >> p == 0).
__device__ __forceinline__ long long recon2(uint32_t m, int p)
{
    if ((m >> p) == 0) return 0;
    return 2ll * (long long)((m >> p) << p) + (p > 0 ? (1ll << p) : 0ll);
}
__device__ __forceinline__ long long derr(uint32_t m, int pb, int pa)
{
    const long long t = 2ll * (long long)m;
    const long long eb = t - (pb > 31 ? 0ll : recon2(m, pb));
    const long long ea = t - recon2(m, pa);
    return eb * eb - ea * ea;
}

// MQ encoder of lane 0 (Annex C, software conventions; the byte at BP is
// held in b until BP moves on).
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
                b = c >> 19;
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
    __device__ __forceinline__ void encode(uint32_t *cxw, int cx, int d)
    {
        const uint32_t w = cxw[cx], qe = w & 0xFFFFu, mps = w >> 31;
        a -= qe;
        if ((uint32_t)d == mps) {
            if (a & 0x8000) {
                c += qe;
                return;
            }
            if (a < qe) a = qe;
            else c += qe;
            cxw[cx] = kMq.w[(w >> 16) & 63u] | (mps << 31);
        } else {
            if (a < qe) c += qe;
            else a = qe;
            cxw[cx] = kMq.w[(w >> 22) & 63u] | ((mps ^ ((w >> 28) & 1u)) << 31);
        }
        renorm();
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

__device__ __forceinline__ int sti(int x, int y) { return (x + 1) * kColS + y + kRowOff; }

// A coefficient became significant: its neighbours' counts (horizontal
// neighbours are a column apart, vertical ones adjacent words).
__device__ __forceinline__ void set_sig(uint16_t *st, int i)
{
    st[i - kColS] += 1;
    st[i + kColS] += 1;
    st[i - 1] += 4;
    st[i + 1] += 4;
    st[i - kColS - 1] += 16;
    st[i - kColS + 1] += 16;
    st[i + kColS - 1] += 16;
    st[i + kColS + 1] += 16;
}

__device__ __forceinline__ void code_sign(T1Warp &s, Mqe &e, int i, uint16_t w)
{
    const uint16_t *st = s.st;
    int hc = contrib(st[i - kColS]) + contrib(st[i + kColS]);
    int vc = contrib(st[i - 1]) + contrib(st[i + 1]);
    hc = hc < -1 ? -1 : (hc > 1 ? 1 : hc);
    vc = vc < -1 ? -1 : (vc > 1 ? 1 : vc);
    const uint8_t sc = kSc[(hc + 1) + 3 * (vc + 1)];
    e.encode(s.cxw, sc & 0x1F, ((w & kNeg) ? 1 : 0) ^ (sc >> 7));
}

// One coding pass of the current plane by the warp: type 0 significance
// propagation, 1 magnitude refinement, 2 cleanup (see the file header);
// e is lane 0's coder.  zc: the zero-coding contexts of the block's
// orientation by the state word's neighbour bits (0-6).  A stripe
// column's four state words are one 64-bit word.
__device__ __forceinline__ void t1_pass(T1Warp &s, Mqe &e, int type, int w, int h, const uint8_t *zc, int lane)
{
    uint16_t *st = s.st;
    constexpr uint64_t kRep = 0x0001000100010001ull;
    for (int y0 = 0; y0 < h; y0 += 4) {
        const int nr = min(4, h - y0);
        // 16-bit lanes of the stripe's rows that exist
        const uint64_t rows = nr >= 4 ? ~0ull : ((1ull << (16 * nr)) - 1);
        if (type == 1) {
            // refinement: every lane forms its columns' symbols (columns
            // lane and lane + 32, rows in order), placed in scan order by a
            // prefix sum over the lanes of each half
            int total = 0;
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int x = half * 32 + lane;
                uint32_t q = 0;  // up to four 3-bit symbols
                int n = 0;
                if (x < w) {
                    const int i0 = sti(x, y0);
                    for (int r = 0; r < nr; r++) {
                        const uint16_t wd = st[i0 + r];
                        if (!(wd & kSig) || (wd & kVis)) continue;
                        const uint32_t ctx = (wd & kRef) ? 2u : ((wd & kNbMask) ? 1u : 0u);
                        const uint32_t bit = (uint32_t)(s.bm[y0 + r] >> x) & 1u;
                        q |= ((ctx << 1) | bit) << (3 * n);
                        n++;
                        st[i0 + r] = wd | kRef | (uint16_t)(2u << kEvShift);
                    }
                }
                int incl = n;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int at = total + incl - n;
                for (int k = 0; k < n; k++) s.mq[at + k] = (uint8_t)((q >> (3 * k)) & 7u);
                total += __shfl_sync(0xffffffffu, incl, 31);
            }
            __syncwarp();
            if (lane == 0)
                for (int k = 0; k < total; k++) {
                    const uint32_t q = s.mq[k];
                    e.encode(s.cxw, 14 + (int)(q >> 1), (int)(q & 1u));
                }
            __syncwarp();
            continue;
        }
        // candidate columns: significance pass, a row with neighbours and
        // without significance; cleanup, a row neither significant nor visited
        uint64_t cand = 0;
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const int x = half * 32 + lane;
            bool c = false;
            if (x < w) {
                const uint64_t q4 = *reinterpret_cast<const uint64_t *>(st + sti(x, y0)) & rows;
                const uint64_t sig4 = q4 & (kRep * kSig), vis4 = q4 & (kRep * kVis), nb4 = q4 & (kRep * kNbMask);
                if (type == 0) {
                    const uint64_t has_nb = (nb4 + kRep * 0x7F) & (kRep * 0x80);  // bit 7 (= kSig) where nb != 0
                    c = (has_nb & ~sig4) != 0;
                } else {
                    c = ((sig4 | (vis4 >> 2)) ^ (kRep * kSig & rows)) != 0;  // kVis = kSig << 2
                }
            }
            cand |= (uint64_t)__ballot_sync(0xffffffffu, c) << (32 * half);
        }
        if (lane == 0) {
            while (cand) {
                const int x = __ffsll((long long)cand) - 1;
                cand &= cand - 1;
                const int i0 = sti(x, y0);
                bool newsig = false;
                int y = y0;
                if (type == 2 && nr == 4) {
                    const uint64_t q4 = *reinterpret_cast<const uint64_t *>(st + i0);
                    if ((q4 & (kRep * (kNbMask | kSig | kVis))) == 0) {
                        // run-length mode: four uncoded, insignificant samples
                        // with all-zero neighbourhoods
                        int r = 4;
#pragma unroll
                        for (int k = 3; k >= 0; k--)
                            if ((s.bm[y0 + k] >> x) & 1) r = k;
                        e.encode(s.cxw, kCtxRL, r < 4);
                        if (r == 4) continue;
                        e.encode(s.cxw, kCtxUni, r >> 1);
                        e.encode(s.cxw, kCtxUni, r & 1);
                        const int i = i0 + r;
                        code_sign(s, e, i, st[i]);
                        st[i] |= kSig | (uint16_t)(3u << kEvShift);
                        set_sig(st, i);
                        y = y0 + r + 1;
                    }
                }
                for (; y < y0 + nr; y++) {
                    const int i = i0 + (y - y0);
                    const uint16_t wd = st[i];
                    if (type == 0) {
                        if ((wd & kSig) || (wd & kNbMask) == 0) continue;
                    } else {
                        if (wd & (kSig | kVis)) continue;
                    }
                    const int bit = (int)((s.bm[y] >> x) & 1);
                    e.encode(s.cxw, zc[wd & kNbMask], bit);
                    uint16_t nw = wd;
                    if (type == 0) nw |= kVis;
                    if (bit) {
                        code_sign(s, e, i, wd);
                        nw |= kSig | (uint16_t)((type == 0 ? 1u : 3u) << kEvShift);
                        st[i] = nw;
                        set_sig(st, i);
                        newsig = true;
                    } else {
                        st[i] = nw;
                    }
                }
                // a new significance gives the next column's samples a
                // neighbour: it joins the significance pass's candidates
                if (type == 0 && newsig && x + 1 < w) cand |= 1ull << (x + 1);
            }
        }
        __syncwarp();
    }
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

// Tier-1 coding: one warp per code-block of the job (taken dynamically).
__global__ void __launch_bounds__(32 * kT1Warps, 3) k_t1(const CsJob *__restrict__ job)
{
    extern __shared__ __align__(16) unsigned char t1sm[];
    __shared__ uint8_t s_zc[4][128];  // zero-coding context by orientation and the state word's bits 0-6
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    T1Warp &s = reinterpret_cast<T1Warp *>(t1sm)[wp];
    for (int i = threadIdx.x; i < 4 * 128; i += blockDim.x) {
        const int o = i >> 7, b = i & 127;
        // counts beyond their range (h, v > 2, d > 4) never occur
        s_zc[o][b] = (uint8_t)zc_rule(o, min(b & 3, 2), min((b >> 2) & 3, 2), min(b >> 4, 4));
    }
    __syncthreads();
    // code-blocks are taken in order from the job's counter, one per warp
    // at a time: their costs differ by orders of magnitude
    for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(job->next, 1);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= job->ncb) break;
    // frame of the code-block (frames' code-block ranges are consecutive)
    int f = 0;
    while (f + 1 < job->nframes && job->frames[f + 1].cb0 <= g) f++;
    const CsFrame &F = job->frames[f];
    const int jb = g - F.cb0;
    int band, ori, x0, y0, cw, ch;
    cb_geometry(jb, F.w, F.h, F.levels, band, ori, x0, y0, cw, ch);
    const int32_t *coef = F.coef + (size_t)y0 * F.w + x0;
    int32_t *info = F.info + (size_t)jb * kCbInfo;
    int32_t *plen = F.plen + (size_t)jb * kMaxPasses;
    double *dist = F.dist + (size_t)jb * kMaxPasses;

    __syncwarp();
    for (int i = lane; i < (kCb + 2) * kColS; i += 32) s.st[i] = 0;
    __syncwarp();
    uint32_t mx = 0;
    for (int y = 0; y < ch; y++)
        for (int x = lane; x < cw; x += 32) {
            const int32_t v = __ldg(coef + (size_t)y * F.w + x);
            const uint32_t m = v < 0 ? (uint32_t)(-(long long)v) : (uint32_t)v;
            mx |= m;
            if (v < 0) s.st[sti(x, y)] = kNeg;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx |= __shfl_xor_sync(0xffffffffu, mx, o);
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
    if (lane < kNctx) s.cxw[lane] = kMq.w[lane == 0 ? 4 : (lane == kCtxRL ? 3 : (lane == kCtxUni ? 46 : 0))];
    uint8_t *const cbytes = F.cbytes + (size_t)jb * job->cbcap;
    Mqe e;
    int k = 0, pos = 0;
    bool over = false;
    // plane p's sweep also settles the distortion of plane p + 1's passes
    for (int p = planes - 1; p >= -1; p--) {
        __syncwarp();
        long long dsp = 0, dmr = 0, dcu = 0;
        const int q = p + 1;  // plane whose events are settled
        for (int y = 0; y < ch; y++) {
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int x = half * 32 + lane;
                bool bit = false;
                if (x < cw) {
                    const int32_t v = __ldg(coef + (size_t)y * F.w + x);
                    const uint32_t m = v < 0 ? (uint32_t)(-(long long)v) : (uint32_t)v;
                    if (p >= 0) bit = (m >> p) & 1;
                    uint16_t &wd = s.st[sti(x, y)];
                    const int ev = (wd >> kEvShift) & 3;
                    if (ev == 1) dsp += derr(m, 32, q);
                    else if (ev == 2) dmr += derr(m, q + 1, q);
                    else if (ev == 3) dcu += derr(m, 32, q);
                    wd &= (uint16_t)~(kEvMask | kVis);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                if (lane == 0) {
                    if (half == 0) s.bm[y] = bal;
                    else s.bm[y] |= (uint64_t)bal << 32;
                }
            }
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
        __syncwarp();
        for (int type = (p == planes - 1 ? 2 : 0); type <= 2; type++, k++) {
            if (lane == 0) e.init(cbytes + pos, job->cbcap - pos);
            t1_pass(s, e, type, cw, ch, s_zc[ori], lane);
            if (lane == 0) {
                const int len = e.flush();
                over = over || e.over;
                plen[k] = len;
                pos += len;
            }
        }
    }
    if (lane == 0) {
        info[1] = k;
        if (over) {
            info[3] = 1;
            if (job->err) atomicExch(job->err, kErrCbRange);
        }
    }
    __syncwarp();
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
        int m = 1;
        hk[0] = 0;
        hs[0] = 0.0;
        for (int k = 1; k <= np; k++) {
            if (!(Dc[k] > Dc[hk[m - 1]])) continue;
            for (;;) {
                const int a = hk[m - 1];
                const double sl = (Dc[k] - Dc[a]) / (double)(R[k] - R[a]);
                if (m >= 2 && sl >= hs[m - 1]) {
                    m--;
                    continue;
                }
                hk[m] = k;
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

    auto kept = [&](int g, double lam, long long *bytes) {
        const int m = F.info[(size_t)g * kCbInfo + 4];
        const int32_t *hk = F.hk + (size_t)g * (kMaxPasses + 1);
        const double *hs = F.hs + (size_t)g * (kMaxPasses + 1);
        int jj = 0;
        while (jj + 1 < m && hs[jj + 1] >= lam) jj++;
        const int nk = hk[jj];
        long long b = 0;
        const int32_t *pl = F.plen + (size_t)g * kMaxPasses;
        for (int k = 0; k < nk; k++) b += pl[k];
        *bytes = b;
        return nk;
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
            put32(28, 0u);
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
        const uint8_t *src = F.cbytes + (size_t)j * job->cbcap;
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
    uint32_t cur, last;
    int n, room, nbytes;
    bool over;
    __device__ __forceinline__ void init(uint8_t *o, long long c, long long p)
    {
        out = o;
        cap = c;
        pos = p;
        cur = last = 0;
        n = nbytes = 0;
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
    __device__ __forceinline__ void put(int b)
    {
        cur = (cur << 1) | (uint32_t)(b & 1);
        if (++n == room) {
            emit(cur);
            room = cur == 0xFF ? 7 : 8;
            cur = 0;
            n = 0;
        }
    }
    __device__ __forceinline__ void put_bits(uint32_t v, int k)
    {
        for (int i = k - 1; i >= 0; i--) put((int)((v >> i) & 1u));
    }
    __device__ __forceinline__ void flush()
    {
        if (n) {
            emit(cur << (room - n));
            n = 0;
        }
        if (nbytes && last == 0xFF) emit(0);
    }
};

// A tag tree over nx x ny leaves in global scratch: per node its value
// (the least leaf below it) and its state (low bound, bit 31: known).
struct TagTree {
    int *val, *st;
    int nlev, lw[20], off[20];
    __device__ void build(int *mem, int nx, int ny)
    {
        int w = nx, h = ny, o = 0;
        nlev = 0;
        for (;;) {
            lw[nlev] = w;
            off[nlev] = o;
            o += w * h;
            nlev++;
            if (w == 1 && h == 1) break;
            w = (w + 1) >> 1;
            h = (h + 1) >> 1;
        }
        val = mem;
        st = mem + o;
        for (int i = 0; i < o; i++) {
            val[i] = 0x3fffffff;
            st[i] = 0;
        }
    }
    __device__ int nodes() const { return off[nlev - 1] + 1; }
    __device__ void set(int x, int y, int v)
    {
        for (int l = 0; l < nlev; l++) {
            int &t = val[off[l] + (y >> l) * lw[l] + (x >> l)];
            if (v < t) t = v;
        }
    }
    __device__ void encode(HdrBits &bw, int x, int y, int threshold)
    {
        int low = 0;
        for (int l = nlev - 1; l >= 0; l--) {
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

__device__ __forceinline__ void passes_codeword(HdrBits &bw, int n)
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
            b8((uint32_t)D); b8(4); b8(4); b8(0x04); b8(F.wavelet == 53 ? 1 : 0);
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
        // packets: resolution 0 holds the low-low band, resolution r the
        // HL, LH, HH bands of level D - r + 1; their code-blocks follow one
        // another in the frame's code-block order
        int j0 = 0;
        int *const tt_mem = F.hk;  // the hulls' scratch, free once rate control is done
        for (int r = 0; r <= D; r++) {
            const int nbands = r == 0 ? 1 : 3, l = r == 0 ? D : D - r + 1;
            const int bw = W >> l, bh = H >> l;
            const int nx = (bw + kCb - 1) / kCb, ny = (bh + kCb - 1) / kCb, per = nx * ny;
            const int j1 = j0 + nbands * per;
            int any = 0;
            for (int j = j0 + lane; j < j1; j += 32) any |= F.info[(size_t)j * kCbInfo + 2] > 0;
            any = __any_sync(0xffffffffu, any);
            if (lane == 0) {
                HdrBits bits;
                bits.init(out, cap, pos);
                if (!any) {
                    bits.put(0);
                } else {
                    bits.put(1);
                    for (int k = 0; k < nbands; k++) {
                        const int band = r == 0 ? 3 * D : 3 * (l - 1) + k;
                        const int Mb = G + (int)F.eps[band] - 1;
                        const int jb = j0 + k * per;
                        TagTree incl, zbp;
                        incl.build(tt_mem, nx, ny);
                        zbp.build(tt_mem + 2 * incl.nodes(), nx, ny);
                        for (int q = 0; q < per; q++) {
                            const int32_t *in = F.info + (size_t)(jb + q) * kCbInfo;
                            incl.set(q % nx, q / nx, in[2] > 0 ? 0 : 1);
                            zbp.set(q % nx, q / nx, Mb - in[0]);
                        }
                        for (int q = 0; q < per; q++) {
                            const int j = jb + q;
                            const int32_t *in = F.info + (size_t)j * kCbInfo;
                            const int cx = q % nx, cy = q / nx;
                            incl.encode(bits, cx, cy, 1);
                            const int nk = in[2];
                            if (nk == 0) continue;
                            zbp.encode(bits, cx, cy, 0x3fffffff);
                            passes_codeword(bits, nk);
                            const int32_t *pl = F.plen + (size_t)j * kMaxPasses;
                            int nbits = 1;
                            for (int t = 0; t < nk; t++) nbits = max(nbits, bit_length((uint32_t)pl[t]));
                            const int inc = max(0, nbits - 3);  // Lblock starts at 3
                            for (int t = 0; t < inc; t++) bits.put(1);
                            bits.put(0);
                            for (int t = 0; t < nk; t++) bits.put_bits((uint32_t)pl[t], 3 + inc);
                        }
                    }
                }
                bits.flush();
                pos = bits.pos;
                over = over || bits.over;
            }
            pos = __shfl_sync(0xffffffffu, pos, 0);
            // bodies: the included blocks' kept pass bytes, in header order
            for (int j = j0; j < j1; j++) {
                const int32_t *in = F.info + (size_t)j * kCbInfo;
                const int nk = in[2];
                if (nk == 0) continue;
                const int nbytes = in[5] - 2 * nk;
                const uint8_t *src = F.cbytes + (size_t)j * job->cbcap;
                for (int i = lane; i < nbytes; i += 32)
                    if (pos + i < cap) out[pos + i] = src[i];
                pos += nbytes;
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

namespace {
void ensure_t1_attr()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaFuncSetAttribute(k_t1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kT1Warps * sizeof(T1Warp)));
    done[dev] = true;
}
}  // namespace

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

void launch_ebcot(const CsJob *job_dev, int nframes, int ncb, cudaStream_t s)
{
    ensure_t1_attr();
    k_t1<<<std::max(1, (ncb + kT1Warps - 1) / kT1Warps), 32 * kT1Warps, kT1Warps * sizeof(T1Warp), s>>>(job_dev);
    k_pcrd<<<std::max(1, nframes), 1024, 0, s>>>(job_dev);
    k_cs_copy<<<std::max(1, (ncb + 7) / 8), 256, 0, s>>>(job_dev);
    k_j2c<<<std::max(1, nframes), 32, 0, s>>>(job_dev);
}

void launch_ebcot_persistent(const CsJob *job_dev, int grid_t1, int grid_copy, cudaStream_t s)
{
    ensure_t1_attr();
    k_t1<<<grid_t1, 32 * kT1Warps, kT1Warps * sizeof(T1Warp), s>>>(job_dev);
    k_pcrd<<<kMaxBatch, 1024, 0, s>>>(job_dev);
    k_cs_copy<<<grid_copy, 256, 0, s>>>(job_dev);
    k_j2c<<<kMaxBatch, 32, 0, s>>>(job_dev);
}

int occupancy_t1()
{
    ensure_t1_attr();
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t1, 32 * kT1Warps, kT1Warps * sizeof(T1Warp));
    return b;
}

}  // namespace flowroi
