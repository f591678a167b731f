// RoI mask from the flow: saliency, normalisation, quantile cut, opening
// and closing.
//
// Paper: §Region of Interest extraction.  Saliency combines the flow
// magnitude with its spatial gradient at weight 0.7:
//     M = |d|,  g = |(dM/dx, dM/dy)| (central differences, replicate border),
//     S = alpha*M + (1 - alpha)*g,
// then is min-max normalised, S^ = (S - min)/(max - min) (0 when max == min).
// Pixels above a quantile threshold are kept: with k = floor(q*N), t is the
// (k+1)-th largest S^ and mask0 = S^ > t (at most k pixels).  Opening
// (erode, dilate) of radius r_open then closing (dilate, erode) of radius
// r_close with square structuring elements; out-of-image pixels take no
// part.
//
// The quantile is exact: radix select over the float bit patterns of S
// (non-negative floats order like their unsigned bits), three digit passes
// (bits 30..20, 19..9, 8..0) with integer histograms.  Normalisation is
// monotone, so the (k+1)-th largest S^ is the normalisation of the
// (k+1)-th largest S; selecting on S lets the first pass run inside the
// saliency kernel, before min and max are known.  Every normalised value
// (threshold included) is computed by the same two IEEE operations.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

// Radix digits over the 31 low bits of a non-negative float.
__host__ __device__ constexpr int digit_shift(int pass) { return pass == 0 ? 20 : (pass == 1 ? 9 : 0); }
__host__ __device__ constexpr int digit_bits(int pass) { return pass == 2 ? 9 : 11; }

__device__ __forceinline__ float normalise(float s, float mn, float mx)
{
    return mx > mn ? __fdiv_rn(__fsub_rn(s, mn), __fsub_rn(mx, mn)) : 0.f;
}

__device__ __forceinline__ int64_t quantile_k(float q, int64_t n)
{
    int64_t k = (int64_t)floor((double)q * (double)n);
    if (k < 0) k = 0;
    if (k > n - 1) k = n - 1;
    return k;
}

}  // namespace

// Reset the per-frame reduction blocks of a batch.
__global__ void k_frame_init(const BatchDesc *__restrict__ bd)
{
    for (int f = blockIdx.x; f < bd->nframes; f += gridDim.x) {
        unsigned *red = bd->f[f].red;
        for (int i = threadIdx.x; i < kRedWords; i += blockDim.x) red[i] = 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            red[kRedMin] = 0x7f800000u;  // +inf
            red[kRedMax] = 0u;
            red[kRedTHat] = 0x7f800000u;
        }
    }
}

// Block-private histogram + min/max kept across the consecutive tiles a
// block takes from the same frame, flushed to the frame's reduction block
// when the frame changes and at the end (persistent grids give each block a
// run of tiles, mostly of one frame).
struct BlockHist {
    unsigned *hist;  // shared, kHistBins
    unsigned *mm;    // shared, [0] min, [1] max
    int frame = -1;

    __device__ void begin(int f)
    {
        if (f == frame) return;
        flush();
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
        if (threadIdx.x == 0) { mm[0] = 0x7f800000u; mm[1] = 0u; }
        frame = f;
        __syncthreads();
    }
    __device__ void flush_to(unsigned *red, bool minmax)
    {
        __syncthreads();
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
            if (hist[i]) atomicAdd(red + kRedHist + i, hist[i]);
        if (minmax && threadIdx.x == 0) {
            atomicMin(red + kRedMin, mm[0]);
            atomicMax(red + kRedMax, mm[1]);
        }
        __syncthreads();
    }
    unsigned *target = nullptr;
    bool with_minmax = false;
    __device__ void flush()
    {
        if (frame >= 0) flush_to(target, with_minmax);
    }
};

// sqrt(x) for x >= 0 as x * rsqrt(x) (relative error a few 1e-7, far inside
// the saliency tolerance; the exact cut is taken on these same values).
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// Saliency S, min/max of S, histogram of the first radix digit.  A
// kSalTW x (kSalSub x FrameDesc::sal_strips) tile is taken in row strips of
// kSalSub rows (its own tiling, BatchDesc::sal2_off): the strip's
// flow plus one row above and below (rows clamped to the image) and its
// 16-byte-aligned column apron is copied with cp.async into one of two
// shared-memory buffers while the previous strip is processed.  One thread
// per column walks down the strip, keeping M = |d| of the rows above, at
// and below in registers; the horizontal neighbours come from the adjacent
// lanes, and the first and last lane of each warp read their outer
// neighbour themselves.  Columns past the right edge repeat the last
// column, rows above and below repeat the edge rows (replicate border).
// One thread gathers each tile's descriptor fields two tiles ahead into a
// shared-memory header.
constexpr int kSalRows = kSalSub + 2;            // staged rows
constexpr int kSalCols = kSalTW + 4;             // staged columns x0-2 .. x0+TW+2 (float2)

struct SalTile {
    const float2 *fl;
    float *S;
    float2 *dbg;
    unsigned *red;
    int x0, y0, w, h, p, fi, nsub, pad;
};

struct SalSmem {
    static constexpr size_t fl_bytes = (size_t)2 * kSalRows * kSalCols * sizeof(float2);
    static constexpr size_t hist_off = fl_bytes;
    static constexpr size_t mm_off = hist_off + kHistBins * sizeof(unsigned);
    static constexpr size_t hdr_off = (mm_off + 2 * sizeof(unsigned) + 15) / 16 * 16;
    static constexpr size_t bytes = hdr_off + 3 * sizeof(SalTile);
};

__global__ void __launch_bounds__(256, 4) k_saliency(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    constexpr int TW = kSalTW, SH = kSalSub;
    static_assert(TW == 256, "one thread per tile column");
    extern __shared__ __align__(16) unsigned char ssm[];
    float2 (*s_fl)[kSalRows][kSalCols] = reinterpret_cast<float2 (*)[kSalRows][kSalCols]>(ssm);
    unsigned *const s_hist = reinterpret_cast<unsigned *>(ssm + SalSmem::hist_off);
    unsigned *const s_mm = reinterpret_cast<unsigned *>(ssm + SalSmem::mm_off);
    SalTile *const s_hdr = reinterpret_cast<SalTile *>(ssm + SalSmem::hdr_off);
    const int nfr = bd->nframes;
    const int *off = bd->sal2_off;
    const int total = __ldg(off + nfr);
    const int buf = bd->final_flow_buf;
    const int tid = threadIdx.x, lane = tid & 31;
    const float wm = mc.alpha, wg = 1.f - mc.alpha;
    BlockHist bh{s_hist, s_mm};
    bh.with_minmax = true;
    unsigned mn = 0x7f800000u, mx = 0u;

    auto fill_hdr = [&](int t, SalTile &H) {
        if (t >= total) return;
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        H.fi = fi;
        H.fl = F.flow[buf];
        H.S = F.S;
        H.dbg = F.dbg_flow;
        H.red = F.red;
        H.w = F.W;
        H.h = F.H;
        H.p = F.lp[0];
        const int ntx = (H.w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        H.nsub = F.sal_strips;
        H.x0 = (lt % ntx) * TW;
        H.y0 = (lt / ntx) * SH * H.nsub;
    };
    // strip `sub` of a tile into buffer b: 16-byte chunks (two flow
    // vectors; x0, the width and the row pitch are even) inside the image
    auto issue = [&](const SalTile &H, int sub, int b) {
        constexpr int NCH = kSalCols / 2;
        for (int i = tid; i < kSalRows * NCH; i += TW) {
            const int r = i / NCH, q = i - r * NCH;
            const int gx = H.x0 - 2 + 2 * q;
            if (gx < 0 || gx + 2 > H.w) continue;
            const int gy = clampi(H.y0 + sub * SH - 1 + r, 0, H.h - 1);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(
                             &s_fl[b][r][2 * q])),
                         "l"(H.fl + (size_t)gy * H.p + gx)
                         : "memory");
        }
    };

    // the block's tiles: one contiguous run, so that its histogram changes
    // frame (clear and flush) rarely
    const int run = (total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t0 = min(total, (int)blockIdx.x * run), t1 = min(total, t0 + run);
    if (tid == 0) {
        if (t0 < t1) fill_hdr(t0, s_hdr[0]);
        if (t0 + 1 < t1) fill_hdr(t0 + 1, s_hdr[1]);
    }
    __syncthreads();
    if (t0 < t1) issue(s_hdr[0], 0, 0);
    asm volatile("cp.async.commit_group;" ::: "memory");

    int k = 0, u = 0;  // tile and strip counters of the block
    for (int t = t0; t < t1; t++, k++) {
        const SalTile &H = s_hdr[k % 3];
        const int fi = H.fi;
        if (fi != bh.frame) {
            // this thread's extrema belong to the frame being left
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0 && bh.frame >= 0) {
                atomicMin(&s_mm[0], mn);
                atomicMax(&s_mm[1], mx);
            }
            mn = 0x7f800000u;
            mx = 0u;
        }
        bh.begin(fi);
        bh.target = H.red;
        const int w = H.w, h = H.h, p = H.p, x0 = H.x0, y0 = H.y0;
        float *const Sp = H.S;
        float2 *const dbg_flow = H.dbg;
        const int gx = x0 + tid;
        // staged columns of the thread's pixel and of the warp's outer
        // neighbours (clamped to the image)
        const int cg = min(gx, w - 1);
        const int cx = cg - (x0 - 2);
        const int ex = (lane == 0 ? max(cg - 1, 0) : min(cg + 1, w - 1)) - (x0 - 2);
        const bool edge = lane == 0 || lane == 31;
        const int nsub = H.nsub;
        for (int sub = 0; sub < nsub; sub++, u++) {
            // this strip has landed; every thread is done with the other buffer
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            if (sub == 0 && tid == 0 && t + 2 < t1) fill_hdr(t + 2, s_hdr[(k + 2) % 3]);
            if (sub + 1 < nsub) issue(H, sub + 1, (u + 1) & 1);
            else if (t + 1 < t1) issue(s_hdr[(k + 1) % 3], 0, (u + 1) & 1);
            asm volatile("cp.async.commit_group;" ::: "memory");

            const float2(*fl)[kSalCols] = s_fl[u & 1];
            auto mag = [&](int r, int c) {
                const float2 v = fl[r][c];
                return fast_sqrt(v.x * v.x + v.y * v.y);
            };
            float Mp = mag(0, cx), Mc = mag(1, cx);
            float Ec = edge ? mag(1, ex) : 0.f;
#pragma unroll
            for (int j = 0; j < SH; j++) {
                const float Mn = mag(j + 2, cx);
                const float En = edge ? mag(j + 2, ex) : 0.f;
                const int gy = y0 + sub * SH + j;
                float Ml = __shfl_up_sync(0xffffffffu, Mc, 1), Mr = __shfl_down_sync(0xffffffffu, Mc, 1);
                if (lane == 0) Ml = Ec;
                if (lane == 31) Mr = Ec;
                if (gx < w && gy < h) {
                    const float gxv = 0.5f * (Mr - Ml), gyv = 0.5f * (Mn - Mp);
                    const float S = wm * Mc + wg * fast_sqrt(gxv * gxv + gyv * gyv);
                    Sp[(size_t)gy * p + gx] = S;
                    if (dbg_flow) dbg_flow[(size_t)gy * w + gx] = fl[j + 1][cx];
                    const unsigned b = __float_as_uint(S);
                    mn = min(mn, b);
                    mx = max(mx, b);
                    atomicAdd(&s_hist[b >> digit_shift(0)], 1u);
                }
                Mp = Mc;
                Mc = Mn;
                Ec = En;
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0 && bh.frame >= 0) {
        atomicMin(&s_mm[0], mn);
        atomicMax(&s_mm[1], mx);
    }
    bh.flush();
}

// Histogram of radix digit 1 over the values whose higher bits equal the
// prefix selected so far.  One thread per tile column: all of its kSalTH
// loads are issued before any is tested.  The matching values are also
// appended to the frame's candidate list (one atomic per warp and tile), so
// the last digit reads only them.
__global__ void __launch_bounds__(256, 4) k_select_pass(const BatchDesc *__restrict__ bd, int pass)
{
    constexpr int TW = kSalTW, TH = kSalTH;
    __shared__ unsigned s_hist[kHistBins];
    __shared__ unsigned s_mm[2];
    const int nfr = bd->nframes;
    const int *off = bd->sal_off;
    const int total = __ldg(off + nfr);
    const int sh = digit_shift(pass), hi = sh + digit_bits(pass);
    const unsigned dmask = (1u << digit_bits(pass)) - 1u;
    const int lane = threadIdx.x & 31;
    BlockHist bh{s_hist, s_mm};
    // the block's tiles: one contiguous run (its histogram changes frame rarely)
    const int run = (total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t0 = min(total, (int)blockIdx.x * run), t1 = min(total, t0 + run);
    for (int t = t0; t < t1; t++) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        bh.begin(fi);
        bh.target = F.red;
        const int w = F.W, h = F.H, p = F.lp[0];
        const int ntx = (w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * TW, y0 = (lt / ntx) * TH;
        const unsigned want = __ldg(F.red + kRedPrefix) >> hi;
        const int gx = x0 + (int)threadIdx.x;
        const int nr = gx < w ? min(TH, h - y0) : 0;
        const unsigned *col = reinterpret_cast<const unsigned *>(F.S) + (size_t)y0 * p + min(gx, w - 1);
        unsigned v[TH];
#pragma unroll
        for (int j = 0; j < TH; j++) v[j] = j < nr ? __ldg(col + (size_t)j * p) : 0u;
        unsigned tot = 0;
#pragma unroll
        for (int j = 0; j < TH; j++) {
            const bool hit = j < nr && (v[j] >> hi) == want;
            if (hit) atomicAdd(&s_hist[(v[j] >> sh) & dmask], 1u);
            tot += __popc(__ballot_sync(0xffffffffu, hit));
        }
        if (tot == 0) continue;  // warp-uniform
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(F.red + kRedCand, tot);
        base = __shfl_sync(0xffffffffu, base, 0);
        // the row's matches are stored contiguously (the row's ballot again)
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int j = 0; j < TH; j++) {
            const bool hit = j < nr && (v[j] >> hi) == want;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) F.cand[base + __popc(m & below)] = v[j];
            base += __popc(m);
        }
    }
    bh.flush();
}

// Histogram of the last radix digit over the frame's candidate list (the
// values in the first digit's selected bin), counting those that are also in
// the second digit's selected bin.  kCandBlocks blocks share a frame; the
// grid (a multiple of kCandBlocks) strides over the frames.
__global__ void __launch_bounds__(256) k_select_cand(const BatchDesc *__restrict__ bd)
{
    constexpr int NB = 1 << digit_bits(2);
    __shared__ unsigned s_hist[NB];
    const int part = blockIdx.x % kCandBlocks, fstride = gridDim.x / kCandBlocks;
    const int sh = digit_shift(2), hi = sh + digit_bits(2);
    for (int f = blockIdx.x / kCandBlocks; f < bd->nframes; f += fstride) {
        const FrameDesc &F = bd->f[f];
        if (!F.has_prev) continue;  // block-uniform
        const unsigned want = F.red[kRedPrefix] >> hi;
        const unsigned n = F.red[kRedCand];
        for (int i = threadIdx.x; i < NB; i += blockDim.x) s_hist[i] = 0u;
        __syncthreads();
        for (unsigned i = part * blockDim.x + threadIdx.x; i < n; i += kCandBlocks * blockDim.x) {
            const unsigned v = __ldg(F.cand + i);
            if ((v >> hi) == want) atomicAdd(&s_hist[(v >> sh) & (NB - 1)], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NB; i += blockDim.x)
            if (s_hist[i]) atomicAdd(F.red + kRedHist + i, s_hist[i]);
        __syncthreads();
    }
}

// One block per frame: locate the bin of the current digit that holds the
// remaining rank (counting from the largest values), extend the prefix,
// clear the histogram.  After the last digit the prefix is t_S exactly.
__global__ void __launch_bounds__(256) k_select_find(const BatchDesc *__restrict__ bd, MethodConsts mc, int pass)
{
    __shared__ unsigned s_part[256];
    __shared__ unsigned s_sel[2];
    const int nfr = bd->nframes;
    const int sh = digit_shift(pass);
    const int nb = 1 << digit_bits(pass);
    const int per = nb / 256;  // bins per thread (8 or 2)
    for (int f = blockIdx.x; f < nfr; f += gridDim.x) {
        const FrameDesc &F = bd->f[f];
        if (!F.has_prev) continue;
        unsigned *red = F.red;
        unsigned rank;
        if (pass == 0) rank = (unsigned)quantile_k(mc.q, (int64_t)F.W * F.H);
        else rank = red[kRedRank];
        // Thread t covers bins nb-1-t*per ... nb-per-t*per (descending).
        unsigned local = 0;
        for (int j = 0; j < per; j++) local += red[kRedHist + nb - 1 - (threadIdx.x * per + j)];
        s_part[threadIdx.x] = local;
        __syncthreads();
        // Exclusive scan (Hillis-Steele on 256 entries).
        for (int o = 1; o < 256; o <<= 1) {
            const unsigned v = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0u;
            __syncthreads();
            s_part[threadIdx.x] += v;
            __syncthreads();
        }
        const unsigned incl = s_part[threadIdx.x];
        const unsigned excl = incl - local;
        if (rank >= excl && rank < incl) {
            unsigned c = excl;
            for (int j = 0; j < per; j++) {
                const int b = nb - 1 - (threadIdx.x * per + j);
                const unsigned hb = red[kRedHist + b];
                if (rank < c + hb) { s_sel[0] = (unsigned)b; s_sel[1] = rank - c; break; }
                c += hb;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) red[kRedHist + i] = 0u;
        if (threadIdx.x == 0) {
            const unsigned prefix = (pass == 0 ? 0u : red[kRedPrefix]) | (s_sel[0] << sh);
            red[kRedPrefix] = prefix;
            red[kRedRank] = s_sel[1];
            if (pass == 2) {
                const float mn = __uint_as_float(red[kRedMin]), mx = __uint_as_float(red[kRedMax]);
                const float th = normalise(__uint_as_float(prefix), mn, mx);
                red[kRedTS] = prefix;
                red[kRedTHat] = __float_as_uint(th);
                // normalise() is monotone in S, so {S : normalise(S) > th} =
                // {S > s*} with s* the largest value normalising to <= th;
                // binary search over the float bits in [t_S, max].
                unsigned lo = prefix, hi = red[kRedMax];
                if (normalise(__uint_as_float(hi), mn, mx) <= th) {
                    lo = hi;
                } else {
                    while (hi - lo > 1u) {
                        const unsigned mid = lo + ((hi - lo) >> 1);
                        if (normalise(__uint_as_float(mid), mn, mx) <= th) lo = mid; else hi = mid;
                    }
                }
                red[kRedSStar] = lo;
                if (F.dbg_thr) *F.dbg_thr = th;
            }
        }
        __syncthreads();
    }
}

// Threshold + opening + closing, bit-packed: 32 horizontally adjacent
// pixels per 32-bit word (bit i = pixel x0 + i).  A block owns a tile of
// kMorWords words x kMorRows rows and loads an apron of one word on each
// side (>= the total radius 2*(r_open + r_close) <= 16) and 16 rows above
// and below.  mask0 is formed with one warp ballot per word from coalesced
// S reads; erosion / dilation of radius r are shifts and AND / OR across
// neighbouring words, then across neighbouring rows.  Words and rows at the
// apron's outer edge see missing neighbours as the neutral element; the
// error this causes moves inwards by r per operation and never reaches the
// tile (apron >= total radius).  Out-of-image pixels take no part: before
// each operation they are set to its neutral element (1 for AND, 0 for OR).
namespace {

constexpr int kMorMaxR = 4;
constexpr int kMorWords = kMorTW / 32, kMorRows = kMorTH;
constexpr int kMorApron = 4 * kMorMaxR;                  // rows above and below
constexpr int kMorEW = kMorWords + 2, kMorEH = kMorRows + 2 * kMorApron;

// Bits of word (wx) of row gy that lie inside the image.
__device__ __forceinline__ unsigned in_image_bits(int wx, int gy, int w, int h)
{
    if (gy < 0 || gy >= h || wx < 0) return 0u;
    const int x = wx * 32;
    if (x >= w) return 0u;
    const int n = w - x;
    return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

__device__ __forceinline__ void morph_op(unsigned (*a)[kMorEW], unsigned (*b)[kMorEW], int r, bool erode, int wx0,
                                         int gy0, int w, int h, bool next_erode, int ylo, int yhi)
{
    const unsigned neutral = erode ? 0xffffffffu : 0u;
    const int n = (yhi - ylo) * kMorEW;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int y = ylo + i / kMorEW, x = i % kMorEW;
        const unsigned m = a[y][x];
        const unsigned l = x > 0 ? a[y][x - 1] : neutral, rr = x + 1 < kMorEW ? a[y][x + 1] : neutral;
        unsigned v = m;
        for (int d = 1; d <= r; d++) {
            const unsigned sl = (m << d) | (l >> (32 - d)), sr = (m >> d) | (rr << (32 - d));
            v = erode ? (v & sl & sr) : (v | sl | sr);
        }
        b[y][x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int y = ylo + i / kMorEW, x = i % kMorEW;
        unsigned v = b[y][x];
        for (int d = 1; d <= r; d++) {
            const unsigned up = y - d >= ylo ? b[y - d][x] : neutral, dn = y + d < yhi ? b[y + d][x] : neutral;
            v = erode ? (v & up & dn) : (v | up | dn);
        }
        const unsigned inb = in_image_bits(wx0 + x, gy0 + y, w, h);
        a[y][x] = (v & inb) | (next_erode ? ~inb : 0u);
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(256) k_morph(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    __shared__ unsigned s_a[kMorEH][kMorEW];
    __shared__ unsigned s_b[kMorEH][kMorEW];
    const int nfr = bd->nframes;
    const int *off = bd->mor_off;
    const int total = __ldg(off + nfr);
    const int ro = mc.r_open, rc = mc.r_close;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.W, h = F.H, p = F.lp[0];
        const int ntx = (w + 32 * kMorWords - 1) / (32 * kMorWords);
        const int lt = t - __ldg(off + fi);
        const int tx = lt % ntx, ty = lt / ntx;
        const int wx0 = tx * kMorWords - 1;         // global word index of apron column 0
        const int gy0 = ty * kMorRows - kMorApron;  // global row of apron row 0
        if (!F.has_prev) {
            // no predecessor: empty mask
            for (int i = threadIdx.x; i < kMorRows * kMorWords * 8; i += blockDim.x) {
                const int r = i / (kMorWords * 8), q = i - r * (kMorWords * 8);
                const int gy = ty * kMorRows + r, gx = (tx * kMorWords) * 32 + q * 4;
                if (gy >= h) continue;
                for (int j = 0; j < 4; j++)
                    if (gx + j < w) {
                        F.mask[(size_t)gy * w + gx + j] = 0;
                        if (F.dbg_mask0) F.dbg_mask0[(size_t)gy * w + gx + j] = 0;
                        if (F.dbg_shat) F.dbg_shat[(size_t)gy * w + gx + j] = 0.f;
                    }
            }
            continue;
        }
        const unsigned sstar = F.red[kRedSStar];
        const bool keep = F.dbg_mask0 != nullptr;
        const float *const Sp = F.S;
        uint8_t *const dbg_mask0 = F.dbg_mask0;
        float *const dbg_shat = F.dbg_shat;
        uint8_t *const maskp = F.mask;
        const float mn = __uint_as_float(F.red[kRedMin]), mx = __uint_as_float(F.red[kRedMax]);
        // Pack mask0 = (S > s*) one row per warp, each lane loading one pixel
        // of every word of the row (all loads of the row in flight together).
        // Out-of-image bits = 1 (the first operation is an erosion; with
        // r_open = 0 the first is a dilation, padded below).  Rows outside
        // the apron actually needed (2*(r_open + r_close)) are left unused.
        const int apron = 2 * (ro + rc);
        for (int y = kMorApron - apron + warp; y < kMorApron + kMorRows + apron; y += nwarps) {
            const int gy = gy0 + y;
            const bool rin = gy >= 0 && gy < h;
            unsigned bits[kMorEW];
#pragma unroll
            for (int x = 0; x < kMorEW; x++) {
                const int gx = (wx0 + x) * 32 + lane;
                bits[x] = (rin && gx >= 0 && gx < w) ? __float_as_uint(Sp[(size_t)gy * p + gx]) : 0xffffffffu;
            }
#pragma unroll
            for (int x = 0; x < kMorEW; x++) {
                const bool inb = bits[x] != 0xffffffffu;
                const bool bit = inb ? bits[x] > sstar : true;
                if (keep && inb && y >= kMorApron && y < kMorApron + kMorRows && x >= 1 && x <= kMorWords) {
                    const int gx = (wx0 + x) * 32 + lane;
                    dbg_mask0[(size_t)gy * w + gx] = bit ? 1 : 0;
                    dbg_shat[(size_t)gy * w + gx] = normalise(__uint_as_float(bits[x]), mn, mx);
                }
                const unsigned word = __ballot_sync(0xffffffffu, bit);
                if (lane == 0) s_a[y][x] = word;
            }
        }
        __syncthreads();
        const int ylo = kMorApron - apron, yhi = kMorApron + kMorRows + apron;
        if (ro > 0) {
            morph_op(s_a, s_b, ro, true, wx0, gy0, w, h, false, ylo, yhi);
            morph_op(s_a, s_b, ro, false, wx0, gy0, w, h, rc == 0, ylo, yhi);
        } else {
            for (int i = threadIdx.x; i < (yhi - ylo) * kMorEW; i += blockDim.x) {
                const int y = ylo + i / kMorEW, x = i % kMorEW;
                s_a[y][x] &= in_image_bits(wx0 + x, gy0 + y, w, h);
            }
            __syncthreads();
        }
        if (rc > 0) {
            morph_op(s_a, s_b, rc, false, wx0, gy0, w, h, true, ylo, yhi);
            morph_op(s_a, s_b, rc, true, wx0, gy0, w, h, false, ylo, yhi);
        }
        // Unpack the tile: 4 pixels (one byte each) per item.
        for (int i = threadIdx.x; i < kMorRows * kMorWords * 8; i += blockDim.x) {
            const int r = i / (kMorWords * 8), q = i - r * (kMorWords * 8);
            const int gy = ty * kMorRows + r, gx = (tx * kMorWords) * 32 + q * 4;
            if (gy >= h || gx >= w) continue;
            const unsigned word = s_a[kMorApron + r][1 + (q >> 3)];
            const unsigned nib = (word >> ((q & 7) * 4)) & 0xfu;
            const unsigned bytes = (nib * 0x00204081u) & 0x01010101u;
            uint8_t *dst = maskp + (size_t)gy * w + gx;
            if (gx + 4 <= w && ((((size_t)gy * w + gx) & 3) == 0)) {
                *reinterpret_cast<unsigned *>(dst) = bytes;
            } else {
                for (int j = 0; j < 4 && gx + j < w; j++) dst[j] = (uint8_t)((bytes >> (8 * j)) & 1u);
            }
        }
        __syncthreads();
    }
}

void launch_frame_init(const BatchDesc *bd, int grid, cudaStream_t s) { k_frame_init<<<grid, 256, 0, s>>>(bd); }
namespace {
// k_saliency takes more than the default 48 KB of dynamic shared memory:
// raise its limit once per device.
void ensure_saliency_attr()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaFuncSetAttribute(k_saliency, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SalSmem::bytes);
    done[dev] = true;
}
}  // namespace

void launch_saliency(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s)
{
    ensure_saliency_attr();
    k_saliency<<<grid, 256, SalSmem::bytes, s>>>(bd, mc);
}
void launch_select_pass(const BatchDesc *bd, int pass, int grid, cudaStream_t s)
{
    if (pass == 1) k_select_pass<<<grid, 256, 0, s>>>(bd, pass);
    else k_select_cand<<<grid, 256, 0, s>>>(bd);
}
void launch_select_find(const BatchDesc *bd, const MethodConsts &mc, int pass, int grid, cudaStream_t s)
{
    k_select_find<<<grid, 256, 0, s>>>(bd, mc, pass);
}
void launch_morph(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s) { k_morph<<<grid, 256, 0, s>>>(bd, mc); }

int occupancy_mask_kernels()
{
    int a = 0, b = 0, c = 0;
    ensure_saliency_attr();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_saliency, 256, SalSmem::bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_select_pass, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_morph, 256, 0);
    return min(a, min(b, c));
}

bool morph_radius_supported(int r) { return r >= 0 && r <= kMorMaxR; }

}  // namespace flowroi
