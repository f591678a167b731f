// JPEG2000 front end of the RoI encoder, one DWT level per launch:
// DC level shift (level 1), 2-D lifting DWT (columns then rows), dead-zone
// quantisation (9/7), wavelet-domain RoI mask, RoI up-shift.
//
// Paper: §Implementation details (JPEG2000 scaling-based RoI: RoI
// coefficients are scaled up by the user's scaling factor) and Table 1.
//   - DC shift: x - 2^(B-1).
//   - Lifting with whole-sample symmetric extension:
//       5/3: H[k] = x[2k+1] - floor((x[2k] + x[2k+2]) / 2)
//            L[k] = x[2k]   + floor((H[k-1] + H[k] + 2) / 4)
//       9/7: four lifting steps (alpha, beta, gamma, delta of the CDF 9/7
//            factorisation), then low / K and high * K.
//   - Quantisation (9/7): q = sign(y) floor(|y| / delta_b), decided in
//     float (IEEE division); 5/3: q = y.
//   - A coefficient is RoI when its synthesis support meets the RoI:
//       5/3: low k <- samples [2k-1, 2k+1], high k <- [2k-1, 2k+3]
//       9/7: low k <- samples [2k-3, 2k+3], high k <- [2k-3, 2k+5]
//     (clipped to the signal), applied to columns then rows of the
//     previous level's low-low mask (level 1: the pixel mask).
//   - RoI coefficients: q <- sign(q) (|q| << s).
//
// Tile scheme: a block owns kDwtTW x kDwtTH coefficients of each of the
// four bands of the level, i.e. a 2*TW x 2*TH input block plus a 4-sample
// apron loaded with the symmetric extension (for the 4-step 9/7 cone;
// 5/3 needs 2).  Each column of the extended tile is lifted in a thread's
// registers; then each (row, 16-sample segment) is lifted in registers
// from a 24-sample window of that row and its 8 low and 8 high
// coefficients are quantised, shifted and stored.  Outputs come from window centres, which
// depend only on in-window samples.  The low-low band goes to a temporary
// plane for the next level (or, at the last level, into the coefficient
// plane).  A batch entry's DWT codes the frame named by its dwt_* fields
// (with an adjacent factor, an earlier frame than the one whose flow the
// entry computes).
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr float kA = -1.586134342059924f, kB = -0.052980118572961f, kG = 0.882911075530934f,
                kD = 0.443506852043971f, kK = 1.230174104914001f;
// 1/K rounded to float: low samples are scaled by a product (one more
// rounding than a division, far inside the 9/7 coefficient tolerance).
constexpr float kInvK = (float)(1.0 / 1.230174104914001);
constexpr int kDwtHalo = 4;

// Whole-sample symmetric extension of index i into [0, n), for any i: one
// reflection where it lands inside, else the periodic form (a tile's apron
// reaches more than a signal length past the edge on small images).
__device__ __forceinline__ int mirror(int i, int n)
{
    if (i >= 0 && i < n) return i;
    if (i < 0 && -i < n) return -i;
    if (i >= n && i <= 2 * (n - 1)) return 2 * (n - 1) - i;
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    i %= period;
    if (i < 0) i += period;
    return i <= n - 1 ? i : period - i;
}

template <typename V>
__device__ __forceinline__ int32_t quantise(V y, float delta, int wav)
{
    if constexpr (std::is_same<V, float>::value) {
        const float a = __fdiv_rn(fabsf(y), delta);
        const int32_t m = (int32_t)floorf(a);
        return y < 0.f ? -m : m;
    } else {
        (void)delta;
        (void)wav;
        return (int32_t)y;
    }
}

__device__ __forceinline__ int32_t roi_up(int32_t q, int s) { return q < 0 ? -((-q) << s) : (q << s); }

__device__ __forceinline__ uint32_t smem_u32_dwt(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The low-low plane's 32-bit words as the level's sample type.
template <typename V>
__device__ __forceinline__ V __int_as_float_or_int(uint32_t u)
{
    if constexpr (std::is_same<V, float>::value) return __uint_as_float(u);
    else return (V)u;
}

}  // namespace

// One 1-D lifting pass over N register values (x[0] has even parity).
// Only positions 1..N-2 are updated (their neighbours exist); the caller's
// apron keeps the outputs it uses away from the stale ends.
template <int N>
__device__ __forceinline__ void lift97(float (&x)[N])
{
#pragma unroll
    for (int i = 1; i < N - 1; i += 2) x[i] += kA * (x[i - 1] + x[i + 1]);
#pragma unroll
    for (int i = 2; i < N - 1; i += 2) x[i] += kB * (x[i - 1] + x[i + 1]);
#pragma unroll
    for (int i = 1; i < N - 1; i += 2) x[i] += kG * (x[i - 1] + x[i + 1]);
#pragma unroll
    for (int i = 2; i < N - 1; i += 2) x[i] += kD * (x[i - 1] + x[i + 1]);
#pragma unroll
    for (int i = 0; i < N; i++) x[i] *= (i & 1) ? kK : kInvK;
}

template <int N>
__device__ __forceinline__ void lift53(int (&x)[N])
{
#pragma unroll
    for (int i = 1; i < N - 1; i += 2) x[i] -= (x[i - 1] + x[i + 1]) >> 1;
#pragma unroll
    for (int i = 2; i < N - 1; i += 2) x[i] += (x[i - 1] + x[i + 1] + 2) >> 2;
}

template <typename V, int N>
__device__ __forceinline__ void lift(V (&x)[N])
{
    if constexpr (std::is_same<V, float>::value) lift97<N>(x);
    else lift53<N>(x);
}

// 1-D mask rule on a register window: low k from [2k+lo0, 2k+lo1], high k
// from [2k+hi0, 2k+hi1] (relative to the window's even sample e = HALO+2k).
// Applied to 0/1 bytes, or to words of four such bytes (four columns).
template <int WAV, typename M, int N>
__device__ __forceinline__ void mask_rule(const M (&m)[N], int e, M &lo, M &hi)
{
    constexpr int lo0 = WAV == 97 ? -3 : -1, lo1 = WAV == 97 ? 3 : 1;
    constexpr int hi0 = WAV == 97 ? -3 : -1, hi1 = WAV == 97 ? 5 : 3;
    M a = 0, b = 0;
#pragma unroll
    for (int d = lo0; d <= lo1; d++) a |= m[e + d];
#pragma unroll
    for (int d = hi0; d <= hi1; d++) b |= m[e + d];
    lo = a;
    hi = b;
}

// A tile's geometry and descriptor fields, gathered by one thread two
// tiles ahead into shared memory, so the other threads take no dependent
// global loads per tile.
struct DwtTile {
    const void *llin;        // previous level's low-low plane (levels > 1)
    const uint8_t *mlin;     // ... and its mask
    const uint8_t *fraw;     // level 1: raw samples
    const uint8_t *fmask;    // level 1: pixel mask
    int32_t *coeffs;
    float *dbg_yf;
    void *llout;             // this level's low-low plane
    uint8_t *llmout;         // ... and its mask
    int W, iw, ih, bw, bh, bx0, by0, raw_pitch, bpp, dc_off, staged, pad;
};

// Shared-memory plan of k_dwt: the vertically lifted tile s_x [EH][EW+1]
// (sample type), the mask rows [NB][EH][MW] bytes, at level 1 the staged
// raw samples [2][EH][EW] (u16), and three tile headers.  Level 1
// double-buffers the mask and samples so the next tile's copies run during
// this tile's lifting.
template <int WAV, bool L1>
struct DwtSmem {
    using V = typename std::conditional<WAV == 97, float, int>::type;
    static constexpr int EW = 2 * kDwtTW + 2 * kDwtHalo, EH = 2 * kDwtTH + 2 * kDwtHalo;  // 136 x 40
    static constexpr int MW = EW + 4;                                                    // mask row stride
    static constexpr int NB = L1 ? 2 : 1;
    static constexpr size_t x_bytes = (size_t)EH * (EW + 1) * sizeof(V);
    static constexpr size_t m_off = (x_bytes + 15) / 16 * 16;
    static constexpr size_t r_off = (m_off + (size_t)NB * EH * MW + 15) / 16 * 16;
    static constexpr size_t h_off = (r_off + (L1 ? (size_t)2 * EH * EW * sizeof(uint16_t) : 0) + 15) / 16 * 16;
    static constexpr size_t bytes = h_off + 3 * sizeof(DwtTile);
};

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32_dwt(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32_dwt(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int WAV, bool L1>
__global__ void __launch_bounds__(256, 3) k_dwt(const BatchDesc *__restrict__ bd, MethodConsts mc, int level)
{
    using SM = DwtSmem<WAV, L1>;
    using V = typename SM::V;
    constexpr int TW = kDwtTW, TH = kDwtTH, HALO = kDwtHalo;
    constexpr int EW = SM::EW, EH = SM::EH, MW = SM::MW;
    constexpr int SEG = 8;                  // band outputs per row item
    constexpr int RW = 2 * SEG + 2 * HALO;  // row window (24)
    extern __shared__ __align__(16) unsigned char dsm[];
    V (*s_x)[EW + 1] = reinterpret_cast<V (*)[EW + 1]>(dsm);
    uint8_t *const s_mb = dsm + SM::m_off;                                  // [NB][EH][MW]
    uint16_t *const s_rb = reinterpret_cast<uint16_t *>(dsm + SM::r_off);  // [2][EH][EW] (level 1)
    DwtTile *const s_hdr = reinterpret_cast<DwtTile *>(dsm + SM::h_off);    // [3]

    const int nfr = bd->nframes;
    const int *off = bd->dwt_off[level - 1];
    const int total = __ldg(off + nfr);
    const bool last = level == mc.dwt_levels;

    // The header of tile t (thread 0).  Level 1: a tile's raw samples and
    // mask bytes are copied to the staging buffers with cp.async, 8 and 4
    // bytes per copy (4 samples, 4 mask bytes): sample rows through the
    // symmetric extension, chunks outside the image left out (the vertical
    // pass reads a column outside from its mirror image inside), mask
    // chunks and rows outside the image zero.
    auto fill_hdr = [&](int t, DwtTile &H) {
        if (t >= total) return;
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        H.W = F.W;
        H.iw = F.W >> (level - 1);
        H.ih = F.H >> (level - 1);
        H.bw = H.iw >> 1;
        H.bh = H.ih >> 1;
        const int ntx = (H.bw + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        H.bx0 = (lt % ntx) * TW;
        H.by0 = (lt / ntx) * TH;
        H.llin = F.ll[level % 2];
        H.mlin = F.llm[level % 2];
        H.fraw = static_cast<const uint8_t *>(F.dwt_raw);
        H.fmask = F.dwt_mask;
        H.raw_pitch = F.raw_pitch;
        H.bpp = F.bpp;
        H.dc_off = F.dc_off;
        H.coeffs = F.dwt_coeffs;
        H.dbg_yf = F.dwt_yf;
        H.llout = F.ll[(level - 1) % 2];
        H.llmout = F.llm[(level - 1) % 2];
        H.staged = L1 && F.bpp == 2 && ((reinterpret_cast<uintptr_t>(F.dwt_raw) | (uintptr_t)F.raw_pitch) & 7) == 0 &&
                   ((reinterpret_cast<uintptr_t>(F.dwt_mask) | (uintptr_t)F.W) & 3) == 0;
    };
    auto issue_async = [&](const DwtTile &H, int buf) {
        constexpr int NQ = EW / 4;  // 8-byte sample chunks (and 4-byte mask chunks) per row
        const int ix0 = 2 * H.bx0 - HALO, iy0 = 2 * H.by0 - HALO;
        uint16_t *rb = s_rb + (size_t)buf * EH * EW;
        uint8_t *mb = s_mb + (size_t)buf * EH * MW;
        for (int i = threadIdx.x; i < EH * NQ; i += blockDim.x) {
            const int r = i / NQ, q = i - r * NQ;
            const int gy = iy0 + r, gx = ix0 + 4 * q;  // ix0 and W are multiples of 4
            const bool xin = gx >= 0 && gx + 4 <= H.W;
            if (xin) cp_async8(rb + r * EW + 4 * q, H.fraw + (size_t)mirror(gy, H.ih) * H.raw_pitch + (size_t)gx * 2);
            if (xin && gy >= 0 && gy < H.ih) cp_async4(mb + r * MW + 4 * q, H.fmask + (size_t)gy * H.W + gx);
            else *reinterpret_cast<uint32_t *>(mb + r * MW + 4 * q) = 0u;
        }
    };
    if (threadIdx.x == 0) {
        fill_hdr(blockIdx.x, s_hdr[0]);
        fill_hdr(blockIdx.x + gridDim.x, s_hdr[1]);
    }
    __syncthreads();
    if (L1) {
        // prologue: the block's first tile
        if ((int)blockIdx.x < total && s_hdr[0].staged) issue_async(s_hdr[0], 0);
        cp_async_commit();
    }

    int k = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, k++) {
        const int cur = L1 ? (k & 1) : 0;
        uint8_t *const s_m = s_mb + (size_t)cur * EH * MW;
        uint16_t *const s_r = s_rb + (size_t)cur * EH * EW;
        const DwtTile &H = s_hdr[k % 3];
        const int W = H.W, iw = H.iw, ih = H.ih, bw = H.bw, bh = H.bh, bx0 = H.bx0, by0 = H.by0;
        const int ix0 = 2 * bx0 - HALO, iy0 = 2 * by0 - HALO;
        // Descriptor fields in registers (the output stores below could
        // otherwise force their reloads).
        const V *llin = static_cast<const V *>(H.llin);
        const uint8_t *mlin = H.mlin;
        const uint8_t *fraw = H.fraw;
        const uint8_t *fmask = H.fmask;
        const int raw_pitch = H.raw_pitch, bpp = H.bpp, dc_off = H.dc_off;
        int32_t *const coeffs = H.coeffs;
        float *const dbg_yf = H.dbg_yf;
        V *const llout = static_cast<V *>(H.llout);
        uint8_t *const llmout = H.llmout;
        const bool staged = L1 && H.staged;

        if (L1) {
            // start the next tile's copies into the other buffers (their last
            // reader, the previous tile's vertical pass, is behind a barrier)
            const DwtTile &Hn = s_hdr[(k + 1) % 3];
            if (t + (int)gridDim.x < total && Hn.staged) issue_async(Hn, cur ^ 1);
            cp_async_commit();
        }

        if (!staged) {
            // Samples with symmetric extension, mask clipped (0 outside).
            // Two adjacent columns per item (ix0 is even, so an in-range pair
            // is one aligned 2-sample / 2-byte load); a thread issues all of
            // its items' loads before any shared-memory store, holding level-1
            // sample pairs packed in one word and every mask pair in one word.
            const bool xin = ix0 >= 0 && ix0 + EW <= iw;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            constexpr int NR = (EH + 7) / 8, NP = (EW / 2 + 31) / 32;
            constexpr int NV = L1 ? 1 : 2;  // registers per sample pair
            uint32_t sv[NR][NP][NV];
            uint32_t mm[NR][NP];
#pragma unroll
            for (int i = 0; i < NR; i++) {
                const int r = warp + 8 * i;
                const int gy = iy0 + r, my = mirror(gy, ih);
                const bool rin = gy >= 0 && gy < ih;
                const uint8_t *mrow = L1 ? fmask + (size_t)gy * W : mlin + (size_t)gy * iw;
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const int c = 2 * (lane + 32 * j), gx = ix0 + c;
#pragma unroll
                    for (int e = 0; e < NV; e++) sv[i][j][e] = 0u;
                    mm[i][j] = 0u;
                    if (r >= EH || c >= EW) continue;
                    if constexpr (L1) {
                        const uint8_t *row = fraw + (size_t)my * raw_pitch;
                        if (xin && bpp == 2) {
                            sv[i][j][0] = __ldg(reinterpret_cast<const unsigned *>(row) + (gx >> 1));
                        } else {
                            const int m0 = mirror(gx, iw), m1 = mirror(gx + 1, iw);
                            const uint32_t r0 = bpp == 1 ? __ldg(row + m0) : __ldg(reinterpret_cast<const uint16_t *>(row) + m0);
                            const uint32_t r1 = bpp == 1 ? __ldg(row + m1) : __ldg(reinterpret_cast<const uint16_t *>(row) + m1);
                            sv[i][j][0] = r0 | (r1 << 16);
                        }
                    } else {
                        const uint32_t *row = reinterpret_cast<const uint32_t *>(llin) + (size_t)my * iw;
                        if (xin) {
                            const uint2 pr = __ldg(reinterpret_cast<const uint2 *>(row + gx));
                            sv[i][j][0] = pr.x;
                            sv[i][j][1] = pr.y;
                        } else {
                            sv[i][j][0] = __ldg(row + mirror(gx, iw));
                            sv[i][j][1] = __ldg(row + mirror(gx + 1, iw));
                        }
                    }
                    if (rin) {
                        if (xin) {
                            mm[i][j] = __ldg(reinterpret_cast<const unsigned short *>(mrow + gx));
                        } else {
                            const uint32_t m0 = gx >= 0 && gx < iw ? __ldg(mrow + gx) : 0;
                            const uint32_t m1 = gx + 1 >= 0 && gx + 1 < iw ? __ldg(mrow + gx + 1) : 0;
                            mm[i][j] = m0 | (m1 << 8);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NR; i++)
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const int r = warp + 8 * i, c = 2 * (lane + 32 * j);
                    if (r >= EH || c >= EW) continue;
                    if constexpr (L1) {
                        *reinterpret_cast<uint32_t *>(s_r + r * EW + c) = sv[i][j][0];
                    } else {
                        s_x[r][c] = __int_as_float_or_int<V>(sv[i][j][0]);
                        s_x[r][c + 1] = __int_as_float_or_int<V>(sv[i][j][1]);
                    }
                    *reinterpret_cast<uint16_t *>(s_m + r * MW + c) = (uint16_t)mm[i][j];
                }
        }
        if (L1) cp_async_wait_prior();  // this tile's staged copies have landed
        __syncthreads();
        // two tiles ahead: its header (the slot's last reader was the
        // previous tile, behind the barrier above)
        if (threadIdx.x == 0) fill_hdr(t + 2 * gridDim.x, s_hdr[(k + 2) % 3]);

        // Vertical: threads [0, EW) lift one column each in registers (level
        // 1 from the staged samples, with the DC shift); the next EW/4
        // threads turn four columns of the mask at a time (the byte lanes of
        // a word, made 0/1 first) into (low, high) row masks with the 1-D
        // rule, in place (the columns are private to their item).
        if (threadIdx.x < EW) {
            const int c = threadIdx.x;
            // a staged column outside the image is read from its mirror image
            // (clamped: columns that far out feed no stored output)
            const int cs = staged ? clampi(mirror(ix0 + c, iw) - ix0, 0, EW - 1) : c;
            V x[EH];
#pragma unroll
            for (int j = 0; j < EH; j++) {
                if constexpr (L1) x[j] = (V)((int)s_r[j * EW + cs] - dc_off);
                else x[j] = s_x[j][c];
            }
            lift<V, EH>(x);
#pragma unroll
            for (int j = 0; j < EH; j++) s_x[j][c] = x[j];
        } else if (threadIdx.x < EW + EW / 4) {
            const int c = 4 * (threadIdx.x - EW);
            uint32_t m[EH];
#pragma unroll
            for (int j = 0; j < EH; j++)
                m[j] = __vcmpne4(*reinterpret_cast<const uint32_t *>(s_m + j * MW + c), 0u) & 0x01010101u;
#pragma unroll
            for (int kk = 0; kk < TH; kk++) {
                uint32_t lo, hi;
                mask_rule<WAV>(m, HALO + 2 * kk, lo, hi);
                *reinterpret_cast<uint32_t *>(s_m + (HALO + 2 * kk) * MW + c) = lo;      // even rows: low-vertical mask
                *reinterpret_cast<uint32_t *>(s_m + (HALO + 2 * kk + 1) * MW + c) = hi;  // odd rows: high-vertical mask
            }
        }
        __syncthreads();

        // Horizontal: one (output row, 16-sample segment) per thread.
        {
            // a warp takes 16 consecutive rows x 2 segments: with the odd row
            // stride of s_x its 32 window reads fall in 32 different banks
            static_assert(2 * TH == 32 && TW / SEG == 8, "row-item map");
            const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
            const int rr = (wq & 1) * 16 + (lane & 15), sg = (wq >> 1) * 2 + (lane >> 4);  // rr in [0, 2*TH)
            const int row = HALO + rr;         // even: low-vertical row, odd: high
            const int gj = by0 + (rr >> 1);
            const int c0 = sg * 2 * SEG;       // window start (covers its apron)
            if (rr < 2 * TH && gj < bh) {
                V x[RW];
#pragma unroll
                for (int j = 0; j < RW; j++) x[j] = s_x[row][c0 + j];
                // the RW mask bytes (0/1) of the window as bits 0..RW-1
                uint32_t mb = 0;
#pragma unroll
                for (int q = 0; q < RW / 4; q++) {
                    const uint32_t wq = *reinterpret_cast<const uint32_t *>(&s_m[row * MW + c0 + 4 * q]);
                    mb |= ((wq * 0x01020408u) >> 24 & 0xfu) << (4 * q);
                }
                lift<V, RW>(x);
                const bool vhigh = rr & 1;
                const int b_lo = vhigh ? 3 * (level - 1) + 1 : 3 * mc.dwt_levels;  // LH or LL
                const int b_hi = vhigh ? 3 * (level - 1) + 2 : 3 * (level - 1);    // HH or HL
                const float d_lo = mc.delta[b_lo], d_hi = mc.delta[b_hi];
                const int ylo = vhigh ? bh + gj : gj;
                // the 1-D rule on bits: low k <- [e+lo0, e+lo1], high k <- [e+hi0, e+hi1], e = HALO+2k
                constexpr int lo0 = WAV == 97 ? -3 : -1, lo1 = WAV == 97 ? 3 : 1;
                constexpr int hi0 = WAV == 97 ? -3 : -1, hi1 = WAV == 97 ? 5 : 3;
                constexpr uint32_t lom = (1u << (lo1 - lo0 + 1)) - 1u, him = (1u << (hi1 - hi0 + 1)) - 1u;
                int32_t qh[SEG], ql[SEG];
#pragma unroll
                for (int k = 0; k < SEG; k++) {
                    const bool mlo = (mb >> (HALO + 2 * k + lo0)) & lom;
                    const bool mhi = (mb >> (HALO + 2 * k + hi0)) & him;
                    const V ylo_v = x[HALO + 2 * k], yhi_v = x[HALO + 2 * k + 1];
                    const int32_t a = quantise(yhi_v, d_hi, WAV);
                    qh[k] = mhi ? roi_up(a, mc.shift) : a;
                    const int32_t b = quantise(ylo_v, d_lo, WAV);
                    ql[k] = mlo ? roi_up(b, mc.shift) : b;
                }
                const int gi0 = bx0 + sg * SEG;
                const bool lo_band = vhigh || last;  // low horizontal band to the coefficients (LH or LL)
                int32_t *const ph = coeffs + (size_t)ylo * W + bw + gi0;
                int32_t *const pl = coeffs + (size_t)ylo * W + gi0;
                if (gi0 + SEG <= bw && (bw & 3) == 0) {
#pragma unroll
                    for (int k = 0; k < SEG; k += 4) {
                        *reinterpret_cast<int4 *>(ph + k) = make_int4(qh[k], qh[k + 1], qh[k + 2], qh[k + 3]);
                        if (lo_band) *reinterpret_cast<int4 *>(pl + k) = make_int4(ql[k], ql[k + 1], ql[k + 2], ql[k + 3]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < SEG; k++) {
                        if (gi0 + k >= bw) break;
                        ph[k] = qh[k];
                        if (lo_band) pl[k] = ql[k];
                    }
                }
                if (!lo_band) {
#pragma unroll
                    for (int k = 0; k < SEG; k++) {
                        if (gi0 + k >= bw) break;
                        llout[(size_t)gj * bw + gi0 + k] = x[HALO + 2 * k];
                        llmout[(size_t)gj * bw + gi0 + k] = (mb >> (HALO + 2 * k + lo0)) & lom ? 1 : 0;
                    }
                }
                if constexpr (WAV == 97) {
                    if (dbg_yf) {
#pragma unroll
                        for (int k = 0; k < SEG; k++) {
                            if (gi0 + k >= bw) break;
                            dbg_yf[(size_t)ylo * W + bw + gi0 + k] = x[HALO + 2 * k + 1];
                            if (lo_band) dbg_yf[(size_t)ylo * W + gi0 + k] = x[HALO + 2 * k];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (L1) cp_async_wait_all();
}

namespace {

// The kernels take more than the default 48 KB of dynamic shared memory:
// raise their limit once per device.
template <int WAV, bool L1>
void dwt_attr()
{
    cudaFuncSetAttribute(k_dwt<WAV, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DwtSmem<WAV, L1>::bytes);
}

void ensure_dwt_attrs()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    dwt_attr<97, true>();
    dwt_attr<97, false>();
    dwt_attr<53, true>();
    dwt_attr<53, false>();
    done[dev] = true;
}

}  // namespace

void launch_dwt(const BatchDesc *bd, const MethodConsts &mc, int level, int grid, cudaStream_t s)
{
    ensure_dwt_attrs();
    if (mc.wavelet == 97) {
        if (level == 1) k_dwt<97, true><<<grid, 256, DwtSmem<97, true>::bytes, s>>>(bd, mc, level);
        else k_dwt<97, false><<<grid, 256, DwtSmem<97, false>::bytes, s>>>(bd, mc, level);
    } else {
        if (level == 1) k_dwt<53, true><<<grid, 256, DwtSmem<53, true>::bytes, s>>>(bd, mc, level);
        else k_dwt<53, false><<<grid, 256, DwtSmem<53, false>::bytes, s>>>(bd, mc, level);
    }
}

int occupancy_dwt(int wavelet)
{
    // the level-1 kernel (staging buffers) bounds the occupancy
    ensure_dwt_attrs();
    int a = 0, b = 0;
    if (wavelet == 97) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_dwt<97, true>, 256, DwtSmem<97, true>::bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dwt<97, false>, 256, DwtSmem<97, false>::bytes);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_dwt<53, true>, 256, DwtSmem<53, true>::bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dwt<53, false>, 256, DwtSmem<53, false>::bytes);
    }
    return a < b ? a : b;
}

}  // namespace flowroi
