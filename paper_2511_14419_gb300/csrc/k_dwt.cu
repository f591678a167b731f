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
// registers; then each (row, 16-coefficient segment) is lifted in
// registers from a 40-sample window of that row and its coefficients are
// quantised, shifted and stored.  Outputs come from window centres, which
// depend only on in-window samples.  The low-low band goes to a temporary
// plane for the next level (or, at the last level, into the coefficient
// plane).
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr float kA = -1.586134342059924f, kB = -0.052980118572961f, kG = 0.882911075530934f,
                kD = 0.443506852043971f, kK = 1.230174104914001f;
constexpr int kDwtHalo = 4;

// Whole-sample symmetric extension of index i into [0, n).  One
// reflection suffices when the apron is shorter than the signal; tiny
// signals take the periodic form.
__device__ __forceinline__ int mirror(int i, int n)
{
    if (i >= 0 && i < n) return i;
    if (n > kDwtHalo) return i < 0 ? -i : 2 * (n - 1) - i;
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
    for (int i = 0; i < N; i++) x[i] = (i & 1) ? x[i] * kK : __fdiv_rn(x[i], kK);
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
template <int WAV, int N>
__device__ __forceinline__ void mask_rule(const uint8_t (&m)[N], int e, uint8_t &lo, uint8_t &hi)
{
    constexpr int lo0 = WAV == 97 ? -3 : -1, lo1 = WAV == 97 ? 3 : 1;
    constexpr int hi0 = WAV == 97 ? -3 : -1, hi1 = WAV == 97 ? 5 : 3;
    uint8_t a = 0, b = 0;
#pragma unroll
    for (int d = lo0; d <= lo1; d++) a |= m[e + d];
#pragma unroll
    for (int d = hi0; d <= hi1; d++) b |= m[e + d];
    lo = a;
    hi = b;
}

template <int WAV>
__global__ void __launch_bounds__(256, 3) k_dwt(const BatchDesc *__restrict__ bd, MethodConsts mc, int level)
{
    using V = typename std::conditional<WAV == 97, float, int>::type;
    constexpr int TW = kDwtTW, TH = kDwtTH, HALO = kDwtHalo;
    constexpr int EW = 2 * TW + 2 * HALO, EH = 2 * TH + 2 * HALO;  // 136 x 72
    constexpr int SEG = 8;                                          // band outputs per row item
    constexpr int RW = 2 * SEG + 2 * HALO;                          // row window (24)
    __shared__ V s_x[EH][EW + 1];
    __shared__ uint8_t s_m[EH][EW + 4];

    const int nfr = bd->nframes;
    const int *off = bd->dwt_off[level - 1];
    const int total = __ldg(off + nfr);
    const bool last = level == mc.dwt_levels;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int W = F.W;
        const int iw = F.W >> (level - 1), ih = F.H >> (level - 1);
        const int bw = iw >> 1, bh = ih >> 1;
        const int ntx = (bw + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        const int bx0 = (lt % ntx) * TW, by0 = (lt / ntx) * TH;
        const int ix0 = 2 * bx0 - HALO, iy0 = 2 * by0 - HALO;
        // Descriptor fields in registers (the output stores below could
        // otherwise force their reloads).
        const V *llin = static_cast<const V *>(F.ll[level % 2]);
        const uint8_t *mlin = F.llm[level % 2];
        const uint8_t *fraw = static_cast<const uint8_t *>(F.raw);
        const uint8_t *fmask = F.mask;
        const int raw_pitch = F.raw_pitch, bpp = F.bpp, dc_off = F.dc_off;
        int32_t *const coeffs = F.coeffs;
        float *const dbg_yf = F.dbg_yf;
        V *const llout = static_cast<V *>(F.ll[(level - 1) % 2]);
        uint8_t *const llmout = F.llm[(level - 1) % 2];

        // Load: samples with symmetric extension, mask clipped (0 outside).
        // Two adjacent columns per item (ix0 is even, so an in-range pair is
        // one aligned 2-sample / 2-byte load); a thread issues all of its
        // items' loads before any shared-memory store.
        {
            const bool xin = ix0 >= 0 && ix0 + EW <= iw;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            constexpr int NR = (EH + 7) / 8, NP = (EW / 2 + 31) / 32;
            V v[NR][NP][2];
            uint8_t mm[NR][NP][2];
#pragma unroll
            for (int i = 0; i < NR; i++) {
                const int r = warp + 8 * i;
                const int gy = iy0 + r, my = mirror(gy, ih);
                const bool rin = gy >= 0 && gy < ih;
                const uint8_t *mrow = level == 1 ? fmask + (size_t)gy * W : mlin + (size_t)gy * iw;
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const int c = 2 * (lane + 32 * j), gx = ix0 + c;
                    v[i][j][0] = v[i][j][1] = (V)0;
                    mm[i][j][0] = mm[i][j][1] = 0;
                    if (r >= EH || c >= EW) continue;
                    if (level == 1) {
                        const uint8_t *row = fraw + (size_t)my * raw_pitch;
                        int r0, r1;
                        if (xin && bpp == 2) {
                            const unsigned pr = __ldg(reinterpret_cast<const unsigned *>(row) + (gx >> 1));
                            r0 = (int)(pr & 0xffffu);
                            r1 = (int)(pr >> 16);
                        } else {
                            const int m0 = mirror(gx, iw), m1 = mirror(gx + 1, iw);
                            r0 = bpp == 1 ? (int)__ldg(row + m0) : (int)__ldg(reinterpret_cast<const uint16_t *>(row) + m0);
                            r1 = bpp == 1 ? (int)__ldg(row + m1) : (int)__ldg(reinterpret_cast<const uint16_t *>(row) + m1);
                        }
                        v[i][j][0] = (V)(r0 - dc_off);
                        v[i][j][1] = (V)(r1 - dc_off);
                    } else {
                        const V *row = llin + (size_t)my * iw;
                        if (xin) {
                            v[i][j][0] = __ldg(row + gx);
                            v[i][j][1] = __ldg(row + gx + 1);
                        } else {
                            v[i][j][0] = __ldg(row + mirror(gx, iw));
                            v[i][j][1] = __ldg(row + mirror(gx + 1, iw));
                        }
                    }
                    if (rin) {
                        if (xin) {
                            const unsigned short m2 = __ldg(reinterpret_cast<const unsigned short *>(mrow + gx));
                            mm[i][j][0] = (uint8_t)(m2 & 0xff);
                            mm[i][j][1] = (uint8_t)(m2 >> 8);
                        } else {
                            if (gx >= 0 && gx < iw) mm[i][j][0] = __ldg(mrow + gx);
                            if (gx + 1 >= 0 && gx + 1 < iw) mm[i][j][1] = __ldg(mrow + gx + 1);
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
                    s_x[r][c] = v[i][j][0];
                    s_x[r][c + 1] = v[i][j][1];
                    s_m[r][c] = mm[i][j][0];
                    s_m[r][c + 1] = mm[i][j][1];
                }
        }
        __syncthreads();

        // Vertical: threads [0, EW) lift one column each in registers; the
        // other threads turn columns of the pixel mask into (low, high) row
        // masks with the 1-D rule, in place (a column is private to its item).
        if (threadIdx.x < EW) {
            const int c = threadIdx.x;
            V x[EH];
#pragma unroll
            for (int j = 0; j < EH; j++) x[j] = s_x[j][c];
            lift<V, EH>(x);
#pragma unroll
            for (int j = 0; j < EH; j++) s_x[j][c] = x[j];
        } else {
            for (int c = threadIdx.x - EW; c < EW; c += blockDim.x - EW) {
                uint8_t m[EH];
#pragma unroll
                for (int j = 0; j < EH; j++) m[j] = s_m[j][c];
#pragma unroll
                for (int k = 0; k < TH; k++) {
                    uint8_t lo, hi;
                    mask_rule<WAV, EH>(m, HALO + 2 * k, lo, hi);
                    s_m[HALO + 2 * k][c] = lo;       // even rows: low-vertical mask
                    s_m[HALO + 2 * k + 1][c] = hi;   // odd rows: high-vertical mask
                }
            }
        }
        __syncthreads();

        // Horizontal: one (output row, 16-coefficient segment) per thread.
        {
            const int rr = threadIdx.x / (TW / SEG), sg = threadIdx.x - rr * (TW / SEG);  // rr in [0, 2*TH)
            const int row = HALO + rr;         // even: low-vertical row, odd: high
            const int gj = by0 + (rr >> 1);
            const int c0 = sg * 2 * SEG;       // window start (covers its apron)
            if (rr < 2 * TH && gj < bh) {
                V x[RW];
                uint8_t m[RW];
#pragma unroll
                for (int j = 0; j < RW; j++) { x[j] = s_x[row][c0 + j]; m[j] = s_m[row][c0 + j]; }
                lift<V, RW>(x);
                const bool vhigh = rr & 1;
                const int b_lo = vhigh ? 3 * (level - 1) + 1 : 3 * mc.dwt_levels;  // LH or LL
                const int b_hi = vhigh ? 3 * (level - 1) + 2 : 3 * (level - 1);    // HH or HL
                const float d_lo = mc.delta[b_lo], d_hi = mc.delta[b_hi];
                const int ylo = vhigh ? bh + gj : gj;
#pragma unroll
                for (int k = 0; k < SEG; k++) {
                    const int gi = bx0 + sg * SEG + k;
                    if (gi >= bw) break;
                    uint8_t mlo, mhi;
                    mask_rule<WAV, RW>(m, HALO + 2 * k, mlo, mhi);
                    const V ylo_v = x[HALO + 2 * k], yhi_v = x[HALO + 2 * k + 1];
                    // high horizontal band (HL or HH)
                    const size_t ph = (size_t)ylo * W + bw + gi;
                    int32_t q = quantise(yhi_v, d_hi, WAV);
                    coeffs[ph] = mhi ? roi_up(q, mc.shift) : q;
                    if constexpr (WAV == 97) { if (dbg_yf) dbg_yf[ph] = yhi_v; }
                    // low horizontal band (LL or LH)
                    if (vhigh || last) {
                        const size_t pl = (size_t)ylo * W + gi;
                        q = quantise(ylo_v, d_lo, WAV);
                        coeffs[pl] = mlo ? roi_up(q, mc.shift) : q;
                        if constexpr (WAV == 97) { if (dbg_yf) dbg_yf[pl] = ylo_v; }
                    } else {
                        llout[(size_t)gj * bw + gi] = ylo_v;
                        llmout[(size_t)gj * bw + gi] = mlo;
                    }
                }
            }
        }
        __syncthreads();
    }
}

void launch_dwt(const BatchDesc *bd, const MethodConsts &mc, int level, int grid, cudaStream_t s)
{
    if (mc.wavelet == 97) k_dwt<97><<<grid, 256, 0, s>>>(bd, mc, level);
    else k_dwt<53><<<grid, 256, 0, s>>>(bd, mc, level);
}

int occupancy_dwt(int wavelet)
{
    int b = 0;
    if (wavelet == 97) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dwt<97>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dwt<53>, 256, 0);
    return b;
}

}  // namespace flowroi
