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
// 5/3 needs 2).  Lifting runs in place in shared memory over the whole
// extended tile; outputs come from its centre, which depends only on
// in-tile samples.  The low-low band goes to a temporary plane for the
// next level (or, at the last level, quantised into the coefficient plane).
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr float kA = -1.586134342059924f, kB = -0.052980118572961f, kG = 0.882911075530934f,
                kD = 0.443506852043971f, kK = 1.230174104914001f;
constexpr int kDwtHalo = 4;
constexpr int kDwtEW = 2 * kDwtTW + 2 * kDwtHalo, kDwtEH = 2 * kDwtTH + 2 * kDwtHalo;

// Whole-sample symmetric extension of index i into [0, n).
__device__ __forceinline__ int mirror(int i, int n)
{
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

template <int WAV>
__global__ void __launch_bounds__(256) k_dwt(const BatchDesc *__restrict__ bd, MethodConsts mc, int level)
{
    using V = typename std::conditional<WAV == 97, float, int>::type;
    constexpr int TW = kDwtTW, TH = kDwtTH, EW = kDwtEW, EH = kDwtEH, HALO = kDwtHalo;
    constexpr int lo0 = WAV == 97 ? -3 : -1, lo1 = WAV == 97 ? 3 : 1;
    constexpr int hi0 = WAV == 97 ? -3 : -1, hi1 = WAV == 97 ? 5 : 3;
    __shared__ V s_x[EH][EW + 1];
    __shared__ uint8_t s_m[EH][EW];
    __shared__ uint8_t s_mv[2 * TH][EW];

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
        const V *llin = static_cast<const V *>(F.ll[level % 2]);
        const uint8_t *mlin = F.llm[level % 2];
        for (int i = threadIdx.x; i < EH * EW; i += blockDim.x) {
            const int r = i / EW, c = i - r * EW;
            const int gy = iy0 + r, gx = ix0 + c;
            const int my = mirror(gy, ih), mx = mirror(gx, iw);
            V v;
            if (level == 1) {
                const uint8_t *row = static_cast<const uint8_t *>(F.raw) + (size_t)my * F.raw_pitch;
                const int raw = F.bpp == 1 ? (int)__ldg(row + mx) : (int)__ldg(reinterpret_cast<const uint16_t *>(row) + mx);
                v = (V)(raw - F.dc_off);
            } else {
                v = llin[(size_t)my * iw + mx];
            }
            s_x[r][c] = v;
            uint8_t m = 0;
            if (gx >= 0 && gx < iw && gy >= 0 && gy < ih) m = level == 1 ? F.mask[(size_t)gy * W + gx] : mlin[(size_t)gy * iw + gx];
            s_m[r][c] = m;
        }
        __syncthreads();

        // Vertical lifting (every column), rows of each parity in turn.
        if constexpr (WAV == 97) {
            const float cst[4] = {kA, kB, kG, kD};
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const int par = (s % 2 == 0) ? 1 : 0;
                const int nr = (EH - 1 - par) / 2;  // rows par, par+2, ... in [1, EH-1)
                for (int i = threadIdx.x; i < nr * EW; i += blockDim.x) {
                    const int k = i / EW, c = i - k * EW;
                    const int r = par + 2 * k + (par == 0 ? 2 : 0);
                    if (r < 1 || r >= EH - 1) continue;
                    s_x[r][c] += cst[s] * (s_x[r - 1][c] + s_x[r + 1][c]);
                }
                __syncthreads();
            }
            for (int i = threadIdx.x; i < EH * EW; i += blockDim.x) {
                const int r = i / EW, c = i - r * EW;
                s_x[r][c] = (r & 1) ? s_x[r][c] * kK : __fdiv_rn(s_x[r][c], kK);
            }
            __syncthreads();
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const int par = (s % 2 == 0) ? 1 : 0;
                const int nc = (EW - 1 - par) / 2;
                for (int i = threadIdx.x; i < EH * nc; i += blockDim.x) {
                    const int r = i / nc, k = i - r * nc;
                    const int c = par + 2 * k + (par == 0 ? 2 : 0);
                    if (c < 1 || c >= EW - 1) continue;
                    s_x[r][c] += cst[s] * (s_x[r][c - 1] + s_x[r][c + 1]);
                }
                __syncthreads();
            }
            for (int i = threadIdx.x; i < EH * EW; i += blockDim.x) {
                const int r = i / EW, c = i - r * EW;
                s_x[r][c] = (c & 1) ? s_x[r][c] * kK : __fdiv_rn(s_x[r][c], kK);
            }
            __syncthreads();
        } else {
            for (int i = threadIdx.x; i < (EH / 2) * EW; i += blockDim.x) {
                const int k = i / EW, c = i - k * EW;
                const int r = 2 * k + 1;
                if (r >= EH - 1) continue;
                s_x[r][c] -= (s_x[r - 1][c] + s_x[r + 1][c]) >> 1;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < (EH / 2) * EW; i += blockDim.x) {
                const int k = i / EW, c = i - k * EW;
                const int r = 2 * k;
                if (r < 1 || r >= EH - 1) continue;
                s_x[r][c] += (s_x[r - 1][c] + s_x[r + 1][c] + 2) >> 2;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < EH * (EW / 2); i += blockDim.x) {
                const int r = i / (EW / 2), k = i - r * (EW / 2);
                const int c = 2 * k + 1;
                if (c >= EW - 1) continue;
                s_x[r][c] -= (s_x[r][c - 1] + s_x[r][c + 1]) >> 1;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < EH * (EW / 2); i += blockDim.x) {
                const int r = i / (EW / 2), k = i - r * (EW / 2);
                const int c = 2 * k;
                if (c < 1 || c >= EW - 1) continue;
                s_x[r][c] += (s_x[r][c - 1] + s_x[r][c + 1] + 2) >> 2;
            }
            __syncthreads();
        }

        // Wavelet-domain mask: vertical rule into s_mv (low rows, then high rows).
        for (int i = threadIdx.x; i < TH * EW; i += blockDim.x) {
            const int j = i / EW, c = i - j * EW;
            const int ce = HALO + 2 * j;
            uint8_t l = 0, hm = 0;
#pragma unroll
            for (int d = lo0; d <= lo1; d++) l |= s_m[ce + d][c];
#pragma unroll
            for (int d = hi0; d <= hi1; d++) hm |= s_m[ce + d][c];
            s_mv[j][c] = l;
            s_mv[TH + j][c] = hm;
        }
        __syncthreads();

        for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
            const int j = i / TW, k = i - j * TW;
            const int gi = bx0 + k, gj = by0 + j;
            if (gi >= bw || gj >= bh) continue;
            const int er = HALO + 2 * j, ec = HALO + 2 * k;
            uint8_t mll = 0, mhl = 0, mlh = 0, mhh = 0;
#pragma unroll
            for (int d = lo0; d <= lo1; d++) { mll |= s_mv[j][ec + d]; mlh |= s_mv[TH + j][ec + d]; }
#pragma unroll
            for (int d = hi0; d <= hi1; d++) { mhl |= s_mv[j][ec + d]; mhh |= s_mv[TH + j][ec + d]; }
            const V yll = s_x[er][ec], yhl = s_x[er][ec + 1], ylh = s_x[er + 1][ec], yhh = s_x[er + 1][ec + 1];
            const int b0 = 3 * (level - 1);
            const size_t phl = (size_t)gj * W + bw + gi, plh = (size_t)(bh + gj) * W + gi, phh = (size_t)(bh + gj) * W + bw + gi;
            int32_t q;
            q = quantise(yhl, mc.delta[b0 + 0], WAV);
            F.coeffs[phl] = mhl ? roi_up(q, mc.shift) : q;
            q = quantise(ylh, mc.delta[b0 + 1], WAV);
            F.coeffs[plh] = mlh ? roi_up(q, mc.shift) : q;
            q = quantise(yhh, mc.delta[b0 + 2], WAV);
            F.coeffs[phh] = mhh ? roi_up(q, mc.shift) : q;
            if constexpr (WAV == 97) {
                if (F.dbg_yf) {
                    F.dbg_yf[phl] = yhl;
                    F.dbg_yf[plh] = ylh;
                    F.dbg_yf[phh] = yhh;
                }
            }
            if (last) {
                const size_t pll = (size_t)gj * W + gi;
                q = quantise(yll, mc.delta[3 * mc.dwt_levels], WAV);
                F.coeffs[pll] = mll ? roi_up(q, mc.shift) : q;
                if constexpr (WAV == 97) {
                    if (F.dbg_yf) F.dbg_yf[pll] = yll;
                }
            } else {
                V *llout = static_cast<V *>(F.ll[(level - 1) % 2]);
                llout[(size_t)gj * bw + gi] = yll;
                F.llm[(level - 1) % 2][(size_t)gj * bw + gi] = mll;
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
