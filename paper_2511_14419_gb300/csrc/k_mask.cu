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

// Saliency S, min/max of S, histogram of the first radix digit.
__global__ void __launch_bounds__(256) k_saliency(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    constexpr int TW = kSalTW, TH = kSalTH;
    __shared__ float s_m[TH + 2][TW + 2];
    __shared__ unsigned s_hist[kHistBins];
    __shared__ unsigned s_mn[8], s_mx[8];
    const int nfr = bd->nframes;
    const int *off = bd->sal_off;
    const int total = __ldg(off + nfr);
    const int buf = bd->final_flow_buf;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.W, h = F.H, p = F.lp[0];
        const int ntx = (w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * TW, y0 = (lt / ntx) * TH;
        const float2 *fl = F.flow[buf];
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) s_hist[i] = 0u;
        for (int i = threadIdx.x; i < (TH + 2) * (TW + 2); i += blockDim.x) {
            const int r = i / (TW + 2), c = i - r * (TW + 2);
            const int gy = clampi(y0 - 1 + r, 0, h - 1), gx = clampi(x0 - 1 + c, 0, w - 1);
            const float2 d = fl[(size_t)gy * p + gx];
            s_m[r][c] = sqrtf(d.x * d.x + d.y * d.y);
        }
        __syncthreads();
        unsigned mn = 0x7f800000u, mx = 0u;
        for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
            const int r = i / TW, c = i - r * TW;
            const int gx = x0 + c, gy = y0 + r;
            if (gx >= w || gy >= h) continue;
            const float gxv = 0.5f * (s_m[r + 1][c + 2] - s_m[r + 1][c]);
            const float gyv = 0.5f * (s_m[r + 2][c + 1] - s_m[r][c + 1]);
            const float S = mc.alpha * s_m[r + 1][c + 1] + (1.f - mc.alpha) * sqrtf(gxv * gxv + gyv * gyv);
            F.S[(size_t)gy * p + gx] = S;
            if (F.dbg_flow) F.dbg_flow[(size_t)gy * w + gx] = fl[(size_t)gy * p + gx];
            const unsigned b = __float_as_uint(S);
            mn = min(mn, b);
            mx = max(mx, b);
            atomicAdd(&s_hist[b >> digit_shift(0)], 1u);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if ((threadIdx.x & 31) == 0) { s_mn[threadIdx.x >> 5] = mn; s_mx[threadIdx.x >> 5] = mx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < (int)(blockDim.x >> 5); k++) { mn = min(mn, s_mn[k]); mx = max(mx, s_mx[k]); }
            atomicMin(F.red + kRedMin, mn);
            atomicMax(F.red + kRedMax, mx);
        }
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
            if (s_hist[i]) atomicAdd(F.red + kRedHist + i, s_hist[i]);
        __syncthreads();
    }
}

// Histogram of radix digit `pass` (1 or 2) over the values whose higher
// bits equal the prefix selected so far.
__global__ void __launch_bounds__(256) k_select_pass(const BatchDesc *__restrict__ bd, int pass)
{
    constexpr int TW = kSalTW, TH = kSalTH;
    __shared__ unsigned s_hist[kHistBins];
    const int nfr = bd->nframes;
    const int *off = bd->sal_off;
    const int total = __ldg(off + nfr);
    const int sh = digit_shift(pass), hi = sh + digit_bits(pass);
    const unsigned dmask = (1u << digit_bits(pass)) - 1u;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.W, h = F.H, p = F.lp[0];
        const int ntx = (w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * TW, y0 = (lt / ntx) * TH;
        const unsigned want = __ldg(F.red + kRedPrefix) >> hi;
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) s_hist[i] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
            const int r = i / TW, c = i - r * TW;
            const int gx = x0 + c, gy = y0 + r;
            if (gx >= w || gy >= h) continue;
            const unsigned b = __float_as_uint(F.S[(size_t)gy * p + gx]);
            if ((b >> hi) == want) atomicAdd(&s_hist[(b >> sh) & dmask], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
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
                if (F.dbg_thr) *F.dbg_thr = th;
            }
        }
        __syncthreads();
    }
}

// Threshold + opening + closing on a tile with an apron of
// 2*(r_open + r_close) pixels, in bytes in shared memory.
namespace {

constexpr int kMorMaxR = 4;
constexpr int kMorHalo = 4 * kMorMaxR;
constexpr int kMorEW = kMorTW + 2 * kMorHalo, kMorEH = kMorTH + 2 * kMorHalo;

// One separable min (erosion) or max (dilation) of radius r over the valid
// region [m, E-m) of `a`, result back in `a` (valid region then [m+r, E-m-r)).
__device__ __forceinline__ void morph_stage(uint8_t (*a)[kMorEW], uint8_t (*b)[kMorEW], int m, int r, bool erode)
{
    const int y0 = m, y1 = kMorEH - m, xa = m + r, xb = kMorEW - m - r;
    for (int i = threadIdx.x; i < (y1 - y0) * (xb - xa); i += blockDim.x) {
        const int y = y0 + i / (xb - xa), x = xa + i % (xb - xa);
        uint8_t v = a[y][x];
        for (int d = 1; d <= r; d++) {
            const uint8_t l = a[y][x - d], rr = a[y][x + d];
            v = erode ? (v & l & rr) : (v | l | rr);
        }
        b[y][x] = v;
    }
    __syncthreads();
    const int ya = m + r, yb = kMorEH - m - r;
    for (int i = threadIdx.x; i < (yb - ya) * (xb - xa); i += blockDim.x) {
        const int y = ya + i / (xb - xa), x = xa + i % (xb - xa);
        uint8_t v = b[y][x];
        for (int d = 1; d <= r; d++) {
            const uint8_t u = b[y - d][x], dd = b[y + d][x];
            v = erode ? (v & u & dd) : (v | u | dd);
        }
        a[y][x] = v;
    }
    __syncthreads();
}

// Out-of-image pixels of the valid region take the neutral value of the
// next operation (1 before an erosion, 0 before a dilation).
__device__ __forceinline__ void morph_pad(uint8_t (*a)[kMorEW], int m, int gx0, int gy0, int w, int h, uint8_t neutral)
{
    for (int i = threadIdx.x; i < kMorEH * kMorEW; i += blockDim.x) {
        const int y = i / kMorEW, x = i - y * kMorEW;
        if (y < m || y >= kMorEH - m || x < m || x >= kMorEW - m) continue;
        const int gx = gx0 + x, gy = gy0 + y;
        if (gx < 0 || gx >= w || gy < 0 || gy >= h) a[y][x] = neutral;
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(256) k_morph(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    __shared__ uint8_t s_a[kMorEH][kMorEW];
    __shared__ uint8_t s_b[kMorEH][kMorEW];
    const int nfr = bd->nframes;
    const int *off = bd->mor_off;
    const int total = __ldg(off + nfr);
    const int ro = mc.r_open, rc = mc.r_close;
    const int H0 = kMorHalo - 2 * (ro + rc);  // unused outer margin of the buffers
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.W, h = F.H, p = F.lp[0];
        const int ntx = (w + kMorTW - 1) / kMorTW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * kMorTW, y0 = (lt / ntx) * kMorTH;
        const int gx0 = x0 - kMorHalo, gy0 = y0 - kMorHalo;
        if (!F.has_prev) {
            for (int i = threadIdx.x; i < kMorTH * kMorTW; i += blockDim.x) {
                const int r = i / kMorTW, c = i - r * kMorTW;
                const int gx = x0 + c, gy = y0 + r;
                if (gx >= w || gy >= h) continue;
                F.mask[(size_t)gy * w + gx] = 0;
                if (F.dbg_mask0) F.dbg_mask0[(size_t)gy * w + gx] = 0;
                if (F.dbg_shat) F.dbg_shat[(size_t)gy * w + gx] = 0.f;
            }
            continue;
        }
        const float mn = __uint_as_float(F.red[kRedMin]), mx = __uint_as_float(F.red[kRedMax]);
        const float th = __uint_as_float(F.red[kRedTHat]);
        // mask0 on the buffer's used region; outside the image: 1 (the
        // first operation is an erosion, or with r_open = 0 a dilation
        // that the pad below fixes).
        for (int i = threadIdx.x; i < kMorEH * kMorEW; i += blockDim.x) {
            const int y = i / kMorEW, x = i - y * kMorEW;
            if (y < H0 || y >= kMorEH - H0 || x < H0 || x >= kMorEW - H0) continue;
            const int gx = gx0 + x, gy = gy0 + y;
            uint8_t v = 1;
            if (gx >= 0 && gx < w && gy >= 0 && gy < h) {
                const float sh = normalise(F.S[(size_t)gy * p + gx], mn, mx);
                v = sh > th ? 1 : 0;
                if (y >= kMorHalo && y < kMorHalo + kMorTH && x >= kMorHalo && x < kMorHalo + kMorTW) {
                    if (F.dbg_mask0) F.dbg_mask0[(size_t)gy * w + gx] = v;
                    if (F.dbg_shat) F.dbg_shat[(size_t)gy * w + gx] = sh;
                }
            }
            s_a[y][x] = v;
        }
        __syncthreads();
        int m = H0;
        if (ro > 0) {
            morph_stage(s_a, s_b, m, ro, true);
            m += ro;
        }
        morph_pad(s_a, m, gx0, gy0, w, h, 0);
        if (ro > 0) {
            morph_stage(s_a, s_b, m, ro, false);
            m += ro;
            morph_pad(s_a, m, gx0, gy0, w, h, 0);
        }
        if (rc > 0) {
            morph_stage(s_a, s_b, m, rc, false);
            m += rc;
        }
        morph_pad(s_a, m, gx0, gy0, w, h, 1);
        if (rc > 0) {
            morph_stage(s_a, s_b, m, rc, true);
            m += rc;
        }
        for (int i = threadIdx.x; i < kMorTH * kMorTW; i += blockDim.x) {
            const int r = i / kMorTW, c = i - r * kMorTW;
            const int gx = x0 + c, gy = y0 + r;
            if (gx >= w || gy >= h) continue;
            F.mask[(size_t)gy * w + gx] = s_a[kMorHalo + r][kMorHalo + c];
        }
        __syncthreads();
    }
}

void launch_frame_init(const BatchDesc *bd, int grid, cudaStream_t s) { k_frame_init<<<grid, 256, 0, s>>>(bd); }
void launch_saliency(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s)
{
    k_saliency<<<grid, 256, 0, s>>>(bd, mc);
}
void launch_select_pass(const BatchDesc *bd, int pass, int grid, cudaStream_t s) { k_select_pass<<<grid, 256, 0, s>>>(bd, pass); }
void launch_select_find(const BatchDesc *bd, const MethodConsts &mc, int pass, int grid, cudaStream_t s)
{
    k_select_find<<<grid, 256, 0, s>>>(bd, mc, pass);
}
void launch_morph(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s) { k_morph<<<grid, 256, 0, s>>>(bd, mc); }

int occupancy_mask_kernels()
{
    int a = 0, b = 0, c = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_saliency, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_select_pass, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_morph, 256, 0);
    return min(a, min(b, c));
}

bool morph_radius_supported(int r) { return r >= 0 && r <= kMorMaxR; }

}  // namespace flowroi
