// Optional denoising of the flow input (paper: §Optical flow extraction,
// a two-step denoising -- median filtering, then bilateral filtering --
// before the flow; Table 1 "Denoise", on or off).  The paper gives no
// sizes; this library's readings (also the oracle's):
//   - median over the 3x3 neighbourhood, replicate border;
//   - bilateral over the (2rb+1)^2 square of the median image, replicate
//     border, w(q) = exp(-|q-p|^2 / (2 sigma_s^2)) exp(-(I(q)-I(p))^2 / (2 sigma_r^2)),
//     out(p) = sum w I / sum w, in 8-bit units.
// The result replaces the raw frame as level 0 of the pyramid (the
// expansion reads it); the JPEG2000 front end still codes the raw frame.
//
// One block per 256x16 tile (the expansion's level-0 tiles): the raw
// samples of the tile plus an apron of rb+1 are staged (replicate border),
// the median image of the tile plus an apron of rb is formed from them
// (each apron position takes the median at its border-clamped pixel, which
// is the replicate border of the median image), then each thread walks
// down one column computing the bilateral sums.  The median is taken on
// the integer samples (scaling to 8-bit units is monotone, so it commutes)
// with a min/max network: sort the three rows, then the median of
// (largest row minimum, median of row medians, smallest row maximum).
// Weights are powers of two, 2^-(ls + lr d^2), through the ex2.approx
// instruction.
#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr int kDenTW = kExpTW, kDenTH = kExpTH;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void sort3(int &a, int &b, int &c)
{
    const int lo = min(a, b), hi = max(a, b);
    const int m = min(hi, c);
    c = max(hi, c);
    a = min(lo, m);
    b = max(lo, m);
}

__device__ __forceinline__ int med3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

}  // namespace

template <typename T, int RB>
__global__ void __launch_bounds__(256) k_denoise(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    constexpr int TW = kDenTW, TH = kDenTH, A = RB + 1;
    constexpr int IW = TW + 2 * A, IH = TH + 2 * A;     // staged raw samples
    constexpr int MW = TW + 2 * RB, MH = TH + 2 * RB;   // median image with the bilateral apron
    constexpr int S = 2 * kDenMaxR + 1;                  // row length of den_ls
    static_assert(TW == 256, "one thread per tile column");
    __shared__ int s_raw[IH][IW];
    __shared__ float s_med[MH][MW + 1];
    using ST = Store<T>;

    float ls[2 * RB + 1][2 * RB + 1];
#pragma unroll
    for (int dy = -RB; dy <= RB; dy++)
#pragma unroll
        for (int dx = -RB; dx <= RB; dx++) ls[dy + RB][dx + RB] = mc.den_ls[(dy + kDenMaxR) * S + dx + kDenMaxR];
    const float lr = mc.den_lr;

    const int nfr = bd->nframes;
    const int *off = bd->exp_off[0];
    const int total = __ldg(off + nfr);
    const int tid = threadIdx.x;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.lw[0], h = F.lh[0], p = F.lp[0];
        const int ntx = (w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * TW, y0 = (lt / ntx) * TH;
        const uint8_t *raw = static_cast<const uint8_t *>(F.raw);
        const int rp = F.raw_pitch, bpp = F.bpp;
        const float scale = F.unit_scale;
        T *const dst = static_cast<T *>(F.pyr[0]);
        float *const dbg = F.dbg_den;

        // stage the raw samples (replicate border)
        for (int i = tid; i < IH * IW; i += blockDim.x) {
            const int r = i / IW, c = i - r * IW;
            const int gy = clampi(y0 - A + r, 0, h - 1), gx = clampi(x0 - A + c, 0, w - 1);
            const uint8_t *row = raw + (size_t)gy * rp;
            s_raw[r][c] = bpp == 1 ? (int)__ldg(row + gx) : (int)__ldg(reinterpret_cast<const uint16_t *>(row) + gx);
        }
        __syncthreads();
        // the median image over the tile and the bilateral apron
        for (int i = tid; i < MH * MW; i += blockDim.x) {
            const int r = i / MW, c = i - r * MW;
            // border-clamped pixel, in staged coordinates
            const int sy = clampi(y0 - RB + r, 0, h - 1) - (y0 - A), sx = clampi(x0 - RB + c, 0, w - 1) - (x0 - A);
            int a0 = s_raw[sy - 1][sx - 1], a1 = s_raw[sy - 1][sx], a2 = s_raw[sy - 1][sx + 1];
            int b0 = s_raw[sy][sx - 1], b1 = s_raw[sy][sx], b2 = s_raw[sy][sx + 1];
            int c0 = s_raw[sy + 1][sx - 1], c1 = s_raw[sy + 1][sx], c2 = s_raw[sy + 1][sx + 1];
            sort3(a0, a1, a2);
            sort3(b0, b1, b2);
            sort3(c0, c1, c2);
            const int m = med3(max(a0, max(b0, c0)), med3(a1, b1, c1), min(a2, min(b2, c2)));
            s_med[r][c] = (float)m * scale;
        }
        __syncthreads();
        // bilateral: thread = column, walking down the rows
        const int gx = x0 + tid;
        if (gx < w) {
            for (int j = 0; j < TH; j++) {
                const int gy = y0 + j;
                if (gy >= h) break;
                const float cv = s_med[j + RB][tid + RB];
                float num = 0.f, den = 0.f;
#pragma unroll
                for (int dy = -RB; dy <= RB; dy++)
#pragma unroll
                    for (int dx = -RB; dx <= RB; dx++) {
                        const float q = s_med[j + RB + dy][tid + RB + dx];
                        const float d = q - cv;
                        const float wq = ex2_approx(-fmaf(lr * d, d, ls[dy + RB][dx + RB]));
                        num = fmaf(wq, q, num);
                        den += wq;
                    }
                const float v = __fdividef(num, den);
                ST::st(dst + (size_t)gy * p + gx, v);
                if (dbg) dbg[(size_t)gy * w + gx] = v;
            }
        }
        __syncthreads();
    }
}

template <typename T, int RB>
static void launch_t(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s)
{
    k_denoise<T, RB><<<grid, 256, 0, s>>>(bd, mc);
}

void launch_denoise(const BatchDesc *bd, const MethodConsts &mc, bool half, int grid, cudaStream_t s)
{
    switch (mc.den_r) {
    case 1: half ? launch_t<__half, 1>(bd, mc, grid, s) : launch_t<float, 1>(bd, mc, grid, s); break;
    case 2: half ? launch_t<__half, 2>(bd, mc, grid, s) : launch_t<float, 2>(bd, mc, grid, s); break;
    case 3: half ? launch_t<__half, 3>(bd, mc, grid, s) : launch_t<float, 3>(bd, mc, grid, s); break;
    default: break;
    }
}

int occupancy_denoise(bool half, int radius)
{
    int b = 0;
    switch (radius) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, half ? k_denoise<__half, 1> : k_denoise<float, 1>, 256, 0); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, half ? k_denoise<__half, 2> : k_denoise<float, 2>, 256, 0); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, half ? k_denoise<__half, 3> : k_denoise<float, 3>, 256, 0); break;
    default: break;
    }
    return b;
}

bool denoise_radius_supported(int r) { return r >= 1 && r <= kDenMaxR; }

}  // namespace flowroi
