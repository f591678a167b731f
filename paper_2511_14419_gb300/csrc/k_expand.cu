// Gaussian pyramid + Farneback polynomial expansion, fused per level.
//
// Paper: §Optical flow extraction (dense Farneback flow).  The expansion
// fits, around every pixel, f(u,v) ~ r1 + r2 u + r3 v + r4 u^2 + r5 v^2 +
// r6 u v by least squares weighted with the separable Gaussian
// applicability a(u) a(v) over a (2n+1)^2 square (replicate border), and
// stores A = [[r4, r6/2], [r6/2, r5]], b = (r2, r3).  Because the weight
// is separable, the six weighted moments of the window are two passes of
// 1-D correlations (row pass: a, a*u, a*u^2; column pass: six outputs) and
// the least-squares solution is a closed form in those moments:
//   r_u = <u,f>/(s0 s2), r_v = <v,f>/(s0 s2), r_uv = <uv,f>/s2^2, and
//   (r_1, r_uu, r_vv) = M^-1 (<1,f>, <u^2,f>, <v^2,f>),
// with s_k = sum_u a(u) u^k (constants computed on the host).
//
// The same input tile (halo 2) also yields the next pyramid level:
// separable [1 4 6 4 1]/16 blur with replicate border, even samples.
//
// Level 0 reads the raw u8/u16 frame and converts to 8-bit units on the
// fly; level l > 0 reads the pyramid image written by level l-1.
// Storage type T (float or __half) holds pyramid images and fields; every
// arithmetic operation is in float.
#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

// Source of one level, with the descriptor fields it needs held in
// registers (read once per tile).
template <typename T>
struct LevelSrc {
    const uint8_t *raw;  // level 0: raw samples
    const T *img;        // level > 0: pyramid image
    int pitch;           // raw row pitch in bytes, or image pitch in elements
    int bpp;
    float scale;
    __device__ __forceinline__ LevelSrc(const FrameDesc &F, int level)
    {
        raw = static_cast<const uint8_t *>(F.raw);
        img = static_cast<const T *>(F.pyr[level]);
        bpp = F.bpp;
        scale = F.unit_scale;
        pitch = level == 0 ? F.raw_pitch : F.lp[level];
        if (level > 0) raw = nullptr;
    }
    __device__ __forceinline__ float at(int x, int y) const
    {
        if (raw) {
            if (bpp == 1) return (float)__ldg(raw + (size_t)y * pitch + x) * scale;
            return (float)__ldg(reinterpret_cast<const uint16_t *>(raw + (size_t)y * pitch) + x) * scale;
        }
        return Store<T>::ld(img + (size_t)y * pitch + x);
    }
};

}  // namespace

template <typename T, int NH>
__global__ void __launch_bounds__(256) k_expand(const BatchDesc *__restrict__ bd, MethodConsts mc, int level)
{
    constexpr int HALO = NH > 2 ? NH : 2;
    constexpr int IW = kExpTW + 2 * HALO, IH = kExpTH + 2 * HALO;
    constexpr int RH = kExpTH + 2 * NH;  // rows the column pass needs
    constexpr int BW = kExpTW / 2;
    __shared__ float s_in[IH][IW + 1];
    __shared__ float s_g[3][RH][kExpTW + 1];
    __shared__ float s_blur[IH][BW + 1];
    using ST = Store<T>;
    using T4 = typename ST::T4;
    const float b5[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};

    const int nfr = bd->nframes;
    const int *off = bd->exp_off[level];
    const int total = __ldg(off + nfr);
    const bool pyr_next = level + 1 < mc.pyr_levels;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.lw[level], h = F.lh[level], p = F.lp[level];
        const int ntx = (w + kExpTW - 1) / kExpTW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * kExpTW, y0 = (lt / ntx) * kExpTH;
        // A per-tile constant is removed before the fit (the fit of a
        // constant is that constant: A and b are unchanged) to keep the
        // single-precision moments small.
        const LevelSrc<T> src(F, level);
        T4 *fq = static_cast<T4 *>(F.fq_cur[level]);
        T *fb = static_cast<T *>(F.fb_cur[level]);
        T *pdst = pyr_next ? static_cast<T *>(F.pyr[level + 1]) : nullptr;
        const int wn = pyr_next ? F.lw[level + 1] : 0, hn = pyr_next ? F.lh[level + 1] : 0, pn = pyr_next ? F.lp[level + 1] : 0;
        const float c0 = src.at(min(x0 + kExpTW / 2, w - 1), min(y0 + kExpTH / 2, h - 1));
        {
            // All of a thread's loads first (up to 3 rows x 3 columns), then
            // the shared-memory stores, so the loads are in flight together.
            const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
            float v[3][3];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int r = ty + 8 * i, c = tx + 32 * j;
                    v[i][j] = 0.f;
                    if (r < IH && c < IW) {
                        const int gy = clampi(y0 - HALO + r, 0, h - 1), gx = clampi(x0 - HALO + c, 0, w - 1);
                        v[i][j] = src.at(gx, gy);
                    }
                }
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int r = ty + 8 * i, c = tx + 32 * j;
                    if (r < IH && c < IW) s_in[r][c] = v[i][j] - c0;
                }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < RH * kExpTW; i += blockDim.x) {
            const int r = i / kExpTW, c = i - r * kExpTW;
            const float *row = &s_in[r + HALO - NH][c + HALO - NH];
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
            for (int u = -NH; u <= NH; u++) {
                const float av = mc.app[u + NH] * row[u + NH];
                g0 += av;
                g1 += (float)u * av;
                g2 += (float)(u * u) * av;
            }
            s_g[0][r][c] = g0;
            s_g[1][r][c] = g1;
            s_g[2][r][c] = g2;
        }
        if (pyr_next) {
            for (int i = threadIdx.x; i < IH * BW; i += blockDim.x) {
                const int r = i / BW, k = i - r * BW;
                const float *row = &s_in[r][HALO + 2 * k - 2];
                s_blur[r][k] = b5[0] * row[0] + b5[1] * row[1] + b5[2] * row[2] + b5[3] * row[3] + b5[4] * row[4];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kExpTH * kExpTW; i += blockDim.x) {
            const int r = i / kExpTW, c = i - r * kExpTW;
            const int gx = x0 + c, gy = y0 + r;
            if (gx >= w || gy >= h) continue;
            float c00 = 0.f, c01 = 0.f, c02 = 0.f, c10 = 0.f, c11 = 0.f, c20 = 0.f;
#pragma unroll
            for (int v = -NH; v <= NH; v++) {
                const float a = mc.app[v + NH];
                const float g0 = s_g[0][r + v + NH][c], g1 = s_g[1][r + v + NH][c], g2 = s_g[2][r + v + NH][c];
                c00 += a * g0;
                c01 += (a * (float)v) * g0;
                c02 += (a * (float)(v * v)) * g0;
                c10 += a * g1;
                c11 += (a * (float)v) * g1;
                c20 += a * g2;
            }
            const float ruu = mc.m_uu[0] * c00 + mc.m_uu[1] * c20 + mc.m_uu[2] * c02;
            const float rvv = mc.m_vv[0] * c00 + mc.m_vv[1] * c20 + mc.m_vv[2] * c02;
            const float ruv = c11 * mc.inv_s2s2;
            const size_t o = (size_t)gy * p + gx;
            ST::st4(fq + o, ruu, 0.5f * ruv, rvv, c10 * mc.inv_s0s2);
            ST::st(fb + o, c01 * mc.inv_s0s2);
        }
        if (pyr_next) {
            for (int i = threadIdx.x; i < (kExpTH / 2) * BW; i += blockDim.x) {
                const int j = i / BW, k = i - j * BW;
                const int gx = x0 / 2 + k, gy = y0 / 2 + j;
                if (gx >= wn || gy >= hn) continue;
                const int r = HALO + 2 * j;
                const float v = b5[0] * s_blur[r - 2][k] + b5[1] * s_blur[r - 1][k] + b5[2] * s_blur[r][k] +
                                b5[3] * s_blur[r + 1][k] + b5[4] * s_blur[r + 2][k];
                ST::st(pdst + (size_t)gy * pn + gx, v + c0);
            }
        }
        __syncthreads();
    }
}

void launch_expand(const BatchDesc *bd, const MethodConsts &mc, int level, bool half, int grid, cudaStream_t s)
{
    const int n = mc.n_half;
    if (half) {
        if (n == 3) k_expand<__half, 3><<<grid, 256, 0, s>>>(bd, mc, level);
        else k_expand<__half, 2><<<grid, 256, 0, s>>>(bd, mc, level);
    } else {
        if (n == 3) k_expand<float, 3><<<grid, 256, 0, s>>>(bd, mc, level);
        else k_expand<float, 2><<<grid, 256, 0, s>>>(bd, mc, level);
    }
}

int occupancy_expand(bool half, int n_half)
{
    int b = 0;
    if (half) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, n_half == 3 ? k_expand<__half, 3> : k_expand<__half, 2>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, n_half == 3 ? k_expand<float, 3> : k_expand<float, 2>, 256, 0);
    return b;
}

}  // namespace flowroi
