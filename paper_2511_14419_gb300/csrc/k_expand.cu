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
// fly (or reads the denoised frame when denoising is on); level l > 0 reads
// the pyramid image written by level l-1.
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
    const T *img;        // level > 0 (or denoised level 0): pyramid image
    int pitch;           // raw row pitch in bytes, or image pitch in elements
    int bpp;
    float scale;
    __device__ __forceinline__ LevelSrc(const uint8_t *raw_, const T *img_, int pitch_, int bpp_, float scale_)
        : raw(raw_), img(img_), pitch(pitch_), bpp(bpp_), scale(scale_)
    {
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

// Per-tile descriptor fields, gathered by one thread two tiles ahead into
// shared memory (the other threads take no dependent global loads per
// tile).
template <typename T>
struct ExpTile {
    using T4 = typename Store<T>::T4;
    const uint8_t *raw;  // level-0 raw samples (null when the level reads an image)
    const T *img;        // pyramid image of the level
    T4 *fq;
    T *fb;
    T *pnext;            // next pyramid level (null at the top)
    float scale;
    int x0, y0, w, h, p, pitch, bpp, staged, wn, hn, pn;
};

// One block per kExpTW x kExpTH tile (kExpTW = the block's 256 threads):
// the tile plus a HALO apron (replicate border) is staged in shared memory
// once; then each thread walks down its column, forming the three row
// moments of each row from 2n+1 neighbours and, from a sliding window of
// 2n+1 rows of them, the six window moments of each output pixel, all in
// registers.  The applicability is even, so both passes fold the taps in
// symmetric pairs (sums for the even moments, differences for the odd).
// The next pyramid level's even samples are blurred from the same staged
// tile: a row pass at even columns into a second buffer, then a column
// pass at even rows.
//
// Level 0 from raw samples (16-byte aligned rows, width a multiple of 16
// bytes): the next tile's rows (row-clamped, 16-byte chunks inside the
// image) are copied with cp.async into one of two raw buffers while this
// tile is expanded; the conversion to 8-bit units then applies the column
// clamp from the staged copy.  Other levels and sources load directly.
template <typename T, int NH>
__global__ void __launch_bounds__(256, 4) k_expand(const BatchDesc *__restrict__ bd, MethodConsts mc, int level)
{
    constexpr int TW = kExpTW, TH = kExpTH;
    constexpr int HALO = NH > 2 ? NH : 2;
    constexpr int IW = TW + 2 * HALO, IH = TH + 2 * HALO;
    constexpr int BW = TW / 2, HR = IH / 2;
    constexpr int NLD = (IH * IW + TW - 1) / TW;  // staged elements per thread
    constexpr int SRB = (TW + 2 * 8) * 2;         // raw row bytes: 16-bit samples, one chunk each side
    static_assert(TW == 256 && IW % 2 == 0 && IH % 2 == 0, "tile geometry");
    static_assert(IH * BW * sizeof(float) <= (size_t)IH * SRB, "pyramid row buffer fits a raw buffer");
    __shared__ __align__(16) float s_in[IH][IW];
    __shared__ __align__(16) uint8_t s_raw[2][IH][SRB];
    __shared__ ExpTile<T> s_hdr[3];
    using ST = Store<T>;
    using T4 = typename ST::T4;

    // applicability taps a(u) and their first / second moments, u = 1..n
    float a0 = mc.app[NH], au[NH + 1], au1[NH + 1], au2[NH + 1];
#pragma unroll
    for (int u = 1; u <= NH; u++) {
        au[u] = mc.app[NH + u];
        au1[u] = (float)u * au[u];
        au2[u] = (float)(u * u) * au[u];
    }

    const int nfr = bd->nframes;
    const int *off = bd->exp_off[level];
    const int total = __ldg(off + nfr);
    const bool pyr_next = level + 1 < mc.pyr_levels;
    const int tid = threadIdx.x;

    auto fill_hdr = [&](int t, ExpTile<T> &H) {
        if (t >= total) return;
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.lw[level], h = F.lh[level];
        const int ntx = (w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        H.x0 = (lt % ntx) * TW;
        H.y0 = (lt / ntx) * TH;
        H.w = w;
        H.h = h;
        H.p = F.lp[level];
        // level 0 is the raw frame, or its denoised image when one exists
        H.img = static_cast<const T *>(F.pyr[level]);
        H.raw = H.img ? nullptr : static_cast<const uint8_t *>(F.raw);
        H.bpp = F.bpp;
        H.scale = F.unit_scale;
        H.pitch = H.raw ? F.raw_pitch : F.lp[level];
        H.fq = static_cast<T4 *>(F.fq_cur[level]);
        H.fb = static_cast<T *>(F.fb_cur[level]);
        H.pnext = pyr_next ? static_cast<T *>(F.pyr[level + 1]) : nullptr;
        H.wn = pyr_next ? F.lw[level + 1] : 0;
        H.hn = pyr_next ? F.lh[level + 1] : 0;
        H.pn = pyr_next ? F.lp[level + 1] : 0;
        H.staged = H.raw && (H.bpp == 1 || H.bpp == 2) &&
                   ((reinterpret_cast<uintptr_t>(H.raw) | (uintptr_t)H.pitch | (uintptr_t)(w * H.bpp)) & 15) == 0;
    };
    // cp.async of a staged tile: rows clamped to the image, 16-byte chunks
    // [x0 - CE, x0 + TW + CE) that lie inside it (CE samples per chunk)
    auto issue_raw = [&](const ExpTile<T> &H, int buf) {
        const int ce = 16 / H.bpp, nch = TW / ce + 2, xs = H.x0 - ce;
        for (int i = tid; i < IH * nch; i += TW) {
            const int r = i / nch, q = i - r * nch, gx = xs + q * ce;
            if (gx < 0 || gx + ce > H.w) continue;
            const int gy = clampi(H.y0 - HALO + r, 0, H.h - 1);
            const uint8_t *src = H.raw + (size_t)gy * H.pitch + (size_t)gx * H.bpp;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(
                             &s_raw[buf][r][q * 16])),
                         "l"(src)
                         : "memory");
        }
    };

    if (tid == 0) {
        fill_hdr(blockIdx.x, s_hdr[0]);
        fill_hdr(blockIdx.x + gridDim.x, s_hdr[1]);
    }
    __syncthreads();
    if ((int)blockIdx.x < total && s_hdr[0].staged) issue_raw(s_hdr[0], 0);
    asm volatile("cp.async.commit_group;" ::: "memory");

    int k = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, k++) {
        const ExpTile<T> &H = s_hdr[k % 3];
        const int w = H.w, h = H.h, p = H.p, x0 = H.x0, y0 = H.y0;
        float c0;
        if (H.staged) {
            // this tile's copies, then the column clamp and the conversion
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            const int bpp = H.bpp, xs = x0 - 16 / bpp;
            const float scale = H.scale;
            const uint8_t *rb = &s_raw[k & 1][0][0];
            auto raw_at = [&](int r, int gx) {
                const int i = gx - xs;
                return (bpp == 2 ? (float)reinterpret_cast<const uint16_t *>(rb + r * SRB)[i] : (float)rb[r * SRB + i]) *
                       scale;
            };
            // A per-tile constant is removed before the fit (the fit of a
            // constant is that constant: A and b are unchanged) to keep the
            // single-precision moments small.
            c0 = raw_at(HALO + TH / 2, min(x0 + TW / 2, w - 1));
            for (int e = tid; e < IH * IW; e += TW) {
                const int r = e / IW, cc = e - r * IW;
                s_in[r][cc] = raw_at(r, clampi(x0 - HALO + cc, 0, w - 1)) - c0;
            }
        } else {
            const LevelSrc<T> src(H.raw, H.img, H.pitch, H.bpp, H.scale);
            c0 = src.at(min(x0 + TW / 2, w - 1), min(y0 + TH / 2, h - 1));
            // every load of the thread first, then the shared-memory stores
            float v[NLD];
#pragma unroll
            for (int i = 0; i < NLD; i++) {
                const int e = i * TW + tid, r = e / IW, cc = e - r * IW;
                v[i] = 0.f;
                if (e < IH * IW) {
                    const int gy = clampi(y0 - HALO + r, 0, h - 1), gx = clampi(x0 - HALO + cc, 0, w - 1);
                    v[i] = src.at(gx, gy);
                }
            }
#pragma unroll
            for (int i = 0; i < NLD; i++) {
                const int e = i * TW + tid, r = e / IW, cc = e - r * IW;
                if (e < IH * IW) s_in[r][cc] = v[i] - c0;
            }
        }
        __syncthreads();
        // two tiles ahead: the header; one tile ahead: the raw copies (their
        // buffer's last reader was the previous tile's conversion)
        if (tid == 0) fill_hdr(t + 2 * gridDim.x, s_hdr[(k + 2) % 3]);
        {
            const ExpTile<T> &Hn = s_hdr[(k + 1) % 3];
            if (t + (int)gridDim.x < total && Hn.staged) issue_raw(Hn, (k + 1) & 1);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        T4 *const fq = H.fq;
        T *const fb = H.fb;

        // expansion: thread = column, walking down the rows
        {
            const int gx = x0 + tid;
            float m0[IH], m1[IH], m2[IH];  // row moments (only a sliding window stays live)
#pragma unroll
            for (int r = HALO - NH; r < HALO + TH + NH; r++) {
                const float *row = &s_in[r][tid + HALO];
                float g0 = a0 * row[0], g1 = 0.f, g2 = 0.f;
#pragma unroll
                for (int u = 1; u <= NH; u++) {
                    const float xp = row[u], xm = row[-u];
                    const float su = xp + xm, du = xp - xm;
                    g0 = fmaf(au[u], su, g0);
                    g1 = fmaf(au1[u], du, g1);
                    g2 = fmaf(au2[u], su, g2);
                }
                m0[r] = g0;
                m1[r] = g1;
                m2[r] = g2;
                const int j = r - HALO - NH;  // output row completed by this row
                if (j >= 0) {
                    const int cr = HALO + j;
                    float c00 = a0 * m0[cr], c01 = 0.f, c02 = 0.f, c10 = a0 * m1[cr], c11 = 0.f, c20 = a0 * m2[cr];
#pragma unroll
                    for (int q = 1; q <= NH; q++) {
                        const float s0 = m0[cr + q] + m0[cr - q], d0 = m0[cr + q] - m0[cr - q];
                        const float s1 = m1[cr + q] + m1[cr - q], d1 = m1[cr + q] - m1[cr - q];
                        const float s2 = m2[cr + q] + m2[cr - q];
                        c00 = fmaf(au[q], s0, c00);
                        c01 = fmaf(au1[q], d0, c01);
                        c02 = fmaf(au2[q], s0, c02);
                        c10 = fmaf(au[q], s1, c10);
                        c11 = fmaf(au1[q], d1, c11);
                        c20 = fmaf(au[q], s2, c20);
                    }
                    const int gy = y0 + j;
                    if (gx < w && gy < h) {
                        const float ruu = mc.m_uu[0] * c00 + mc.m_uu[1] * c20 + mc.m_uu[2] * c02;
                        const float rvv = mc.m_vv[0] * c00 + mc.m_vv[1] * c20 + mc.m_vv[2] * c02;
                        const float ruv = c11 * mc.inv_s2s2;
                        const size_t o = (size_t)gy * p + gx;
                        ST::st4(fq + o, ruu, 0.5f * ruv, rvv, c10 * mc.inv_s0s2);
                        ST::st(fb + o, c01 * mc.inv_s0s2);
                    }
                }
            }
        }

        if (pyr_next) {
            // [1 4 6 4 1]/16 along rows at even columns (half the rows per
            // thread), into this tile's raw buffer (its samples are converted)
            float(*s_hb)[BW] = reinterpret_cast<float(*)[BW]>(&s_raw[k & 1][0][0]);
            const int kk = tid & (BW - 1), r0 = (tid / BW) * HR;
#pragma unroll
            for (int i = 0; i < HR; i++) {
                const float *row = &s_in[r0 + i][HALO + 2 * kk];
                s_hb[r0 + i][kk] = (6.f * row[0] + 4.f * (row[-1] + row[1]) + (row[-2] + row[2])) * (1.f / 16.f);
            }
            __syncthreads();
            // ... and along columns at even rows
            T *pdst = H.pnext;
            const int wn = H.wn, hn = H.hn, pn = H.pn;
            const int gi = x0 / 2 + kk;
#pragma unroll
            for (int q = 0; q < TH / 4; q++) {
                const int jj = (tid / BW) * (TH / 4) + q, gj = y0 / 2 + jj;
                const int cr = HALO + 2 * jj;
                const float vv = (6.f * s_hb[cr][kk] + 4.f * (s_hb[cr - 1][kk] + s_hb[cr + 1][kk]) +
                                  (s_hb[cr - 2][kk] + s_hb[cr + 2][kk])) * (1.f / 16.f);
                if (gi < wn && gj < hn) ST::st(pdst + (size_t)gj * pn + gi, vv + c0);
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
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
