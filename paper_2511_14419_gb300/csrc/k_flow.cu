// Farneback displacement estimation: one iteration at one pyramid level,
// fused (update, box window, 2x2 solve) in one pass over a tile.
//
// Paper: §Optical flow extraction (dense Farneback flow between adjacent
// frames).  With f1 = the current frame and f2 = its predecessor, and a
// prior displacement d~ (the coarser level's flow, bilinearly upsampled at
// (x/2, y/2) and doubled, at the first iteration of a level; the previous
// iteration's flow after that):
//     A  = (A1(x) + A2(x + d~)) / 2             (A2, b2 read bilinearly,
//     db = -(b2(x + d~) - b1(x)) / 2 + A d~      position clamped to the image)
//     G  = A^T A,  h = A^T db
//     G_, h_ = means over the (2r+1)^2 box around x (clipped to the image)
//     d  = adj(G_) h_ / (det G_ + lambda)
//
// Two kernels per iteration: k_update computes G and h per pixel into five
// planes (no apron recompute, no shared memory: full occupancy hides the
// gather latency); k_window forms the box means over a shared-memory tile
// and solves.  Box sums keep a column (row segment) in registers and form
// every window from a block suffix sum and a block prefix sum (no running
// sums: every window is a fresh sum of its own 2r+1 terms, so no
// cancellation between far-apart values).
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace flowroi {

namespace {

// out[i] = v[i] + ... + v[i + WN - 1] for i < N - WN + 1.  The column is
// cut into blocks of WN starting at 0; a window starting at i either is
// one whole block (i a multiple of WN) or ends in the next block, so it is
// the suffix sum of i's block from i plus the prefix sum of the next block
// up to i + WN - 1 (the van Herk / Gil-Werman decomposition, here for sums
// instead of extrema).  About three additions per output instead of
// log2(WN) per output plus the partial-sum pyramid, and each window is
// still a fresh sum of its own WN terms.  All indices are compile-time
// after unrolling; sums nothing reads are removed by the compiler.
template <int N, int WN>
__device__ __forceinline__ void box_sums(const float (&v)[N], float (&out)[N - WN + 1])
{
    constexpr int M = N - WN + 1;
    float suf[N], pre[N];
#pragma unroll
    for (int j = N - 1; j >= 0; j--) {
        if (j % WN == WN - 1 || j == N - 1) suf[j] = v[j];
        else suf[j] = v[j] + suf[j + 1];
    }
#pragma unroll
    for (int j = 0; j < N; j++) {
        if (j % WN == 0) pre[j] = v[j];
        else pre[j] = pre[j - 1] + v[j];
    }
#pragma unroll
    for (int i = 0; i < M; i++) out[i] = (i % WN == 0) ? suf[i] : suf[i] + pre[i + WN - 1];
}

// a*b - c*d with one rounding error at most a few ulps (FMA error-free
// transformation of c*d).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d)
{
    const float cd = c * d;
    const float err = fmaf(-c, d, cd);
    const float dop = fmaf(a, b, -cd);
    return dop + err;
}

}  // namespace

// ---------------------------------------------------------------- update
// Per pixel G = A^T A and h = A^T db (5 values) into five planes.  One
// thread owns a column of kUpdRows rows of a 256-wide row band, so its
// loads for those pixels are in flight together; no shared memory, full
// occupancy hides the gather latency.
template <typename T>
__global__ void __launch_bounds__(256) k_update(const BatchDesc *__restrict__ bd, MethodConsts mc, int level, int iter,
                                              int src)
{
    using ST = Store<T>;
    using T4 = typename ST::T4;
    const int nfr = bd->nframes;
    const int *off = bd->flow_off[level];
    const int total = __ldg(off + nfr);
    const bool top = level == mc.pyr_levels - 1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.lw[level], h = F.lh[level], p = F.lp[level];
        const int ntx = (w + kUpdTW - 1) / kUpdTW;
        const int lt = t - __ldg(off + fi);
        const int gx = (lt % ntx) * kUpdTW + threadIdx.x, y0 = (lt / ntx) * kUpdRows;
        if (gx >= w) continue;
        const T4 *q1 = static_cast<const T4 *>(F.fq_cur[level]);
        const T *b1p = static_cast<const T *>(F.fb_cur[level]);
        const T4 *q2 = static_cast<const T4 *>(F.fq_prev[level]);
        const T *b2p = static_cast<const T *>(F.fb_prev[level]);
        const float2 *fsrc = F.flow[src];
        T *gh = static_cast<T *>(F.gh[level]);
        const size_t plane = (size_t)p * h;
        float ddx[kUpdRows], ddy[kUpdRows];
#pragma unroll
        for (int j = 0; j < kUpdRows; j++) {
            const int gy = y0 + j;
            ddx[j] = 0.f;
            ddy[j] = 0.f;
            if (gy >= h) continue;
            if (iter > 0) {
                const float2 v = fsrc[(size_t)gy * p + gx];
                ddx[j] = v.x;
                ddy[j] = v.y;
            } else if (!top) {
                const int wc = F.lw[level + 1], hc = F.lh[level + 1], pc = F.lp[level + 1];
                const int cx = gx >> 1, cy = gy >> 1;
                const int cx1 = min(cx + 1, wc - 1), cy1 = min(cy + 1, hc - 1);
                const float fx = (gx & 1) ? 0.5f : 0.f, fy = (gy & 1) ? 0.5f : 0.f;
                const float2 a = fsrc[(size_t)cy * pc + cx], b = fsrc[(size_t)cy * pc + cx1];
                const float2 c = fsrc[(size_t)cy1 * pc + cx], d = fsrc[(size_t)cy1 * pc + cx1];
                ddx[j] = 2.f * ((1.f - fy) * ((1.f - fx) * a.x + fx * b.x) + fy * ((1.f - fx) * c.x + fx * d.x));
                ddy[j] = 2.f * ((1.f - fy) * ((1.f - fx) * a.y + fx * b.y) + fy * ((1.f - fx) * c.y + fx * d.y));
            }
        }
#pragma unroll
        for (int j = 0; j < kUpdRows; j++) {
            const int gy = y0 + j;
            if (gy >= h) continue;
            const float dx = ddx[j], dy = ddy[j];
            // Position x + d~ as integer + fraction (full-precision
            // fraction), clamped to the image.
            const float flx = floorf(dx), fly = floorf(dy);
            int ix = gx + (int)flx, iy = gy + (int)fly;
            float fx = dx - flx, fy = dy - fly;
            if (ix < 0) { ix = 0; fx = 0.f; } else if (ix >= w - 1) { ix = w - 1; fx = 0.f; }
            if (iy < 0) { iy = 0; fy = 0.f; } else if (iy >= h - 1) { iy = h - 1; fy = 0.f; }
            const int ix1 = min(ix + 1, w - 1), iy1 = min(iy + 1, h - 1);
            const size_t r0 = (size_t)iy * p, r1 = (size_t)iy1 * p, o = (size_t)gy * p + gx;
            const float4 qa = ST::f4(ST::ld4(q2 + r0 + ix)), qb = ST::f4(ST::ld4(q2 + r0 + ix1));
            const float4 qc = ST::f4(ST::ld4(q2 + r1 + ix)), qd = ST::f4(ST::ld4(q2 + r1 + ix1));
            const float ba = ST::ld(b2p + r0 + ix), bb = ST::ld(b2p + r0 + ix1);
            const float bc = ST::ld(b2p + r1 + ix), bdd = ST::ld(b2p + r1 + ix1);
            const float4 qs = ST::f4(ST::ld4(q1 + o));
            const float b2a = ST::ld(b1p + o);
            const float gx0 = 1.f - fx, gy0 = 1.f - fy;
            const float A11b = gy0 * (gx0 * qa.x + fx * qb.x) + fy * (gx0 * qc.x + fx * qd.x);
            const float A12b = gy0 * (gx0 * qa.y + fx * qb.y) + fy * (gx0 * qc.y + fx * qd.y);
            const float A22b = gy0 * (gx0 * qa.z + fx * qb.z) + fy * (gx0 * qc.z + fx * qd.z);
            const float b1b = gy0 * (gx0 * qa.w + fx * qb.w) + fy * (gx0 * qc.w + fx * qd.w);
            const float b2b = gy0 * (gx0 * ba + fx * bb) + fy * (gx0 * bc + fx * bdd);
            const float a11 = 0.5f * (qs.x + A11b), a12 = 0.5f * (qs.y + A12b), a22 = 0.5f * (qs.z + A22b);
            const float db1 = -0.5f * (b1b - qs.w) + (a11 * dx + a12 * dy);
            const float db2 = -0.5f * (b2b - b2a) + (a12 * dx + a22 * dy);
            ST::st(gh + 0 * plane + o, a11 * a11 + a12 * a12);
            ST::st(gh + 1 * plane + o, a11 * a12 + a12 * a22);
            ST::st(gh + 2 * plane + o, a12 * a12 + a22 * a22);
            ST::st(gh + 3 * plane + o, a11 * db1 + a12 * db2);
            ST::st(gh + 4 * plane + o, a12 * db1 + a22 * db2);
        }
    }
}

// ---------------------------------------------------------------- window
// Box means of G and h over (2r+1)^2 (clipped to the image) and the 2x2
// solve.  One TMA copy brings the five planes of a kWinTW x kWinTH tile
// plus its r-pixel apron into shared memory (elements outside the image
// arrive as zeros, which is exactly the clipped sum).  Every column is then
// summed over 2r+1 rows, fields 0-2 in a first round of threads and fields
// 3-4 in a second; each round sums its columns in registers before any
// thread writes, so the sums can be packed in place (fp32) at a row stride
// SW with SW/4 odd.  Then each thread sums 8 adjacent outputs of a row over
// 2r+1 columns for all five fields, reading its row segment as 16-byte
// words: the 8 threads of a quarter-warp take 8 different rows, whose
// words fall in 8 different bank groups, so the reads are conflict-free.
template <typename T, int R>
struct WinGeom {
    static constexpr int EPC = 16 / sizeof(T);                         // elements per 16 bytes
    static constexpr int XO = (R + EPC - 1) / EPC * EPC;               // box starts XO left of the tile
    static constexpr int BW = (kWinTW + XO + R + EPC - 1) / EPC * EPC; // box width (elements)
    static constexpr int EH = kWinTH + 2 * R;
    static constexpr int EW = kWinTW + 2 * R;
    static constexpr int SEG = 8;                                      // outputs per thread in a row
    static constexpr int SV = (SEG + 2 * R + 3) / 4;                   // float4 words a thread reads per row
    static constexpr int SW0 = EW > kWinTW - SEG + 4 * SV ? (EW + 3) / 4 * 4 : kWinTW - SEG + 4 * SV;
    static constexpr int SW = (SW0 / 4) % 2 ? SW0 : SW0 + 4;           // sums row stride (floats)
    static constexpr size_t box_bytes = (size_t)5 * EH * BW * sizeof(T);
    // float sums buffer (half storage only; fp32 packs the sums in place)
    static constexpr size_t sum_bytes = sizeof(T) == 4 ? 0 : (size_t)5 * kWinTH * SW * sizeof(float);
    static constexpr size_t smem = 128 + box_bytes + sum_bytes;
    static_assert(sizeof(T) != 4 || kWinTH * SW <= EH * BW, "packed sums fit each field's box");
    static_assert(3 * EW <= 256, "a round of three fields' columns fits the block");
    static_assert(kWinTW % SEG == 0 && (kWinTW / SEG) * kWinTH == 256, "one row segment per thread");
};

template <typename T, int R>
__global__ void __launch_bounds__(256, 3) k_window(const BatchDesc *__restrict__ bd, MethodConsts mc, int level, int dst)
{
    using G = WinGeom<T, R>;
    constexpr int TW = kWinTW, TH = kWinTH, EW = G::EW, EH = G::EH, BW = G::BW, WN = 2 * R + 1;
    constexpr int SEG = G::SEG, SW = G::SW, SV = G::SV;
    constexpr bool kF32 = sizeof(T) == 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    T *box = reinterpret_cast<T *>(smem_raw + 128);  // [5][EH][BW]
    // field k's column sums: [TH][SW] at sums + k * SFS
    float *sums = kF32 ? reinterpret_cast<float *>(box) : reinterpret_cast<float *>(smem_raw + 128 + G::box_bytes);
    constexpr int SFS = kF32 ? EH * BW : TH * SW;

    // row-segment owner of this thread: quarter-warps span 8 rows
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int r = (wp & 3) * 8 + (lane & 7), sg = (wp >> 2) * 4 + (lane >> 3);

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const int nfr = bd->nframes;
    const int *off = bd->win_off[level];
    const int total = __ldg(off + nfr);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.lw[level], h = F.lh[level], p = F.lp[level];
        const int ntx = (w + TW - 1) / TW;
        const int lt = t - __ldg(off + fi);
        const int x0 = (lt % ntx) * TW, y0 = (lt / ntx) * TH;
        if (threadIdx.x == 0) {
            const CUtensorMap *map = &F.gh_map[level];
            tensormap_acquire(map);
            fence_proxy_async_smem();
            mbar_expect_tx(bar, (uint32_t)G::box_bytes);
            tma_load_3d(box, map, x0 - G::XO, y0 - R, 0, bar);
        }
        const bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {
            // Give up: flag the batch, give the copy one more bounded wait, leave.
            if (threadIdx.x == 0) atomicExch(bd->err, kErrTmaTimeout);
            mbar_wait(bar, phase);
            return;
        }
        phase ^= 1u;

        // vertical sums of every ext column, two rounds of fields
#pragma unroll
        for (int round = 0; round < 2; round++) {
            const int k0 = round ? 3 : 0, nk = round ? 2 : 3;
            const int k = k0 + (int)threadIdx.x / EW, ex = (int)threadIdx.x % EW;
            const bool mine = (int)threadIdx.x < nk * EW;
            float sm[TH];
            if (mine) {
                const T *col = box + k * EH * BW + ex + (G::XO - R);
                float v[EH];
#pragma unroll
                for (int j = 0; j < EH; j++) v[j] = (float)col[j * BW];
                box_sums<EH, WN>(v, sm);
            }
            if (kF32) __syncthreads();  // every column of the round is read before the packed sums overwrite it
            if (mine) {
                float *dcol = sums + k * SFS + ex;
#pragma unroll
                for (int j = 0; j < TH; j++) dcol[j * SW] = sm[j];
            }
        }
        __syncthreads();

        {
            const int gy = y0 + r, gxs = x0 + sg * SEG;
            if (gy < h && gxs < w) {
                float acc[5][SEG];
#pragma unroll
                for (int k = 0; k < 5; k++) {
                    const float4 *row = reinterpret_cast<const float4 *>(sums + k * SFS + r * SW + sg * SEG);
                    float v[4 * SV], sm[SEG];
#pragma unroll
                    for (int q = 0; q < SV; q++) {
                        const float4 u = row[q];
                        v[4 * q] = u.x;
                        v[4 * q + 1] = u.y;
                        v[4 * q + 2] = u.z;
                        v[4 * q + 3] = u.w;
                    }
                    const float(&vv)[SEG + 2 * R] = *reinterpret_cast<const float(*)[SEG + 2 * R]>(v);
                    box_sums<SEG + 2 * R, WN>(vv, sm);
#pragma unroll
                    for (int j = 0; j < SEG; j++) acc[k][j] = sm[j];
                }
                // With c = the window's in-image pixel count, G_ = S_G / c and
                // h_ = S_h / c, so adj(G_) h_ / (det G_ + lambda) =
                // adj(S_G) S_h / (det S_G + lambda c^2): one division.
                const int cy = min(gy + R, h - 1) - max(gy - R, 0) + 1;
                float2 *frow = F.flow[dst] + (size_t)gy * p + gxs;
                const bool whole = gxs + SEG <= w;
#pragma unroll
                for (int j = 0; j < SEG; j += 2) {
                    float d[4];
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int gx = gxs + j + e;
                        const int cx = min(gx + R, w - 1) - max(gx - R, 0) + 1;
                        const float c = (float)(cx * cy);
                        const float g11 = acc[0][j + e], g12 = acc[1][j + e], g22 = acc[2][j + e];
                        const float h1 = acc[3][j + e], h2 = acc[4][j + e];
                        const float idet = 1.f / (diff_of_products(g11, g22, g12, g12) + mc.lambda * c * c);
                        d[2 * e] = diff_of_products(g22, h1, g12, h2) * idet;
                        d[2 * e + 1] = diff_of_products(g11, h2, g12, h1) * idet;
                    }
                    if (whole) {
                        *reinterpret_cast<float4 *>(frow + j) = make_float4(d[0], d[1], d[2], d[3]);
                    } else {
                        if (gxs + j < w) frow[j] = make_float2(d[0], d[1]);
                        if (gxs + j + 1 < w) frow[j + 1] = make_float2(d[2], d[3]);
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int R>
static void launch_window_t(const BatchDesc *bd, const MethodConsts &mc, int level, int dst, int grid, cudaStream_t s)
{
    // The dynamic shared-memory limit was raised by occ_window_t at set-up.
    k_window<T, R><<<grid, 256, WinGeom<T, R>::smem, s>>>(bd, mc, level, dst);
}

template <typename T, int R>
static int occ_window_t()
{
    const size_t sm = WinGeom<T, R>::smem;
    cudaFuncSetAttribute(k_window<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_window<T, R>, 256, sm);
    return b;
}

#define FLOWROI_FLOW_RADII(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

void launch_update(const BatchDesc *bd, const MethodConsts &mc, int level, int iter, int src, bool half, int grid,
                   cudaStream_t s)
{
    if (half) k_update<__half><<<grid, 256, 0, s>>>(bd, mc, level, iter, src);
    else k_update<float><<<grid, 256, 0, s>>>(bd, mc, level, iter, src);
}

int window_box(bool half, int win_r, int *xo, int *bw, int *eh)
{
    switch (win_r) {
#define CASE(RR)                                                                                              \
    case RR:                                                                                                  \
        if (half) { *xo = WinGeom<__half, RR>::XO; *bw = WinGeom<__half, RR>::BW; *eh = WinGeom<__half, RR>::EH; } \
        else { *xo = WinGeom<float, RR>::XO; *bw = WinGeom<float, RR>::BW; *eh = WinGeom<float, RR>::EH; }       \
        return 0;
        FLOWROI_FLOW_RADII(CASE)
#undef CASE
    default: return -1;
    }
}

void launch_window(const BatchDesc *bd, const MethodConsts &mc, int level, int dst, bool half, int grid, cudaStream_t s)
{
    switch (mc.win_r) {
#define CASE(RR)                                                                 \
    case RR:                                                                     \
        if (half) launch_window_t<__half, RR>(bd, mc, level, dst, grid, s);      \
        else launch_window_t<float, RR>(bd, mc, level, dst, grid, s);            \
        break;
        FLOWROI_FLOW_RADII(CASE)
#undef CASE
    default: break;
    }
}

int occupancy_update(bool half)
{
    int b = 0;
    if (half) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update<__half>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update<float>, 256, 0);
    return b;
}

int occupancy_window(bool half, int win_r)
{
    switch (win_r) {
#define CASE(RR) \
    case RR: return half ? occ_window_t<__half, RR>() : occ_window_t<float, RR>();
        FLOWROI_FLOW_RADII(CASE)
#undef CASE
    default: return 0;
    }
}

bool flow_radius_supported(int r) { return r >= 2 && r <= 10; }

}  // namespace flowroi
