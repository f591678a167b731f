// Farneback displacement estimation: one iteration at one pyramid level,
// as two kernels (per-pixel update of G and h, then box window and 2x2
// solve).
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
// Per pixel G = A^T A and h = A^T db (5 values) into five planes.  A tile
// is 256 columns x (kUpdRows x GROUPS) rows; one thread owns a column of it
// and takes its rows kUpdRows at a time, so the loads of those pixels are
// in flight together; no shared memory, full occupancy hides the gather
// latency.  With GROUPS > 1 a block walks consecutive rows, whose bilinear
// reads of the predecessor's fields overlap (L1 hits instead of L2
// requests); the tile table chooses GROUPS per context.
template <typename T, int GROUPS>
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
        const int gx = (lt % ntx) * kUpdTW + threadIdx.x, ty0 = (lt / ntx) * kUpdRows * GROUPS;
        if (gx >= w) continue;
        const T4 *q1 = static_cast<const T4 *>(F.fq_cur[level]);
        const T *b1p = static_cast<const T *>(F.fb_cur[level]);
        const T4 *q2 = static_cast<const T4 *>(F.fq_prev[level]);
        const T *b2p = static_cast<const T *>(F.fb_prev[level]);
        const float2 *fsrc = F.flow[src];
        T *gh = static_cast<T *>(F.gh[level]);
        // registration: the predecessor translated by the drift s is read at x + d~ - s / 2^level
        float ox = 0.f, oy = 0.f;
        if (mc.reg_on) {
            const float sc = -ldexpf(1.f, -level);
            ox = __uint_as_float(__ldg(F.red + kRedRegDrift)) * sc;
            oy = __uint_as_float(__ldg(F.red + kRedRegDrift + 1)) * sc;
        }
        const size_t plane = (size_t)p * h;
#pragma unroll 1
        for (int grp = 0; grp < GROUPS; grp++) {
        const int y0 = ty0 + grp * kUpdRows;
        if (GROUPS > 1 && y0 >= h) break;
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
            // Position x + d~ (+ the registration offset) as integer +
            // fraction (full-precision fraction), clamped to the image.
            const float px = dx + ox, py = dy + oy;
            const float flx = floorf(px), fly = floorf(py);
            int ix = gx + (int)flx, iy = gy + (int)fly;
            float fx = px - flx, fy = py - fly;
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
}

// ---------------------------------------------------------------- window
// Box means of G and h over (2r+1)^2 (clipped to the image) and the 2x2
// solve, over kWinTW x kWinTH tiles.  Warp-specialised: a producer warp
// streams each tile's five G, h planes (each with the r-pixel apron, one
// TMA copy per plane) through a ring of NS >= 5 shared-memory slots
// guarded by full / empty mbarriers, so the next tile's planes are in
// flight while the current tile is summed.  Elements outside the image
// arrive as zeros, which is exactly the clipped sum.
//
// Per tile, each plane's 64 + 2r extended columns are cut into three
// warp-sized pieces (the last one partial), and the 15 pieces are dealt to
// the eight consumer warps, two rounds; each lane sums its whole column
// over 2r+1 rows in one pass (every slot value is read once).  A warp's
// piece lies in one plane, so its lanes take 32 different banks.  With fp32 planes the column sums overwrite the column
// they came from (each column has one owner, and it has read the column
// before it writes it), so the slot itself holds the plane's sums; with
// fp16 planes each slot has a separate fp32 sums area.  After one barrier
// every consumer thread sums 16 adjacent outputs of a row over 2r+1
// columns into registers, plane by plane, each warp releasing a plane's
// slot when its reads of it are done; then it solves.  Sums rows are an
// odd number of 16-byte words apart and the 8 threads of a quarter-warp
// take 8 different rows, so the float4 row reads are conflict-free.
// Square 64 x 64 tiles with 16 outputs a thread take about 0.83
// shared-memory wavefronts per pixel (column loads 0.29, in-place stores
// 0.23, row loads 0.31) against 1.2 for 64 x 32 tiles with 8; the ring of
// such tiles fills one block per SM.
//
// Ordering: a consumer waits for a slot's fill only for the tile that
// uses it, after the barrier of the previous tile, by which every earlier
// fill of every slot has completed; the producer refills a slot only after
// all eight warps released it.  So the parity waits cannot alias.  Every
// wait is bounded: a consumer whose wait runs out skips the work, the
// consumers agree at the barrier and leave with the batch error word set,
// and the producer waits (bounded) for the copies it issued before it
// leaves.
constexpr int kWinConsumers = 256;
constexpr int kWinThreads = kWinConsumers + 32;
constexpr size_t kWinSmem = 220 * 1024;  // one block per SM: a deep ring of large tiles
constexpr int kWinMaxSlots = 10;
constexpr int kWinHdrs = 4;                   // tile headers in flight

// A tile's geometry, written by the producer with the tile's first plane
// copy (published to the consumers by that copy's mbarrier and the
// consumers' barrier), so that consumer warps take no dependent global
// loads per tile.  Header j mod kWinHdrs is rewritten for tile j + 4 only
// after the slot of a plane of tile j + 2 was released, i.e. after every
// consumer has finished tile j.
struct WinTile {
    int x0, y0, w, h, p, pad;
    float2 *flow;
};
constexpr size_t kWinHdrOff = 2 * kWinMaxSlots * sizeof(uint64_t);
constexpr size_t kWinSlotsOff = (kWinHdrOff + kWinHdrs * sizeof(WinTile) + 127) / 128 * 128;

template <typename T, int R>
struct WinGeom {
    static constexpr bool inplace = sizeof(T) == 4;                    // sums overwrite the fp32 plane
    static constexpr int EPC = 16 / sizeof(T);                         // elements per 16 bytes
    static constexpr int XO = (R + EPC - 1) / EPC * EPC;               // box starts XO left of the tile
    static constexpr int EH = kWinTH + 2 * R;
    static constexpr int EW = kWinTW + 2 * R;
    static constexpr int SEG = 16;                                     // outputs per thread in a row
    static constexpr int SO = inplace ? XO - R : 0;                    // sums column of extended column 0
    static constexpr int SV = (SO + SEG + 2 * R + 3) / 4;              // float4 words a thread reads per row
    static constexpr int SNEED = kWinTW - SEG + 4 * SV;                // sums row span of the row reads
    // Box width: the tile and its apron in whole 16-byte words; in place it
    // also spans the row reads and is an odd number of 16-byte words.
    static constexpr int BW0 = (kWinTW + XO + R + EPC - 1) / EPC * EPC;
    static constexpr int BW1 = inplace && SNEED > BW0 ? SNEED : BW0;
    static constexpr int BW = inplace && (BW1 / 4) % 2 == 0 ? BW1 + 4 : BW1;
    static constexpr int SW0 = EW > SNEED ? (EW + 3) / 4 * 4 : SNEED;
    static constexpr int SW = inplace ? BW : ((SW0 / 4) % 2 ? SW0 : SW0 + 4);  // sums row stride (floats)
    static constexpr size_t plane_bytes = (size_t)EH * BW * sizeof(T); // one TMA copy
    static constexpr size_t data_bytes = (plane_bytes + 127) / 128 * 128;
    static constexpr size_t sums_bytes = inplace ? 0 : ((size_t)kWinTH * SW * sizeof(float) + 127) / 128 * 128;
    static constexpr size_t slot_stride = data_bytes + sums_bytes;
    static constexpr int NS0 = (int)((kWinSmem - kWinSlotsOff) / slot_stride);
    static constexpr int NS = NS0 > kWinMaxSlots ? kWinMaxSlots : NS0; // ring slots
    static constexpr size_t slots_off = kWinSlotsOff;
    static constexpr size_t smem = slots_off + NS * slot_stride;
    static_assert(NS >= 5, "a whole tile's planes in flight");
    static_assert(5 * ((EW + 31) / 32) <= 2 * (kWinConsumers / 32), "at most two column pieces per consumer warp");
    static_assert((kWinTW / SEG) * kWinTH == kWinConsumers, "one row segment per consumer thread");
    static_assert(kWinConsumers == 256, "row-segment thread map assumes 8 warps");
    static_assert(!inplace || (SO + EW <= BW && SNEED <= BW && EH >= kWinTH), "in-place sums fit the plane");
    static_assert(inplace || (EW <= SW && SNEED <= SW), "sums rows span the columns and the row reads");
};

template <typename T, int R>
__global__ void __launch_bounds__(kWinThreads, 1) k_window(const BatchDesc *__restrict__ bd, MethodConsts mc, int level,
                                                          int dst)
{
    using G = WinGeom<T, R>;
    constexpr int TW = kWinTW, TH = kWinTH, EW = G::EW, EH = G::EH, BW = G::BW, WN = 2 * R + 1;
    constexpr int SEG = G::SEG, SW = G::SW, SV = G::SV, SO = G::SO, NS = G::NS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + NS;
    WinTile *hdr = reinterpret_cast<WinTile *>(smem_raw + kWinHdrOff);
    unsigned char *slots = smem_raw + G::slots_off;
    auto sums_of = [&](int slot) {
        return reinterpret_cast<float *>(slots + slot * G::slot_stride + (G::inplace ? 0 : G::data_bytes));
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < NS; b++) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kWinConsumers / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int nfr = bd->nframes;
    const int *off = bd->win_off[level];
    const int total = __ldg(off + nfr);
    const int mine = total > (int)blockIdx.x ? (total - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

    if (threadIdx.x >= kWinConsumers) {
        // ---- producer: one lane issues the plane copies in order
        if (threadIdx.x == kWinConsumers) {
            int i = 0;
            bool ok = true;
            const uint32_t spin = bd->tma_spin;
            for (int j = 0; j < mine && ok; j++) {
                // test only (FLOWROI_TEST_EXPIRE_TMA): this tile's copies are
                // never issued, so the waits for them run out
                const bool skip = bd->test_skip_tile && level == 0 && blockIdx.x == 0 && j == 0;
                const int t = blockIdx.x + j * gridDim.x;
                const int fi = find_frame(off, nfr, t);
                const FrameDesc &F = bd->f[fi];
                const int w = F.lw[level];
                const int ntx = (w + TW - 1) / TW;
                const int lt = t - __ldg(off + fi);
                const int x0 = (lt % ntx) * TW, y0 = (lt / ntx) * TH;
                const CUtensorMap *map = &F.gh_map[level];
                tensormap_acquire(map);
                for (int k = 0; k < 5; k++, i++) {
                    const int slot = i % NS;
                    if (i >= NS && !mbar_wait(&empty[slot], (uint32_t)((i / NS - 1) & 1), spin)) {
                        atomicExch(bd->err, kErrTmaTimeout);
                        ok = false;
                        break;
                    }
                    if (k == 0) {
                        WinTile &ht = hdr[j % kWinHdrs];
                        ht.x0 = x0;
                        ht.y0 = y0;
                        ht.w = w;
                        ht.h = F.lh[level];
                        ht.p = F.lp[level];
                        ht.flow = F.flow[dst];
                    }
                    if (skip) continue;
                    fence_proxy_async_smem();
                    mbar_expect_tx(&full[slot], (uint32_t)G::plane_bytes);
                    tma_load_3d(slots + slot * G::slot_stride, map, x0 - G::XO, y0 - R, k, &full[slot]);
                }
            }
            // No copy may still be writing shared memory when the block leaves.
            for (int q = i - NS < 0 ? 0 : i - NS; q < i; q++) mbar_wait(&full[q % NS], (uint32_t)((q / NS) & 1), spin);
        }
        return;
    }

    // ---- consumers
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    // column pieces wp and wp + 8: plane ck[u], the lane's extended column cx[u]
    constexpr int PARTS = (EW + 31) / 32, PIECES = 5 * PARTS;
    int ck[2], cx[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int m = wp + u * (kWinConsumers / 32);
        ck[u] = m < PIECES ? m / PARTS : 5;
        cx[u] = (m - ck[u] * PARTS) * 32 + lane;
    }
    // row-segment owner: warp wp takes rows 8wp .. 8wp + 7, a quarter-warp one row each
    const int r = wp * 8 + (lane & 7), sg = lane >> 3;
    int i = 0;  // ring index of the tile's plane 0
    const uint32_t spin = bd->tma_spin;
    for (int j = 0; j < mine; j++, i += 5) {
        bool ok = true;
#pragma unroll
        for (int u = 0; u < 2; u++) {
            if (ck[u] >= 5) break;
            const int ii = i + ck[u];
            const int slot = ii % NS;
            ok = ok && mbar_wait(&full[slot], (uint32_t)((ii / NS) & 1), spin);
            if (!ok) break;
            if (cx[u] >= EW) continue;
            const T *col = reinterpret_cast<const T *>(slots + slot * G::slot_stride) + cx[u] + (G::XO - R);
            float v[EH], sm[TH];
#pragma unroll
            for (int q = 0; q < EH; q++) v[q] = (float)col[q * BW];
            box_sums<EH, WN>(v, sm);
            float *dcol = sums_of(slot) + cx[u] + SO;
#pragma unroll
            for (int q = 0; q < TH; q++) dcol[q * SW] = sm[q];
        }
        // Generic-proxy writes to a slot precede the TMA refill of it.
        if (G::inplace) fence_proxy_async_smem();
        if (named_sync_or(1, kWinConsumers, !ok)) {
            if (tid == 0) atomicExch(bd->err, kErrTmaTimeout);
            return;
        }

        // horizontal sums of each plane for the thread's SEG outputs
        float acc[5][SEG];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int slot = (i + k) % NS;
            const float4 *row = reinterpret_cast<const float4 *>(sums_of(slot) + r * SW + sg * SEG);
            float v[4 * SV], hs[SEG];
#pragma unroll
            for (int q = 0; q < SV; q++) {
                const float4 u4 = row[q];
                v[4 * q] = u4.x;
                v[4 * q + 1] = u4.y;
                v[4 * q + 2] = u4.z;
                v[4 * q + 3] = u4.w;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            const float(&vv)[SEG + 2 * R] = *reinterpret_cast<const float(*)[SEG + 2 * R]>(v + SO);
            box_sums<SEG + 2 * R, WN>(vv, hs);
#pragma unroll
            for (int q = 0; q < SEG; q++) acc[k][q] = hs[q];
        }

        const WinTile &ht = hdr[j % kWinHdrs];
        const int w = ht.w, h = ht.h;
        const int gy = ht.y0 + r, gxs = ht.x0 + sg * SEG;
        if (gy < h && gxs < w) {
            // With c = the window's in-image pixel count, G_ = S_G / c and
            // h_ = S_h / c, so adj(G_) h_ / (det G_ + lambda) =
            // adj(S_G) S_h / (det S_G + lambda c^2): one division.
            const int cy = min(gy + R, h - 1) - max(gy - R, 0) + 1;
            float2 *frow = ht.flow + (size_t)gy * ht.p + gxs;
            const bool whole = gxs + SEG <= w;
#pragma unroll
            for (int q = 0; q < SEG; q += 2) {
                float d[4];
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int gx = gxs + q + e;
                    const int cx = min(gx + R, w - 1) - max(gx - R, 0) + 1;
                    const float c = (float)(cx * cy);
                    const float g11 = acc[0][q + e], g12 = acc[1][q + e], g22 = acc[2][q + e];
                    const float h1 = acc[3][q + e], h2 = acc[4][q + e];
                    // det + lambda c^2 >= lambda > 0 (G_ is a sum of A^T A), far
                    // below the range where the fast reciprocal flushes
                    const float idet = __fdividef(1.f, diff_of_products(g11, g22, g12, g12) + mc.lambda * c * c);
                    d[2 * e] = fmaf(g22, h1, -g12 * h2) * idet;
                    d[2 * e + 1] = fmaf(g11, h2, -g12 * h1) * idet;
                }
                if (whole) {
                    *reinterpret_cast<float4 *>(frow + q) = make_float4(d[0], d[1], d[2], d[3]);
                } else {
                    if (gxs + q < w) frow[q] = make_float2(d[0], d[1]);
                    if (gxs + q + 1 < w) frow[q + 1] = make_float2(d[2], d[3]);
                }
            }
        }
    }
}

template <typename T, int R>
static void launch_window_t(const BatchDesc *bd, const MethodConsts &mc, int level, int dst, int grid, cudaStream_t s)
{
    // The dynamic shared-memory limit was raised by occ_window_t at set-up.
    k_window<T, R><<<grid, kWinThreads, WinGeom<T, R>::smem, s>>>(bd, mc, level, dst);
}

template <typename T, int R>
static int occ_window_t()
{
    const size_t sm = WinGeom<T, R>::smem;
    cudaFuncSetAttribute(k_window<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_window<T, R>, kWinThreads, sm);
    return b;
}

#define FLOWROI_FLOW_RADII(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

void launch_update(const BatchDesc *bd, const MethodConsts &mc, int level, int iter, int src, bool half, int rows,
                   int grid, cudaStream_t s)
{
    switch (rows) {
#define CASE(G)                                                                              \
    case kUpdRows * G:                                                                       \
        if (half) k_update<__half, G><<<grid, 256, 0, s>>>(bd, mc, level, iter, src);         \
        else k_update<float, G><<<grid, 256, 0, s>>>(bd, mc, level, iter, src);               \
        break;
        CASE(2)
        CASE(4)
        CASE(8)
#undef CASE
    default:
        if (half) k_update<__half, 1><<<grid, 256, 0, s>>>(bd, mc, level, iter, src);
        else k_update<float, 1><<<grid, 256, 0, s>>>(bd, mc, level, iter, src);
    }
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

int occupancy_update(bool half, int rows)
{
    int b = 0;
    switch (rows) {
#define CASE(G)                                                                                            \
    case kUpdRows * G:                                                                                     \
        if (half) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update<__half, G>, 256, 0);           \
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update<float, G>, 256, 0);                 \
        break;
        CASE(2)
        CASE(4)
        CASE(8)
#undef CASE
    default:
        if (half) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update<__half, 1>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update<float, 1>, 256, 0);
    }
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
