// Removal of small connected components of the RoI mask (paper: §Region of
// Interest extraction -- after opening and closing, residual small
// connected components are removed by an area criterion).  Readings (also
// the oracle's): 8-connectivity; components with fewer than min_area pixels
// are cleared; off when min_area <= 1.
//
// Union-find over pixel indices, in four launches over the 256x32 tiles of
// the mask stage (frames with a predecessor only):
//   1. k_cc_local: per tile, in shared memory, every foreground pixel is
//      united with its raster-earlier 8-neighbours of the tile (lock-free
//      union by atomicMin: a root is linked under the smaller root, so a
//      parent index never exceeds its child's); each pixel's label L is the
//      frame index of its tile-local root (the smallest index of its local
//      component), C holds each local root's pixel count, A is cleared at
//      local roots;
//   2. k_cc_merge: tile-border pixels are united with their neighbours in
//      the tiles above and to the left, on L in global memory (same union);
//   3. k_cc_count: each local root finds its final root (path written back)
//      and adds its count to A[root];
//   4. k_cc_filter: pixels whose final root's area is below min_area are
//      cleared from the mask.
// Every find / union loop is bounded; one that runs out sets the batch's
// error word (the labels only ever point to smaller indices, so it cannot
// run out unless memory is corrupt).
#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr int kCcTW = kSalTW, kCcTH = kSalTH;
constexpr int kCcN = kCcTW * kCcTH;
constexpr unsigned kErrCcLoop = 2u;  // error word: a union-find loop ran out
constexpr int kCcLimit = 1 << 24;

__device__ __forceinline__ int find_s(const int *P, int x, bool &bad)
{
    for (int k = 0; k < kCcLimit; k++) {
        const int p = P[x];
        if (p == x) return x;
        x = p;
    }
    bad = true;
    return x;
}

__device__ __forceinline__ void union_s(int *P, int a, int b, bool &bad)
{
    for (int k = 0; k < kCcLimit; k++) {
        a = find_s(P, a, bad);
        b = find_s(P, b, bad);
        if (a == b || bad) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&P[a], b);
        if (old == a) return;  // a was a root and is now under b
        a = old;               // a was re-linked meanwhile: continue from its new parent
    }
    bad = true;
}

// The same on the frame's label array in global memory (volatile reads:
// other blocks link roots concurrently).
__device__ __forceinline__ int find_g(int *L, int x, bool &bad)
{
    for (int k = 0; k < kCcLimit; k++) {
        const int p = *reinterpret_cast<volatile int *>(L + x);
        if (p == x) return x;
        x = p;
    }
    bad = true;
    return x;
}

__device__ __forceinline__ void union_g(int *L, int a, int b, bool &bad)
{
    for (int k = 0; k < kCcLimit; k++) {
        a = find_g(L, a, bad);
        b = find_g(L, b, bad);
        if (a == b || bad) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(L + a, b);
        if (old == a) return;
        a = old;
    }
    bad = true;
}

struct CcTile {
    const FrameDesc *F;
    int w, h, x0, y0;
};

__device__ __forceinline__ CcTile cc_tile(const BatchDesc *bd, int t)
{
    const int nfr = bd->nframes;
    const int *off = bd->sal_off;
    const int fi = find_frame(off, nfr, t);
    CcTile c;
    c.F = &bd->f[fi];
    c.w = c.F->W;
    c.h = c.F->H;
    const int ntx = (c.w + kCcTW - 1) / kCcTW;
    const int lt = t - __ldg(off + fi);
    c.x0 = (lt % ntx) * kCcTW;
    c.y0 = (lt / ntx) * kCcTH;
    return c;
}

}  // namespace

// 1. tile-local labelling (dynamic shared memory: parents and counts)
__global__ void __launch_bounds__(256) k_cc_local(const BatchDesc *__restrict__ bd)
{
    extern __shared__ int sm_cc[];
    int *P = sm_cc;          // [kCcN] parent (local index), -1 = background
    int *cnt = sm_cc + kCcN; // [kCcN] pixel count of each local root
    const int total = __ldg(bd->sal_off + bd->nframes);
    const int c = threadIdx.x;
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        const uint8_t *mask = T.F->mask;
        const int gx = T.x0 + c;
#pragma unroll 4
        for (int r = 0; r < kCcTH; r++) {
            const int gy = T.y0 + r, i = r * kCcTW + c;
            const bool fg = gx < T.w && gy < T.h && mask[(size_t)gy * T.w + gx] != 0;
            P[i] = fg ? i : -1;
            cnt[i] = 0;
        }
        __syncthreads();
        for (int r = 0; r < kCcTH; r++) {
            const int i = r * kCcTW + c;
            if (P[i] < 0) continue;
            if (c > 0 && P[i - 1] >= 0) union_s(P, i, i - 1, bad);
            if (r > 0) {
                const int u = i - kCcTW;
                if (c > 0 && P[u - 1] >= 0) union_s(P, i, u - 1, bad);
                if (P[u] >= 0) union_s(P, i, u, bad);
                if (c + 1 < kCcTW && P[u + 1] >= 0) union_s(P, i, u + 1, bad);
            }
        }
        __syncthreads();
        int root[kCcTH];
#pragma unroll
        for (int r = 0; r < kCcTH; r++) {
            const int i = r * kCcTW + c;
            root[r] = P[i] >= 0 ? find_s(P, i, bad) : -1;
        }
        __syncthreads();  // every find is done before counts and compression
#pragma unroll
        for (int r = 0; r < kCcTH; r++)
            if (root[r] >= 0) {
                // one atomic per distinct root in the warp
                const unsigned grp = __match_any_sync(__activemask(), root[r]);
                if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&cnt[root[r]], __popc(grp));
            }
        __syncthreads();
        int *L = T.F->cc_lab, *C = T.F->cc_cnt, *A = T.F->cc_area;
        if (gx < T.w) {
            for (int r = 0; r < kCcTH; r++) {
                const int gy = T.y0 + r;
                if (gy >= T.h) break;
                const int i = r * kCcTW + c;
                const size_t g = (size_t)gy * T.w + gx;
                const int ro = root[r];
                // frame index of the local root (same raster order as the local index)
                const int lab = ro < 0 ? -1 : (T.y0 + ro / kCcTW) * T.w + T.x0 + ro % kCcTW;
                L[g] = lab;
                C[g] = ro == i ? cnt[i] : 0;
                if (ro == i) A[g] = 0;
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

// 2. unions across the top and left tile borders
__global__ void __launch_bounds__(256) k_cc_merge(const BatchDesc *__restrict__ bd)
{
    const int total = __ldg(bd->sal_off + bd->nframes);
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        int *L = T.F->cc_lab;
        const int w = T.w, h = T.h;
        // top row against the row above (three neighbours each)
        if (T.y0 > 0) {
            const int gx = T.x0 + threadIdx.x, gy = T.y0;
            if (gx < w && gy < h) {
                const int p = gy * w + gx;
                if (L[p] >= 0)
                    for (int dx = -1; dx <= 1; dx++) {
                        const int qx = gx + dx;
                        if (qx < 0 || qx >= w) continue;
                        const int q = (gy - 1) * w + qx;
                        if (L[q] >= 0) union_g(L, L[p], L[q], bad);
                    }
            }
        }
        // left column against the column to the left
        if (T.x0 > 0 && threadIdx.x < kCcTH) {
            const int gx = T.x0, gy = T.y0 + threadIdx.x;
            if (gx < w && gy < h) {
                const int p = gy * w + gx;
                if (L[p] >= 0)
                    for (int dy = -1; dy <= 1; dy++) {
                        const int qy = gy + dy;
                        if (qy < 0 || qy >= h) continue;
                        const int q = qy * w + gx - 1;
                        if (L[q] >= 0) union_g(L, L[p], L[q], bad);
                    }
            }
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

// 3. areas of the final components
__global__ void __launch_bounds__(256) k_cc_count(const BatchDesc *__restrict__ bd)
{
    const int total = __ldg(bd->sal_off + bd->nframes);
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        int *L = T.F->cc_lab, *C = T.F->cc_cnt, *A = T.F->cc_area;
        const int gx = T.x0 + threadIdx.x;
        if (gx >= T.w) continue;
        for (int r = 0; r < kCcTH; r++) {
            const int gy = T.y0 + r;
            if (gy >= T.h) break;
            const int g = gy * T.w + gx;
            const int n = C[g];
            if (n == 0) continue;
            const int root = find_g(L, g, bad);
            L[g] = root;  // shortcut for the filter (root <= g)
            atomicAdd(A + root, n);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

// 4. clear the pixels of components below min_area
__global__ void __launch_bounds__(256) k_cc_filter(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    const int total = __ldg(bd->sal_off + bd->nframes);
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        int *L = T.F->cc_lab, *A = T.F->cc_area;
        uint8_t *mask = T.F->mask;
        const int gx = T.x0 + threadIdx.x;
        if (gx >= T.w) continue;
        for (int r = 0; r < kCcTH; r++) {
            const int gy = T.y0 + r;
            if (gy >= T.h) break;
            const int g = gy * T.w + gx;
            const int lab = L[g];
            if (lab < 0) continue;
            const int root = find_g(L, lab, bad);
            if (__ldg(A + root) < mc.min_area) mask[g] = 0;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

void launch_cc(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s)
{
    static const size_t smem = 2 * kCcN * sizeof(int);
    k_cc_local<<<grid, 256, smem, s>>>(bd);
    k_cc_merge<<<grid, 256, 0, s>>>(bd);
    k_cc_count<<<grid, 256, 0, s>>>(bd);
    k_cc_filter<<<grid, 256, 0, s>>>(bd, mc);
}

int occupancy_cc()
{
    const size_t smem = 2 * kCcN * sizeof(int);
    cudaFuncSetAttribute(k_cc_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cc_local, 256, smem);
    return a;
}

}  // namespace flowroi
