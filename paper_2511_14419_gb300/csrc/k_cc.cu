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

// Root of x, halving the path on the way (a non-root's parent may be
// replaced by any ancestor: roots are only ever linked, never unlinked).
__device__ __forceinline__ int find_s(int *P, int x, bool &bad, int lim)
{
    for (int k = 0; k < lim; k++) {
        const int p = P[x];
        if (p == x) return x;
        const int gp = P[p];
        if (gp != p) P[x] = gp;
        x = gp;
    }
    bad = true;
    return x;
}

__device__ __forceinline__ void union_s(int *P, int a, int b, bool &bad, int lim)
{
    for (int k = 0; k < lim; k++) {
        a = find_s(P, a, bad, lim);
        b = find_s(P, b, bad, lim);
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
__device__ __forceinline__ int find_g(int *L, int x, bool &bad, int lim)
{
    volatile int *V = L;
    for (int k = 0; k < lim; k++) {
        const int p = V[x];
        if (p == x) return x;
        const int gp = V[p];
        if (gp != p) V[x] = gp;
        x = gp;
    }
    bad = true;
    return x;
}

// Root of x once no union runs any more (read-only path).
__device__ __forceinline__ int find_ro(const int *L, int x, bool &bad, int lim)
{
    for (int k = 0; k < lim; k++) {
        const int p = __ldg(L + x);
        if (p == x) return x;
        x = p;
    }
    bad = true;
    return x;
}

__device__ __forceinline__ void union_g(int *L, int a, int b, bool &bad, int lim)
{
    for (int k = 0; k < lim; k++) {
        a = find_g(L, a, bad, lim);
        b = find_g(L, b, bad, lim);
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

// 1. tile-local labelling (shared memory: parents, then the counts)
__global__ void __launch_bounds__(256) k_cc_local(const BatchDesc *__restrict__ bd)
{
    const int lim = bd->loop_limit;
    __shared__ int P[kCcN];  // parent (local index), -1 = background; then the count of each local root
    const int total = __ldg(bd->sal_off + bd->nframes);
    const int c = threadIdx.x;
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        const uint8_t *mask = T.F->mask;
        const int gx = T.x0 + c;
#pragma unroll 8
        for (int r = 0; r < kCcTH; r++) {
            const int gy = T.y0 + r, i = r * kCcTW + c;
            const bool fg = gx < T.w && gy < T.h && mask[(size_t)gy * T.w + gx] != 0;
            P[i] = fg ? i : -1;
        }
        __syncthreads();
        // Raster-earlier neighbours, with the unions other pixels make
        // anyway left out: the north pixel, when set, is 8-adjacent to the
        // west and both diagonal ones (their own unions join them to it);
        // otherwise the west pixel, when set, covers the north-west one.
        for (int r = 0; r < kCcTH; r++) {
            const int i = r * kCcTW + c;
            if (P[i] < 0) continue;
            const int u = i - kCcTW;
            const bool n = r > 0 && P[u] >= 0;
            const bool wst = c > 0 && P[i - 1] >= 0;
            if (n) {
                union_s(P, i, u, bad, lim);
                continue;
            }
            if (wst) union_s(P, i, i - 1, bad, lim);
            else if (r > 0 && c > 0 && P[u - 1] >= 0) union_s(P, i, u - 1, bad, lim);
            if (r > 0 && c + 1 < kCcTW && P[u + 1] >= 0) union_s(P, i, u + 1, bad, lim);
        }
        __syncthreads();
        int root[kCcTH];
#pragma unroll
        for (int r = 0; r < kCcTH; r++) {
            const int i = r * kCcTW + c;
            root[r] = P[i] >= 0 ? find_s(P, i, bad, lim) : -1;
        }
        __syncthreads();  // every find is done: the parents are not needed any more
#pragma unroll
        for (int r = 0; r < kCcTH; r++) P[r * kCcTW + c] = 0;
        __syncthreads();
        // counts: one atomic per run of equal roots down the column
        {
            int cur = -1, run = 0;
#pragma unroll
            for (int r = 0; r < kCcTH; r++) {
                if (root[r] == cur) {
                    run++;
                } else {
                    if (cur >= 0) atomicAdd(&P[cur], run);
                    cur = root[r];
                    run = 1;
                }
            }
            if (cur >= 0) atomicAdd(&P[cur], run);
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
                C[g] = ro == i ? P[i] : 0;
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
    const int lim = bd->loop_limit;
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
                        if (L[q] >= 0) union_g(L, L[p], L[q], bad, lim);
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
                        if (L[q] >= 0) union_g(L, L[p], L[q], bad, lim);
                    }
            }
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

// 3. areas of the final components (each local root adds its count; the
// column's counts are all read before any root is looked up)
__global__ void __launch_bounds__(256) k_cc_count(const BatchDesc *__restrict__ bd)
{
    const int lim = bd->loop_limit;
    const int total = __ldg(bd->sal_off + bd->nframes);
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        int *L = T.F->cc_lab, *A = T.F->cc_area;
        const int *C = T.F->cc_cnt;
        const int gx = T.x0 + threadIdx.x;
        if (gx >= T.w) continue;
        const int nr = min(kCcTH, T.h - T.y0);
        static_assert(kCcTH <= 32, "rows of a column as bits");
        unsigned rows = 0u;  // rows holding a local root
#pragma unroll
        for (int r = 0; r < kCcTH; r++)
            if (r < nr && __ldg(C + (size_t)(T.y0 + r) * T.w + gx) != 0) rows |= 1u << r;
        while (rows) {
            const int r = __ffs(rows) - 1;
            rows &= rows - 1u;
            const int g = (T.y0 + r) * T.w + gx;
            const int root = find_g(L, g, bad, lim);
            L[g] = root;  // the filter reaches the root in one step (root <= g)
            atomicAdd(A + root, __ldg(C + g));
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

// 4. clear the pixels of components below min_area.  After step 3 a pixel's
// label is its local root, whose label is the final root: the column's
// labels, roots and areas are read in three batches.
__global__ void __launch_bounds__(256) k_cc_filter(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    const int lim = bd->loop_limit;
    const int total = __ldg(bd->sal_off + bd->nframes);
    bool bad = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const CcTile T = cc_tile(bd, t);
        const int *L = T.F->cc_lab, *A = T.F->cc_area;
        uint8_t *mask = T.F->mask;
        const int gx = T.x0 + threadIdx.x;
        if (gx >= T.w) continue;
        const int nr = min(kCcTH, T.h - T.y0);
        int rt[kCcTH];
#pragma unroll
        for (int r = 0; r < kCcTH; r++) rt[r] = r < nr ? __ldg(L + (size_t)(T.y0 + r) * T.w + gx) : -1;
#pragma unroll
        for (int r = 0; r < kCcTH; r++)
            if (rt[r] >= 0) rt[r] = __ldg(L + rt[r]);
#pragma unroll
        for (int r = 0; r < kCcTH; r++)
            if (rt[r] >= 0 && __ldg(L + rt[r]) != rt[r]) rt[r] = find_ro(L, rt[r], bad, lim);  // not expected
#pragma unroll
        for (int r = 0; r < kCcTH; r++)
            if (rt[r] >= 0 && __ldg(A + rt[r]) < mc.min_area) mask[(size_t)(T.y0 + r) * T.w + gx] = 0;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(bd->err, kErrCcLoop);
}

// Adjacent-factor merge (paper: §Region of Interest extraction, masks of
// neighbouring frames incorporated; Table 1 "Adjacent factor").  Reading:
// the RoI mask of frame j is the union (OR) of the per-frame masks of
// frames j-k .. j+k that exist.  16 bytes per thread, 4096-byte units.
__global__ void __launch_bounds__(256) k_merge(const BatchDesc *__restrict__ bd)
{
    const int nfr = bd->nframes;
    const int *off = bd->mrg_off;
    const int total = __ldg(off + nfr);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const size_t npx = (size_t)F.W * F.H;
        const size_t o = (size_t)(t - __ldg(off + fi)) * 4096 + threadIdx.x * 16;
        if (o >= npx) continue;
        const int n = F.n_adj;
        if (o + 16 <= npx) {
            uint4 acc = make_uint4(0u, 0u, 0u, 0u);
            for (int j = 0; j < n; j++) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(F.adj[j] + o));
                acc.x |= v.x;
                acc.y |= v.y;
                acc.z |= v.z;
                acc.w |= v.w;
            }
            *reinterpret_cast<uint4 *>(F.dwt_mask + o) = acc;
        } else {
            for (size_t q = o; q < npx; q++) {
                uint8_t a = 0;
                for (int j = 0; j < n; j++) a |= F.adj[j][q];
                F.dwt_mask[q] = a;
            }
        }
    }
}

void launch_merge(const BatchDesc *bd, int grid, cudaStream_t s) { k_merge<<<grid, 256, 0, s>>>(bd); }

void launch_cc(const BatchDesc *bd, const MethodConsts &mc, int step, int grid, cudaStream_t s)
{
    switch (step) {
    case 0: k_cc_local<<<grid, 256, 0, s>>>(bd); break;
    case 1: k_cc_merge<<<grid, 256, 0, s>>>(bd); break;
    case 2: k_cc_count<<<grid, 256, 0, s>>>(bd); break;
    default: k_cc_filter<<<grid, 256, 0, s>>>(bd, mc); break;
    }
}

int occupancy_cc()
{
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cc_local, 256, 0);
    return a;
}

}  // namespace flowroi
