// Registration of each frame to its predecessor (paper: §Optical flow
// extraction -- global translational drift corrected by phase-correlation
// alignment to the predecessor).  Readings (also the oracle's):
//   - phase correlation of the pyramid images of level l = reg_level of the
//     two flow inputs, each made mean-free and multiplied by a symmetric
//     Hann window over the image size, zero-padded to powers of two;
//   - X = F_cur conj(F_prev), R = X / (|X| + 0.01 max|X|), r = Re IFFT(R);
//   - the first maximum of r (row-major), wrapped to (-N/2, N/2], refined
//     per axis by the vertex of the parabola through r at the peak and its
//     two circular neighbours (when it opens downwards; clamped to +-0.5);
//   - the drift s = shift * 2^l (cur(x) ~ prev(x - s)); the flow is that of
//     the registered pair: the predecessor's expansion is read at
//     x + d~ - s / 2^l (k_update).
// The current frame's spectrum is kept for the next frame.
//
// Launches, all over the batch's registered frames: the level image's sum;
// forward FFT of rows, then of columns (the spectrum); for frames with a
// predecessor the cross-power spectrum (and its largest magnitude), the
// inverse FFT of rows (normalising on load) and of columns, the peak, and
// the drift.  FFTs are radix-2 in shared memory: a row per block, or eight
// columns per block, with the data loaded in bit-reversed order.
#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr int kRegCols = 8;      // columns per block of the column FFTs
constexpr int kRegMaxLog = 10;   // padded sizes up to 1024
constexpr int kRegUnit = 4096;   // elements per block-unit of the element-wise launches

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__device__ __forceinline__ int brev(int i, int ln) { return ln ? (int)(__brev((unsigned)i) >> (32 - ln)) : 0; }

// tw[k] = exp(-2 pi i k / n), k < n/2
__device__ __forceinline__ void twiddles(float2 *tw, int ln)
{
    const int n = 1 << ln;
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.f * (float)k / (float)n, &sn, &cs);
        tw[k] = make_float2(cs, sn);
    }
}

// In-place radix-2 FFTs of `m` sequences of n = 2^ln values each (sequence
// q at x + q * n), entered in bit-reversed order.  All threads of the block
// take part; the block is synchronised after every stage.
template <bool INV>
__device__ __forceinline__ void fft_smem(float2 *x, const float2 *tw, int ln, int m)
{
    const int n = 1 << ln, nb = m * (n / 2);
    for (int st = 1; st <= ln; st++) {
        const int half = 1 << (st - 1), tstride = n >> st;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int q = b / (n / 2), bb = b - q * (n / 2);
            const int j = bb & (half - 1);
            const int i0 = q * n + ((bb >> (st - 1)) << st) + j, i1 = i0 + half;
            float2 w = tw[j * tstride];
            if (INV) w.y = -w.y;
            const float2 t = cmul(w, x[i1]), u = x[i0];
            x[i0] = make_float2(u.x + t.x, u.y + t.y);
            x[i1] = make_float2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float hann(int i, int m)
{
    return m > 1 ? 0.5f - 0.5f * cospif(2.f * (float)i / (float)(m - 1)) : 1.f;
}

template <typename T>
__device__ __forceinline__ float level_px(const FrameDesc &F, int level, int x, int y)
{
    return Store<T>::ld(static_cast<const T *>(F.pyr[level]) + (size_t)y * F.lp[level] + x);
}

// orderable key of a float (larger float -> larger unsigned)
__device__ __forceinline__ unsigned fkey(float v)
{
    const unsigned u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace

// sum of the level image (double atomics), per frame
template <typename T>
__global__ void __launch_bounds__(256) k_reg_sum(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    const int nfr = bd->nframes;
    const int *off = bd->reg_el_off;
    const int total = __ldg(off + nfr);
    const int l = mc.reg_level;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int w = F.lw[l], h = F.lh[l];
        const int u = t - __ldg(off + fi);
        double acc = 0.0;
        for (int e = u * kRegUnit + threadIdx.x; e < min((u + 1) * kRegUnit, w * h); e += blockDim.x)
            acc += (double)level_px<T>(F, l, e % w, e / w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(reinterpret_cast<double *>(F.red + kRedRegSum), acc);
    }
}

// forward FFT of the rows of the windowed, mean-free level image
template <typename T>
__global__ void __launch_bounds__(256) k_reg_rows_fwd(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    __shared__ float2 buf[1 << kRegMaxLog];
    __shared__ float2 tw[1 << (kRegMaxLog - 1)];
    const int nfr = bd->nframes;
    const int *off = bd->reg_row_off;
    const int total = __ldg(off + nfr);
    const int l = mc.reg_level;
    int cur_ln = -1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        const int ln = F.reg_lnx, nx = 1 << ln;
        const int y = t - __ldg(off + fi);
        const int w = F.lw[l], h = F.lh[l];
        if (ln != cur_ln) {
            twiddles(tw, ln);
            cur_ln = ln;
        }
        const float mean = (float)(*reinterpret_cast<const double *>(F.red + kRedRegSum) / ((double)w * h));
        const float wy = y < h ? hann(y, h) : 0.f;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const float v = (y < h && x < w) ? (level_px<T>(F, l, x, y) - mean) * hann(x, w) * wy : 0.f;
            buf[brev(x, ln)] = make_float2(v, 0.f);
        }
        __syncthreads();
        fft_smem<false>(buf, tw, ln, 1);
        float2 *row = F.reg_cur + (size_t)y * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) row[x] = buf[x];
        __syncthreads();
    }
}

// FFT of columns, eight per block, in place (plane `which`: 0 = the frame's
// spectrum, 1 = the correlation work plane)
template <bool INV>
__global__ void __launch_bounds__(256) k_reg_cols(const BatchDesc *__restrict__ bd, int which)
{
    extern __shared__ float2 cbuf[];  // [kRegCols][ny] then the twiddles
    const int nfr = bd->nframes;
    const int *off = bd->reg_col_off;
    const int total = __ldg(off + nfr);
    int cur_ln = -1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        if (which == 1 && !F.has_prev) continue;  // block-uniform
        const int lnx = F.reg_lnx, lny = F.reg_lny, nx = 1 << lnx, ny = 1 << lny;
        float2 *tw = cbuf + kRegCols * (1 << kRegMaxLog);
        if (lny != cur_ln) {
            twiddles(tw, lny);
            cur_ln = lny;
        }
        const int c0 = (t - __ldg(off + fi)) * kRegCols;
        float2 *plane = which ? F.reg_work : F.reg_cur;
        for (int i = threadIdx.x; i < kRegCols * ny; i += blockDim.x) {
            const int y = i / kRegCols, k = i - y * kRegCols;
            cbuf[k * ny + brev(y, lny)] = c0 + k < nx ? plane[(size_t)y * nx + c0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        fft_smem<INV>(cbuf, tw, lny, kRegCols);
        for (int i = threadIdx.x; i < kRegCols * ny; i += blockDim.x) {
            const int y = i / kRegCols, k = i - y * kRegCols;
            if (c0 + k < nx) plane[(size_t)y * nx + c0 + k] = cbuf[k * ny + y];
        }
        __syncthreads();
    }
}

// cross-power spectrum X = F_cur conj(F_prev) and its largest magnitude
__global__ void __launch_bounds__(256) k_reg_cross(const BatchDesc *__restrict__ bd)
{
    const int nfr = bd->nframes;
    const int *off = bd->reg_el_off;
    const int total = __ldg(off + nfr);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        if (!F.has_prev) continue;
        const int n = 1 << (F.reg_lnx + F.reg_lny);
        const int u = t - __ldg(off + fi);
        float mx = 0.f;
        for (int e = u * kRegUnit + threadIdx.x; e < min((u + 1) * kRegUnit, n); e += blockDim.x) {
            const float2 a = F.reg_cur[e], b = F.reg_prev[e];
            const float2 x = make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
            F.reg_work[e] = x;
            mx = fmaxf(mx, sqrtf(x.x * x.x + x.y * x.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(F.red + kRedRegXMax, __float_as_uint(mx));
    }
}

// inverse FFT of the rows of R = X / (|X| + 0.01 max|X|), in place
__global__ void __launch_bounds__(256) k_reg_rows_inv(const BatchDesc *__restrict__ bd)
{
    __shared__ float2 buf[1 << kRegMaxLog];
    __shared__ float2 tw[1 << (kRegMaxLog - 1)];
    const int nfr = bd->nframes;
    const int *off = bd->reg_row_off;
    const int total = __ldg(off + nfr);
    int cur_ln = -1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        if (!F.has_prev) continue;
        const int ln = F.reg_lnx, nx = 1 << ln;
        const int y = t - __ldg(off + fi);
        if (ln != cur_ln) {
            twiddles(tw, ln);
            cur_ln = ln;
        }
        const float reg = 0.01f * __uint_as_float(F.red[kRedRegXMax]);
        float2 *row = F.reg_work + (size_t)y * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const float2 v = row[x];
            const float m = sqrtf(v.x * v.x + v.y * v.y) + reg;
            buf[brev(x, ln)] = m > 0.f ? make_float2(v.x / m, v.y / m) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        fft_smem<true>(buf, tw, ln, 1);
        for (int x = threadIdx.x; x < nx; x += blockDim.x) row[x] = buf[x];
        __syncthreads();
    }
}

// first maximum of the real part of the correlation (key: value, then the
// smaller index)
__global__ void __launch_bounds__(256) k_reg_peak(const BatchDesc *__restrict__ bd)
{
    const int nfr = bd->nframes;
    const int *off = bd->reg_el_off;
    const int total = __ldg(off + nfr);
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int fi = find_frame(off, nfr, t);
        const FrameDesc &F = bd->f[fi];
        if (!F.has_prev) continue;
        const int n = 1 << (F.reg_lnx + F.reg_lny);
        const int u = t - __ldg(off + fi);
        unsigned long long best = 0ull;
        for (int e = u * kRegUnit + threadIdx.x; e < min((u + 1) * kRegUnit, n); e += blockDim.x) {
            const unsigned long long k = ((unsigned long long)fkey(F.reg_work[e].x) << 32) | (0xffffffffu - (unsigned)e);
            best = k > best ? k : best;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v > best ? v : best;
        }
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long *>(F.red + kRedRegPeak), best);
    }
}

// integer peak, wrap, parabolic refinement, drift in level-0 pixels
__global__ void k_reg_drift(const BatchDesc *__restrict__ bd, MethodConsts mc)
{
    for (int fi = blockIdx.x * blockDim.x + threadIdx.x; fi < bd->nframes; fi += gridDim.x * blockDim.x) {
        const FrameDesc &F = bd->f[fi];
        if (!F.do_reg || !F.has_prev) continue;
        const int nx = 1 << F.reg_lnx, ny = 1 << F.reg_lny;
        const unsigned long long key = *reinterpret_cast<const unsigned long long *>(F.red + kRedRegPeak);
        const int e = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
        const int ky = e / nx, kx = e - ky * nx;
        auto r = [&](int y, int x) { return F.reg_work[(size_t)((y + ny) % ny) * nx + (x + nx) % nx].x; };
        auto sub = [](float c0, float cm, float cp) {
            const float den = cm - 2.f * c0 + cp;
            if (!(den < 0.f)) return 0.f;
            return fminf(0.5f, fmaxf(-0.5f, (cm - cp) / (2.f * den)));
        };
        const float c0 = r(ky, kx);
        const float dx = sub(c0, r(ky, kx - 1), r(ky, kx + 1));
        const float dy = sub(c0, r(ky - 1, kx), r(ky + 1, kx));
        const float sc = (float)(1 << mc.reg_level);
        const float sx = ((float)(kx > nx / 2 ? kx - nx : kx) + dx) * sc;
        const float sy = ((float)(ky > ny / 2 ? ky - ny : ky) + dy) * sc;
        F.red[kRedRegDrift] = __float_as_uint(sx);
        F.red[kRedRegDrift + 1] = __float_as_uint(sy);
        if (F.dbg_drift) {
            F.dbg_drift[0] = sx;
            F.dbg_drift[1] = sy;
        }
    }
}

void launch_register(const BatchDesc *bd, const MethodConsts &mc, bool half, int step, int grid, cudaStream_t s)
{
    const int max_ny = 1 << kRegMaxLog;
    const size_t col_smem = (size_t)(kRegCols * max_ny + max_ny / 2) * sizeof(float2);
    switch (step) {
    case 0:
        if (half) k_reg_sum<__half><<<grid, 256, 0, s>>>(bd, mc);
        else k_reg_sum<float><<<grid, 256, 0, s>>>(bd, mc);
        break;
    case 1:
        if (half) k_reg_rows_fwd<__half><<<grid, 256, 0, s>>>(bd, mc);
        else k_reg_rows_fwd<float><<<grid, 256, 0, s>>>(bd, mc);
        break;
    case 2: k_reg_cols<false><<<grid, 256, col_smem, s>>>(bd, 0); break;
    case 3: k_reg_cross<<<grid, 256, 0, s>>>(bd); break;
    case 4: k_reg_rows_inv<<<grid, 256, 0, s>>>(bd); break;
    case 5: k_reg_cols<true><<<grid, 256, col_smem, s>>>(bd, 1); break;
    case 6: k_reg_peak<<<grid, 256, 0, s>>>(bd); break;
    default: k_reg_drift<<<1, 64, 0, s>>>(bd, mc); break;
    }
}

int occupancy_register()
{
    const int max_ny = 1 << kRegMaxLog;
    const size_t col_smem = (size_t)(kRegCols * max_ny + max_ny / 2) * sizeof(float2);
    cudaFuncSetAttribute(k_reg_cols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem);
    cudaFuncSetAttribute(k_reg_cols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem);
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_reg_cols<false>, 256, col_smem);
    return a;
}

int register_max_log() { return kRegMaxLog; }
int register_cols() { return kRegCols; }
int register_unit() { return kRegUnit; }

}  // namespace flowroi
