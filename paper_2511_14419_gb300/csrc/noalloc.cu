// JPEG2000 front end for one frame without any allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// pre-reserved memory budget, plug-ins whose host owns the device heap, or
// real-time loops that must not call cudaMalloc (it can synchronise the
// device and its latency is unbounded).  flowroi_dwt_roi_noalloc serves
// them: it runs the library's DWT kernel (DC shift, lifting DWT,
// quantisation, wavelet-domain RoI mask, RoI up-shift) on caller-owned
// device buffers, and keeps the only memory it needs besides those - a
// one-frame batch descriptor and the two low-low planes (and their masks)
// passed between DWT levels - in the fixed array below, which every GPU
// that loads the library holds until the process exits.
//
// The array is shared by every call: calls whose work overlaps on the GPU
// (different streams, or different host threads on different streams)
// race on it.  Nothing in it has to start at zero: each call writes the
// descriptor and every low-low element before it reads them.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/flowroi.h"
#include "common.cuh"
#include "kernels.h"

namespace flowroi {
namespace {

// Largest frame (pixels) whose low-low planes fit the array.
constexpr size_t kNaMaxPixels = size_t(1) << 20;
constexpr size_t kNaDescBytes = (offsetof(BatchDesc, f) + sizeof(FrameDesc) + 255) / 256 * 256;
constexpr size_t kNaLLBytes = (kNaMaxPixels / 4) * sizeof(float);  // one low-low plane (float or int32)
constexpr size_t kNaLLMBytes = kNaMaxPixels / 4;                   // its mask
constexpr size_t kNaBytes = kNaDescBytes + 2 * kNaLLBytes + 2 * kNaLLMBytes;

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;                                 // guards the table below
unsigned char *g_na_dev_ptr[kNaMaxDevices] = {};    // device address of the array, per device

// What the DWT kernel reads of a batch descriptor, passed by value.
struct NaDesc {
    int tiles[kMaxLevels];
    FrameDesc f;
};
static_assert(sizeof(FrameDesc) % 4 == 0, "descriptor copied in 32-bit words");
static_assert(sizeof(NaDesc) <= 4000, "kernel parameter size");

// Writes the one-frame batch descriptor into the array (queued on the
// caller's stream ahead of the DWT launches, so no host staging is needed).
__global__ void k_na_desc(NaDesc d, BatchDesc *bd)
{
    if (threadIdx.x == 0) {
        bd->nframes = 1;
        for (int l = 0; l < kMaxLevels; l++) {
            bd->dwt_off[l][0] = 0;
            bd->dwt_off[l][1] = d.tiles[l];
        }
    }
    const unsigned *src = reinterpret_cast<const unsigned *>(&d.f);
    unsigned *dst = reinterpret_cast<unsigned *>(&bd->f[0]);
    for (int i = threadIdx.x; i < (int)(sizeof(FrameDesc) / 4); i += blockDim.x) dst[i] = src[i];
}

}  // namespace
}  // namespace flowroi

using namespace flowroi;

extern "C" int flowroi_dwt_roi_noalloc(const void *raw, int width, int height, int pitch_bytes, int dtype, int bit_depth,
                                       const uint8_t *mask, int wavelet, int levels, int scale_shift, const float *delta,
                                       int32_t *coeffs, void *cuda_stream)
{
    if (!raw || !mask || !coeffs) return FLOWROI_EINVAL;
    if (dtype != FLOWROI_U8 && dtype != FLOWROI_U16) return FLOWROI_EINVAL;
    const int bpp = dtype == FLOWROI_U8 ? 1 : 2;
    if (bit_depth < 1 || bit_depth > 8 * bpp) return FLOWROI_EINVAL;
    if (wavelet != FLOWROI_W53 && wavelet != FLOWROI_W97) return FLOWROI_EINVAL;
    if (levels < 1 || levels > kMaxLevels || scale_shift < 0 || scale_shift > 15) return FLOWROI_EINVAL;
    if (wavelet == FLOWROI_W97 && !delta) return FLOWROI_EINVAL;
    const int align = 1 << levels;
    if (width < 16 || height < 16 || width % align || height % align) return FLOWROI_EINVAL;
    if ((size_t)width * (size_t)height > kNaMaxPixels) return FLOWROI_EINVAL;  // larger than the fixed array holds
    const int pitch = pitch_bytes ? pitch_bytes : width * bpp;
    if (pitch < width * bpp) return FLOWROI_EINVAL;
    // The kernel reads 16-bit samples in aligned pairs and mask bytes in
    // aligned pairs, and stores 32-bit coefficients.
    if (bpp == 2 && ((reinterpret_cast<uintptr_t>(raw) & 3) || (pitch & 3))) return FLOWROI_EINVAL;
    if ((reinterpret_cast<uintptr_t>(mask) & 1) || (reinterpret_cast<uintptr_t>(coeffs) & 3)) return FLOWROI_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return FLOWROI_EDEVICE;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_dev_ptr[dev]) {
        // Set-up, once per device, with that device current: the host-side
        // name of a __device__ array is not its device address.
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FLOWROI_EDEVICE;
        }
        g_na_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    unsigned char *base = g_na_dev_ptr[dev];

    MethodConsts mc;
    memset(&mc, 0, sizeof mc);
    mc.wavelet = wavelet;
    mc.dwt_levels = levels;
    mc.shift = scale_shift;
    for (int b = 0; b < kMaxSubbands; b++) mc.delta[b] = 1.f;
    if (wavelet == FLOWROI_W97)
        for (int b = 0; b <= 3 * levels; b++) {
            if (!(delta[b] > 0.f) || !(delta[b] < 1e30f)) return FLOWROI_EINVAL;
            mc.delta[b] = delta[b];
        }
    for (int b = 0; b < kMaxSubbands; b++) mc.rdelta[b] = 1.f / mc.delta[b];  // IEEE float division: rounded to nearest

    NaDesc nd;
    memset(&nd, 0, sizeof nd);
    FrameDesc &F = nd.f;
    F.W = width;
    F.H = height;
    F.bpp = bpp;
    F.bit_depth = bit_depth;
    F.raw_pitch = pitch;
    F.dc_off = 1 << (bit_depth - 1);
    F.raw = raw;
    F.mask = const_cast<uint8_t *>(mask);
    F.coeffs = coeffs;
    F.dwt_raw = raw;
    F.dwt_mask = const_cast<uint8_t *>(mask);
    F.dwt_coeffs = coeffs;
    F.do_dwt = 1;
    F.ll[0] = base + kNaDescBytes;
    F.ll[1] = base + kNaDescBytes + kNaLLBytes;
    F.llm[0] = base + kNaDescBytes + 2 * kNaLLBytes;
    F.llm[1] = base + kNaDescBytes + 2 * kNaLLBytes + kNaLLMBytes;
    for (int l = 1; l <= levels; l++) {
        F.dwt_seg[l - 1] = dwt_default_seg(width >> l, height >> l);
        nd.tiles[l - 1] = dwt_units(width >> l, height >> l, F.dwt_seg[l - 1]);
    }
    BatchDesc *bdd = reinterpret_cast<BatchDesc *>(base);
    // An error left pending by an earlier, unrelated call on this thread
    // would otherwise be reported as this call's; a launch that fails stops
    // the sequence there (the levels after it are not queued).
    cudaGetLastError();
    k_na_desc<<<1, 128, 0, st>>>(nd, bdd);
    if (cudaGetLastError() != cudaSuccess) return FLOWROI_EDEVICE;
    for (int l = 1; l <= levels; l++) {
        launch_dwt(bdd, mc, l, dwt_grid(nd.tiles[l - 1], 1 << 20), 5, st);
        if (cudaGetLastError() != cudaSuccess) return FLOWROI_EDEVICE;
    }
    return FLOWROI_OK;
}
