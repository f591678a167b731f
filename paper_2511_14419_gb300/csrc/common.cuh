// Device-visible descriptors and small device helpers shared by the
// FlowRoI kernels and the runtime that fills them.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace flowroi {

constexpr int kMaxLevels = 8;    // pyramid and DWT levels
constexpr int kMaxBatch = 64;    // frames per batched launch
constexpr int kHistBins = 2048;  // radix-select digit of 11 bits
constexpr int kCandBlocks = 32;  // blocks per frame of the last radix digit
constexpr int kMaxSubbands = 3 * kMaxLevels + 1;
constexpr int kLoopLimit = 1 << 24;          // union-find loop steps before a loop gives up
constexpr unsigned kTestTmaSpin = 1u << 12;  // FLOWROI_TEST_EXPIRE_TMA: polls of a bounded TMA wait
constexpr int kTestLoopLimit = 1;            // FLOWROI_TEST_EXPIRE_LOOP: union-find loop steps

// Tile shapes (output pixels per block) of each kernel family.
constexpr int kDenMaxR = 3;                // largest bilateral radius of the optional denoising
constexpr int kMaxAdj = 4;                 // largest adjacent factor (masks of frames t-k..t+k merged)
constexpr int kExpTW = 256, kExpTH = 16;   // pyramid + polynomial expansion
constexpr int kUpdTW = 256, kUpdRows = 4; // displacement update (G, h per pixel)
constexpr int kWinTW = 64, kWinTH = 64;   // box window + 2x2 solve
constexpr int kSalTW = 256, kSalTH = 32;   // radix-select passes (saliency: kSalSub-row strips, per frame)
constexpr int kSalSub = 8;                 // saliency: rows per staged strip
constexpr int kMorTW = 256, kMorTH = 64;  // threshold + opening + closing (8 words x 64 rows)
constexpr int kDwtStrip = 60;             // DWT: band columns per warp unit (lanes 1..30, two each)
constexpr int kDwtWarps = 4;              // DWT: warps (independent units) per block
constexpr int kDwtRing = 4;               // DWT: row pairs in a warp's staging ring (kDwtRing - 1 in flight)

// Per-frame reduction block (device), one per frame slot.
//   [0] min of S (float bits), [1] max of S, [2] select prefix,
//   [3] remaining rank, [4] t_S bits, [5] t_hat bits, [6] s* bits (the
//   largest S whose normalised value is <= t_hat: mask0 = S > s*),
//   [kRedHist .. +kHistBins) histogram of the current radix digit.
constexpr int kRedMin = 0, kRedMax = 1, kRedPrefix = 2, kRedRank = 3, kRedTS = 4, kRedTHat = 5, kRedSStar = 6;
constexpr int kRedCand = 7;  // S values left after the second digit, in FrameDesc::cand
constexpr int kRedHist = 8;
//   [kRedReg ..) registration: the level image's sum (double), max |X|
//   (float bits), the correlation peak key (u64) and the drift (2 floats).
constexpr int kRedReg = kRedHist + kHistBins;
constexpr int kRedRegSum = kRedReg, kRedRegXMax = kRedReg + 2, kRedRegPeak = kRedReg + 4, kRedRegDrift = kRedReg + 6;
constexpr int kRedWords = kRedReg + 8;

// Method constants of a context (passed by value to every kernel).
struct MethodConsts {
    // polynomial expansion: 1-D applicability a(u), u = -n..n, and the
    // closed-form projection constants of the separable fit.
    int n_half;
    float app[7];
    float inv_s0s2;   // r_u = <u,f> / (s0 s2), r_v likewise
    float inv_s2s2;   // r_uv = <uv,f> / s2^2
    float m_uu[3];    // r_uu = m_uu . (<1,f>, <u^2,f>, <v^2,f>)
    float m_vv[3];    // r_vv likewise
    // displacement
    int pyr_levels, iters, win_r;
    float lambda;
    // saliency / threshold / morphology
    float alpha;      // weight of |d|
    float q;          // RoI threshold
    int r_open, r_close;
    // JPEG2000 front end
    int wavelet, dwt_levels, shift;
    float delta[kMaxSubbands];
    float rdelta[kMaxSubbands];  // float32 reciprocals of delta, rounded to nearest (the quantiser's divisor)
    // optional denoising of the flow input: bilateral radius; the weights
    // as powers of two, w = 2^-(den_ls[offset] + den_lr * (I(q) - I(p))^2),
    // den_ls = -log2 of the spatial weight over the (2 kDenMaxR + 1)^2
    // square (row-major, centred), den_lr = log2(e) / (2 sigma_r^2)
    int min_area;  // components of the final mask below this many pixels removed (<= 1: off)
    int reg_on, reg_level;  // registration to the predecessor by phase correlation of pyramid level reg_level
    int denoise, den_r;
    float den_ls[(2 * kDenMaxR + 1) * (2 * kDenMaxR + 1)];
    float den_lr;
};

// Embedded block coding (k_ebcot.cu): one frame of a coder job, with the
// scratch of its code-blocks, and the job.
constexpr int kCb = 64;                        // code-block side
constexpr int kMaxPlanes = 24;                 // magnitudes below 2^24
constexpr int kMaxPasses = 3 * kMaxPlanes - 2;
constexpr int kCbInfo = 8;                     // per code-block: planes, passes, kept, status, hull size, data size, data offset
constexpr int kCsHeader = 32, kCsEntry = 16;   // container header and per-code-block entry bytes
// JPEG2000 codestream: bytes of the markers (with 3 x 8 + 1 bands) and of
// a code-block's packet-header bits at most (tag-tree paths, pass count,
// Lblock, 70 lengths of up to 16 bits, one stuffed bit per byte)
constexpr int kJ2cHeader = 256, kJ2cPerBlock = 192;
constexpr unsigned kErrCbRange = 3u;           // error word: a code-block or container exceeded its buffer or range
constexpr int kCbBytes = 32768;                // pass bytes a code-block may produce
// Coding decisions a code-block's passes may produce, one byte each
// (context << 1 | decision): per bit-plane and stripe column at most six
// that are not signs (four samples, or run-length mode's run symbol, two
// position symbols and the three samples below), and one sign per sample
// over all planes; each pass starts 16-byte aligned.
constexpr int kSymCap = kMaxPlanes * 6 * (kCb * kCb / 4) + kCb * kCb + 16 * kMaxPasses;
// Bytes of a code-block's pass-byte region: each pass is first coded into
// a slot of floor(S / 7) + 3 bytes (S its renormalisation shifts; a pass of
// L bytes has S <= 8 L + 12), and the slots of a block whose passes fit
// kCbBytes sum to less than 8/7 kCbBytes + 5 per pass; then moved down to
// be contiguous.
constexpr int kCbRegion = 40960;
constexpr int kMqWords = 20;  // a pass's starting MQ context states (19 contexts, padded)
// device bytes of a code-block's scratch (pass bytes, decision stream and
// per-pass counts, lengths, distortions, context states and slot table,
// info, hull)
constexpr size_t kCbScratch = (size_t)kCbRegion + (size_t)kSymCap + kMaxPasses * (4 + 4 + 8 + 4 * kMqWords + 16) +
                              kCbInfo * 4 + (kMaxPasses + 1) * (4 + 8);

struct CsFrame {
    const int32_t *coef;  // Mallat plane, row pitch = w
    uint8_t *out;         // container
    long long cap;        // container capacity (bytes)
    long long budget;     // pass-data budget (bytes); <= 0 keeps every pass
    int w, h, levels, wavelet, shift, bit_depth;
    int cb0, ncb;         // the frame's code-blocks in the job
    // per code-block scratch of the frame, [ncb][...]
    uint8_t *cbytes;      // [kCbRegion] pass bytes (the first kCbBytes hold them back to back)
    int32_t *plen;        // [kMaxPasses]
    uint8_t *sym;         // [kSymCap] the passes' coding decisions, in coding order
    int32_t *nsym;        // [kMaxPasses] decisions per pass
    uint32_t *mqs;        // [kMaxPasses][kMqWords] MQ context states at each pass's start
    int4 *ptab;           // [kMaxPasses] per pass: first decision, slot offset, slot bytes
    double *dist;         // [kMaxPasses]
    int32_t *info;        // [kCbInfo]
    int32_t *hk;          // [kMaxPasses + 1] hull scratch
    double *hs;           // [kMaxPasses + 1]
    long long *flen;      // the container's length (negative: it needs that many bytes; -1: a code-block out of range)
    int format;           // 0: the library's frame container, 1: JPEG2000 Part 1 codestream
    int reset;            // 1: the MQ contexts reset at every pass (code-block style 0x02)
    uint8_t eps[kMaxSubbands];   // 1: the bands' quantisation exponents (table index as delta[])
    uint16_t mu[kMaxSubbands];   // 1: and mantissas (9/7)
};
struct CsJob {
    int nframes, ncb;
    const CsFrame *frames;  // device array [nframes]
    int cbcap;              // kCbBytes
    unsigned *err;          // error word, or null
    int *next;              // work counters, zeroed before the coder runs: [0] modelling, [1] MQ state chains,
                            // [2] MQ codewords, [3] MQ states of passes coded apart (reset)
};

// One frame of a batch.  Level geometry: lw/lh = level size, lp = pitch in
// elements.  All planes of the previous frame of the same stream are read
// through fq_prev / fb_prev.
struct FrameDesc {
    // TMA maps of the five G, h planes per level (3-D: x, y, plane).
    CUtensorMap gh_map[kMaxLevels];
    int W, H, bpp, bit_depth;
    int has_prev, keep, raw_pitch, dc_off;  // raw_pitch in bytes; dc_off = 2^(B-1)
    float unit_scale;                        // 255 / (2^B - 1)
    int pad0, pad1, pad2;
    const void *raw;
    int lw[kMaxLevels], lh[kMaxLevels], lp[kMaxLevels];
    void *pyr[kMaxLevels];          // level images 1..L-1 (storage type)
    void *fq_cur[kMaxLevels];       // A11, A12, A22, b1 (4 x storage type per pixel)
    void *fb_cur[kMaxLevels];       // b2 (storage type per pixel)
    void *gh[kMaxLevels];           // G11, G12, G22, h1, h2: five planes (storage type)
    const void *fq_prev[kMaxLevels];
    const void *fb_prev[kMaxLevels];
    float2 *flow[2];                // ping-pong flow buffers, level-0 capacity
    float *S;                       // saliency, pitch lp[0]
    unsigned *red;                  // reduction block (kRedWords)
    unsigned *cand;                 // the S bits of the pixels the last digit pass reads (W*H words)
    uint8_t *mask;                  // result mask, W*H
    int32_t *coeffs;                // result coefficients, W*H (Mallat)
    float2 *dbg_flow;               // keep: level-0 flow, W*H (else null)
    float *dbg_shat;                // keep: normalised saliency, W*H
    uint8_t *dbg_mask0;             // keep: mask before morphology, W*H
    float *dbg_yf;                  // keep + 9/7: float coefficients, W*H
    float *dbg_thr;                 // keep: threshold on S^ (1 float)
    float *dbg_den;                 // keep + denoise: denoised flow input, W*H
    float *dbg_drift;               // keep + registration: the drift (2 floats)
    int *cc_lab, *cc_cnt, *cc_area; // min_area > 1: component labels, local-root counts, areas (W*H each)
    // JPEG2000 front end of this entry: the frame it codes (the flow frame
    // itself, or with an adjacent factor k > 0 the frame k earlier), its
    // samples, RoI mask and outputs
    const void *dwt_raw;
    uint8_t *dwt_mask;
    int32_t *dwt_coeffs;
    float *dwt_yf;                  // keep + 9/7: float coefficients of that frame
    int do_flow, do_dwt;
    // registration (do_reg): padded FFT size 2^reg_lnx x 2^reg_lny of the
    // level image, this frame's spectrum (kept for the next frame), the
    // predecessor's, and the correlation work plane
    int do_reg, reg_lnx, reg_lny;
    float2 *reg_cur, *reg_prev, *reg_work;
    int do_cs;                      // the JPEG2000 target's coefficients are coded into a container
    CsFrame cs;
    int n_adj;                      // per-frame masks ORed into dwt_mask (0: none, dwt_mask is the frame's own)
    const uint8_t *adj[2 * kMaxAdj + 1];
    void *ll[2];                    // DWT low-low temporaries ((W/2)*(H/2) elements)
    int dwt_seg[kMaxLevels];        // DWT: band rows per warp unit at each level
    int sal_strips;                 // saliency: tiles of kSalSub x sal_strips rows
    uint8_t *llm[2];                // their RoI masks
};

// A batch: per kernel family and level, an exclusive prefix over frames of
// their tile counts (blocks binary-search it to find their frame).
struct BatchDesc {
    int nframes;
    int final_flow_buf;             // ping-pong index holding the level-0 flow
    unsigned *err;                  // error word (mapped host memory); kernels set it on a failed wait
    unsigned tma_spin;              // polls of a bounded TMA wait before it gives up
    int loop_limit;                 // steps of a bounded union-find loop before it gives up
    int test_skip_tile;             // test only: the level-0 window producer of block 0 skips its first tile's copies
    int exp_off[kMaxLevels][kMaxBatch + 1];
    int flow_off[kMaxLevels][kMaxBatch + 1];   // update tiles
    int win_off[kMaxLevels][kMaxBatch + 1];    // window tiles
    int dwt_off[kMaxLevels][kMaxBatch + 1];
    int sal_off[kMaxBatch + 1];     // frames with a predecessor only (kSalTW x kSalTH tiles)
    int sal2_off[kMaxBatch + 1];    // the saliency kernel's own tiles (kSalTW x kSalSub * sal_strips)
    int mor_off[kMaxBatch + 1];     // every flow frame
    int frm_off[kMaxBatch + 1];     // one unit per frame (init / select-find)
    int mrg_off[kMaxBatch + 1];     // adjacent-mask merge: 4096-byte units of entries with n_adj > 0
    int reg_row_off[kMaxBatch + 1]; // registration: padded rows, 8-column groups, 4096-element units
    int reg_col_off[kMaxBatch + 1];
    int reg_el_off[kMaxBatch + 1];
    FrameDesc f[kMaxBatch];
    CsJob cs;                       // the batch's coder job over csf (frames with do_cs)
    CsFrame csf[kMaxBatch];
    int cs_next[4];                 // the coder's work counters
};

#ifdef __CUDACC__
// Frame owning global tile t: largest i with off[i] <= t (off[0] = 0).
__device__ __forceinline__ int find_frame(const int *off, int nframes, int t)
{
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Storage conversions.
template <typename T> struct Store;
template <> struct Store<float> {
    using T4 = float4;
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float4 ld4(const float4 *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
    static __device__ __forceinline__ void st4(float4 *p, float a, float b, float c, float d) { *p = make_float4(a, b, c, d); }
    static __device__ __forceinline__ float4 f4(float4 v) { return v; }
};
template <> struct Store<__half> {
    using T4 = uint2;  // four halves
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ uint2 ld4(const uint2 *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void st4(uint2 *p, float a, float b, float c, float d)
    {
        __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&lo);
        u.y = *reinterpret_cast<unsigned *>(&hi);
        *p = u;
    }
    static __device__ __forceinline__ float4 f4(uint2 u)
    {
        __half2 lo = *reinterpret_cast<__half2 *>(&u.x), hi = *reinterpret_cast<__half2 *>(&u.y);
        float2 a = __half22float2(lo), b = __half22float2(hi);
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
#endif

}  // namespace flowroi
