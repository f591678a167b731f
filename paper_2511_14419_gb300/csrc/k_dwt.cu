// JPEG2000 front end of the RoI encoder, one DWT level per launch:
// DC level shift (level 1), 2-D lifting DWT (columns then rows), dead-zone
// quantisation (9/7), wavelet-domain RoI mask, RoI up-shift.
//
// Paper: §Implementation details (JPEG2000 scaling-based RoI: RoI
// coefficients are scaled up by the user's scaling factor) and Table 1.
//   - DC shift: x - 2^(B-1).
//   - Lifting with whole-sample symmetric extension:
//       5/3: H[k] = x[2k+1] - floor((x[2k] + x[2k+2]) / 2)
//            L[k] = x[2k]   + floor((H[k-1] + H[k] + 2) / 4)
//       9/7: four lifting steps (alpha, beta, gamma, delta of the CDF 9/7
//            factorisation), then low / K and high * K.
//   - Quantisation (9/7): q = sign(y) floor(|y| / delta_b), the quotient
//     rounded to float32 as an IEEE division would; 5/3: q = y.
//   - A coefficient is RoI when its synthesis support meets the RoI:
//       5/3: low k <- samples [2k-1, 2k+1], high k <- [2k-1, 2k+3]
//       9/7: low k <- samples [2k-3, 2k+3], high k <- [2k-3, 2k+5]
//     (clipped to the signal), applied to columns then rows of the
//     previous level's low-low mask (level 1: the pixel mask).
//   - RoI coefficients: q <- sign(q) (|q| << s).
//
// Work decomposition: one warp per unit (frame, strip, segment), no shared
// memory and no barriers.  A strip is 60 band columns: lane j (0..31) owns
// the 4 input columns 2*bc..2*bc+3 with bc = 60*strip + 2*(j-1), so lanes
// 0 and 31 hold the symmetric-extension apron of lanes 1..30, whose 2
// low and 2 high band columns are stored.  A segment is `seg` band rows
// (per frame and level, FrameDesc::dwt_seg).
//   - Vertical: the warp walks its input rows in pairs (2n, 2n+1), one pair
//     per step.  The pairs are staged by cp.async into a warp-private ring
//     of kDwtRing pairs in shared memory, kDwtRing - 1 pairs ahead; each
//     lane copies and later reads only its own columns, so no barrier is
//     needed.  A lane whose columns lie outside the image on the left
//     (right) copies the two aligned chunks holding their mirror images
//     and permutes them when it reads.  Each column is
//     lifted as a stream: the lifting steps of the 9/7 (5/3) factorisation
//     run with a lag of two pairs (one pair), keeping five (three) values
//     per column in registers, so each step completes one low and one
//     high row.  The segment's first 2 (1) steps only fill the pipeline
//     (the apron rows above it); rows outside the image are read from
//     their mirror image.
//   - Horizontal: each completed row is lifted across the warp, lane j
//     holding (even, odd, even, odd) samples and taking its neighbours'
//     from lanes j-1 and j+1 by shuffles.
//   - Masks: mask words (4 columns as bytes) of the pairs needed by the
//     vertical rule are kept ORed per pair; the horizontal rule works on a
//     12-bit window of 4-bit column masks from lanes j-1, j, j+1.
//   - Stores: per step, two 32-bit band coefficients per lane and band
//     (8-byte stores), the low-low band to a temporary plane for the next
//     level (or, at the last level, quantised into the coefficient plane).
// A batch entry's DWT codes the frame named by its dwt_* fields (with an
// adjacent factor, an earlier frame than the one whose flow the entry
// computes).
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace flowroi {

namespace {

constexpr float kA = -1.586134342059924f, kB = -0.052980118572961f, kG = 0.882911075530934f,
                kD = 0.443506852043971f, kK = 1.230174104914001f;
// The normalisation (low / K, high * K in each direction) is applied once
// per 2-D band: HL and LH carry K / K = 1, LL 1/K^2, HH K^2 (each a float
// rounded from the double product; one rounding per coefficient instead of
// two, far inside the 9/7 coefficient tolerance).
constexpr float kInvK2 = (float)(1.0 / (1.230174104914001 * 1.230174104914001));
constexpr float kK2 = (float)(1.230174104914001 * 1.230174104914001);
constexpr unsigned kFull = 0xffffffffu;

enum { kSrcU8 = 0, kSrcU16 = 1, kSrcLL = 2 };

// Whole-sample symmetric extension of index i into [0, n), for any i: one
// reflection where it lands inside, else the periodic form (a strip's apron
// reaches more than a signal length past the edge on small images).
__device__ __noinline__ int mirror_far(int i, int n)
{
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    i %= period;
    if (i < 0) i += period;
    return i <= n - 1 ? i : period - i;
}
__device__ __forceinline__ int mirror(int i, int n)
{
    if (i >= 0 && i < n) return i;
    if (i < 0 && -i < n) return -i;
    if (i >= n && i <= 2 * (n - 1)) return 2 * (n - 1) - i;
    return mirror_far(i, n);
}

// Four samples of one row, columns cx..cx+3, as loaded (u8: .x holds four
// bytes; u16: .x, .y two samples each; low-low plane: one 32-bit value per
// component).  Columns outside the image come from their mirror image.
template <int SRC>
__device__ __noinline__ uint4 load_row_slow(const unsigned char *row, int cx, int iw);
template <int SRC>
__device__ __forceinline__ uint4 load_row(const unsigned char *row, int cx, int iw, bool vec)
{
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (!(vec && cx >= 0 && cx + 4 <= iw)) return load_row_slow<SRC>(row, cx, iw);
    {
        if constexpr (SRC == kSrcU8) {
            r.x = __ldg(reinterpret_cast<const unsigned *>(row + cx));
        } else if constexpr (SRC == kSrcU16) {
            const uint2 t = __ldg(reinterpret_cast<const uint2 *>(row + 2 * cx));
            r.x = t.x;
            r.y = t.y;
        } else {
            r = __ldg(reinterpret_cast<const uint4 *>(row + 4 * cx));
        }
        return r;
    }
}
template <int SRC>
__device__ __noinline__ uint4 load_row_slow(const unsigned char *row, int cx, int iw)
{
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    unsigned v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = mirror(cx + k, iw);
        if constexpr (SRC == kSrcU8) v[k] = __ldg(row + c);
        else if constexpr (SRC == kSrcU16) v[k] = __ldg(reinterpret_cast<const unsigned short *>(row) + c);
        else v[k] = __ldg(reinterpret_cast<const unsigned *>(row) + c);
    }
    if constexpr (SRC == kSrcU8) {
        r.x = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
    } else if constexpr (SRC == kSrcU16) {
        r.x = v[0] | (v[1] << 16);
        r.y = v[2] | (v[3] << 16);
    } else {
        r = make_uint4(v[0], v[1], v[2], v[3]);
    }
    return r;
}

// Mask bytes of row y at columns cx..cx+3 (any nonzero byte is RoI); 0
// outside the image (the support rules are clipped to the signal).
__device__ __noinline__ uint32_t load_mask_slow(const uint8_t *row, int cx, int iw)
{
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = cx + k;
        if (c >= 0 && c < iw && __ldg(row + c)) m |= 1u << (8 * k);
    }
    return m;
}
__device__ __forceinline__ uint32_t load_mask(const uint8_t *base, int pitch, int y, int ih, int cx, int iw, bool vec)
{
    if (y < 0 || y >= ih || cx + 4 <= 0 || cx >= iw) return 0u;
    const uint8_t *row = base + (size_t)y * pitch;
    if (vec && cx >= 0 && cx + 4 <= iw) return __ldg(reinterpret_cast<const unsigned *>(row + cx));
    return load_mask_slow(row, cx, iw);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bytes per lane and row of a source: 4 samples (u8 4, u16 8, float/int 16).
template <int SRC> struct Chunk {
    static constexpr int bytes = SRC == kSrcU8 ? 4 : (SRC == kSrcU16 ? 8 : 16);
};

template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(B) : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_s(uint32_t dst, const void *src)
{
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int SRC>
__device__ __forceinline__ uint4 lds_chunk(const unsigned char *p)
{
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (SRC == kSrcU8) {
        r.x = *reinterpret_cast<const unsigned *>(p);
    } else if constexpr (SRC == kSrcU16) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        r.x = t.x;
        r.y = t.y;
    } else {
        r = *reinterpret_cast<const uint4 *>(p);
    }
    return r;
}
template <int SRC>
__device__ __forceinline__ void sts_chunk(unsigned char *p, const uint4 &r)
{
    if constexpr (SRC == kSrcU8) *reinterpret_cast<unsigned *>(p) = r.x;
    else if constexpr (SRC == kSrcU16) *reinterpret_cast<uint2 *>(p) = make_uint2(r.x, r.y);
    else *reinterpret_cast<uint4 *>(p) = r;
}

// Lane kinds of a unit's source columns cx..cx+3.
enum { kColPacked = 0, kColLeft = 1, kColRight = 2, kColNone = 3 };

// Columns -4..-1 mirror to 4, 3, 2, 1 (chunks c0 = columns 0..3, c1 =
// 4..7); columns iw..iw+3 mirror to iw-2..iw-5 (c0 = iw-8..iw-5, c1 =
// iw-4..iw-1).
template <int SRC>
__device__ __forceinline__ uint4 mirror_chunks(const uint4 &c0, const uint4 &c1, bool left)
{
    uint4 r;
    if constexpr (SRC == kSrcU8) {
        r = make_uint4(__byte_perm(c0.x, c1.x, left ? 0x1234 : 0x3456), 0u, 0u, 0u);
    } else if constexpr (SRC == kSrcU16) {
        if (left) r = make_uint4(__byte_perm(c1.x, c0.y, 0x7610), __byte_perm(c0.y, c0.x, 0x7610), 0u, 0u);
        else r = make_uint4(__byte_perm(c1.y, c1.x, 0x7610), __byte_perm(c1.x, c0.y, 0x7610), 0u, 0u);
    } else {
        r = left ? make_uint4(c1.x, c0.w, c0.z, c0.y) : make_uint4(c1.z, c1.y, c1.x, c0.w);
    }
    return r;
}

// Loaded samples -> the level's arithmetic type (level 1: DC-shifted).
// A 16-bit sample u becomes a float exactly as the bit pattern
// 0x4B000000 | u (= 2^23 + u) minus 2^23 + dc.
template <int WAV, int SRC, typename V>
__device__ __forceinline__ void to_vals(const uint4 &r, int dc, float dcf, V (&v)[4])
{
    if constexpr (SRC == kSrcLL) {
        if constexpr (WAV == 97) {
            v[0] = __uint_as_float(r.x), v[1] = __uint_as_float(r.y), v[2] = __uint_as_float(r.z), v[3] = __uint_as_float(r.w);
        } else {
            v[0] = (int)r.x, v[1] = (int)r.y, v[2] = (int)r.z, v[3] = (int)r.w;
        }
    } else if constexpr (WAV == 97) {
        if constexpr (SRC == kSrcU8) {
            v[0] = __uint_as_float(__byte_perm(r.x, 0x4B00u, 0x5440)) - dcf;
            v[1] = __uint_as_float(__byte_perm(r.x, 0x4B00u, 0x5441)) - dcf;
            v[2] = __uint_as_float(__byte_perm(r.x, 0x4B00u, 0x5442)) - dcf;
            v[3] = __uint_as_float(__byte_perm(r.x, 0x4B00u, 0x5443)) - dcf;
        } else {
            v[0] = __uint_as_float(__byte_perm(r.x, 0x4B00u, 0x5410)) - dcf;
            v[1] = __uint_as_float(__byte_perm(r.x, 0x4B00u, 0x5432)) - dcf;
            v[2] = __uint_as_float(__byte_perm(r.y, 0x4B00u, 0x5410)) - dcf;
            v[3] = __uint_as_float(__byte_perm(r.y, 0x4B00u, 0x5432)) - dcf;
        }
    } else {
        if constexpr (SRC == kSrcU8) {
            v[0] = (int)(r.x & 0xffu) - dc, v[1] = (int)((r.x >> 8) & 0xffu) - dc;
            v[2] = (int)((r.x >> 16) & 0xffu) - dc, v[3] = (int)(r.x >> 24) - dc;
        } else {
            v[0] = (int)(r.x & 0xffffu) - dc, v[1] = (int)(r.x >> 16) - dc;
            v[2] = (int)(r.y & 0xffffu) - dc, v[3] = (int)(r.y >> 16) - dc;
        }
    }
}

// 4 column masks (bytes, nonzero = RoI) -> bits 0..3.
__device__ __forceinline__ uint32_t nibble(uint32_t w)
{
    // bit 7 of each byte becomes "byte != 0": its low 7 bits plus 0x7f
    // carry into bit 7 exactly when they are nonzero, and never beyond
    // the byte (at most 0x7f + 0x7f); OR-ing the byte keeps a set bit 7.
    // The four bit 7s are then gathered into bits 0..3 by one multiply.
    const uint32_t t = (((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;
    return ((t >> 7) * 0x01020408u) >> 24;
}

// Horizontal lifting of one row across the warp: this lane holds samples
// (e0, o0, e1, o1) at columns 4j..4j+3; the even sample right of o1 is
// lane j+1's e0, the odd sample left of e0 is lane j-1's o1.  9/7: the four
// lifting steps only; the caller applies the band's normalisation.
__device__ __forceinline__ void hlift(float &e0, float &o0, float &e1, float &o1)
{
    o0 += kA * (e0 + e1);
    o1 += kA * (e1 + __shfl_down_sync(kFull, e0, 1));
    e0 += kB * (__shfl_up_sync(kFull, o1, 1) + o0);
    e1 += kB * (o0 + o1);
    o0 += kG * (e0 + e1);
    o1 += kG * (e1 + __shfl_down_sync(kFull, e0, 1));
    e0 += kD * (__shfl_up_sync(kFull, o1, 1) + o0);
    e1 += kD * (o0 + o1);
}
__device__ __forceinline__ void hlift(int &e0, int &o0, int &e1, int &o1)
{
    o0 -= (e0 + e1) >> 1;
    o1 -= (e1 + __shfl_down_sync(kFull, e0, 1)) >> 1;
    e0 += (__shfl_up_sync(kFull, o1, 1) + o0 + 2) >> 2;
    e1 += (o0 + o1 + 2) >> 2;
}

// Quantised, RoI-shifted coefficient.  9/7: floor(RN(|y| / d)) with RN
// the float32 round-to-nearest quotient, formed from rd = RN(1/d) by one
// residual correction (Markstein, "Computation of elementary functions on
// the IBM RISC System/6000 processor", IBM J. Res. Dev. 34(1), 1990: with
// rd the correctly rounded reciprocal and q0 within an ulp of the
// quotient, q0 + (|y| - d q0) rd rounded once is the correctly rounded
// quotient; the residual is exact in a fused multiply-add).  5/3: y itself.
__device__ __forceinline__ int32_t qroi(float y, float d, float rd, bool roi, int s)
{
    const float a = fabsf(y);
    const float q0 = __fmul_rn(a, rd);
    const float e = __fmaf_rn(-q0, d, a);
    const float q1 = __fmaf_rn(e, rd, q0);
    const int32_t mag = __float2int_rd(q1) << (roi ? s : 0);
    return y < 0.f ? -mag : mag;
}
__device__ __forceinline__ int32_t qroi(int y, float, float, bool roi, int s)
{
    return (int32_t)((uint32_t)y << (roi ? s : 0));
}

template <typename T>
__device__ __forceinline__ bool aligned(const void *p, int n)
{
    return (reinterpret_cast<uintptr_t>(p) & (uintptr_t)(n - 1)) == 0;
}

// Stores a pair of adjacent values at p (8-byte store when allowed).
template <typename T>
__device__ __forceinline__ void st2(T *p, T a, T b, bool vec, bool both)
{
    if (vec) {
        if constexpr (std::is_same<T, float>::value) *reinterpret_cast<float2 *>(p) = make_float2(a, b);
        else *reinterpret_cast<int2 *>(p) = make_int2((int)a, (int)b);
    } else {
        p[0] = a;
        if (both) p[1] = b;
    }
}

// One unit: frame fi, unit index lt within the frame's units of this level.
template <int WAV, int SRC>
__device__ __forceinline__ void dwt_unit(const FrameDesc &F, const MethodConsts &mc, int level, int lt, int lane,
                                         unsigned char *ring)
{
    using V = typename std::conditional<WAV == 97, float, int>::type;
    constexpr int A = WAV == 97 ? 2 : 1;  // apron pairs above the segment = output lag in pairs
    const int W = F.W;
    const int iw = W >> (level - 1), ih = F.H >> (level - 1), bw = iw >> 1, bh = ih >> 1;
    const int seg = F.dwt_seg[level - 1];
    const int nst = (bw + kDwtStrip - 1) / kDwtStrip;
    const int sgi = lt / nst, sti = lt - sgi * nst;
    const int r0 = sgi * seg, r1 = min(r0 + seg, bh);  // band rows [r0, r1)
    const int bc = sti * kDwtStrip + 2 * (lane - 1);    // first band column of this lane's outputs
    const int cx = 2 * bc;                              // first of its 4 input columns
    const bool last = level == mc.dwt_levels;
    const bool outl = lane >= 1 && lane <= 30 && bc < bw;
    const bool both = bc + 1 < bw;

    // Sources: level 1 the raw frame and pixel mask, above it the previous
    // level's low-low plane (pitch iw) and its mask.
    const unsigned char *src;
    size_t spitch;
    const uint8_t *msrc;
    int mpitch;
    bool svec;
    if constexpr (SRC == kSrcLL) {
        src = static_cast<const unsigned char *>(F.ll[level % 2]);
        spitch = (size_t)iw * 4;
        msrc = F.llm[level % 2];
        mpitch = iw;
        svec = aligned<int>(src, 16) && (iw & 3) == 0;
    } else {
        src = static_cast<const unsigned char *>(F.dwt_raw);
        spitch = (size_t)F.raw_pitch;
        msrc = F.dwt_mask;
        mpitch = W;
        const int sa = SRC == kSrcU8 ? 4 : 8;
        svec = aligned<int>(src, sa) && (F.raw_pitch & (sa - 1)) == 0;
    }
    const bool mvec = aligned<int>(msrc, 4) && (mpitch & 3) == 0;
    const int dc = SRC == kSrcLL ? 0 : F.dc_off;
    const float dcf = 8388608.f + (float)dc;

    // Outputs.
    int32_t *const coeffs = F.dwt_coeffs;
    float *const yf = WAV == 97 ? F.dwt_yf : nullptr;
    V *const llo = static_cast<V *>(F.ll[(level - 1) % 2]);
    uint8_t *const llmo = F.llm[(level - 1) % 2];
    const bool ovec = (bw & 1) == 0 && aligned<int>(coeffs, 8) && (!yf || aligned<int>(yf, 8)) &&
                      (last || (aligned<int>(llo, 8) && aligned<int>(llmo, 2)));
    const int b_ll = 3 * mc.dwt_levels, b_hl = 3 * (level - 1), b_lh = b_hl + 1, b_hh = b_hl + 2;
    const float d_ll = mc.delta[b_ll], d_hl = mc.delta[b_hl], d_lh = mc.delta[b_lh], d_hh = mc.delta[b_hh];
    const float r_ll = mc.rdelta[b_ll], r_hl = mc.rdelta[b_hl], r_lh = mc.rdelta[b_lh], r_hh = mc.rdelta[b_hh];
    const int sh = mc.shift;
    const int ohl = bw + bc;                  // column of this lane's high-horizontal outputs
    const size_t hoff = (size_t)bh * W;       // offset of the vertical-high half of the plane
    // horizontal rules on the 12-bit window (bit i = column 4j - 4 + i)
    constexpr uint32_t kE0 = WAV == 97 ? 0x0FEu : 0x038u, kE1 = WAV == 97 ? 0x3F8u : 0x0E0u;
    constexpr uint32_t kO0 = WAV == 97 ? 0x3FEu : 0x0F8u, kO1 = WAV == 97 ? 0xFF8u : 0x3E0u;

    // Pipeline state per column (see the header).  9/7: the partial sums of
    // lifting steps 1-4 that the next pair completes (x_odd + a x_even,
    // x_even + b o1, o1 + g e2, e2 + d o3 of the rows above); 5/3: the
    // previous pair and the last high sample.
    V xe[4], xo[4], s1[4], s2[4], s3[4];
#pragma unroll
    for (int c = 0; c < 4; c++) xe[c] = xo[c] = s1[c] = s2[c] = s3[c] = (V)0;
    // mask history: ORs of the last three pairs, odd rows of the last four
    uint32_t p1 = 0, p2 = 0, p3 = 0, od1 = 0, od2 = 0, od3 = 0, od4 = 0;

    // Staging kinds of this lane's columns (constant over the unit).
    constexpr int CH = Chunk<SRC>::bytes, E = CH / 4;  // chunk bytes, bytes per sample
    int kind;
    bool sync_load = false;  // copied by plain loads at issue time (unaligned source, partial lanes)
    if (cx >= 0 && cx + 4 <= iw) kind = kColPacked, sync_load = !svec;
    else if (cx >= iw + 4) kind = kColNone;  // feeds no stored output
    else if (svec && cx == -4 && iw >= 8) kind = kColLeft;
    else if (svec && cx == iw && iw >= 8 && (iw & 3) == 0) kind = kColRight;
    else kind = kColPacked, sync_load = true;
    const bool mask_async = mvec && cx >= 0 && cx + 4 <= iw;
    // ring layout: raw [kDwtRing][2 rows][2 chunks][32 lanes][CH], masks [kDwtRing][2 rows][32 lanes] words
    unsigned char *const rraw = ring + lane * CH;
    uint32_t *const rmask = reinterpret_cast<uint32_t *>(ring + kDwtRing * 4 * 32 * CH) + lane;

    const int n0 = r0 - A, n1 = r1 - 1 + A;  // pair steps n0..n1
    // Queues the copies of pair n (rows 2n, 2n+1) into its ring slot.
    int islot = 0, cslot = 0;  // ring slots of the next pair to issue and to consume
    // common case: this lane's columns inside the image, aligned sources:
    // column pointers and shared-space addresses kept, four copies a pair
    const bool fast = kind == kColPacked && !sync_load && mask_async;
    const unsigned char *const scol = src + (size_t)cx * E;
    const uint8_t *const mcol = msrc + cx;
    const uint32_t rraw_s = smem_u32(rraw), rmask_s = smem_u32(rmask);
    auto issue = [&](int n) {
        const int slot = islot;
        islot = islot == kDwtRing - 1 ? 0 : islot + 1;
        if (fast && n >= 0 && 2 * n + 1 < ih) {
            const unsigned char *r0 = scol + (size_t)(2 * n) * spitch;
            const uint8_t *m0 = mcol + (size_t)(2 * n) * mpitch;
            const uint32_t d = rraw_s + (uint32_t)(slot * 2 * 2 * 32 * CH), dm = rmask_s + (uint32_t)(slot * 2 * 32 * 4);
            cp_async_s<CH>(d, r0);
            cp_async_s<CH>(d + 2 * 32 * CH, r0 + spitch);
            cp_async_s<4>(dm, m0);
            cp_async_s<4>(dm + 32 * 4, m0 + mpitch);
            cp_async_commit();
            return;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int y = 2 * n + h;
            const unsigned char *rowp = src + (size_t)mirror(y, ih) * spitch;
            unsigned char *d0 = rraw + (slot * 2 + h) * 2 * 32 * CH, *d1 = d0 + 32 * CH;
            if (kind == kColPacked) {
                if (!sync_load) cp_async<CH>(d0, rowp + (size_t)cx * E);
                else sts_chunk<SRC>(d0, load_row<SRC>(rowp, cx, iw, false));
            } else if (kind == kColLeft) {
                cp_async<CH>(d0, rowp);
                cp_async<CH>(d1, rowp + 4 * E);
            } else if (kind == kColRight) {
                cp_async<CH>(d0, rowp + (size_t)(iw - 8) * E);
                cp_async<CH>(d1, rowp + (size_t)(iw - 4) * E);
            }
            uint32_t *md = rmask + (slot * 2 + h) * 32;
            if (mask_async && y >= 0 && y < ih) cp_async<4>(md, msrc + (size_t)y * mpitch + cx);
            else *md = load_mask(msrc, mpitch, y, ih, cx, iw, false);
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int k = 0; k < kDwtRing - 1; k++) {
        if (n0 + k <= n1) issue(n0 + k);
        else cp_async_commit();
    }
#pragma unroll 1
    for (int n = n0; n <= n1; n++) {
        if (n + kDwtRing - 1 <= n1) issue(n + kDwtRing - 1);
        else cp_async_commit();
        cp_async_wait<kDwtRing - 1>();  // pair n has landed
        const int slot = cslot;
        cslot = cslot == kDwtRing - 1 ? 0 : cslot + 1;
        uint4 ra, rb;
        {
            const unsigned char *q = rraw + slot * 2 * 2 * 32 * CH;
            if (kind == kColPacked) {
                ra = lds_chunk<SRC>(q);
                rb = lds_chunk<SRC>(q + 2 * 32 * CH);
            } else if (kind == kColNone) {
                ra = rb = make_uint4(0u, 0u, 0u, 0u);
            } else {
                ra = mirror_chunks<SRC>(lds_chunk<SRC>(q), lds_chunk<SRC>(q + 32 * CH), kind == kColLeft);
                rb = mirror_chunks<SRC>(lds_chunk<SRC>(q + 2 * 32 * CH), lds_chunk<SRC>(q + 3 * 32 * CH), kind == kColLeft);
            }
        }
        const uint32_t ma = rmask[slot * 2 * 32], mb = rmask[(slot * 2 + 1) * 32];
        V e[4], o[4], lo[4], hi[4];
        to_vals<WAV, SRC>(ra, dc, dcf, e);
        to_vals<WAV, SRC>(rb, dc, dcf, o);
        uint32_t lowm, highm;
        const uint32_t pn = ma | mb;
        if constexpr (WAV == 97) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                // each lifting step's sum with its earlier operand is formed
                // one step ahead, so four values per column carry over
                const float O1 = s1[c] + kA * e[c];   // odd 2n-1, step 1
                const float E2 = s2[c] + kB * O1;     // even 2n-2, step 2
                const float O3 = s3[c] + kG * E2;     // odd 2n-3, step 3 (final)
                const float E4 = xe[c] + kD * O3;     // even 2n-4, step 4 (final)
                lo[c] = E4;  // normalised per band after the rows are lifted
                hi[c] = O3;
                s1[c] = o[c] + kA * e[c];             // odd 2n+1 with its left even sample
                s2[c] = e[c] + kB * O1;               // even 2n with its upper odd sample
                s3[c] = O1 + kG * E2;                 // odd 2n-1 with its upper even sample
                xe[c] = E2 + kD * O3;                 // even 2n-2 with its upper odd sample
            }
            // band row n-2: low from rows [2n-7, 2n-1], high from [2n-7, 2n+1]
            lowm = od4 | p3 | p2 | p1;
            highm = lowm | pn;
            od4 = od3, od3 = od2, od2 = od1, od1 = mb;
            p3 = p2, p2 = p1, p1 = pn;
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int H = xo[c] - ((xe[c] + e[c]) >> 1);      // odd 2n-1
                const int L = xe[c] + ((s1[c] + H + 2) >> 2);     // even 2n-2
                lo[c] = L;
                hi[c] = H;
                xe[c] = e[c];
                xo[c] = o[c];
                s1[c] = H;
            }
            // band row n-1: low from rows [2n-3, 2n-1], high from [2n-3, 2n+1]
            lowm = od2 | p1;
            highm = lowm | pn;
            od2 = od1, od1 = mb;
            p1 = pn;
        }
        const int m = n - A;  // band row completed by this step
        if (m >= r0) {
            hlift(lo[0], lo[1], lo[2], lo[3]);
            hlift(hi[0], hi[1], hi[2], hi[3]);
            if constexpr (WAV == 97) {
                lo[0] *= kInvK2;  // LL
                lo[2] *= kInvK2;
                hi[1] *= kK2;     // HH
                hi[3] *= kK2;
            }
            const uint32_t nl = nibble(lowm), nh = nibble(highm);
            const uint32_t pk = nl | (nh << 16);
            const uint32_t pl = __shfl_up_sync(kFull, pk, 1), pr = __shfl_down_sync(kFull, pk, 1);
            const uint32_t wl = (pl & 0xfu) | (nl << 4) | ((pr & 0xfu) << 8);
            const uint32_t wh = ((pl >> 16) & 0xfu) | (nh << 4) | (((pr >> 16) & 0xfu) << 8);
            if (outl) {
                int32_t *const cl = coeffs + (size_t)m * W;  // band row m of the vertical-low half
                int32_t *const ch = cl + hoff;               // ... and of the vertical-high half
                // vertical-low row: LL (even) and HL (odd)
                st2<int32_t>(cl + ohl, qroi(lo[1], d_hl, r_hl, wl & kO0, sh), qroi(lo[3], d_hl, r_hl, wl & kO1, sh), ovec,
                             both);
                if (last) {
                    st2<int32_t>(cl + bc, qroi(lo[0], d_ll, r_ll, wl & kE0, sh), qroi(lo[2], d_ll, r_ll, wl & kE1, sh), ovec,
                                 both);
                } else {
                    const size_t lo_at = (size_t)m * bw + bc;
                    st2<V>(llo + lo_at, lo[0], lo[2], ovec, both);
                    const uint8_t m0 = (wl & kE0) ? 1 : 0, m1 = (wl & kE1) ? 1 : 0;
                    if (ovec) {
                        *reinterpret_cast<uint16_t *>(llmo + lo_at) = (uint16_t)(m0 | (m1 << 8));
                    } else {
                        llmo[lo_at] = m0;
                        if (both) llmo[lo_at + 1] = m1;
                    }
                }
                // vertical-high row: LH (even) and HH (odd)
                st2<int32_t>(ch + bc, qroi(hi[0], d_lh, r_lh, wh & kE0, sh), qroi(hi[2], d_lh, r_lh, wh & kE1, sh), ovec,
                             both);
                st2<int32_t>(ch + ohl, qroi(hi[1], d_hh, r_hh, wh & kO0, sh), qroi(hi[3], d_hh, r_hh, wh & kO1, sh), ovec,
                             both);
                if constexpr (WAV == 97) {
                    if (yf) {
                        float *const fl = yf + (size_t)m * W, *const fh = fl + hoff;
                        st2<float>(fl + ohl, lo[1], lo[3], ovec, both);
                        if (last) st2<float>(fl + bc, lo[0], lo[2], ovec, both);
                        st2<float>(fh + bc, hi[0], hi[2], ovec, both);
                        st2<float>(fh + ohl, hi[1], hi[3], ovec, both);
                    }
                }
            }
        }
    }
}

}  // namespace

// Shared-memory ring of one warp: level 1 sized for 16-bit samples, higher
// levels for 32-bit low-low values.
__host__ __device__ constexpr int dwt_ring_bytes(bool l1) { return kDwtRing * 2 * (2 * 32 * (l1 ? 8 : 16) + 32 * 4); }

// MB: resident blocks per SM the register budget is sized for (5: no
// spills; 6: more warps, a few spilled values).
template <int WAV, bool L1, int MB>
__global__ void __launch_bounds__(32 * kDwtWarps, MB) k_dwt(const BatchDesc *__restrict__ bd, MethodConsts mc, int level)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    unsigned char *const ring = dsm + (size_t)(threadIdx.x >> 5) * dwt_ring_bytes(L1);
    const int nfr = bd->nframes;
    const int *off = bd->dwt_off[level - 1];
    const int total = __ldg(off + nfr);
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < total; u += gridDim.x * wpb) {
        const int fi = find_frame(off, nfr, u);
        const int lt = u - __ldg(off + fi);
        const FrameDesc &F = bd->f[fi];
        if constexpr (L1) {
            if (F.bpp == 1) dwt_unit<WAV, kSrcU8>(F, mc, level, lt, lane, ring);
            else dwt_unit<WAV, kSrcU16>(F, mc, level, lt, lane, ring);
        } else {
            dwt_unit<WAV, kSrcLL>(F, mc, level, lt, lane, ring);
        }
    }
}

int dwt_default_seg(int bw, int bh)
{
    (void)bw;
    // Short units where a level has few rows: a unit's first steps only
    // fill its lifting pipeline, and a warp walks its rows one pair at a time.
    return bh >= 1024 ? 32 : (bh >= 256 ? 16 : 8);
}

int dwt_units(int bw, int bh, int seg)
{
    if (bw <= 0 || bh <= 0) return 0;
    return ((bw + kDwtStrip - 1) / kDwtStrip) * ((bh + seg - 1) / seg);
}

int dwt_grid(int units, int persistent_blocks)
{
    const int need = (units + kDwtWarps - 1) / kDwtWarps;
    return need < persistent_blocks ? (need > 0 ? need : 1) : persistent_blocks;
}

namespace {
template <int MB>
void launch_dwt_mb(const BatchDesc *bd, const MethodConsts &mc, int level, int grid, cudaStream_t s)
{
    if (mc.wavelet == 97) {
        if (level == 1) k_dwt<97, true, MB><<<grid, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(true), s>>>(bd, mc, level);
        else k_dwt<97, false, MB><<<grid, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(false), s>>>(bd, mc, level);
    } else {
        if (level == 1) k_dwt<53, true, MB><<<grid, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(true), s>>>(bd, mc, level);
        else k_dwt<53, false, MB><<<grid, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(false), s>>>(bd, mc, level);
    }
}
template <int MB>
int occupancy_dwt_mb(int wavelet)
{
    int a = 0, b = 0;
    if (wavelet == 97) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_dwt<97, true, MB>, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(true));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dwt<97, false, MB>, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(false));
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_dwt<53, true, MB>, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(true));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dwt<53, false, MB>, 32 * kDwtWarps, kDwtWarps * dwt_ring_bytes(false));
    }
    return a < b ? a : b;
}
}  // namespace

void launch_dwt(const BatchDesc *bd, const MethodConsts &mc, int level, int grid, int variant, cudaStream_t s)
{
    if (variant == 6) launch_dwt_mb<6>(bd, mc, level, grid, s);
    else launch_dwt_mb<5>(bd, mc, level, grid, s);
}

int occupancy_dwt(int wavelet, int variant)
{
    return variant == 6 ? occupancy_dwt_mb<6>(wavelet) : occupancy_dwt_mb<5>(wavelet);
}

}  // namespace flowroi
