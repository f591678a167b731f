/*
 * flowroi.h: C ABI of the GB300 (sm_103a) FlowRoI hot-path library.
 *
 * FlowRoI ("FlowRoI: A Fast Optical-Flow-Driven Region-of-Interest
 * Extraction Framework for High-Throughput Image Compression in Immune Cell
 * Migration Analysis", arXiv 2511.14419) turns a stream of grey frames into,
 * per frame, a binary region-of-interest mask and the JPEG2000 wavelet
 * coefficients that a scaling-based RoI encoder codes:
 *
 *   §Method / §Optical flow extraction: dense two-frame Farneback optical
 *       flow between the frame and its predecessor (Gaussian pyramid,
 *       polynomial expansion, iterated windowed displacement solve, coarse
 *       to fine);
 *   §Region of Interest extraction: saliency from the flow magnitude and
 *       its spatial gradient (weight 0.7), min-max normalisation, a
 *       quantile cut keeping the top "RoI threshold" fraction, opening and
 *       closing;
 *   §Implementation details + Table 1: JPEG2000 scaling-based RoI coding
 *       of the raw frame under that mask: DC level shift, lifting DWT
 *       (reversible 5/3 or irreversible 9/7), quantisation, and the up-shift
 *       of RoI coefficients by the scaling factor.
 *
 * Optionally (§Implementation details, Table 1 "compression rate") the
 * coefficients are also coded: EBCOT tier-1 with the MQ coder, rate control
 * to a byte budget, and a frame container of this library's own layout
 * (flowroi_encode_codestreams, or config.codestream_bpp in the stream
 * path).  The standard JPEG2000 codestream syntax (tier-2 packets, markers)
 * is not produced.
 *
 * Every step runs in this library's CUDA kernels on one GPU; the host side
 * only validates, copies and schedules.  The library owns its device
 * memory (one allocation per admitted stream, from the CUDA stream-ordered
 * allocator) and its CUDA streams.
 *
 * Conventions
 *   - Every int-returning call returns FLOWROI_OK (0) or a negative status.
 *   - Pointers are plain host or device pointers; whether a data pointer is
 *     on the device is stated by an explicit flag next to it.  Device
 *     pointers must belong to the context's device.
 *   - Images are row-major, x (columns) fastest.  Flow is stored as
 *     interleaved (dx, dy) float pairs.
 *   - Strings returned by flowroi_last_error stay valid until the next call
 *     on the same context from the same thread.
 *   - A context is safe to use from several host threads.
 */
#ifndef FLOWROI_H
#define FLOWROI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLOWROI_ABI_VERSION 6

/* Exported symbols (the library is built with hidden default visibility). */
#if defined(__GNUC__)
#define FLOWROI_API __attribute__((visibility("default")))
#else
#define FLOWROI_API
#endif

/* ---- status codes ---------------------------------------------------- */
#define FLOWROI_OK 0
#define FLOWROI_EINVAL (-1)     /* bad argument, descriptor, size or frame order */
#define FLOWROI_ENOSTREAM (-2)  /* unknown stream, or frame never submitted */
#define FLOWROI_EBUSY (-3)      /* retry later: HBM budget (stream not admitted yet) or
                                   the stream's frame ring is full of unfinished frames */
#define FLOWROI_ENOMEM (-4)     /* device or host allocation failed */
#define FLOWROI_ETIMEDOUT (-5)  /* a bounded wait expired; nothing was copied */
#define FLOWROI_EDEVICE (-6)    /* a CUDA error was seen; the context is poisoned */
#define FLOWROI_EGONE (-7)      /* result overwritten: the stream's result ring wrapped */
#define FLOWROI_ENOTKEPT (-8)   /* intermediate requested without FLOWROI_KEEP_INTERMEDIATES */
#define FLOWROI_ERANGE (-9)     /* output buffer too small, or a value outside the coder's range */

/* ---- enumerations ------------------------------------------------------ */
#define FLOWROI_U8 1            /* 8-bit unsigned samples */
#define FLOWROI_U16 2           /* 16-bit unsigned samples (e.g. 12-bit data) */
#define FLOWROI_W53 53          /* reversible integer 5/3 lifting DWT (no quantisation) */
#define FLOWROI_W97 97          /* irreversible 9/7 lifting DWT, single precision, quantised */
#define FLOWROI_FP32 32         /* pyramid and expansion fields stored in float */
#define FLOWROI_FP16 16         /* ... stored in half, all arithmetic in float */

/* codestream formats (flowroi_config.codestream_format, flowroi_cs_job.format) */
#define FLOWROI_CS_CONTAINER 0  /* the library's frame container (layout below) */
#define FLOWROI_CS_J2C 1        /* JPEG2000 Part 1 codestream (ISO/IEC 15444-1) */

/* flowroi_config.flags */
#define FLOWROI_KEEP_INTERMEDIATES 0x1u /* keep flow, saliency, pre-morphology mask and
                                           (9/7) float coefficients per result slot */
#define FLOWROI_PLAIN 0x2u              /* plain per-frame path: each frame runs alone,
                                           one grid per frame, no CUDA graphs */
#define FLOWROI_MANUAL 0x4u             /* no scheduler thread: the caller launches batches
                                           with flowroi_step (deterministic batch makeup) */
/* Test only: exercise the failure path of the bounded device waits and
 * loops without a fault.  Every batch run under one of these flags sets the
 * error word and poisons the context (FLOWROI_EDEVICE; the device and other
 * contexts stay usable); results of those batches are not valid. */
#define FLOWROI_TEST_EXPIRE_TMA 0x100u  /* the window kernel's producer (block 0,
                                           level 0) never issues its first tile's
                                           copies; TMA waits give up after 2^12 polls */
#define FLOWROI_TEST_EXPIRE_LOOP 0x200u /* union-find loops of the component filter
                                           (config.min_area > 1) give up after 1 step */

/* flowroi_get_intermediate: `which` */
#define FLOWROI_I_FLOW 1        /* float[2*W*H]: level-0 flow (dx, dy) interleaved */
#define FLOWROI_I_SALIENCY 2    /* float[W*H]: normalised saliency S^ in [0, 1] */
#define FLOWROI_I_MASK0 3       /* uint8[W*H]: mask before opening/closing (0/1) */
#define FLOWROI_I_COEFF_F32 4   /* float[W*H]: 9/7 coefficients before quantisation, Mallat */
#define FLOWROI_I_THRESHOLD 5   /* float[1]: the cut t on S^ (mask0 = S^ > t) */
#define FLOWROI_I_DENOISED 6    /* float[W*H]: denoised flow input in 8-bit units (config.denoise = 1) */
#define FLOWROI_I_DRIFT 7       /* float[2]: registration drift (sx, sy), level-0 pixels (config.register_frames = 1) */

/* ---- configuration ----------------------------------------------------- */
/* Method parameters.  Table 1 of the paper names the user parameters (RoI
 * threshold, scaling factor, denoise, adjacent factor, compression rate:
 * codestream_bpp below).  The estimator constants are not
 * given by the paper; the defaults are the values this library documents
 * (pyramid 5 levels, 3 iterations, 15x15 box window, 5x5 expansion with
 * sigma 1.1, lambda 1e-3 in 8-bit units, opening radius 1, closing
 * radius 2). */
typedef struct flowroi_config {
    uint32_t struct_size;      /* = sizeof(flowroi_config) */
    float roi_q;               /* RoI threshold q in (0,1): keep at most floor(q*W*H) pixels (0.2) */
    int32_t scale_shift;       /* scaling factor s in [0, 15]: RoI coefficients times 2^s (5) */
    int32_t wavelet;           /* FLOWROI_W53 or FLOWROI_W97 */
    int32_t dwt_levels;        /* D in [1, 8] */
    int32_t pyr_levels;        /* L in [1, 8] */
    int32_t iters;             /* displacement iterations per pyramid level, [1, 8] (3) */
    int32_t win_r;             /* box window radius r in [2, 10]: side 2r+1 (7) */
    int32_t poly_n_half;       /* expansion radius n in {2, 3}: side 2n+1 (2) */
    float poly_sigma;          /* applicability sigma (1.1) */
    float lambda;              /* solve regulariser (> 0), added to det (1e-3) */
    float sal_weight;          /* alpha: S = alpha*|d| + (1-alpha)*|grad|d|| (0.7) */
    int32_t r_open;            /* opening radius in [0, 4] (1) */
    int32_t r_close;           /* closing radius in [0, 4] (2) */
    int32_t precision;         /* FLOWROI_FP32 or FLOWROI_FP16 */
    float delta_base;          /* 9/7: base quantisation step (1.0) */
    int32_t max_batch_frames;  /* frames per batched launch, [1, 64] (64) */
    int32_t result_ring;       /* frames kept per stream (input and result slots), [2, 16] (4) */
    uint32_t flags;            /* FLOWROI_KEEP_INTERMEDIATES | FLOWROI_PLAIN | FLOWROI_MANUAL */
    int32_t device;            /* CUDA device ordinal (0) */
    uint64_t hbm_budget_bytes; /* admission budget for all streams' device state;
                                  0 = 80% of the device memory free at create */
    /* Table 1 "Denoise" (§Optical flow extraction: median filtering, then
     * bilateral filtering, of the flow input; the JPEG2000 front end still
     * codes the raw frame).  Sizes are not given by the paper. */
    int32_t denoise;           /* 0 = off (a valid setting of the paper), 1 = on (0) */
    int32_t den_radius;        /* bilateral square radius rb in [1, 3]: side 2rb+1 (2) */
    float den_sigma_s;         /* bilateral spatial sigma in pixels, > 0 (2.0) */
    float den_sigma_r;         /* bilateral range sigma in 8-bit units, > 0 (20.0) */
    /* §Region of Interest extraction: residual small connected components
     * removed by area after opening and closing (8-connectivity). */
    int32_t min_area;          /* components with fewer pixels are removed; 0 = off, [0, 2^20] (0) */
    /* Table 1 "Adjacent factor" (§Region of Interest extraction: masks of
     * neighbouring frames incorporated).  The RoI mask of frame j is the
     * union of the per-frame masks of frames j-k .. j+k, so frame j's mask
     * and coefficients are ready once frame j+k has been processed, or
     * after flowroi_flush / flowroi_end_stream, which finish the last k
     * frames of a stream with the frames there are.  Needs
     * result_ring >= 2k + 2. */
    int32_t adjacent;          /* k in [0, 4] (0) */
    /* §Optical flow extraction: each frame registered to its predecessor
     * by phase correlation (global translational drift); the flow is that
     * of the registered pair.  The correlation runs on pyramid level
     * reg_level, whose padded size must be at most 1024 per side. */
    int32_t register_frames;   /* 0 = off, 1 = on (0) */
    int32_t reg_level;         /* in [1, pyr_levels - 1] (2) */
    /* JPEG2000 coder in the stream path (§Implementation details, Table 1:
     * the codestream cut to a target compression rate): when > 0, every
     * frame's coefficient plane is also coded into a rate-controlled
     * container (the format of flowroi_encode_codestreams) of this many
     * bits per pixel of pass data; fetch it with flowroi_get_codestream.
     * 0 = off. (0) */
    float codestream_bpp;
    /* Format of those codestreams: FLOWROI_CS_CONTAINER (the library's
     * frame container) or FLOWROI_CS_J2C (a JPEG2000 Part 1 codestream, see
     * flowroi_encode_codestreams).  (FLOWROI_CS_CONTAINER) */
    int32_t codestream_format;
    /* Tile table (launch and tile shapes per frame width class, see
     * flowroi_autotune): path of a JSON file read at create, or NULL for
     * the built-in shapes.  Not a method parameter: results do not depend
     * on it, only the time they take.  (NULL) */
    const char *tile_table;
    /* Code-block style of those codestreams: 0 = every pass terminated, the
     * MQ coder's context states carried from pass to pass; 1 = also reset
     * the context states at every pass (JPEG2000 Part 1's code-block style
     * option "reset context probabilities on coding pass boundaries", COD
     * style byte 0x06 instead of 0x04, the container's flags word 1).  With
     * reset every pass is coded apart from the others, so no chain of
     * context states runs through a code-block; the passes cost a few more
     * bytes each, while their contexts learn again.  (0) */
    int32_t codestream_reset;
} flowroi_config;

/* One input frame.  Frames of a stream keep their width, height, dtype and
 * bit depth; frame_idx strictly increases.  width and height must be
 * multiples of 2^max(dwt_levels, pyr_levels - 1) and at least 16. */
typedef struct flowroi_frame {
    uint32_t struct_size;      /* = sizeof(flowroi_frame) */
    int32_t width, height;
    int32_t pitch_bytes;       /* row pitch of `data`; 0 = width * sample size */
    int32_t dtype;             /* FLOWROI_U8 or FLOWROI_U16 */
    int32_t bit_depth;         /* significant bits B: 1..8 (U8) or 1..16 (U16) */
    int64_t frame_idx;
    const void *data;          /* samples; host or device (see data_on_device) */
    int32_t data_on_device;    /* 1: `data` is a device pointer */
} flowroi_frame;

typedef struct flowroi_stats {
    uint32_t struct_size;      /* = sizeof(flowroi_stats) */
    int64_t frames_submitted, frames_done, batches;
    int64_t streams_admitted;  /* streams currently holding device state */
    int64_t admissions_refused;
    uint64_t bytes_admitted, budget_bytes;
    double lat_p50_ms, lat_p99_ms, lat_mean_ms; /* submit -> result ready, frames done so far */
    int64_t kernel_launches;   /* this library's kernels launched so far (graph nodes counted) */
} flowroi_stats;

/* Opaque context: one GPU, its streams, its scheduler. */
typedef struct flowroi_ctx flowroi_ctx;

/* Fill *cfg with the documented defaults (5/3, D = 3, L = 3, FP32,
 * scheduler thread on). */
FLOWROI_API void flowroi_default_config(flowroi_config *cfg);

/* Create a context on cfg->device.  Every field is validated
 * (FLOWROI_EINVAL; flowroi_last_error(NULL) names the field).  Starts the
 * scheduler thread unless FLOWROI_MANUAL.  *out receives the context,
 * owned by the caller until flowroi_destroy.  No device memory is held
 * until the first stream is admitted. */
FLOWROI_API int flowroi_create(const flowroi_config *cfg, flowroi_ctx **out);

/* Submit frame `f` of stream `stream_id` (§Method: the image sequence of
 * one well/lens).  A new stream_id creates a stream on its first frame and
 * is admitted only if its device state fits the HBM budget; otherwise
 * FLOWROI_EBUSY (nothing kept; retry after other streams end).  The frame
 * is copied before the call returns (host data: host-to-device copy
 * completed; device data: device-to-device copy ordered before its use), so
 * the caller keeps ownership of f->data.  FLOWROI_EBUSY too when the
 * stream already has result_ring frames not yet processed.  The first frame
 * of a stream has no predecessor: its mask is empty and its coefficients
 * are the plain (unshifted) JPEG2000 front end. */
FLOWROI_API int flowroi_submit_frame(flowroi_ctx *ctx, int64_t stream_id, const flowroi_frame *f);

/* Submit n frames, frames[k] to stream stream_ids[k], in order, with the
 * rules of flowroi_submit_frame for each; the copies are queued back to
 * back and waited for once (one wait per batch of wells instead of one per
 * frame).  Returns the number of frames accepted, k <= n: frames [0, k)
 * are submitted and their buffers may be reused; when k < n, frames[k] was
 * refused with *status (if status is not NULL: FLOWROI_EBUSY,
 * FLOWROI_EINVAL, ...) and flowroi_last_error says why, and frames after
 * it were not looked at.  Negative on a NULL ctx, n < 0 or a NULL array
 * (FLOWROI_EINVAL), with nothing submitted.  *status is FLOWROI_OK when
 * all n were accepted. */
FLOWROI_API int flowroi_submit_frames(flowroi_ctx *ctx, int n, const int64_t *stream_ids, const flowroi_frame *frames,
                                      int *status);

/* Launch one batch now: for every stream with a pending frame, its oldest
 * one, at most max_batch_frames frames (FLOWROI_PLAIN: one frame per
 * launch sequence, still all pending streams).  Returns the number of
 * frames launched (>= 0) or a negative status.  Needed only with
 * FLOWROI_MANUAL; harmless otherwise. */
FLOWROI_API int flowroi_step(flowroi_ctx *ctx);

/* Copy out the RoI mask of (stream_id, frame_idx): W*H bytes, 0 or 1,
 * row-major, into caller-owned `out` (device memory if out_on_device).
 * Waits at most timeout_ms (< 0: no limit) for the frame to finish, then
 * copies; FLOWROI_ETIMEDOUT if it did not finish in time (nothing copied).
 * FLOWROI_EGONE if the stream's result ring has since been overwritten. */
FLOWROI_API int flowroi_get_mask(flowroi_ctx *ctx, int64_t stream_id, int64_t frame_idx, uint8_t *out,
                     int out_on_device, int timeout_ms);

/* Copy out the wavelet coefficients of (stream_id, frame_idx): W*H int32,
 * Mallat layout (per level the low-low band top-left, HL right of it, LH
 * below, HH diagonal), after quantisation (9/7) and the RoI up-shift
 * q <- sign(q) * (|q| << s) of every coefficient whose synthesis support
 * meets the mask (§Implementation details, scaling-based RoI).  Same
 * waiting, ownership and errors as flowroi_get_mask. */
FLOWROI_API int flowroi_get_coeffs(flowroi_ctx *ctx, int64_t stream_id, int64_t frame_idx, int32_t *out,
                       int out_on_device, int timeout_ms);

/* The masks and coefficients of n frames in one call (one step's
 * results of a batch of wells): frame frame_idx[k] of stream
 * stream_ids[k] into masks[k] (W*H bytes, as flowroi_get_mask) and
 * coeffs[k] (W*H int32, as flowroi_get_coeffs); masks or coeffs, or an
 * element of either, may be NULL to skip that output.  Each frame is
 * waited for like flowroi_get_mask (at most timeout_ms each, < 0: no
 * limit); then every copy is queued back to back on the library's
 * copy-out stream and waited for once (one wait per batch instead of two
 * per frame).  status[k] (if status is not NULL) receives frame k's result
 * (FLOWROI_OK, FLOWROI_ETIMEDOUT, FLOWROI_EGONE, FLOWROI_ENOSTREAM, ...);
 * a failed frame's outputs are not written, and the other frames are still
 * copied.  Returns FLOWROI_OK when every frame's outputs were written, else
 * the first failing frame's code; FLOWROI_EINVAL for a NULL ctx, n < 0 or
 * NULL stream_ids / frame_idx, with nothing copied. */
FLOWROI_API int flowroi_get_results(flowroi_ctx *ctx, int n, const int64_t *stream_ids, const int64_t *frame_idx,
                                    uint8_t *const *masks, int32_t *const *coeffs, int out_on_device, int timeout_ms,
                                    int *status);

/* Copy out an intermediate of (stream_id, frame_idx) (`which`: one of
 * FLOWROI_I_*, sizes as listed there) for inspection and tests.  Needs
 * FLOWROI_KEEP_INTERMEDIATES (else FLOWROI_ENOTKEPT).  A first frame has
 * no flow: its flow and saliency are zero and its threshold is +inf. */
FLOWROI_API int flowroi_get_intermediate(flowroi_ctx *ctx, int64_t stream_id, int64_t frame_idx, int which,
                             void *out, int out_on_device, int timeout_ms);

/* Launch everything pending and wait (at most timeout_ms, < 0: no limit)
 * until every submitted frame has finished.  With an adjacent factor k > 0
 * this also finishes the last k frames of every stream, merging only the
 * neighbours submitted so far. */
FLOWROI_API int flowroi_flush(flowroi_ctx *ctx, int timeout_ms);

/* End a stream: waits for its frames in flight, then frees its device
 * state and returns its bytes to the admission budget.  Later frames with
 * the same id start a new stream. */
FLOWROI_API int flowroi_end_stream(flowroi_ctx *ctx, int64_t stream_id);

/* Counters and latency percentiles since create. */
FLOWROI_API int flowroi_get_stats(flowroi_ctx *ctx, flowroi_stats *out);

/* Forget the latency samples collected so far (counters keep counting),
 * so that flowroi_get_stats reports percentiles of a measurement window. */
FLOWROI_API int flowroi_reset_stats(flowroi_ctx *ctx);

/* Stop the scheduler, wait for the device, free everything.  NULL is a
 * no-op. */
FLOWROI_API void flowroi_destroy(flowroi_ctx *ctx);

/* Human-readable reason for the last failing call of this thread on ctx
 * (ctx may be NULL for flowroi_create failures). */
FLOWROI_API const char *flowroi_last_error(flowroi_ctx *ctx);

/* The 9/7 quantisation steps (§Implementation details: quantisation of the
 * irreversible path; the paper gives no step sizes).  For subband b the step
 * is delta_base / sqrt(G_b), G_b the squared norm of b's 2-D synthesis basis
 * function, written in the JPEG2000 form 2^(R_b - eps) * (1 + mu / 2^11)
 * with R_b = bit_depth + gain_b (gain 0 LL, 1 HL/LH, 2 HH).  Output arrays
 * (caller-owned host memory, length 3*levels + 1) are indexed
 * 3*(level-1) + orientation (0 HL, 1 LH, 2 HH) and 3*levels for the final
 * low-low band; any of them may be NULL.  Host-only, no device use. */
FLOWROI_API int flowroi_quant_steps(int levels, int bit_depth, float delta_base, float *delta, int32_t *eps,
                        int32_t *mu, double *gain_norm);

/* The CUDA stream (cudaStream_t, as void*) on which every batch of ctx
 * runs, for callers that time or order work against it (e.g. record CUDA
 * events around steps).  Owned by the context; do not destroy. */
FLOWROI_API int flowroi_compute_stream(flowroi_ctx *ctx, void **out);

/* Per-kernel timing (tracing).  With profiling on, batches launch their
 * kernels directly (no graph replay) with a CUDA event pair around every
 * launch on the compute stream.  flowroi_get_kernel_times waits for the
 * device, folds the recorded pairs into per-(kernel, level) totals and
 * copies at most `cap` rows into caller-owned `out`; returns the number of
 * rows (or a negative status).  Turning profiling off keeps the totals;
 * flowroi_set_profiling(ctx, 2) clears them and turns profiling on. */
typedef struct flowroi_kernel_time {
    char name[24];       /* "frame_init", "expand", "update", "window", "saliency", "select_find",
                            "select_pass" (digit 2 over the plane, digit 3 over its candidates),
                            "morph", "dwt", "denoise", "components", "merge", "register",
                            "codestream" (the coder's three kernels) */
    int32_t level;       /* pyramid level (expand, update, window), DWT level (dwt), digit pass
                            (select_*), step (components, register), or -1 */
    int32_t iter;        /* displacement iteration (update, window), else -1 */
    int64_t launches;
    double total_ms;
} flowroi_kernel_time;
FLOWROI_API int flowroi_set_profiling(flowroi_ctx *ctx, int on);
FLOWROI_API int flowroi_get_kernel_times(flowroi_ctx *ctx, flowroi_kernel_time *out, int cap);

/* JPEG2000 front end of one frame that allocates nothing.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (code running inside a fixed, pre-reserved
 * device budget, plug-ins whose host application owns the device heap,
 * real-time loops that must not call cudaMalloc, whose latency is unbounded
 * and which can synchronise the device).  It runs the same DWT kernel as the
 * streaming path - DC shift, `levels` levels of lifting DWT, quantisation
 * (9/7), the wavelet-domain RoI mask of `mask` and the up-shift of RoI
 * coefficients by `scale_shift` bits - on buffers the caller owns, and
 * calls no cudaMalloc, cudaFree or allocating routine.  The memory it needs
 * besides the caller's buffers (a one-frame descriptor and the low-low
 * planes between levels) is one fixed array in the library, about 2.6 MB,
 * that every GPU which loads the library holds until the process exits.
 *
 *   raw          device pointer: width x height samples, rows pitch_bytes
 *                apart (0 = tight); dtype FLOWROI_U8 or FLOWROI_U16 (then
 *                raw and pitch 4-byte aligned), bit_depth significant bits
 *   mask         device pointer: width x height bytes, 0/1, tight rows,
 *                2-byte aligned (e.g. from flowroi_get_mask with
 *                out_on_device = 1)
 *   delta        host array of 3*levels + 1 quantisation steps for 9/7 (from
 *                flowroi_quant_steps); may be NULL for 5/3
 *   coeffs       device pointer: width x height int32, Mallat layout (the
 *                layout of flowroi_get_coeffs), 4-byte aligned
 *   cuda_stream  cudaStream_t (as void*) the work is queued on; NULL = the
 *                legacy default stream.  The call returns once the work is
 *                queued.
 *
 * Limits: width * height <= 2^20 pixels (the fixed array holds the low-low
 * planes of frames that large), width and height >= 16 and multiples of
 * 2^levels, levels in [1, 8].  Larger or malformed requests return
 * FLOWROI_EINVAL and queue nothing.  A failed launch returns FLOWROI_EDEVICE:
 * the launches before it (the descriptor and the DWT levels below the
 * failing one) may already be queued, so coeffs is then undefined.  An
 * error left pending by an earlier, unrelated CUDA call on the calling
 * thread is cleared first and not reported here.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU (queued on different streams without ordering between them) race
 * and give undefined coefficients; order them on one stream or with events.
 * Host threads are serialised by an internal lock. */
FLOWROI_API int flowroi_dwt_roi_noalloc(const void *raw, int width, int height, int pitch_bytes, int dtype,
                                        int bit_depth, const uint8_t *mask, int wavelet, int levels,
                                        int scale_shift, const float *delta, int32_t *coeffs, void *cuda_stream);

/* Embedded block coding of coefficient planes into frame containers.
 *
 * Paper: §Implementation details and Table 1 - the RoI-shifted JPEG2000
 * coefficients are coded by a JPEG2000 coder and the codestream is cut to
 * the target compression rate.  This is that coder's block coder and rate
 * control, from the JPEG2000 Part 1 definitions: 64 x 64 code-blocks from
 * each sub-band's origin; bit-plane coding passes (significance
 * propagation, magnitude refinement, cleanup with run-length mode) with the
 * MQ arithmetic coder, every pass terminated (its own byte segment);
 * per-pass distortion decreases of the midpoint reconstruction on the
 * quantised, RoI-shifted coefficients; rate control by the lower convex
 * hull of each code-block's truncation points and a slope threshold found
 * by bisection so that the kept pass bytes fit budget_bytes.
 *
 * Container (little-endian): a 32-byte header {"FRJ2", u32 version 1, u32
 * width, u32 height, u8 wavelet, u8 levels, u8 shift, u8 bit_depth, u32
 * code-blocks, u32 data bytes, u32 flags (bit 0: the contexts were reset at
 * every pass)}; per code-block a 16-byte entry {u32
 * data offset, u16 x0, u16 y0 (in the plane), u8 width-1, u8 height-1, u8
 * band (HL, LH, HH of level l at 3(l-1), +1, +2; low-low at 3 levels), u8
 * bit-planes, u8 passes coded, u8 passes kept, u16 0}, in codestream order
 * (low-low band, then HL, LH, HH of each level from the coarsest, raster
 * order within a band); then the data: per code-block the kept passes'
 * u16 lengths and their bytes.
 *
 * JPEG2000 Part 1 codestream (format FLOWROI_CS_J2C; ISO/IEC 15444-1, the
 * same kept passes): SOC; SIZ (one tile of the whole frame, one unsigned
 * component of bit_depth bits); COD (LRCP, one quality layer, no
 * multi-component transform, `levels` decomposition levels, 64 x 64
 * code-blocks, code-block style "termination on each coding pass" (and
 * "reset context probabilities on coding pass boundaries" with reset),
 * transform 5/3 reversible or 9/7 irreversible, no precinct partition);
 * QCD (5/3: no quantisation, exponent bit_depth + the band's log2 gain;
 * 9/7: scalar expounded, each band's (exponent, mantissa) of the steps
 * flowroi_quant_steps gives for the context's delta_base; guard bits the
 * fewest, 1 to 7, that make every code-block's bit-planes fit); one
 * tile-part (SOT, SOD) of one packet per resolution level (packet headers
 * with inclusion and zero-bit-plane tag trees, pass counts, Lblock and one
 * length per pass); EOC.  No RGN marker: Part 1 signals only the
 * maximum-shift RoI method, so the RoI coefficients' up-shift by `shift`
 * bits stays in the data; a Part 1 decoder returns the shifted
 * coefficients, and undoing the shift needs the RoI mask.  A frame whose
 * bit-planes would need more than 7 guard bits gets FLOWROI_ERANGE.
 *
 * One job per frame:
 *   coeffs        width x height int32 Mallat plane (the layout of
 *                 flowroi_get_coeffs), magnitudes below 2^24
 *   width, height multiples of 2^levels, at most 65535
 *   levels        DWT levels of the plane, [1, 8]
 *   wavelet, shift, bit_depth   recorded in the header (53 or 97, [0, 15],
 *                 [1, 16])
 *   budget_bytes  pass-data budget; <= 0 keeps every pass
 *   out, out_cap  destination of the codestream and its capacity
 *   format        FLOWROI_CS_CONTAINER or FLOWROI_CS_J2C
 *   out_len       set to the container's length (or, when it does not fit,
 *                 to the length it needs, with FLOWROI_ERANGE)
 * on_device: coeffs and out are device pointers of the context's device
 * (else host pointers; the library copies).  Runs synchronously on a
 * stream of its own (device inputs must be complete when the call is made:
 * it does not wait on the caller's streams), with scratch memory that the
 * context keeps between calls (about 34 KB per code-block of the largest
 * call so far); n in [1, 64].  Returns FLOWROI_OK, FLOWROI_EINVAL
 * (malformed job), FLOWROI_ENOMEM, FLOWROI_ERANGE (a container did not fit
 * or a code-block exceeded the coder's limits) or FLOWROI_EDEVICE. */
typedef struct {
    const int32_t *coeffs;
    int32_t width, height;
    int32_t levels, wavelet, shift, bit_depth;
    int64_t budget_bytes;
    uint8_t *out;
    uint64_t out_cap;
    uint64_t out_len;
    int32_t format;      /* FLOWROI_CS_CONTAINER or FLOWROI_CS_J2C */
    int32_t reset;       /* 0 or 1: the code-block style of config.codestream_reset */
} flowroi_cs_job;
FLOWROI_API int flowroi_encode_codestreams(flowroi_ctx *ctx, int n, flowroi_cs_job *jobs, int on_device);
/* The container of a frame coded in the stream path (config.codestream_bpp
 * > 0): waits like flowroi_get_coeffs, then copies the container (host or
 * device out, capacity out_cap) and sets *out_len to its length.  A
 * container that does not fit out_cap, or a frame whose coefficients the
 * coder cannot take (a magnitude of 2^24 or more), returns FLOWROI_ERANGE
 * (with *out_len the length it needs, or 0); FLOWROI_EINVAL when the
 * coder is off. */
FLOWROI_API int flowroi_get_codestream(flowroi_ctx *ctx, int64_t stream_id, int64_t frame_idx, uint8_t *out,
                                       uint64_t out_cap, uint64_t *out_len, int out_on_device, int timeout_ms);
/* A container capacity that always suffices for a width x height plane of
 * `levels` levels (0 for a malformed geometry). */
FLOWROI_API uint64_t flowroi_codestream_bound(int width, int height, int levels);

/* ---- tile shapes -------------------------------------------------------
 * The paper has no counterpart: these calls choose how the kernels cut
 * their work, not what they compute (every choice gives bit-identical
 * results).  A tile table is JSON text:
 *   {"format": "flowroi-tiles-1", "device": "...", "entries": [ENTRY, ...]}
 * with ENTRY one of (storage 32 or 16; w the width class 256, 512, 1024,
 * 2048, 4096 or 8192 that holds the frames of level-0 width <= w and
 * > w/2, the last one every wider frame):
 *   {"param": "dwt_seg", "w": W, "storage": S, "level": l, "value": v}
 *        DWT band rows per warp unit at level l, v in [4, 256]
 *   {"param": "update_rows", "storage": S, "value": v}
 *        rows of a displacement-update tile (4, 8, 16 or 32), which
 *        a block takes 4 at a time
 *   {"param": "saliency_rows", "w": W, "storage": S, "value": v}
 *        rows of a saliency tile, a multiple of 8 up to 128
 *   {"param": "blocks_per_sm", "kernel": K, "storage": S, "value": v}
 *        persistent grid of K (expand, update, window, mask, dwt): min(v,
 *        occupancy) blocks per SM, v in [1, 32]
 *   {"param": "dwt_variant", "storage": S, "value": v}
 *        register budget of the DWT kernel: 5 or 6 resident blocks per SM
 * (entries may also carry "ms", ignored).  Shapes without an entry keep
 * the built-in choice.  Per-width entries apply to each frame of a batch
 * by its own width; the others to the context.
 *
 * flowroi_tiles_check: validates a table (no device needed); FLOWROI_OK or
 * FLOWROI_EINVAL with a message in err (caller-owned, err_cap bytes).
 * flowroi_set_tiles: replaces ctx's table (NULL = built-in shapes); waits
 * for the context's queued work, and its captured graphs are rebuilt at
 * the next batch.  FLOWROI_EINVAL on a malformed table (ctx unchanged).
 * flowroi_get_tiles: ctx's table as JSON into out (cap bytes, NUL
 * included); *out_len = its length; FLOWROI_ERANGE when it does not fit.
 * flowroi_autotune: times candidate shapes on synthetic 12-bit frames of
 * each of the nsizes sizes (`streams` streams per batch, `steps` batches
 * per candidate) with cfg's method settings on cfg's device, by coordinate
 * descent on the summed device time of the kernels each shape affects,
 * and writes the chosen table (JSON) into out; *out_len = its length
 * (FLOWROI_ERANGE when out_cap is too small).  Takes seconds to minutes
 * and the device memory of `streams` streams of the largest size. */
FLOWROI_API int flowroi_tiles_check(const char *json, char *err, uint64_t err_cap);
FLOWROI_API int flowroi_set_tiles(flowroi_ctx *ctx, const char *json);
FLOWROI_API int flowroi_get_tiles(flowroi_ctx *ctx, char *out, uint64_t cap, uint64_t *out_len);
FLOWROI_API int flowroi_autotune(const flowroi_config *cfg, int nsizes, const int *widths, const int *heights,
                                 int streams, int steps, char *out, uint64_t out_cap, uint64_t *out_len);

/* Stream -> device routing for several devices, one context each (streams
 * are independent: a stream's state is its own previous frame, so the path
 * shards by stream with no exchange between devices).  Returns the device
 * index in [0, n_devices) of stream_id: Lamping and Veach's jump consistent
 * hash ("A Fast, Minimal Memory, Consistent Hash Algorithm", 2014) of the
 * id after the splitmix64 finaliser.  The same id always maps to the same
 * device; going from n to n + 1 devices moves a stream only to the new
 * device, and about 1/(n + 1) of them.  Host only, no device call, thread
 * safe.  n_devices == 0: returns UINT32_MAX. */
FLOWROI_API uint32_t flowroi_route(int64_t stream_id, uint32_t n_devices);

/* Library ABI version (FLOWROI_ABI_VERSION). */
FLOWROI_API int flowroi_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
