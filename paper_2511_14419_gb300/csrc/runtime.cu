// FlowRoI runtime and C ABI (see include/flowroi.h for the contract).
//
// One context = one GPU.  Every stream (one microscope well / lens, the
// paper's "image sequence") owns one device block, allocated on admission
// from the stream-ordered allocator and sized from its frame geometry:
//   - a ring of R input frames and R result slots (mask, coefficients,
//     optional intermediates);
//   - two sets of polynomial-expansion fields (this frame's and the
//     previous frame's, alternating by frame parity): the previous
//     frame's expansion stays resident, so each frame expands only itself;
//   - the per-frame temporaries of one frame in flight (pyramid, flow
//     ping-pong, saliency, reduction block, DWT low-low planes).
// Streams are admitted while the sum of their blocks fits the HBM budget.
//
// Batches: a scheduler thread (or flowroi_step in manual mode) takes, for
// every stream, its oldest pending frame, fills a batch descriptor (frames,
// per-kernel tile prefixes) in pinned memory, copies it to the device and
// replays a CUDA graph of the whole hot path whose kernels read the
// descriptor.  Every kernel loops over (frame, tile) work with a fixed
// persistent grid, so one captured graph serves any batch makeup: streams
// of different resolutions are continuously batched without recapture.
// At most two batches are in flight; a host function after each batch
// stamps completion times.  The plain path (FLOWROI_PLAIN) runs each frame
// alone with exact grids and direct launches, for comparison.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>
#include <nvtx3/nvToolsExtCudaRt.h>

#include "../../include/flowroi.h"
#include "common.cuh"
#include "kernels.h"
#include "tiles.h"
#include "tma.cuh"

using namespace flowroi;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
// stderr logging, on when the environment variable FLOWROI_LOG is set (to
// anything but "0"): refusals and errors, admissions, context life.
bool log_on()
{
    static const bool on = [] {
        const char *v = std::getenv("FLOWROI_LOG");
        return v && *v && std::strcmp(v, "0") != 0;
    }();
    return on;
}

void logf(const char *fmt, ...) __attribute__((format(printf, 1, 2)));
void logf(const char *fmt, ...)
{
    if (!log_on()) return;
    va_list ap;
    va_start(ap, fmt);
    std::fputs("[flowroi] ", stderr);
    std::vfprintf(stderr, fmt, ap);
    std::fputc('\n', stderr);
    va_end(ap);
}

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    logf("status %d: %s", code, buf);
    return code;
}

// NVTX range for the duration of a scope (no cost without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

enum EntryState { E_EMPTY = 0, E_PENDING = 2, E_LAUNCHED = 3, E_DONE = 4 };

struct Entry {
    int64_t frame_idx = -1;
    int64_t seq = -1;
    std::atomic<int> state{E_EMPTY};
    bool has_prev = false;
    double t_submit = 0.0, t_done = 0.0;
    int readers = 0;
    cudaEvent_t uploaded = nullptr;
    void *raw = nullptr;
    uint8_t *mask = nullptr;       // the delivered RoI mask (merged with neighbours' when adjacent > 0)
    uint8_t *mask_own = nullptr;   // adjacent > 0: this frame's own mask (after morphology / components)
    int32_t *coeffs = nullptr;
    float2 *dbg_flow = nullptr;
    float *dbg_shat = nullptr;
    uint8_t *dbg_mask0 = nullptr;
    float *dbg_yf = nullptr;
    float *dbg_thr = nullptr;
    float *dbg_den = nullptr;
    float *dbg_drift = nullptr;
    uint8_t *cs = nullptr;          // the coder's container (codestream_bpp > 0)
    long long *cs_len = nullptr;    // its length (device)
};

struct Stream {
    CUtensorMap gh_map[kMaxLevels];
    int64_t id = 0;
    int W = 0, H = 0, bpp = 0, bit_depth = 0;
    size_t bytes = 0;
    char *block = nullptr;
    int64_t next_seq = 0;
    int64_t last_frame_idx = 0;
    bool any_frame = false;
    int64_t launched_seq = -1;     // last frame whose flow was launched
    int64_t dwt_seq = 0;           // next frame whose JPEG2000 front end is not launched yet
    bool draining = false;         // finish the last frames' merges with the frames there are
    bool ending = false;
    std::vector<std::unique_ptr<Entry>> ring;
    int lw[kMaxLevels] = {}, lh[kMaxLevels] = {}, lp[kMaxLevels] = {};
    void *fq[2][kMaxLevels] = {};
    void *fb[2][kMaxLevels] = {};
    void *pyr[kMaxLevels] = {};
    void *gh[kMaxLevels] = {};
    float2 *flow[2] = {};
    int *cc[3] = {};  // component labels, local-root counts, areas (min_area > 1)
    int reg_lnx = 0, reg_lny = 0;                  // registration: log2 of the padded FFT size
    float2 *reg_spec[2] = {}, *reg_work = nullptr; // spectra (by frame parity) and the correlation plane
    float *S = nullptr;
    unsigned *red = nullptr;
    unsigned *cand = nullptr;  // select candidates (W*H words)
    void *ll[2] = {};
    uint8_t *llm[2] = {};
    // JPEG2000 coder (codestream_bpp > 0): code-block scratch, container geometry
    char *cs_scratch = nullptr;
    int cs_ncb = 0;
    long long cs_cap = 0, cs_budget = 0;
    uint8_t cs_eps[kMaxSubbands] = {};   // the bands' quantisation exponents and mantissas (JPEG2000 codestream)
    uint16_t cs_mu[kMaxSubbands] = {};
};

struct BatchRec;

}  // namespace

struct flowroi_ctx {
    flowroi_config cfg{};
    MethodConsts mc{};
    int device = 0, num_sms = 0;
    bool half = false, plain = false, keep = false, manual = false;
    cudaStream_t s_comp = nullptr, s_copy = nullptr, s_d2h = nullptr, s_cap = nullptr;
    std::mutex mu;       // host state: streams, entries, descriptors
    std::mutex d2h_mu;   // serialises copies out on s_d2h
    std::mutex cmu;      // completion state + scheduler wake-ups (never held across CUDA calls)
    std::condition_variable ccv;
    std::map<int64_t, std::unique_ptr<Stream>> streams;
    int64_t rr_cursor = INT64_MIN;
    uint64_t budget = 0, admitted = 0;
    // Descriptor slots: the host can enqueue this many batches ahead of the
    // device, so a host stall shorter than that many batch times does not
    // leave the device idle.
    static constexpr int kDesc = 8;
    BatchDesc *desc_host[kDesc] = {};
    BatchDesc *desc_dev[kDesc] = {};
    cudaEvent_t desc_ev[kDesc] = {};
    cudaGraphExec_t graph[kDesc] = {};
    int graph_launches = 0;
    int desc_next = 0;
    int grid_exp = 0, grid_upd = 0, grid_win = 0, grid_mask = 0, grid_dwt = 0, grid_frames = 0, grid_den = 0, grid_cc = 0, grid_mrg = 0, grid_reg = 0;
    int grid_t1 = 0, grid_mq = 0, grid_csc = 0;
    int occ[TK_COUNT] = {};         // resident blocks per SM of the tunable persistent kernels
    int dwt_variant = 5;            // DWT register budget in use (resident blocks per SM)
    int upd_rows = kUpdRows;        // rows per thread of the update kernel's tile columns
    TileTable tiles{};              // launch and tile shapes (flowroi_set_tiles / config.tile_table)
    int inflight = 0;               // guarded by cmu
    int max_inflight = 2;
    bool work_flag = false;         // guarded by cmu
    bool shutdown = false;          // guarded by cmu
    std::thread sched;
    std::atomic<bool> poisoned{false};
    std::string poison_msg;
    int64_t frames_submitted = 0, frames_cancelled = 0;  // guarded by mu
    int64_t frames_done = 0;                              // guarded by cmu
    std::atomic<int64_t> batches{0}, refused{0}, launches{0};
    std::vector<double> lat_ms;                           // guarded by cmu
    unsigned *err_host = nullptr, *err_dev = nullptr;     // kernel error word (mapped pinned memory)
    // per-kernel event timing (guarded by mu)
    bool profiling = false;
    struct ProfRec { int kid, level, iter; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_pending;
    std::map<std::tuple<int, int, int>, std::pair<int64_t, double>> prof_tot;
    // codestream coder: scratch kept between calls (grow-only) and its stream
    std::mutex cs_mu;
    unsigned char *cs_scratch = nullptr;
    size_t cs_bytes = 0;
    cudaStream_t cs_stream = nullptr;
};

namespace {

struct BatchRec {
    flowroi_ctx *ctx;
    std::vector<Entry *> entries;
};

int cuda_fail(flowroi_ctx *c, cudaError_t e, const char *what)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    if (c) {
        c->poisoned = true;
        c->poison_msg = buf;
    }
    g_err = buf;
    logf("device error, context poisoned: %s", buf);
    return FLOWROI_EDEVICE;
}

#define CK(ctx, call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// ------------------------------------------------------------ validation --
// The bands' exponents and mantissas of a JPEG2000 codestream (table index
// as the quantisation steps): 9/7 the steps' (eps, mu); 5/3 (no
// quantisation) eps = bit depth + log2 of the band's nominal gain (0 LL,
// 1 HL and LH, 2 HH), mu = 0.
bool band_exponents(int levels, int wavelet, int bit_depth, float delta_base, uint8_t *eps, uint16_t *mu)
{
    std::memset(eps, 0, kMaxSubbands);
    std::memset(mu, 0, kMaxSubbands * sizeof(uint16_t));
    const int nb = 3 * levels + 1;
    if (wavelet == FLOWROI_W97) {
        int e[kMaxSubbands], m[kMaxSubbands];
        if (quant_steps(levels, bit_depth, delta_base, nullptr, e, m, nullptr) != 0) return false;
        for (int b = 0; b < nb; b++) {
            if (e[b] < 0 || e[b] > 31) return false;
            eps[b] = (uint8_t)e[b];
            mu[b] = (uint16_t)m[b];
        }
    } else {
        for (int b = 0; b < nb; b++) eps[b] = (uint8_t)(bit_depth + (b == 3 * levels ? 0 : (b % 3 < 2 ? 1 : 2)));
    }
    return true;
}

bool read_text_file(const char *path, std::string &out)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t n;
    out.clear();
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) {
        out.append(buf, n);
        if (out.size() > (1u << 20)) break;
    }
    std::fclose(f);
    return out.size() <= (1u << 20);
}

int validate_config(const flowroi_config *c)
{
    if (!c) return fail(FLOWROI_EINVAL, "config is NULL");
    if (c->struct_size != sizeof(flowroi_config)) return fail(FLOWROI_EINVAL, "config.struct_size mismatch");
    if (!(c->roi_q > 0.f && c->roi_q < 1.f)) return fail(FLOWROI_EINVAL, "config.roi_q must be in (0,1)");
    if (c->scale_shift < 0 || c->scale_shift > 15) return fail(FLOWROI_EINVAL, "config.scale_shift must be in [0,15]");
    if (c->wavelet != FLOWROI_W53 && c->wavelet != FLOWROI_W97) return fail(FLOWROI_EINVAL, "config.wavelet must be 53 or 97");
    if (c->dwt_levels < 1 || c->dwt_levels > kMaxLevels) return fail(FLOWROI_EINVAL, "config.dwt_levels must be in [1,8]");
    if (c->pyr_levels < 1 || c->pyr_levels > kMaxLevels) return fail(FLOWROI_EINVAL, "config.pyr_levels must be in [1,8]");
    if (c->iters < 1 || c->iters > 8) return fail(FLOWROI_EINVAL, "config.iters must be in [1,8]");
    if (!flow_radius_supported(c->win_r)) return fail(FLOWROI_EINVAL, "config.win_r must be in [2,10]");
    if (c->poly_n_half != 2 && c->poly_n_half != 3) return fail(FLOWROI_EINVAL, "config.poly_n_half must be 2 or 3");
    if (!(c->poly_sigma > 0.f)) return fail(FLOWROI_EINVAL, "config.poly_sigma must be > 0");
    if (!(c->lambda > 0.f)) return fail(FLOWROI_EINVAL, "config.lambda must be > 0");
    if (!(c->sal_weight >= 0.f && c->sal_weight <= 1.f)) return fail(FLOWROI_EINVAL, "config.sal_weight must be in [0,1]");
    if (!morph_radius_supported(c->r_open) || !morph_radius_supported(c->r_close))
        return fail(FLOWROI_EINVAL, "config.r_open/r_close must be in [0,4]");
    if (c->precision != FLOWROI_FP32 && c->precision != FLOWROI_FP16) return fail(FLOWROI_EINVAL, "config.precision must be 32 or 16");
    if (!(c->delta_base > 0.f)) return fail(FLOWROI_EINVAL, "config.delta_base must be > 0");
    if (c->max_batch_frames < 1 || c->max_batch_frames > kMaxBatch) return fail(FLOWROI_EINVAL, "config.max_batch_frames must be in [1,64]");
    if (c->result_ring < 2 || c->result_ring > 16) return fail(FLOWROI_EINVAL, "config.result_ring must be in [2,16]");
    if (c->flags & ~(FLOWROI_KEEP_INTERMEDIATES | FLOWROI_PLAIN | FLOWROI_MANUAL | FLOWROI_TEST_EXPIRE_TMA |
                     FLOWROI_TEST_EXPIRE_LOOP))
        return fail(FLOWROI_EINVAL, "config.flags has unknown bits");
    if (c->min_area < 0 || c->min_area > (1 << 20)) return fail(FLOWROI_EINVAL, "config.min_area must be in [0, 2^20]");
    if (c->adjacent < 0 || c->adjacent > kMaxAdj) return fail(FLOWROI_EINVAL, "config.adjacent must be in [0,4]");
    if (c->register_frames != 0 && c->register_frames != 1) return fail(FLOWROI_EINVAL, "config.register_frames must be 0 or 1");
    if (c->register_frames && (c->reg_level < 1 || c->reg_level >= c->pyr_levels))
        return fail(FLOWROI_EINVAL, "config.reg_level must be in [1, pyr_levels - 1]");
    if (c->result_ring < 2 * c->adjacent + 2)
        return fail(FLOWROI_EINVAL, "config.result_ring must be at least 2*adjacent + 2");
    if (c->denoise != 0 && c->denoise != 1) return fail(FLOWROI_EINVAL, "config.denoise must be 0 or 1");
    if (!denoise_radius_supported(c->den_radius)) return fail(FLOWROI_EINVAL, "config.den_radius must be in [1,3]");
    if (!(c->den_sigma_s > 0.f) || !(c->den_sigma_r > 0.f)) return fail(FLOWROI_EINVAL, "config.den_sigma_s/den_sigma_r must be > 0");
    if (!(c->codestream_bpp >= 0.f && c->codestream_bpp <= 64.f))
        return fail(FLOWROI_EINVAL, "config.codestream_bpp must be in [0, 64]");
    if (c->codestream_format != FLOWROI_CS_CONTAINER && c->codestream_format != FLOWROI_CS_J2C)
        return fail(FLOWROI_EINVAL, "config.codestream_format must be FLOWROI_CS_CONTAINER or FLOWROI_CS_J2C");
    if (c->codestream_reset != 0 && c->codestream_reset != 1)
        return fail(FLOWROI_EINVAL, "config.codestream_reset must be 0 or 1");
    if (c->tile_table) {
        std::string text, err;
        TileTable t;
        tiles_clear(t);
        if (!read_text_file(c->tile_table, text)) return fail(FLOWROI_EINVAL, "config.tile_table: cannot read %s", c->tile_table);
        if (!tiles_parse(text.c_str(), t, err)) return fail(FLOWROI_EINVAL, "config.tile_table %s: %s", c->tile_table, err.c_str());
    }
    return FLOWROI_OK;
}

// Closed-form constants of the separable polynomial expansion.
void expansion_consts(int n, double sigma, MethodConsts &mc)
{
    double a[7] = {}, s0 = 0, s2 = 0, s4 = 0;
    for (int u = -n; u <= n; u++) {
        a[u + n] = std::exp(-(double)(u * u) / (2.0 * sigma * sigma));
        s0 += a[u + n];
        s2 += a[u + n] * u * u;
        s4 += a[u + n] * u * u * u * u;
    }
    for (int i = 0; i < 7; i++) mc.app[i] = (float)a[i];
    mc.n_half = n;
    mc.inv_s0s2 = (float)(1.0 / (s0 * s2));
    mc.inv_s2s2 = (float)(1.0 / (s2 * s2));
    // M = [[s0^2, s0 s2, s0 s2], [s0 s2, s0 s4, s2^2], [s0 s2, s2^2, s0 s4]]
    // acting on (r_1, r_uu, r_vv); rows 1 and 2 of its inverse by cofactors.
    double M[3][3] = {{s0 * s0, s0 * s2, s0 * s2}, {s0 * s2, s0 * s4, s2 * s2}, {s0 * s2, s2 * s2, s0 * s4}};
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    double inv[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
            inv[i][j] = (M[r0][c0] * M[r1][c1] - M[r0][c1] * M[r1][c0]) / det;
        }
    for (int j = 0; j < 3; j++) {
        mc.m_uu[j] = (float)inv[1][j];
        mc.m_vv[j] = (float)inv[2][j];
    }
}

int tiles(int w, int h, int tw, int th) { return ((w + tw - 1) / tw) * ((h + th - 1) / th); }

int64_t stream_is_launchable(Stream *s)
{
    if (s->ending) return -1;
    const int64_t next = s->launched_seq + 1;
    if (next >= s->next_seq) return -1;
    Entry *e = s->ring[next % (int64_t)s->ring.size()].get();
    // (Readers never block a launch: a reader of this slot waits for this very
    // frame; submit refuses to reuse a slot that is being read.)
    if (e->seq != next || e->state.load() != E_PENDING) return -1;
    return next;
}

// The frame whose JPEG2000 front end runs with flow frame `seq` of s: the
// same frame, or with adjacent factor k the frame seq - k once it exists
// (its window d-k..d+k is then complete); -1 if none.
int64_t dwt_target_with_flow(flowroi_ctx *c, Stream *s, int64_t seq)
{
    const int k = c->cfg.adjacent;
    if (k == 0) return seq;
    const int64_t d = seq - k;
    return d >= 0 && d >= s->dwt_seq ? d : -1;
}

// A drain entry of s (no flow frame): the next frame whose front end has
// not run, when s is draining (flush, end of stream) and has no flow frame
// to launch; its window is cut at the last frame with a flow.
int64_t stream_drain_target(flowroi_ctx *c, Stream *s)
{
    if (c->cfg.adjacent == 0 || !s->draining || stream_is_launchable(s) >= 0) return -1;
    return s->dwt_seq <= s->launched_seq ? s->dwt_seq : -1;
}

// Byte plan of a stream's device block (carves pointers when base != null).
size_t plan_stream(flowroi_ctx *c, Stream *s, char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        off = align_up(off, 256);
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const int L = c->cfg.pyr_levels, R = c->cfg.result_ring;
    const size_t esz = c->half ? 2 : 4;
    const size_t npx = (size_t)s->W * s->H;
    for (int l = 0; l < L; l++) {
        s->lw[l] = s->W >> l;
        s->lh[l] = s->H >> l;
        s->lp[l] = (int)align_up((size_t)s->lw[l], 32);
    }
    for (int k = 0; k < 2; k++)
        for (int l = 0; l < L; l++) {
            s->fq[k][l] = take((size_t)s->lp[l] * s->lh[l] * 4 * esz);
            s->fb[k][l] = take((size_t)s->lp[l] * s->lh[l] * esz);
        }
    // level 0 is read from the raw frame unless the flow input is denoised
    for (int l = c->cfg.denoise ? 0 : 1; l < L; l++) s->pyr[l] = take((size_t)s->lp[l] * s->lh[l] * esz);
    for (int l = 0; l < L; l++) s->gh[l] = take((size_t)s->lp[l] * s->lh[l] * 5 * esz);
    for (int k = 0; k < 2; k++) s->flow[k] = reinterpret_cast<float2 *>(take((size_t)s->lp[0] * s->H * sizeof(float2)));
    s->S = reinterpret_cast<float *>(take((size_t)s->lp[0] * s->H * sizeof(float)));
    s->red = reinterpret_cast<unsigned *>(take(kRedWords * sizeof(unsigned)));
    s->cand = reinterpret_cast<unsigned *>(take(npx * sizeof(unsigned)));
    if (c->cfg.min_area > 1)
        for (int k = 0; k < 3; k++) s->cc[k] = reinterpret_cast<int *>(take(npx * sizeof(int)));
    if (c->cfg.register_frames) {
        const int rl = c->cfg.reg_level;
        auto lg = [](int n) { int k = 0; while ((1 << k) < n) k++; return k; };
        s->reg_lnx = lg(s->lw[rl]);
        s->reg_lny = lg(s->lh[rl]);
        const size_t nsp = (size_t)1 << (s->reg_lnx + s->reg_lny);
        for (int k = 0; k < 2; k++) s->reg_spec[k] = reinterpret_cast<float2 *>(take(nsp * sizeof(float2)));
        s->reg_work = reinterpret_cast<float2 *>(take(nsp * sizeof(float2)));
    }
    for (int k = 0; k < 2; k++) {
        s->ll[k] = take((npx / 4) * 4);
        s->llm[k] = reinterpret_cast<uint8_t *>(take(npx / 4));
    }
    const bool cs_on = c->cfg.codestream_bpp > 0.f;
    if (cs_on) {
        s->cs_ncb = ebcot_codeblocks(s->W, s->H, c->cfg.dwt_levels);
        s->cs_budget = (long long)std::floor((double)c->cfg.codestream_bpp * (double)npx / 8.0);
        s->cs_cap = c->cfg.codestream_format == FLOWROI_CS_J2C
                        ? kJ2cHeader + (long long)s->cs_ncb * kJ2cPerBlock + s->cs_budget
                        : kCsHeader + (long long)s->cs_ncb * (kCsEntry + 2 * kMaxPasses) + s->cs_budget;
        band_exponents(c->cfg.dwt_levels, c->cfg.wavelet, s->bit_depth, c->cfg.delta_base, s->cs_eps, s->cs_mu);
        s->cs_scratch = take((size_t)s->cs_ncb * kCbScratch);
    }
    for (int r = 0; r < R; r++) {
        Entry *e = s->ring[r].get();
        e->raw = take(npx * s->bpp);
        e->mask = reinterpret_cast<uint8_t *>(take(npx));
        e->mask_own = c->cfg.adjacent > 0 ? reinterpret_cast<uint8_t *>(take(npx)) : nullptr;
        e->coeffs = reinterpret_cast<int32_t *>(take(npx * 4));
        if (c->keep) {
            e->dbg_flow = reinterpret_cast<float2 *>(take(npx * sizeof(float2)));
            e->dbg_shat = reinterpret_cast<float *>(take(npx * 4));
            e->dbg_mask0 = reinterpret_cast<uint8_t *>(take(npx));
            e->dbg_yf = c->cfg.wavelet == FLOWROI_W97 ? reinterpret_cast<float *>(take(npx * 4)) : nullptr;
            e->dbg_thr = reinterpret_cast<float *>(take(sizeof(float)));
            e->dbg_den = c->cfg.denoise ? reinterpret_cast<float *>(take(npx * 4)) : nullptr;
            e->dbg_drift = c->cfg.register_frames ? reinterpret_cast<float *>(take(2 * sizeof(float))) : nullptr;
        }
        if (cs_on) {
            e->cs = reinterpret_cast<uint8_t *>(take((size_t)s->cs_cap));
            e->cs_len = reinterpret_cast<long long *>(take(sizeof(long long)));
        }
    }
    return align_up(off, 256);
}

// TMA maps of a stream's G, h planes (one 3-D map per pyramid level).
bool encode_stream_maps(flowroi_ctx *c, Stream *s)
{
    int xo = 0, bw = 0, eh = 0;
    if (window_box(c->half, c->cfg.win_r, &xo, &bw, &eh) != 0) return false;
    const size_t esz = c->half ? 2 : 4;
    for (int l = 0; l < c->cfg.pyr_levels; l++) {
        const uint64_t dims[3] = {(uint64_t)s->lw[l], (uint64_t)s->lh[l], 5};
        const uint64_t strides[2] = {(uint64_t)s->lp[l] * esz, (uint64_t)s->lp[l] * s->lh[l] * esz};
        const uint32_t box[3] = {(uint32_t)bw, (uint32_t)eh, 1};  // one plane per copy
        if (!tma_encode(&s->gh_map[l], c->half, 3, s->gh[l], dims, strides, box)) return false;
    }
    return true;
}

// One batch entry of stream s: the flow (and mask) of frame `e` if not
// null, and the JPEG2000 front end of frame `d` if not null (the same frame
// when adjacent = 0; with adjacent = k, frame e's seq - k, or during a drain
// an earlier frame alone), with the per-frame masks of d's window.
void fill_frame(flowroi_ctx *c, Stream *s, Entry *e, Entry *d, FrameDesc &F)
{
    std::memset(&F, 0, sizeof F);
    for (int l = 0; l < c->cfg.pyr_levels; l++) F.gh_map[l] = s->gh_map[l];
    F.W = s->W;
    F.H = s->H;
    F.bpp = s->bpp;
    F.bit_depth = s->bit_depth;
    F.do_flow = e ? 1 : 0;
    F.has_prev = e && e->has_prev ? 1 : 0;
    F.keep = c->keep ? 1 : 0;
    F.raw_pitch = s->W * s->bpp;
    F.dc_off = 1 << (s->bit_depth - 1);
    F.unit_scale = (float)(255.0 / (double)((1 << s->bit_depth) - 1));
    const int cur = e ? (int)(e->seq & 1) : 0, prv = cur ^ 1;
    for (int l = 0; l < c->cfg.pyr_levels; l++) {
        F.lw[l] = s->lw[l];
        F.lh[l] = s->lh[l];
        F.lp[l] = s->lp[l];
        F.pyr[l] = s->pyr[l];
        F.fq_cur[l] = s->fq[cur][l];
        F.fb_cur[l] = s->fb[cur][l];
        F.fq_prev[l] = s->fq[prv][l];
        F.fb_prev[l] = s->fb[prv][l];
        F.gh[l] = s->gh[l];
    }
    F.flow[0] = s->flow[0];
    F.flow[1] = s->flow[1];
    F.S = s->S;
    F.red = s->red;
    F.cand = s->cand;
    F.cc_lab = s->cc[0];
    F.cc_cnt = s->cc[1];
    F.cc_area = s->cc[2];
    F.ll[0] = s->ll[0];
    F.ll[1] = s->ll[1];
    for (int l = 0; l < kMaxLevels; l++)
        F.dwt_seg[l] = tiles_dwt_seg(c->tiles, c->half, s->W, l + 1, s->W >> (l + 1), s->H >> (l + 1));
    F.sal_strips = tiles_saliency_strips(c->tiles, c->half, s->W);
    F.llm[0] = s->llm[0];
    F.llm[1] = s->llm[1];
    if (e && c->cfg.register_frames) {
        F.do_reg = 1;
        F.reg_lnx = s->reg_lnx;
        F.reg_lny = s->reg_lny;
        F.reg_cur = s->reg_spec[cur];
        F.reg_prev = s->reg_spec[prv];
        F.reg_work = s->reg_work;
    }
    if (e) {
        F.raw = e->raw;
        F.mask = c->cfg.adjacent > 0 ? e->mask_own : e->mask;
        F.coeffs = e->coeffs;
        F.dbg_flow = e->dbg_flow;
        F.dbg_shat = e->dbg_shat;
        F.dbg_mask0 = e->dbg_mask0;
        F.dbg_thr = e->dbg_thr;
        F.dbg_den = e->dbg_den;
        F.dbg_drift = e->dbg_drift;
    }
    if (d) {
        F.do_dwt = 1;
        F.dwt_raw = d->raw;
        F.dwt_mask = d->mask;
        F.dwt_coeffs = d->coeffs;
        F.dwt_yf = d->dbg_yf;
        if (d->cs) {
            // the coder takes the coefficients this batch's front end writes
            F.do_cs = 1;
            CsFrame &C = F.cs;
            C.coef = d->coeffs;
            C.out = d->cs;
            C.cap = s->cs_cap;
            C.budget = s->cs_budget;
            C.w = s->W;
            C.h = s->H;
            C.levels = c->cfg.dwt_levels;
            C.wavelet = c->cfg.wavelet;
            C.shift = c->cfg.scale_shift;
            C.bit_depth = s->bit_depth;
            C.ncb = s->cs_ncb;
            const size_t n = (size_t)s->cs_ncb;
            char *b = s->cs_scratch;
            C.cbytes = reinterpret_cast<uint8_t *>(b);
            b += n * kCbRegion;
            C.sym = reinterpret_cast<uint8_t *>(b);  // 16-byte aligned: the MQ coder reads it in 16-byte pieces
            b += n * kSymCap;
            C.ptab = reinterpret_cast<int4 *>(b);
            b += n * kMaxPasses * sizeof(int4);
            C.mqs = reinterpret_cast<uint32_t *>(b);
            b += n * kMaxPasses * kMqWords * sizeof(uint32_t);
            C.dist = reinterpret_cast<double *>(b);
            b += n * kMaxPasses * sizeof(double);
            C.hs = reinterpret_cast<double *>(b);
            b += n * (kMaxPasses + 1) * sizeof(double);
            C.plen = reinterpret_cast<int32_t *>(b);
            b += n * kMaxPasses * sizeof(int32_t);
            C.nsym = reinterpret_cast<int32_t *>(b);
            b += n * kMaxPasses * sizeof(int32_t);
            C.info = reinterpret_cast<int32_t *>(b);
            b += n * kCbInfo * sizeof(int32_t);
            C.hk = reinterpret_cast<int32_t *>(b);
            C.flen = d->cs_len;
            C.format = c->cfg.codestream_format;
            C.reset = c->cfg.codestream_reset;
            std::memcpy(C.eps, s->cs_eps, sizeof C.eps);
            std::memcpy(C.mu, s->cs_mu, sizeof C.mu);
        }
        const int k = c->cfg.adjacent;
        if (k > 0) {
            // own masks of frames d-k .. d+k that exist and have their flow launched
            const int64_t last = e ? e->seq : s->launched_seq;
            const int64_t R = (int64_t)s->ring.size();
            for (int64_t m = std::max<int64_t>(0, d->seq - k); m <= std::min(last, d->seq + k); m++) {
                Entry *o = s->ring[m % R].get();
                if (o->seq == m) F.adj[F.n_adj++] = o->mask_own;
            }
        }
    }
}


// Persistent grids and the DWT variant from the context's tile table.
void apply_context_tiles(flowroi_ctx *c)
{
    const int sh = c->half ? 1 : 0;
    const int dv = c->tiles.dwt_variant[sh];
    c->dwt_variant = dv == 6 ? 6 : 5;
    c->occ[TK_DWT] = occupancy_dwt(c->cfg.wavelet, c->dwt_variant);
    c->upd_rows = c->tiles.update_rows[sh] > 0 ? c->tiles.update_rows[sh] : kUpdRows;
    c->occ[TK_UPDATE] = occupancy_update(c->half, c->upd_rows);
    auto grid = [&](int k) {
        const int occ = std::max(1, c->occ[k]);
        const int want = c->tiles.blocks_per_sm[sh][k];
        return (want > 0 ? std::min(want, occ) : occ) * c->num_sms;
    };
    c->grid_exp = grid(TK_EXPAND);
    c->grid_upd = grid(TK_UPDATE);
    c->grid_win = grid(TK_WINDOW);
    c->grid_mask = grid(TK_MASK);
    c->grid_dwt = grid(TK_DWT);
}

// Prefix tables of the batch (also the exact grids of the plain path).
void fill_offsets(flowroi_ctx *c, BatchDesc &bd)
{
    const int n = bd.nframes;
    const int L = c->cfg.pyr_levels, D = c->cfg.dwt_levels;
    for (int l = 0; l < kMaxLevels; l++) {
        bd.exp_off[l][0] = bd.flow_off[l][0] = bd.win_off[l][0] = bd.dwt_off[l][0] = 0;
    }
    bd.sal_off[0] = bd.sal2_off[0] = bd.mor_off[0] = bd.frm_off[0] = bd.mrg_off[0] = 0;
    bd.reg_row_off[0] = bd.reg_col_off[0] = bd.reg_el_off[0] = 0;
    for (int i = 0; i < n; i++) {
        const FrameDesc &F = bd.f[i];
        for (int l = 0; l < L; l++) {
            bd.exp_off[l][i + 1] = bd.exp_off[l][i] + (F.do_flow ? tiles(F.lw[l], F.lh[l], kExpTW, kExpTH) : 0);
            bd.flow_off[l][i + 1] = bd.flow_off[l][i] + (F.has_prev ? tiles(F.lw[l], F.lh[l], kUpdTW, c->upd_rows) : 0);
            bd.win_off[l][i + 1] = bd.win_off[l][i] + (F.has_prev ? tiles(F.lw[l], F.lh[l], kWinTW, kWinTH) : 0);
        }
        for (int l = 1; l <= D; l++)
            bd.dwt_off[l - 1][i + 1] =
                bd.dwt_off[l - 1][i] + (F.do_dwt ? dwt_units(F.W >> l, F.H >> l, F.dwt_seg[l - 1]) : 0);
        bd.sal_off[i + 1] = bd.sal_off[i] + (F.has_prev ? tiles(F.W, F.H, kSalTW, kSalTH) : 0);
        bd.sal2_off[i + 1] = bd.sal2_off[i] + (F.has_prev ? tiles(F.W, F.H, kSalTW, kSalSub * F.sal_strips) : 0);
        bd.mor_off[i + 1] = bd.mor_off[i] + (F.do_flow ? tiles(F.W, F.H, kMorTW, kMorTH) : 0);
        bd.mrg_off[i + 1] = bd.mrg_off[i] + (F.n_adj > 0 ? (int)(((size_t)F.W * F.H + 4095) / 4096) : 0);
        const int rnx = F.do_reg ? 1 << F.reg_lnx : 0, rny = F.do_reg ? 1 << F.reg_lny : 0;
        bd.reg_row_off[i + 1] = bd.reg_row_off[i] + rny;
        bd.reg_col_off[i + 1] = bd.reg_col_off[i] + (rnx + register_cols() - 1) / register_cols();
        bd.reg_el_off[i + 1] = bd.reg_el_off[i] + (rnx * rny + register_unit() - 1) / register_unit();
        bd.frm_off[i + 1] = i + 1;
    }
    // the coder's frames (those whose front end runs), code-blocks numbered in order
    int m = 0, ncb = 0;
    for (int i = 0; i < n; i++)
        if (bd.f[i].do_cs) {
            bd.csf[m] = bd.f[i].cs;
            bd.csf[m].cb0 = ncb;
            ncb += bd.csf[m].ncb;
            m++;
        }
    bd.cs.nframes = m;
    bd.cs.ncb = ncb;
    bd.cs.cbcap = kCbBytes;
    bd.cs.err = nullptr;
}

const char *const kKernelNames[] = {"frame_init", "expand", "update", "window", "saliency", "select_find", "select_pass",
                                    "morph", "dwt", "denoise", "components", "merge", "register", "codestream"};
enum KernelId { K_INIT = 0, K_EXPAND, K_UPDATE, K_WINDOW, K_SAL, K_FIND, K_PASS, K_MORPH, K_DWT, K_DENOISE, K_CC, K_MERGE, K_REG, K_CS };

// Runs one launch, bracketed by an event pair when profiling.
template <class Fn>
void timed(flowroi_ctx *c, cudaStream_t st, bool prof, int kid, int level, int iter, Fn fn)
{
    if (!prof) {
        fn();
        return;
    }
    flowroi_ctx::ProfRec r{kid, level, iter, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, st);
    fn();
    cudaEventRecord(r.b, st);
    c->prof_pending.push_back(r);
}

// The hot path for one batch descriptor.  `hd` (host copy) gives exact grids
// on the plain path; the batched path uses fixed persistent grids.
int enqueue_pipeline(flowroi_ctx *c, const BatchDesc *dd, const BatchDesc *hd, cudaStream_t st, int *nlaunch, bool prof)
{
    const MethodConsts &mc = c->mc;
    const int L = c->cfg.pyr_levels, D = c->cfg.dwt_levels, I = c->cfg.iters;
    const int n = hd->nframes;
    const bool pl = c->plain;
    // Plain path: one frame per launch, the same persistent kernels with a
    // grid no larger than the frame's tile count.
    auto g = [&](int exact, int persistent) { return pl ? std::max(1, std::min(exact, persistent)) : persistent; };
    int cnt = 0;
    const bool any_prev = !pl || hd->sal_off[n] > 0;
    timed(c, st, prof, K_INIT, -1, -1, [&] { launch_frame_init(dd, g(n, c->grid_frames), st); });
    cnt++;
    if (mc.denoise) {
        // the flow input of every frame (its expansion is the next frame's predecessor)
        timed(c, st, prof, K_DENOISE, -1, -1, [&] { launch_denoise(dd, mc, c->half, g(hd->exp_off[0][n], c->grid_den), st); });
        cnt++;
    }
    for (int l = 0; l < L; l++) {
        timed(c, st, prof, K_EXPAND, l, -1, [&] { launch_expand(dd, mc, l, c->half, g(hd->exp_off[l][n], c->grid_exp), st); });
        cnt++;
    }
    if (mc.reg_on) {
        // registration to the predecessor (its spectrum is kept for the next frame)
        const int units[8] = {hd->reg_el_off[n], hd->reg_row_off[n], hd->reg_col_off[n], hd->reg_el_off[n],
                              hd->reg_row_off[n], hd->reg_col_off[n], hd->reg_el_off[n], 1};
        for (int step = 0; step < 8; step++) {
            timed(c, st, prof, K_REG, step, -1,
                  [&] { launch_register(dd, mc, c->half, step, step == 7 ? 1 : g(units[step], c->grid_reg), st); });
            cnt++;
        }
    }
    if (any_prev) {
        int k = 0;
        for (int l = L - 1; l >= 0; l--)
            for (int it = 0; it < I; it++, k++) {
                const int dst = k & 1;
                timed(c, st, prof, K_UPDATE, l, it, [&] {
                    launch_update(dd, mc, l, it, dst ^ 1, c->half, c->upd_rows, g(hd->flow_off[l][n], c->grid_upd), st);
                });
                timed(c, st, prof, K_WINDOW, l, it, [&] {
                    launch_window(dd, mc, l, dst, c->half, g(hd->win_off[l][n], c->grid_win), st);
                });
                cnt += 2;
            }
        timed(c, st, prof, K_SAL, -1, -1, [&] { launch_saliency(dd, mc, g(hd->sal2_off[n], c->grid_mask), st); });
        for (int pass = 0; pass < 3; pass++) {
            // pass 2 reads the candidates pass 1 kept: kCandBlocks blocks a frame
            const int gp = pass == 1 ? g(hd->sal_off[n], c->grid_mask)
                                     : (pl ? n * kCandBlocks : std::max(1, c->grid_mask / kCandBlocks) * kCandBlocks);
            if (pass > 0) timed(c, st, prof, K_PASS, pass, -1, [&] { launch_select_pass(dd, pass, gp, st); });
            timed(c, st, prof, K_FIND, pass, -1, [&] { launch_select_find(dd, mc, pass, g(n, c->grid_frames), st); });
        }
        cnt += 6;
    }
    timed(c, st, prof, K_MORPH, -1, -1, [&] { launch_morph(dd, mc, g(hd->mor_off[n], c->grid_mask), st); });
    cnt++;
    if (mc.min_area > 1 && any_prev) {
        for (int step = 0; step < 4; step++) {
            timed(c, st, prof, K_CC, step, -1, [&] { launch_cc(dd, mc, step, g(hd->sal_off[n], c->grid_cc), st); });
            cnt++;
        }
    }
    if (c->cfg.adjacent > 0) {
        timed(c, st, prof, K_MERGE, -1, -1, [&] { launch_merge(dd, g(hd->mrg_off[n], c->grid_mrg), st); });
        cnt++;
    }
    for (int l = 1; l <= D; l++) {
        timed(c, st, prof, K_DWT, l, -1, [&] {
            launch_dwt(dd, mc, l, pl ? dwt_grid(hd->dwt_off[l - 1][n], c->grid_dwt) : c->grid_dwt, c->dwt_variant, st);
        });
        cnt++;
    }
    if (c->cfg.codestream_bpp > 0.f) {
        // tier-1 coding, rate control and containers of the batch's front-end frames
        timed(c, st, prof, K_CS, -1, -1, [&] {
            cudaMemsetAsync(const_cast<int *>(dd->cs_next), 0, sizeof dd->cs_next, st);
            launch_ebcot_persistent(&dd->cs, c->grid_t1, c->grid_mq, c->grid_csc, c->cfg.codestream_reset != 0, st);
        });
        cnt += 9;
    }
    *nlaunch = cnt;
    return FLOWROI_OK;
}

void CUDART_CB on_batch_done(void *p)
{
    BatchRec *r = static_cast<BatchRec *>(p);
    flowroi_ctx *c = r->ctx;
    const double t = now_ms();
    if (c->err_host && *(volatile unsigned *)c->err_host) {
        // A kernel gave up a bounded wait or loop: results of this batch are not valid.
        const unsigned code = *(volatile unsigned *)c->err_host;
        c->poison_msg = code == 1u ? "a kernel's bounded wait for a TMA copy ran out"
                                   : "a kernel's bounded union-find loop ran out";
        c->poisoned = true;
        logf("context poisoned: %s", c->poison_msg.c_str());
    }
    {
        std::lock_guard<std::mutex> lk(c->cmu);
        for (Entry *e : r->entries) {
            e->t_done = t;
            e->state.store(E_DONE);
            c->lat_ms.push_back(t - e->t_submit);
            c->frames_done++;
        }
        c->inflight--;
    }
    c->ccv.notify_all();
    delete r;
}

// Launch one batch (mu held).  Returns frames launched or a negative status.
int step_locked(flowroi_ctx *c)
{
    NvtxRange range("flowroi.step");
    if (c->poisoned) return fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
    const int maxb = c->plain ? 1 : c->cfg.max_batch_frames;
    struct Pick {
        Stream *s;
        Entry *e;  // flow frame (null: drain entry)
        Entry *d;  // frame whose JPEG2000 front end runs (null: none yet)
    };
    std::vector<Pick> sel;
    // Round-robin over streams, starting after the last one served.
    auto it = c->streams.upper_bound(c->rr_cursor);
    for (size_t visited = 0; visited < c->streams.size() && (int)sel.size() < maxb; visited++) {
        if (it == c->streams.end()) it = c->streams.begin();
        Stream *s = it->second.get();
        const int64_t R = (int64_t)s->ring.size();
        const int64_t seq = stream_is_launchable(s);
        if (seq >= 0) {
            const int64_t j = dwt_target_with_flow(c, s, seq);
            sel.push_back({s, s->ring[seq % R].get(), j >= 0 ? s->ring[j % R].get() : nullptr});
        } else {
            const int64_t j = stream_drain_target(c, s);
            if (j >= 0) sel.push_back({s, nullptr, s->ring[j % R].get()});
        }
        ++it;
    }
    if (sel.empty()) return 0;
    c->rr_cursor = sel.back().s->id;

    const int k = c->desc_next;
    c->desc_next = (k + 1) % flowroi_ctx::kDesc;
    CK(c, cudaEventSynchronize(c->desc_ev[k]));
    BatchDesc &hd = *c->desc_host[k];
    hd.nframes = (int)sel.size();
    hd.err = c->err_dev;
    hd.tma_spin = (c->cfg.flags & FLOWROI_TEST_EXPIRE_TMA) ? kTestTmaSpin : kTmaSpinLimit;
    hd.loop_limit = (c->cfg.flags & FLOWROI_TEST_EXPIRE_LOOP) ? kTestLoopLimit : kLoopLimit;
    hd.test_skip_tile = (c->cfg.flags & FLOWROI_TEST_EXPIRE_TMA) ? 1 : 0;
    const int nflow = c->cfg.pyr_levels * c->cfg.iters;
    hd.final_flow_buf = (nflow - 1) & 1;
    for (size_t i = 0; i < sel.size(); i++) fill_frame(c, sel[i].s, sel[i].e, sel[i].d, hd.f[i]);
    fill_offsets(c, hd);
    hd.cs.frames = c->desc_dev[k]->csf;
    hd.cs.next = c->desc_dev[k]->cs_next;
    for (auto &pk : sel)
        if (pk.e) CK(c, cudaStreamWaitEvent(c->s_comp, pk.e->uploaded, 0));
    const size_t bytes = offsetof(BatchDesc, f) + sizeof(FrameDesc) * sel.size();
    CK(c, cudaMemcpyAsync(c->desc_dev[k], c->desc_host[k], bytes, cudaMemcpyHostToDevice, c->s_comp));
    if (c->cfg.codestream_bpp > 0.f) {
        const size_t cs_bytes = offsetof(BatchDesc, csf) - offsetof(BatchDesc, cs) + sizeof(CsFrame) * (size_t)hd.cs.nframes;
        CK(c, cudaMemcpyAsync(&c->desc_dev[k]->cs, &hd.cs, cs_bytes, cudaMemcpyHostToDevice, c->s_comp));
    }
    CK(c, cudaEventRecord(c->desc_ev[k], c->s_comp));
    int nl = 0;
    if (c->plain || c->profiling) {
        enqueue_pipeline(c, c->desc_dev[k], &hd, c->s_comp, &nl, c->profiling);
        CK(c, cudaGetLastError());
    } else {
        if (!c->graph[k]) {
            // Capture every slot's graph at once (the graphs differ only in
            // the descriptor they read), so no later step pays for a capture.
            for (int g = 0; g < flowroi_ctx::kDesc; g++) {
                if (c->graph[g]) continue;
                cudaGraph_t gr = nullptr;
                int ng = 0;
                CK(c, cudaStreamBeginCapture(c->s_cap, cudaStreamCaptureModeThreadLocal));
                enqueue_pipeline(c, c->desc_dev[g], &hd, c->s_cap, &ng, false);
                cudaError_t e1 = cudaGetLastError();
                cudaError_t e2 = cudaStreamEndCapture(c->s_cap, &gr);
                if (e1 != cudaSuccess) return cuda_fail(c, e1, "kernel launch during capture");
                if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
                cudaError_t e3 = cudaGraphInstantiate(&c->graph[g], gr, 0);
                cudaGraphDestroy(gr);
                if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaGraphInstantiate");
                c->graph_launches = ng;
            }
        }
        nl = c->graph_launches;
        CK(c, cudaGraphLaunch(c->graph[k], c->s_comp));
    }
    BatchRec *rec = new BatchRec{c, {}};
    for (auto &pk : sel) {
        if (pk.e) {
            pk.e->state.store(E_LAUNCHED);
            pk.s->launched_seq = pk.e->seq;
        }
        if (pk.d) {
            // the frame is complete once this batch's front end has run
            pk.s->dwt_seq = pk.d->seq + 1;
            rec->entries.push_back(pk.d);
        }
    }
    {
        std::lock_guard<std::mutex> lk(c->cmu);
        c->inflight++;
    }
    cudaError_t eh = cudaLaunchHostFunc(c->s_comp, on_batch_done, rec);
    if (eh != cudaSuccess) {
        delete rec;
        return cuda_fail(c, eh, "cudaLaunchHostFunc");
    }
    c->batches++;
    c->launches += nl;
    return (int)sel.size();
}

bool any_launchable(flowroi_ctx *c)
{
    for (auto &kv : c->streams)
        if (stream_is_launchable(kv.second.get()) >= 0 || stream_drain_target(c, kv.second.get()) >= 0) return true;
    return false;
}

void scheduler_main(flowroi_ctx *c)
{
    cudaSetDevice(c->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(c->cmu);
            c->ccv.wait_for(lk, std::chrono::milliseconds(20),
                            [&] { return c->shutdown || (c->work_flag && c->inflight < c->max_inflight); });
            if (c->shutdown) return;
            if (!(c->work_flag && c->inflight < c->max_inflight)) continue;
            c->work_flag = false;
        }
        std::lock_guard<std::mutex> lk(c->mu);
        step_locked(c);
        if (any_launchable(c)) {
            std::lock_guard<std::mutex> lk2(c->cmu);
            c->work_flag = true;
        }
    }
}

void wake_scheduler(flowroi_ctx *c)
{
    {
        std::lock_guard<std::mutex> lk(c->cmu);
        c->work_flag = true;
    }
    c->ccv.notify_all();
}

Entry *find_entry(Stream *s, int64_t frame_idx)
{
    for (auto &e : s->ring)
        if (e->state.load() != E_EMPTY && e->frame_idx == frame_idx) return e.get();
    return nullptr;
}

// A device error stops host callbacks from ever running; waits poll the
// compute stream (non-blocking) so they end with FLOWROI_EDEVICE instead.
void poll_device(flowroi_ctx *c)
{
    const cudaError_t e = cudaStreamQuery(c->s_comp);
    if (e != cudaSuccess && e != cudaErrorNotReady) cuda_fail(c, e, "device error");
}

// Waits (bounded) for an entry to be done.
bool wait_done(flowroi_ctx *c, Entry *e, int timeout_ms)
{
    const double t0 = now_ms();
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(c->cmu);
            c->ccv.wait_for(lk, std::chrono::milliseconds(20), [&] { return e->state.load() == E_DONE || c->poisoned.load(); });
            if (e->state.load() == E_DONE) return true;
            if (c->poisoned) return false;
        }
        poll_device(c);
        if (timeout_ms >= 0 && now_ms() - t0 >= timeout_ms) return e->state.load() == E_DONE;
    }
}

int get_common(flowroi_ctx *c, int64_t stream_id, int64_t frame_idx, int which, void *out, int out_on_device,
               int timeout_ms, uint64_t out_cap = 0, uint64_t *out_len = nullptr)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    if (!out) return fail(FLOWROI_EINVAL, "out is NULL");
    if (c->poisoned) return fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
    Entry *e = nullptr;
    Stream *s = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->streams.find(stream_id);
        if (it == c->streams.end()) return fail(FLOWROI_ENOSTREAM, "unknown stream %lld", (long long)stream_id);
        s = it->second.get();
        e = find_entry(s, frame_idx);
        if (!e) {
            if (s->any_frame && frame_idx <= s->last_frame_idx)
                return fail(FLOWROI_EGONE, "frame %lld of stream %lld is no longer held", (long long)frame_idx,
                            (long long)stream_id);
            return fail(FLOWROI_ENOSTREAM, "frame %lld of stream %lld was not submitted", (long long)frame_idx,
                        (long long)stream_id);
        }
        if (which >= FLOWROI_I_FLOW && !c->keep) return fail(FLOWROI_ENOTKEPT, "intermediates not kept (FLOWROI_KEEP_INTERMEDIATES)");
        if (which == FLOWROI_I_COEFF_F32 && c->cfg.wavelet != FLOWROI_W97)
            return fail(FLOWROI_EINVAL, "float coefficients exist only for the 9/7 path");
        if (which == FLOWROI_I_DENOISED && !c->cfg.denoise) return fail(FLOWROI_EINVAL, "denoising is off (config.denoise)");
        if (which == FLOWROI_I_DRIFT && !c->cfg.register_frames)
            return fail(FLOWROI_EINVAL, "registration is off (config.register_frames)");
        if (which == -2 && !(c->cfg.codestream_bpp > 0.f)) return fail(FLOWROI_EINVAL, "the coder is off (config.codestream_bpp)");
        e->readers++;
    }
    const bool ok = wait_done(c, e, timeout_ms);
    int rc = FLOWROI_OK;
    if (!ok) {
        rc = c->poisoned ? fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str())
                         : fail(FLOWROI_ETIMEDOUT, "frame %lld not finished within %d ms", (long long)frame_idx, timeout_ms);
    } else {
        const size_t npx = (size_t)s->W * s->H;
        const void *src = nullptr;
        size_t bytes = 0;
        switch (which) {
        case 0: src = e->mask; bytes = npx; break;
        case -1: src = e->coeffs; bytes = npx * 4; break;
        case FLOWROI_I_FLOW: src = e->dbg_flow; bytes = npx * 8; break;
        case FLOWROI_I_SALIENCY: src = e->dbg_shat; bytes = npx * 4; break;
        case FLOWROI_I_MASK0: src = e->dbg_mask0; bytes = npx; break;
        case FLOWROI_I_COEFF_F32: src = e->dbg_yf; bytes = npx * 4; break;
        case FLOWROI_I_THRESHOLD: src = e->dbg_thr; bytes = 4; break;
        case FLOWROI_I_DENOISED: src = e->dbg_den; bytes = npx * 4; break;
        case FLOWROI_I_DRIFT: src = e->dbg_drift; bytes = 2 * sizeof(float); break;
        case -2: {
            // the container: its length first
            long long L = 0;
            std::lock_guard<std::mutex> lk(c->d2h_mu);
            cudaError_t ce = cudaMemcpyAsync(&L, e->cs_len, sizeof L, cudaMemcpyDeviceToHost, c->s_d2h);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->s_d2h);
            if (ce != cudaSuccess) {
                rc = cuda_fail(c, ce, "copy out");
            } else if (L < 0) {
                if (out_len) *out_len = 0;
                rc = fail(FLOWROI_ERANGE, "frame %lld: a coefficient magnitude of 2^24 or more, or a code-block over %d bytes",
                          (long long)frame_idx, kCbBytes);
            } else {
                if (out_len) *out_len = (uint64_t)L;
                if ((uint64_t)L > out_cap) rc = fail(FLOWROI_ERANGE, "container of %lld bytes, out_cap is %llu", L,
                                                      (unsigned long long)out_cap);
                src = e->cs;
                bytes = (size_t)L;
            }
            break;
        }
        default: rc = fail(FLOWROI_EINVAL, "unknown intermediate %d", which); break;
        }
        if (rc == FLOWROI_OK && which >= FLOWROI_I_FLOW && !e->has_prev) {
            // A first frame has no flow: report zeros and an infinite cut.
            std::lock_guard<std::mutex> lk(c->d2h_mu);
            if (which == FLOWROI_I_THRESHOLD) {
                const float inf = INFINITY;
                cudaError_t ce = cudaMemcpyAsync(out, &inf, 4, out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, c->s_d2h);
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->s_d2h);
                if (ce != cudaSuccess) rc = cuda_fail(c, ce, "copy out");
                src = nullptr;
            } else if (which == FLOWROI_I_FLOW || which == FLOWROI_I_SALIENCY || which == FLOWROI_I_DRIFT) {
                cudaError_t ce = out_on_device ? cudaMemsetAsync(out, 0, bytes, c->s_d2h) : cudaSuccess;
                if (!out_on_device) std::memset(out, 0, bytes);
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->s_d2h);
                if (ce != cudaSuccess) rc = cuda_fail(c, ce, "copy out");
                src = nullptr;
            }
        }
        if (rc == FLOWROI_OK && src) {
            std::lock_guard<std::mutex> lk(c->d2h_mu);
            cudaError_t ce = cudaMemcpyAsync(out, src, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                             c->s_d2h);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->s_d2h);
            if (ce != cudaSuccess) rc = cuda_fail(c, ce, "copy out");
        }
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        e->readers--;
    }
    if (!c->manual) wake_scheduler(c);
    return rc;
}

}  // namespace

// ========================================================= TMA encode ==
namespace flowroi {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

bool tma_available()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

bool tma_encode(CUtensorMap *map, bool half, int rank, void *base, const uint64_t *dims, const uint64_t *strides_bytes,
                const uint32_t *box)
{
    if (!tma_available() || rank < 1 || rank > 5) return false;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], es[5];
    for (int i = 0; i < rank; i++) {
        d[i] = dims[i];
        b[i] = box[i];
        es[i] = 1;
    }
    for (int i = 0; i + 1 < rank; i++) st[i] = strides_bytes[i];
    const CUresult r = g_encode(map, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                                base, d, st, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace flowroi

// ================================================================ C ABI ==
extern "C" {

int flowroi_abi_version(void) { return FLOWROI_ABI_VERSION; }

uint32_t flowroi_route(int64_t stream_id, uint32_t n_devices)
{
    if (n_devices == 0) return UINT32_MAX;
    // splitmix64 finaliser: consecutive ids become unrelated keys
    uint64_t key = (uint64_t)stream_id + 0x9E3779B97F4A7C15ull;
    key = (key ^ (key >> 30)) * 0xBF58476D1CE4E5B9ull;
    key = (key ^ (key >> 27)) * 0x94D049BB133111EBull;
    key ^= key >> 31;
    // jump consistent hash: the last bucket the key jumps to below n_devices
    int64_t b = -1, j = 0;
    while (j < (int64_t)n_devices) {
        b = j;
        key = key * 2862933555777941757ull + 1;
        j = (int64_t)((double)(b + 1) * ((double)(1ll << 31) / (double)((key >> 33) + 1)));
    }
    return (uint32_t)b;
}

void flowroi_default_config(flowroi_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->struct_size = sizeof(flowroi_config);
    cfg->roi_q = 0.2f;
    cfg->scale_shift = 5;
    cfg->wavelet = FLOWROI_W53;
    cfg->dwt_levels = 3;
    cfg->pyr_levels = 3;
    cfg->iters = 3;
    cfg->win_r = 7;
    cfg->poly_n_half = 2;
    cfg->poly_sigma = 1.1f;
    cfg->lambda = 1e-3f;
    cfg->sal_weight = 0.7f;
    cfg->r_open = 1;
    cfg->r_close = 2;
    cfg->precision = FLOWROI_FP32;
    cfg->delta_base = 1.0f;
    cfg->max_batch_frames = 64;
    cfg->result_ring = 4;
    cfg->flags = 0;
    cfg->device = 0;
    cfg->hbm_budget_bytes = 0;
    cfg->denoise = 0;
    cfg->den_radius = 2;
    cfg->den_sigma_s = 2.0f;
    cfg->den_sigma_r = 20.0f;
    cfg->min_area = 0;
    cfg->adjacent = 0;
    cfg->register_frames = 0;
    cfg->reg_level = 2;
    cfg->codestream_bpp = 0.f;
    cfg->codestream_format = FLOWROI_CS_CONTAINER;
    cfg->codestream_reset = 0;
}

int flowroi_quant_steps(int levels, int bit_depth, float delta_base, float *delta, int32_t *eps, int32_t *mu,
                        double *gain_norm)
{
    if (quant_steps(levels, bit_depth, delta_base, delta, eps, mu, gain_norm) != 0)
        return fail(FLOWROI_EINVAL, "quantisation steps out of range for levels=%d bit_depth=%d", levels, bit_depth);
    return FLOWROI_OK;
}

int flowroi_create(const flowroi_config *cfg, flowroi_ctx **out)
{
    if (!out) return fail(FLOWROI_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_config(cfg);
    if (rc) return rc;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return cuda_fail(nullptr, e == cudaSuccess ? cudaErrorNoDevice : e, "no CUDA device");
    if (cfg->device < 0 || cfg->device >= ndev) return fail(FLOWROI_EINVAL, "config.device out of range");
    std::unique_ptr<flowroi_ctx> c(new flowroi_ctx);
    c->cfg = *cfg;
    c->device = cfg->device;
    c->half = cfg->precision == FLOWROI_FP16;
    c->plain = (cfg->flags & FLOWROI_PLAIN) != 0;
    c->keep = (cfg->flags & FLOWROI_KEEP_INTERMEDIATES) != 0;
    c->manual = (cfg->flags & FLOWROI_MANUAL) != 0;
    MethodConsts &mc = c->mc;
    std::memset(&mc, 0, sizeof mc);
    expansion_consts(cfg->poly_n_half, cfg->poly_sigma, mc);
    mc.pyr_levels = cfg->pyr_levels;
    mc.iters = cfg->iters;
    mc.win_r = cfg->win_r;
    mc.lambda = cfg->lambda;
    mc.alpha = cfg->sal_weight;
    mc.q = cfg->roi_q;
    mc.r_open = cfg->r_open;
    mc.r_close = cfg->r_close;
    mc.wavelet = cfg->wavelet;
    mc.dwt_levels = cfg->dwt_levels;
    mc.shift = cfg->scale_shift;
    mc.min_area = cfg->min_area;
    mc.reg_on = cfg->register_frames;
    mc.reg_level = cfg->reg_level;
    mc.denoise = cfg->denoise;
    mc.den_r = cfg->den_radius;
    const double log2e = 1.4426950408889634;
    for (int dy = -cfg->den_radius; dy <= cfg->den_radius; dy++)
        for (int dx = -cfg->den_radius; dx <= cfg->den_radius; dx++)
            mc.den_ls[(dy + kDenMaxR) * (2 * kDenMaxR + 1) + dx + kDenMaxR] =
                (float)(log2e * (double)(dx * dx + dy * dy) / (2.0 * (double)cfg->den_sigma_s * cfg->den_sigma_s));
    mc.den_lr = (float)(log2e / (2.0 * (double)cfg->den_sigma_r * cfg->den_sigma_r));
    for (int b = 0; b < kMaxSubbands; b++) mc.delta[b] = 1.f;
    if (cfg->wavelet == FLOWROI_W97 && quant_steps(cfg->dwt_levels, 12, cfg->delta_base, mc.delta, nullptr, nullptr, nullptr) != 0)
        return fail(FLOWROI_EINVAL, "config.delta_base gives quantisation steps out of range");
    for (int b = 0; b < kMaxSubbands; b++) mc.rdelta[b] = 1.f / mc.delta[b];  // IEEE float division: rounded to nearest

    flowroi_ctx *cp = c.get();
    CK(nullptr, cudaSetDevice(c->device));
    CK(nullptr, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    CK(nullptr, cudaStreamCreateWithFlags(&c->s_comp, cudaStreamNonBlocking));
    nvtxNameCudaStreamA(c->s_comp, "flowroi.compute");
    CK(nullptr, cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking));
    CK(nullptr, cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking));
    CK(nullptr, cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking));
    for (int k = 0; k < flowroi_ctx::kDesc; k++) {
        CK(nullptr, cudaMallocHost(reinterpret_cast<void **>(&c->desc_host[k]), sizeof(BatchDesc)));
        CK(nullptr, cudaMalloc(reinterpret_cast<void **>(&c->desc_dev[k]), sizeof(BatchDesc)));
        CK(nullptr, cudaEventCreateWithFlags(&c->desc_ev[k], cudaEventDisableTiming));
        std::memset(c->desc_host[k], 0, sizeof(BatchDesc));
    }
    CK(nullptr, cudaHostAlloc(reinterpret_cast<void **>(&c->err_host), sizeof(unsigned), cudaHostAllocMapped));
    *c->err_host = 0u;
    CK(nullptr, cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->err_dev), c->err_host, 0));
    if (!tma_available()) return fail(FLOWROI_EDEVICE, "cuTensorMapEncodeTiled is not available from the driver");
    if (cfg->tile_table) {
        std::string text, err;
        if (!read_text_file(cfg->tile_table, text)) return fail(FLOWROI_EINVAL, "config.tile_table: cannot read %s", cfg->tile_table);
        if (!tiles_parse(text.c_str(), c->tiles, err))
            return fail(FLOWROI_EINVAL, "config.tile_table %s: %s", cfg->tile_table, err.c_str());
    }
    c->cfg.tile_table = nullptr;  // the caller's string is not kept
    c->occ[TK_EXPAND] = occupancy_expand(c->half, cfg->poly_n_half);
    c->occ[TK_WINDOW] = occupancy_window(c->half, cfg->win_r);
    c->occ[TK_MASK] = occupancy_mask_kernels();
    apply_context_tiles(c.get());
    CK(nullptr, cudaGetLastError());
    c->grid_den = cfg->denoise ? std::max(1, occupancy_denoise(c->half, cfg->den_radius)) * c->num_sms : 0;
    c->grid_cc = cfg->min_area > 1 ? std::max(1, occupancy_cc()) * c->num_sms : 0;
    c->grid_mrg = 8 * c->num_sms;
    c->grid_reg = cfg->register_frames ? std::max(1, occupancy_register()) * c->num_sms : 0;
    c->grid_t1 = cfg->codestream_bpp > 0.f ? std::max(1, occupancy_t1()) * c->num_sms : 0;
    c->grid_mq = 4 * c->num_sms;
    c->grid_csc = 8 * c->num_sms;
    c->grid_frames = kMaxBatch;
    size_t freeb = 0, totalb = 0;
    CK(nullptr, cudaMemGetInfo(&freeb, &totalb));
    c->budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : (uint64_t)(0.8 * (double)freeb);
    if (!c->manual) c->sched = std::thread(scheduler_main, cp);
    *out = c.release();
    (void)cp;
    return FLOWROI_OK;
}

// Validates frame f of stream_id and enqueues its copy into the stream's
// ring (mu taken inside); *ev receives the copy's completion event.
static int submit_enqueue(flowroi_ctx *c, int64_t stream_id, const flowroi_frame *f, cudaEvent_t *ev)
{
    NvtxRange range("flowroi.submit");
    if (!f || f->struct_size != sizeof(flowroi_frame)) return fail(FLOWROI_EINVAL, "frame descriptor NULL or struct_size mismatch");
    if (c->poisoned) return fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
    if (f->dtype != FLOWROI_U8 && f->dtype != FLOWROI_U16) return fail(FLOWROI_EINVAL, "frame.dtype must be U8 or U16");
    const int bpp = f->dtype == FLOWROI_U8 ? 1 : 2;
    if (f->bit_depth < 1 || f->bit_depth > 8 * bpp) return fail(FLOWROI_EINVAL, "frame.bit_depth out of range for dtype");
    const int align = 1 << std::max(c->cfg.dwt_levels, c->cfg.pyr_levels - 1);
    if (f->width < 16 || f->height < 16 || f->width % align || f->height % align)
        return fail(FLOWROI_EINVAL, "frame %dx%d: width and height must be >= 16 and multiples of %d", f->width, f->height, align);
    if ((int64_t)f->width * f->height > (1LL << 28)) return fail(FLOWROI_EINVAL, "frame larger than 2^28 pixels");
    if (!f->data) return fail(FLOWROI_EINVAL, "frame.data is NULL");
    const int pitch = f->pitch_bytes ? f->pitch_bytes : f->width * bpp;
    if (pitch < f->width * bpp) return fail(FLOWROI_EINVAL, "frame.pitch_bytes smaller than a row");
    cudaSetDevice(c->device);

    Entry *e = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->streams.find(stream_id);
        Stream *s = nullptr;
        if (it == c->streams.end()) {
            std::unique_ptr<Stream> ns(new Stream);
            ns->id = stream_id;
            ns->W = f->width;
            ns->H = f->height;
            ns->bpp = bpp;
            ns->bit_depth = f->bit_depth;
            for (int r = 0; r < c->cfg.result_ring; r++) ns->ring.emplace_back(new Entry);
            const size_t bytes = plan_stream(c, ns.get(), nullptr);
            if (c->cfg.register_frames && (ns->reg_lnx > register_max_log() || ns->reg_lny > register_max_log()))
                return fail(FLOWROI_EINVAL, "frame %dx%d: pyramid level %d exceeds %d pixels per side for registration",
                            f->width, f->height, c->cfg.reg_level, 1 << register_max_log());
            if (c->admitted + bytes > c->budget) {
                c->refused++;
                return fail(FLOWROI_EBUSY, "stream %lld needs %zu bytes; %llu of %llu budget in use", (long long)stream_id, bytes,
                            (unsigned long long)c->admitted, (unsigned long long)c->budget);
            }
            if (c->cfg.wavelet == FLOWROI_W97 && quant_steps(c->cfg.dwt_levels, f->bit_depth, c->cfg.delta_base, nullptr, nullptr, nullptr, nullptr) != 0)
                return fail(FLOWROI_EINVAL, "bit depth %d gives quantisation exponents out of range", f->bit_depth);
            void *blk = nullptr;
            cudaError_t ae = cudaMallocAsync(&blk, bytes, c->s_copy);
            if (ae != cudaSuccess) {
                cudaGetLastError();
                return fail(FLOWROI_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(ae));
            }
            ns->block = static_cast<char *>(blk);
            ns->bytes = bytes;
            plan_stream(c, ns.get(), ns->block);
            if (!encode_stream_maps(c, ns.get())) {
                cudaFreeAsync(blk, c->s_copy);
                return fail(FLOWROI_EDEVICE, "TMA tensor map encoding failed");
            }
            for (auto &en : ns->ring) CK(c, cudaEventCreateWithFlags(&en->uploaded, cudaEventDisableTiming));
            c->admitted += bytes;
            logf("stream %lld admitted: %dx%d, %zu bytes (%llu of %llu in use)", (long long)stream_id, f->width,
                 f->height, bytes, (unsigned long long)c->admitted, (unsigned long long)c->budget);
            s = ns.get();
            c->streams[stream_id] = std::move(ns);
        } else {
            s = it->second.get();
            if (s->ending) return fail(FLOWROI_EINVAL, "stream %lld is ending", (long long)stream_id);
            if (s->W != f->width || s->H != f->height || s->bpp != bpp || s->bit_depth != f->bit_depth)
                return fail(FLOWROI_EINVAL, "stream %lld: frame geometry or format changed", (long long)stream_id);
            if (s->any_frame && f->frame_idx <= s->last_frame_idx)
                return fail(FLOWROI_EINVAL, "stream %lld: frame_idx %lld not after %lld", (long long)stream_id,
                            (long long)f->frame_idx, (long long)s->last_frame_idx);
        }
        const int64_t seq = s->next_seq;
        e = s->ring[seq % (int64_t)s->ring.size()].get();
        const int st = e->state.load();
        if ((st != E_EMPTY && st != E_DONE) || e->readers > 0)
            return fail(FLOWROI_EBUSY, "stream %lld: %zu frames not yet processed or being read", (long long)stream_id, s->ring.size());
        e->frame_idx = f->frame_idx;
        e->seq = seq;
        e->has_prev = seq > 0;
        e->t_submit = now_ms();
        e->t_done = 0.0;
        const cudaMemcpyKind kind = f->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (pitch == s->W * bpp)  // contiguous rows: one linear copy
            CK(c, cudaMemcpyAsync(e->raw, f->data, (size_t)s->W * bpp * s->H, kind, c->s_copy));
        else
            CK(c, cudaMemcpy2DAsync(e->raw, (size_t)s->W * bpp, f->data, pitch, (size_t)s->W * bpp, s->H, kind, c->s_copy));
        CK(c, cudaEventRecord(e->uploaded, c->s_copy));
        e->state.store(E_PENDING);
        s->draining = false;
        s->next_seq = seq + 1;
        s->last_frame_idx = f->frame_idx;
        s->any_frame = true;
        c->frames_submitted++;
    }
    *ev = e->uploaded;
    return FLOWROI_OK;
}

int flowroi_submit_frame(flowroi_ctx *c, int64_t stream_id, const flowroi_frame *f)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    cudaEvent_t ev = nullptr;
    const int rc = submit_enqueue(c, stream_id, f, &ev);
    if (rc != FLOWROI_OK) return rc;
    // The caller may reuse its buffer as soon as this returns.
    CK(c, cudaEventSynchronize(ev));
    if (!c->manual) wake_scheduler(c);
    return FLOWROI_OK;
}

int flowroi_submit_frames(flowroi_ctx *c, int n, const int64_t *stream_ids, const flowroi_frame *frames, int *status)
{
    if (status) *status = FLOWROI_OK;
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    if (n < 0 || (n > 0 && (!stream_ids || !frames))) return fail(FLOWROI_EINVAL, "n < 0 or a NULL array");
    cudaEvent_t last = nullptr;
    int k = 0;
    for (; k < n; k++) {
        cudaEvent_t ev = nullptr;
        const int rc = submit_enqueue(c, stream_ids[k], &frames[k], &ev);
        if (rc != FLOWROI_OK) {
            if (status) *status = rc;
            break;
        }
        last = ev;
    }
    // Every accepted copy is on the one copy stream: the last one's event
    // covers them all.  The caller may reuse those buffers once this returns.
    if (last) {
        const cudaError_t e = cudaEventSynchronize(last);
        if (e != cudaSuccess) {
            cuda_fail(c, e, "cudaEventSynchronize");
            if (status) *status = FLOWROI_EDEVICE;
            return k;
        }
    }
    if (k > 0 && !c->manual) wake_scheduler(c);
    return k;  // k < n: frames[k] failed with *status, flowroi_last_error says why
}

int flowroi_step(flowroi_ctx *c)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    cudaSetDevice(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    return step_locked(c);
}

int flowroi_get_mask(flowroi_ctx *c, int64_t stream_id, int64_t frame_idx, uint8_t *out, int out_on_device, int timeout_ms)
{
    if (c) cudaSetDevice(c->device);
    return get_common(c, stream_id, frame_idx, 0, out, out_on_device, timeout_ms);
}

int flowroi_get_coeffs(flowroi_ctx *c, int64_t stream_id, int64_t frame_idx, int32_t *out, int out_on_device, int timeout_ms)
{
    if (c) cudaSetDevice(c->device);
    return get_common(c, stream_id, frame_idx, -1, out, out_on_device, timeout_ms);
}

int flowroi_get_results(flowroi_ctx *c, int n, const int64_t *stream_ids, const int64_t *frame_idx, uint8_t *const *masks,
                        int32_t *const *coeffs, int out_on_device, int timeout_ms, int *status)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    if (n < 0 || (n > 0 && (!stream_ids || !frame_idx))) return fail(FLOWROI_EINVAL, "n < 0 or a NULL array");
    cudaSetDevice(c->device);
    std::vector<Entry *> held((size_t)n, nullptr);
    std::vector<size_t> npx((size_t)n, 0);
    std::vector<int> rc((size_t)n, FLOWROI_OK);
    // look up and hold every frame (its ring slot is not reused while held)
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (int k = 0; k < n; k++) {
            if (c->poisoned) {
                rc[(size_t)k] = fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
                continue;
            }
            auto it = c->streams.find(stream_ids[k]);
            if (it == c->streams.end()) {
                rc[(size_t)k] = fail(FLOWROI_ENOSTREAM, "unknown stream %lld", (long long)stream_ids[k]);
                continue;
            }
            Stream *s = it->second.get();
            Entry *e = find_entry(s, frame_idx[k]);
            if (!e) {
                rc[(size_t)k] = s->any_frame && frame_idx[k] <= s->last_frame_idx
                                    ? fail(FLOWROI_EGONE, "frame %lld of stream %lld is no longer held",
                                           (long long)frame_idx[k], (long long)stream_ids[k])
                                    : fail(FLOWROI_ENOSTREAM, "frame %lld of stream %lld was not submitted",
                                           (long long)frame_idx[k], (long long)stream_ids[k]);
                continue;
            }
            e->readers++;
            held[(size_t)k] = e;
            npx[(size_t)k] = (size_t)s->W * s->H;
        }
    }
    for (int k = 0; k < n; k++) {
        Entry *e = held[(size_t)k];
        if (e && !wait_done(c, e, timeout_ms))
            rc[(size_t)k] = c->poisoned ? fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str())
                                        : fail(FLOWROI_ETIMEDOUT, "frame %lld not finished within %d ms",
                                               (long long)frame_idx[k], timeout_ms);
    }
    {
        std::lock_guard<std::mutex> lk(c->d2h_mu);
        const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaError_t ce = cudaSuccess;
        int queued = 0;
        for (int k = 0; k < n && ce == cudaSuccess; k++) {
            Entry *e = held[(size_t)k];
            if (!e || rc[(size_t)k] != FLOWROI_OK) continue;
            if (masks && masks[k]) ce = cudaMemcpyAsync(masks[k], e->mask, npx[(size_t)k], kind, c->s_d2h), queued++;
            if (ce == cudaSuccess && coeffs && coeffs[k])
                ce = cudaMemcpyAsync(coeffs[k], e->coeffs, npx[(size_t)k] * 4, kind, c->s_d2h), queued++;
        }
        if (ce == cudaSuccess && queued) ce = cudaStreamSynchronize(c->s_d2h);
        if (ce != cudaSuccess) {
            const int code = cuda_fail(c, ce, "copy out");
            for (int k = 0; k < n; k++)
                if (held[(size_t)k] && rc[(size_t)k] == FLOWROI_OK) rc[(size_t)k] = code;
        }
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (Entry *e : held)
            if (e) e->readers--;
    }
    if (!c->manual) wake_scheduler(c);
    int first = FLOWROI_OK;
    for (int k = 0; k < n; k++) {
        if (status) status[k] = rc[(size_t)k];
        if (first == FLOWROI_OK) first = rc[(size_t)k];
    }
    return first;
}

int flowroi_get_intermediate(flowroi_ctx *c, int64_t stream_id, int64_t frame_idx, int which, void *out, int out_on_device,
                             int timeout_ms)
{
    if (which < FLOWROI_I_FLOW || which > FLOWROI_I_DRIFT) return fail(FLOWROI_EINVAL, "unknown intermediate %d", which);
    if (c) cudaSetDevice(c->device);
    return get_common(c, stream_id, frame_idx, which, out, out_on_device, timeout_ms);
}

int flowroi_flush(flowroi_ctx *c, int timeout_ms)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    cudaSetDevice(c->device);
    const double t0 = now_ms();
    int64_t target;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(c->mu);
            // the last adjacent-factor frames of every stream finish with the frames there are
            for (auto &kv : c->streams) kv.second->draining = true;
            if (c->manual) {
                for (;;) {
                    int n = step_locked(c);
                    if (n < 0) return n;
                    if (n == 0) break;
                    // two batches in flight at most; let the device drain
                    std::unique_lock<std::mutex> lk2(c->cmu);
                    c->ccv.wait_for(lk2, std::chrono::milliseconds(50), [&] { return c->inflight < c->max_inflight; });
                }
            }
            target = c->frames_submitted - c->frames_cancelled;
        }
        if (!c->manual) wake_scheduler(c);
        std::unique_lock<std::mutex> lk(c->cmu);
        c->ccv.wait_for(lk, std::chrono::milliseconds(10), [&] { return c->frames_done >= target || c->poisoned.load(); });
        if (c->poisoned) return fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
        if (c->frames_done >= target) {
            lk.unlock();
            std::lock_guard<std::mutex> lk3(c->mu);
            if (c->frames_submitted - c->frames_cancelled <= target) return FLOWROI_OK;
            continue;
        }
        lk.unlock();
        poll_device(c);
        if (timeout_ms >= 0 && now_ms() - t0 > timeout_ms) return fail(FLOWROI_ETIMEDOUT, "flush did not finish in %d ms", timeout_ms);
    }
}

int flowroi_end_stream(flowroi_ctx *c, int64_t stream_id)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    cudaSetDevice(c->device);
    Stream *s = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->streams.find(stream_id);
        if (it == c->streams.end()) return fail(FLOWROI_ENOSTREAM, "unknown stream %lld", (long long)stream_id);
        s = it->second.get();
        s->ending = true;
        s->draining = true;
        for (auto &e : s->ring)
            if (e->state.load() == E_PENDING) {
                e->state.store(E_EMPTY);
                c->frames_cancelled++;
            }
    }
    for (;;) {
        bool busy = false;
        {
            std::lock_guard<std::mutex> lk(c->mu);
            for (auto &e : s->ring)
                if (e->state.load() == E_LAUNCHED || e->readers > 0) busy = true;
            if (!busy) {
                if (c->poisoned) {
                    // leave the block to flowroi_destroy's device reset path
                } else {
                    cudaFreeAsync(s->block, c->s_comp);
                }
                for (auto &e : s->ring)
                    if (e->uploaded) cudaEventDestroy(e->uploaded);
                c->admitted -= s->bytes;
                c->streams.erase(stream_id);
                return FLOWROI_OK;
            }
        }
        if (c->cfg.adjacent > 0) {
            // frames still waiting for their merged mask: run their drain steps
            if (c->manual) {
                std::lock_guard<std::mutex> lk(c->mu);
                const int n = step_locked(c);
                if (n < 0) return n;
            } else {
                wake_scheduler(c);
            }
        }
        {
            std::unique_lock<std::mutex> lk(c->cmu);
            c->ccv.wait_for(lk, std::chrono::milliseconds(5));
        }
        poll_device(c);
        if (c->poisoned) return fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
    }
}

int flowroi_get_stats(flowroi_ctx *c, flowroi_stats *out)
{
    if (!c || !out) return fail(FLOWROI_EINVAL, "ctx or out is NULL");
    if (out->struct_size != sizeof(flowroi_stats)) return fail(FLOWROI_EINVAL, "stats.struct_size mismatch");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        out->frames_submitted = c->frames_submitted;
        out->streams_admitted = (int64_t)c->streams.size();
        out->bytes_admitted = c->admitted;
        out->budget_bytes = c->budget;
    }
    {
        std::lock_guard<std::mutex> lk(c->cmu);
        out->frames_done = c->frames_done;
        lat = c->lat_ms;
    }
    out->batches = c->batches;
    out->admissions_refused = c->refused;
    out->kernel_launches = c->launches;
    out->lat_p50_ms = out->lat_p99_ms = out->lat_mean_ms = 0.0;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double q) {
            const double pos = q * (double)(lat.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return i + 1 < lat.size() ? lat[i] * (1 - f) + lat[i + 1] * f : lat[i];
        };
        out->lat_p50_ms = pct(0.5);
        out->lat_p99_ms = pct(0.99);
        double s = 0;
        for (double v : lat) s += v;
        out->lat_mean_ms = s / (double)lat.size();
    }
    return FLOWROI_OK;
}

int flowroi_reset_stats(flowroi_ctx *c)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->cmu);
    c->lat_ms.clear();
    return FLOWROI_OK;
}

void flowroi_destroy(flowroi_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    {
        std::lock_guard<std::mutex> lk(c->cmu);
        c->shutdown = true;
    }
    c->ccv.notify_all();
    if (c->sched.joinable()) c->sched.join();
    cudaStreamSynchronize(c->s_comp);
    cudaStreamSynchronize(c->s_copy);
    cudaStreamSynchronize(c->s_d2h);
    for (auto &kv : c->streams) {
        cudaFreeAsync(kv.second->block, c->s_comp);
        for (auto &e : kv.second->ring)
            if (e->uploaded) cudaEventDestroy(e->uploaded);
    }
    cudaStreamSynchronize(c->s_comp);
    for (int k = 0; k < flowroi_ctx::kDesc; k++) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        if (c->desc_host[k]) cudaFreeHost(c->desc_host[k]);
        if (c->desc_dev[k]) cudaFree(c->desc_dev[k]);
        if (c->desc_ev[k]) cudaEventDestroy(c->desc_ev[k]);
    }
    if (c->err_host) cudaFreeHost(c->err_host);
    if (c->cs_stream) {
        cudaStreamSynchronize(c->cs_stream);
        cudaStreamDestroy(c->cs_stream);
    }
    if (c->cs_scratch) cudaFree(c->cs_scratch);
    cudaStreamDestroy(c->s_comp);
    cudaStreamDestroy(c->s_copy);
    cudaStreamDestroy(c->s_d2h);
    cudaStreamDestroy(c->s_cap);
    delete c;
}

int flowroi_compute_stream(flowroi_ctx *c, void **out)
{
    if (!c || !out) return fail(FLOWROI_EINVAL, "ctx or out is NULL");
    *out = (void *)c->s_comp;
    return FLOWROI_OK;
}

int flowroi_set_tiles(flowroi_ctx *c, const char *json)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    TileTable t;
    tiles_clear(t);
    std::string err;
    if (json && !tiles_parse(json, t, err)) return fail(FLOWROI_EINVAL, "tile table: %s", err.c_str());
    cudaSetDevice(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    // queued batches replay graphs captured with the old shapes: let them finish
    CK(c, cudaStreamSynchronize(c->s_comp));
    for (int g = 0; g < flowroi_ctx::kDesc; g++)
        if (c->graph[g]) {
            cudaGraphExecDestroy(c->graph[g]);
            c->graph[g] = nullptr;
        }
    c->tiles = t;
    apply_context_tiles(c);
    CK(c, cudaGetLastError());
    return FLOWROI_OK;
}

int flowroi_get_tiles(flowroi_ctx *c, char *out, uint64_t cap, uint64_t *out_len)
{
    if (!c || !out_len) return fail(FLOWROI_EINVAL, "ctx or out_len is NULL");
    std::string j;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        cudaDeviceProp prop;
        const bool named = cudaGetDeviceProperties(&prop, c->device) == cudaSuccess;
        j = tiles_json(c->tiles, named ? prop.name : nullptr);
    }
    *out_len = j.size();
    if (!out || cap < j.size() + 1) return fail(FLOWROI_ERANGE, "tile table of %zu bytes, cap is %llu", j.size(),
                                                (unsigned long long)cap);
    std::memcpy(out, j.c_str(), j.size() + 1);
    return FLOWROI_OK;
}

int flowroi_set_profiling(flowroi_ctx *c, int on)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (on == 2) c->prof_tot.clear();
    c->profiling = on != 0;
    return FLOWROI_OK;
}

int flowroi_get_kernel_times(flowroi_ctx *c, flowroi_kernel_time *out, int cap)
{
    if (!c || (!out && cap > 0)) return fail(FLOWROI_EINVAL, "ctx or out is NULL");
    cudaSetDevice(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    CK(c, cudaStreamSynchronize(c->s_comp));
    for (auto &r : c->prof_pending) {
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, r.a, r.b));
        auto &t = c->prof_tot[std::make_tuple(r.kid, r.level, r.iter)];
        t.first += 1;
        t.second += ms;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->prof_pending.clear();
    int n = 0;
    for (auto &kv : c->prof_tot) {
        if (n < cap) {
            flowroi_kernel_time &o = out[n];
            std::memset(&o, 0, sizeof o);
            snprintf(o.name, sizeof o.name, "%s", kKernelNames[std::get<0>(kv.first)]);
            o.level = std::get<1>(kv.first);
            o.iter = std::get<2>(kv.first);
            o.launches = kv.second.first;
            o.total_ms = kv.second.second;
        }
        n++;
    }
    return std::min(n, cap);
}

const char *flowroi_last_error(flowroi_ctx *c)
{
    (void)c;
    return g_err.c_str();
}

int flowroi_get_codestream(flowroi_ctx *c, int64_t stream_id, int64_t frame_idx, uint8_t *out, uint64_t out_cap,
                           uint64_t *out_len, int out_on_device, int timeout_ms)
{
    return get_common(c, stream_id, frame_idx, -2, out, out_on_device, timeout_ms, out_cap, out_len);
}

uint64_t flowroi_codestream_bound(int width, int height, int levels)
{
    if (levels < 1 || levels > kMaxLevels || width < 1 || height < 1 || width > 65535 || height > 65535 ||
        width % (1 << levels) || height % (1 << levels))
        return 0;
    const uint64_t ncb = (uint64_t)ebcot_codeblocks(width, height, levels);
    // the larger of the two formats' bounds (the codestream's)
    return (uint64_t)kJ2cHeader + ncb * ((uint64_t)kJ2cPerBlock + kCbBytes);
}

int flowroi_encode_codestreams(flowroi_ctx *c, int n, flowroi_cs_job *jobs, int on_device)
{
    if (!c) return fail(FLOWROI_EINVAL, "ctx is NULL");
    if (c->poisoned) return fail(FLOWROI_EDEVICE, "context poisoned: %s", c->poison_msg.c_str());
    if (n < 1 || n > kMaxBatch || !jobs) return fail(FLOWROI_EINVAL, "n must be in [1,64] and jobs non-NULL");
    std::vector<CsFrame> fr((size_t)n);
    int ncb = 0;
    size_t coef_bytes = 0, out_bytes = 0;
    bool any_reset = false, any_carry = false;  // code-block styles present: the launches they need
    for (int i = 0; i < n; i++) {
        const flowroi_cs_job &J = jobs[i];
        if (!J.coeffs || !J.out) return fail(FLOWROI_EINVAL, "job %d: coeffs and out must be non-NULL", i);
        if (flowroi_codestream_bound(J.width, J.height, J.levels) == 0)
            return fail(FLOWROI_EINVAL, "job %d: width/height must be in [1,65535], multiples of 2^levels, levels in [1,8]", i);
        if (J.wavelet != FLOWROI_W53 && J.wavelet != FLOWROI_W97) return fail(FLOWROI_EINVAL, "job %d: wavelet must be 53 or 97", i);
        if (J.shift < 0 || J.shift > 15 || J.bit_depth < 1 || J.bit_depth > 16)
            return fail(FLOWROI_EINVAL, "job %d: shift must be in [0,15] and bit_depth in [1,16]", i);
        CsFrame &F = fr[(size_t)i];
        F.coef = J.coeffs;
        F.out = J.out;
        F.cap = (long long)std::min<uint64_t>(J.out_cap, (uint64_t)INT64_MAX);
        F.budget = J.budget_bytes;
        F.w = J.width;
        F.h = J.height;
        F.levels = J.levels;
        F.wavelet = J.wavelet;
        F.shift = J.shift;
        F.bit_depth = J.bit_depth;
        if (J.format != FLOWROI_CS_CONTAINER && J.format != FLOWROI_CS_J2C)
            return fail(FLOWROI_EINVAL, "job %d: format must be FLOWROI_CS_CONTAINER or FLOWROI_CS_J2C", i);
        F.format = J.format;
        if (J.reset != 0 && J.reset != 1) return fail(FLOWROI_EINVAL, "job %d: reset must be 0 or 1", i);
        F.reset = J.reset;
        (J.reset ? any_reset : any_carry) = true;
        if (J.format == FLOWROI_CS_J2C && !band_exponents(J.levels, J.wavelet, J.bit_depth, c->cfg.delta_base, F.eps, F.mu))
            return fail(FLOWROI_EINVAL, "job %d: quantisation steps out of range for bit_depth %d", i, J.bit_depth);
        F.cb0 = ncb;
        F.ncb = ebcot_codeblocks(J.width, J.height, J.levels);
        ncb += F.ncb;
        coef_bytes += (size_t)J.width * J.height * sizeof(int32_t);
        out_bytes += (size_t)J.out_cap;
    }
    // scratch: one allocation carved in 256-byte aligned pieces
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t at = total;
        total += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_frames = take(sizeof(CsFrame) * (size_t)n), o_job = take(sizeof(CsJob));
    const size_t o_bytes = take((size_t)ncb * kCbRegion);
    const size_t o_plen = take((size_t)ncb * kMaxPasses * sizeof(int32_t));
    const size_t o_nsym = take((size_t)ncb * kMaxPasses * sizeof(int32_t));
    const size_t o_ptab = take((size_t)ncb * kMaxPasses * sizeof(int4));
    const size_t o_mqs = take((size_t)ncb * kMaxPasses * kMqWords * sizeof(uint32_t));
    const size_t o_sym = take((size_t)ncb * kSymCap);
    const size_t o_dist = take((size_t)ncb * kMaxPasses * sizeof(double));
    const size_t o_info = take((size_t)ncb * kCbInfo * sizeof(int32_t));
    const size_t o_hk = take((size_t)ncb * (kMaxPasses + 1) * sizeof(int32_t));
    const size_t o_hs = take((size_t)ncb * (kMaxPasses + 1) * sizeof(double));
    const size_t o_flen = take((size_t)n * sizeof(long long)), o_err = take(5 * sizeof(unsigned));
    const size_t o_coef = on_device ? 0 : take(coef_bytes), o_out = on_device ? 0 : take(out_bytes);

    int rc = FLOWROI_OK;
    std::lock_guard<std::mutex> lk(c->cs_mu);
    CK(c, cudaSetDevice(c->device));
    if (!c->cs_stream) CK(c, cudaStreamCreateWithFlags(&c->cs_stream, cudaStreamNonBlocking));
    cudaStream_t st = c->cs_stream;
    if (c->cs_bytes < total) {
        if (c->cs_scratch) cudaFree(c->cs_scratch);
        c->cs_scratch = nullptr;
        c->cs_bytes = 0;
        if (cudaMalloc(&c->cs_scratch, total) != cudaSuccess) {
            cudaGetLastError();
            c->cs_scratch = nullptr;
            return fail(FLOWROI_ENOMEM, "codestream scratch of %zu bytes", total);
        }
        c->cs_bytes = total;
    }
    unsigned char *dev = c->cs_scratch;
    std::vector<long long> flen((size_t)n, 0);
    unsigned err = 0;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    if (!on_device) {
        size_t co = 0, oo = 0;
        for (int i = 0; i < n; i++) {
            const size_t cb = (size_t)fr[(size_t)i].w * fr[(size_t)i].h * sizeof(int32_t);
            step(cudaMemcpyAsync(dev + o_coef + co, jobs[i].coeffs, cb, cudaMemcpyHostToDevice, st));
            fr[(size_t)i].coef = reinterpret_cast<const int32_t *>(dev + o_coef + co);
            fr[(size_t)i].out = dev + o_out + oo;
            co += cb;
            oo += (size_t)jobs[i].out_cap;
        }
    }
    for (int i = 0; i < n; i++) {
        CsFrame &F = fr[(size_t)i];
        const size_t b0 = (size_t)F.cb0;
        F.cbytes = dev + o_bytes + b0 * kCbRegion;
        F.plen = reinterpret_cast<int32_t *>(dev + o_plen) + b0 * kMaxPasses;
        F.nsym = reinterpret_cast<int32_t *>(dev + o_nsym) + b0 * kMaxPasses;
        F.ptab = reinterpret_cast<int4 *>(dev + o_ptab) + b0 * kMaxPasses;
        F.mqs = reinterpret_cast<uint32_t *>(dev + o_mqs) + b0 * kMaxPasses * kMqWords;
        F.sym = dev + o_sym + b0 * kSymCap;
        F.dist = reinterpret_cast<double *>(dev + o_dist) + b0 * kMaxPasses;
        F.info = reinterpret_cast<int32_t *>(dev + o_info) + b0 * kCbInfo;
        F.hk = reinterpret_cast<int32_t *>(dev + o_hk) + b0 * (kMaxPasses + 1);
        F.hs = reinterpret_cast<double *>(dev + o_hs) + b0 * (kMaxPasses + 1);
        F.flen = reinterpret_cast<long long *>(dev + o_flen) + i;
    }
    CsJob job{};
    job.nframes = n;
    job.ncb = ncb;
    job.frames = reinterpret_cast<const CsFrame *>(dev + o_frames);
    job.cbcap = kCbBytes;
    job.err = reinterpret_cast<unsigned *>(dev + o_err);
    job.next = reinterpret_cast<int *>(dev + o_err) + 1;
    step(cudaMemcpyAsync(dev + o_frames, fr.data(), sizeof(CsFrame) * (size_t)n, cudaMemcpyHostToDevice, st));
    step(cudaMemcpyAsync(dev + o_job, &job, sizeof job, cudaMemcpyHostToDevice, st));
    step(cudaMemsetAsync(dev + o_err, 0, 5 * sizeof(unsigned), st));
    if (e == cudaSuccess) {
        launch_ebcot(reinterpret_cast<const CsJob *>(dev + o_job), n, ncb, any_carry, any_reset, st);
        step(cudaGetLastError());
    }
    step(cudaMemcpyAsync(flen.data(), dev + o_flen, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToHost, st));
    step(cudaMemcpyAsync(&err, dev + o_err, sizeof err, cudaMemcpyDeviceToHost, st));
    step(cudaStreamSynchronize(st));
    if (e == cudaSuccess && !on_device) {
        size_t oo = 0;
        for (int i = 0; i < n; i++) {
            if (flen[(size_t)i] > 0)
                step(cudaMemcpyAsync(jobs[i].out, dev + o_out + oo, (size_t)flen[(size_t)i], cudaMemcpyDeviceToHost, st));
            oo += (size_t)jobs[i].out_cap;
        }
        step(cudaStreamSynchronize(st));
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "flowroi_encode_codestreams");
    for (int i = 0; i < n; i++) {
        const long long L = flen[(size_t)i];
        jobs[i].out_len = (uint64_t)(L == -1 ? 0 : (L < 0 ? -L : L));
        if (L == -1 && rc == FLOWROI_OK)
            rc = fail(FLOWROI_ERANGE, "job %d: a coefficient magnitude of 2^24 or more, or a code-block over %d bytes", i, kCbBytes);
        else if (L < 0 && rc == FLOWROI_OK)
            rc = fail(FLOWROI_ERANGE, "job %d: container needs %lld bytes, out_cap is %llu", i, -L,
                      (unsigned long long)jobs[i].out_cap);
    }
    if (rc == FLOWROI_OK && err != 0)
        rc = fail(FLOWROI_ERANGE, "a code-block has a magnitude of 2^24 or more, or exceeded %d bytes", kCbBytes);
    return rc;
}

}  // extern "C"
