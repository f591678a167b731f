// Tile table (see tiles.h): defaults, JSON form, and the search that
// chooses it (flowroi_autotune).
//
// The search is a coordinate descent on measured kernel time: for each
// tunable in turn, every candidate value is set on a live context (run with
// per-kernel CUDA-event timing, which launches kernels directly, so grid
// sizes and tile shapes change between steps without graph captures), a
// few steps of synthetic frames run, the summed device time of the kernels
// the tunable affects is read back, and the fastest value is kept before
// the next tunable is searched.  Per-frame tunables are searched for every
// requested frame size (its width class); per-context ones on the largest.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/flowroi.h"
#include "kernels.h"
#include "tiles.h"

namespace flowroi {

int width_class(int w)
{
    int c = 0;
    while (c < kWClasses - 1 && w > (256 << c)) c++;
    return c;
}

int class_width(int c) { return 256 << c; }

const char *tile_kernel_name(int k)
{
    static const char *const n[TK_COUNT] = {"expand", "update", "window", "mask", "dwt"};
    return k >= 0 && k < TK_COUNT ? n[k] : "?";
}

void tiles_clear(TileTable &t) { std::memset(&t, 0, sizeof t); }

int tiles_dwt_seg(const TileTable &t, bool half, int W, int level, int bw, int bh)
{
    const int v = t.dwt_seg[half][width_class(W)][level - 1];
    return v > 0 ? v : dwt_default_seg(bw, bh);
}

int tiles_saliency_strips(const TileTable &t, bool half, int W)
{
    const int v = t.saliency_rows[half][width_class(W)];
    return v > 0 ? v / kSalSub : 4;
}

namespace {

// ------------------------------------------------------------- JSON reader
// Objects, arrays, strings (no escapes beyond \" \\ \/), numbers, true,
// false, null; nesting at most 8 deep.
struct JVal {
    enum Kind { Null, Bool, Num, Str, Arr, Obj } kind = Null;
    double num = 0.0;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
};

struct JParser {
    const char *p;
    std::string err;
    void ws()
    {
        while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') p++;
    }
    bool fail(const char *m)
    {
        if (err.empty()) err = m;
        return false;
    }
    bool str(std::string &out)
    {
        if (*p != '"') return fail("expected a string");
        p++;
        out.clear();
        while (*p && *p != '"') {
            if (*p == '\\') {
                p++;
                if (*p != '"' && *p != '\\' && *p != '/') return fail("unsupported string escape");
            }
            if ((unsigned char)*p < 0x20) return fail("control character in a string");
            out.push_back(*p++);
        }
        if (*p != '"') return fail("unterminated string");
        p++;
        return true;
    }
    bool value(JVal &v, int depth)
    {
        if (depth > 8) return fail("nesting too deep");
        ws();
        if (*p == '{') {
            p++;
            v.kind = JVal::Obj;
            ws();
            if (*p == '}') {
                p++;
                return true;
            }
            for (;;) {
                ws();
                std::string k;
                if (!str(k)) return false;
                ws();
                if (*p != ':') return fail("expected ':'");
                p++;
                JVal x;
                if (!value(x, depth + 1)) return false;
                v.obj.emplace_back(std::move(k), std::move(x));
                ws();
                if (*p == ',') {
                    p++;
                    continue;
                }
                if (*p == '}') {
                    p++;
                    return true;
                }
                return fail("expected ',' or '}'");
            }
        }
        if (*p == '[') {
            p++;
            v.kind = JVal::Arr;
            ws();
            if (*p == ']') {
                p++;
                return true;
            }
            for (;;) {
                JVal x;
                if (!value(x, depth + 1)) return false;
                v.arr.push_back(std::move(x));
                ws();
                if (*p == ',') {
                    p++;
                    continue;
                }
                if (*p == ']') {
                    p++;
                    return true;
                }
                return fail("expected ',' or ']'");
            }
        }
        if (*p == '"') {
            v.kind = JVal::Str;
            return str(v.str);
        }
        if (!std::strncmp(p, "true", 4) || !std::strncmp(p, "false", 5)) {
            v.kind = JVal::Bool;
            v.num = *p == 't' ? 1.0 : 0.0;
            p += *p == 't' ? 4 : 5;
            return true;
        }
        if (!std::strncmp(p, "null", 4)) {
            p += 4;
            return true;
        }
        if (*p == '-' || std::isdigit((unsigned char)*p)) {
            char *e = nullptr;
            v.num = std::strtod(p, &e);
            if (e == p) return fail("bad number");
            v.kind = JVal::Num;
            p = e;
            return true;
        }
        return fail("unexpected character");
    }
};

const JVal *member(const JVal &o, const char *k)
{
    for (auto &kv : o.obj)
        if (kv.first == k) return &kv.second;
    return nullptr;
}

bool as_int(const JVal *v, int &out)
{
    if (!v || v->kind != JVal::Num || v->num != std::floor(v->num) || std::fabs(v->num) > 1e9) return false;
    out = (int)v->num;
    return true;
}

}  // namespace

bool tiles_parse(const char *json, TileTable &t, std::string &err)
{
    if (!json) {
        err = "table text is NULL";
        return false;
    }
    JParser ps{json, {}};
    JVal root;
    if (!ps.value(root, 0)) {
        err = "malformed JSON: " + ps.err;
        return false;
    }
    ps.ws();
    if (*ps.p) {
        err = "malformed JSON: text after the table";
        return false;
    }
    if (root.kind != JVal::Obj) {
        err = "the table must be a JSON object";
        return false;
    }
    const JVal *fmt = member(root, "format");
    if (!fmt || fmt->kind != JVal::Str || fmt->str != "flowroi-tiles-1") {
        err = "format must be \"flowroi-tiles-1\"";
        return false;
    }
    for (auto &kv : root.obj)
        if (kv.first != "format" && kv.first != "device" && kv.first != "note" && kv.first != "entries") {
            err = "unknown key \"" + kv.first + "\"";
            return false;
        }
    const JVal *ents = member(root, "entries");
    if (!ents || ents->kind != JVal::Arr) {
        err = "entries must be an array";
        return false;
    }
    TileTable n = t;
    int idx = 0;
    for (const JVal &e : ents->arr) {
        char where[64];
        snprintf(where, sizeof where, "entry %d: ", idx++);
        if (e.kind != JVal::Obj) {
            err = std::string(where) + "not an object";
            return false;
        }
        for (auto &kv : e.obj)
            if (kv.first != "param" && kv.first != "w" && kv.first != "storage" && kv.first != "level" &&
                kv.first != "kernel" && kv.first != "value" && kv.first != "ms") {
                err = std::string(where) + "unknown key \"" + kv.first + "\"";
                return false;
            }
        const JVal *pv = member(e, "param");
        if (!pv || pv->kind != JVal::Str) {
            err = std::string(where) + "param must be a string";
            return false;
        }
        const std::string &param = pv->str;
        int storage = 0, value = 0;
        if (!as_int(member(e, "storage"), storage) || (storage != 32 && storage != 16)) {
            err = std::string(where) + "storage must be 32 or 16";
            return false;
        }
        if (!as_int(member(e, "value"), value)) {
            err = std::string(where) + "value must be an integer";
            return false;
        }
        const int sh = storage == 16 ? 1 : 0;
        auto wclass = [&](int &c) {
            int w = 0;
            if (!as_int(member(e, "w"), w)) return false;
            for (c = 0; c < kWClasses; c++)
                if (class_width(c) == w) return true;
            return false;
        };
        int c = 0;
        if (param == "dwt_seg") {
            int level = 0;
            if (!wclass(c)) {
                err = std::string(where) + "w must be 256, 512, 1024, 2048, 4096 or 8192";
                return false;
            }
            if (!as_int(member(e, "level"), level) || level < 1 || level > kMaxLevels) {
                err = std::string(where) + "level must be in [1, 8]";
                return false;
            }
            if (value < 4 || value > 256) {
                err = std::string(where) + "dwt_seg must be in [4, 256]";
                return false;
            }
            n.dwt_seg[sh][c][level - 1] = value;
        } else if (param == "saliency_rows") {
            if (!wclass(c)) {
                err = std::string(where) + "w must be 256, 512, 1024, 2048, 4096 or 8192";
                return false;
            }
            if (value < kSalSub || value > 16 * kSalSub || value % kSalSub) {
                err = std::string(where) + "saliency_rows must be a multiple of 8 up to 128";
                return false;
            }
            n.saliency_rows[sh][c] = value;
        } else if (param == "update_rows") {
            if (value != 4 && value != 8 && value != 16 && value != 32) {
                err = std::string(where) + "update_rows must be 4, 8, 16 or 32";
                return false;
            }
            n.update_rows[sh] = value;
        } else if (param == "blocks_per_sm") {
            const JVal *kn = member(e, "kernel");
            int k = -1;
            for (int i = 0; i < TK_COUNT && kn && kn->kind == JVal::Str; i++)
                if (kn->str == tile_kernel_name(i)) k = i;
            if (k < 0) {
                err = std::string(where) + "kernel must be expand, update, window, mask or dwt";
                return false;
            }
            if (value < 1 || value > 32) {
                err = std::string(where) + "blocks_per_sm must be in [1, 32]";
                return false;
            }
            n.blocks_per_sm[sh][k] = value;
        } else if (param == "dwt_variant") {
            if (value != 5 && value != 6) {
                err = std::string(where) + "dwt_variant must be 5 or 6";
                return false;
            }
            n.dwt_variant[sh] = value;
        } else {
            err = std::string(where) + "unknown param \"" + param + "\"";
            return false;
        }
    }
    t = n;
    return true;
}

std::string tiles_json(const TileTable &t, const char *device_name)
{
    std::string s = "{\n  \"format\": \"flowroi-tiles-1\",\n";
    if (device_name) {
        std::string d;
        for (const char *q = device_name; *q; q++)
            if (*q != '"' && *q != '\\' && (unsigned char)*q >= 0x20) d.push_back(*q);
        s += "  \"device\": \"" + d + "\",\n";
    }
    s += "  \"entries\": [";
    bool first = true;
    char buf[192];
    auto add = [&](const char *txt) {
        s += first ? "\n    " : ",\n    ";
        s += txt;
        first = false;
    };
    for (int sh = 0; sh < 2; sh++) {
        const int st = sh ? 16 : 32;
        for (int c = 0; c < kWClasses; c++) {
            for (int l = 0; l < kMaxLevels; l++)
                if (t.dwt_seg[sh][c][l]) {
                    snprintf(buf, sizeof buf, "{\"param\": \"dwt_seg\", \"w\": %d, \"storage\": %d, \"level\": %d, \"value\": %d}",
                             class_width(c), st, l + 1, t.dwt_seg[sh][c][l]);
                    add(buf);
                }
            if (t.saliency_rows[sh][c]) {
                snprintf(buf, sizeof buf, "{\"param\": \"saliency_rows\", \"w\": %d, \"storage\": %d, \"value\": %d}",
                         class_width(c), st, t.saliency_rows[sh][c]);
                add(buf);
            }
        }
        for (int k = 0; k < TK_COUNT; k++)
            if (t.blocks_per_sm[sh][k]) {
                snprintf(buf, sizeof buf, "{\"param\": \"blocks_per_sm\", \"kernel\": \"%s\", \"storage\": %d, \"value\": %d}",
                         tile_kernel_name(k), st, t.blocks_per_sm[sh][k]);
                add(buf);
            }
        if (t.update_rows[sh]) {
            snprintf(buf, sizeof buf, "{\"param\": \"update_rows\", \"storage\": %d, \"value\": %d}", st, t.update_rows[sh]);
            add(buf);
        }
        if (t.dwt_variant[sh]) {
            snprintf(buf, sizeof buf, "{\"param\": \"dwt_variant\", \"storage\": %d, \"value\": %d}", st, t.dwt_variant[sh]);
            add(buf);
        }
    }
    s += first ? "]\n}\n" : "\n  ]\n}\n";
    return s;
}

namespace {

// ------------------------------------------------------------- the search

// Synthetic 12-bit frames for timing: a texture moving by (1.5, -0.8) px
// per frame with a per-stream phase, plus hashed noise.  The kernels' time
// does not depend on the content beyond the radix select's candidate count,
// which any textured, moving content keeps typical.
__global__ void k_tune_frame(uint16_t *out, int w, int h, int t, int s)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= w || y >= h) return;
    const float fx = (float)x - 1.5f * (float)t + 17.f * (float)s, fy = (float)y + 0.8f * (float)t;
    const float v = 1200.f + 900.f * __sinf(fx * 0.17f) * __sinf(fy * 0.11f) + 400.f * __sinf((fx + fy) * 0.031f);
    uint32_t hsh = (uint32_t)x * 73856093u ^ (uint32_t)y * 19349663u ^ (uint32_t)(t * 83492791 + s);
    hsh ^= hsh >> 13;
    hsh *= 0x5bd1e995u;
    hsh ^= hsh >> 15;
    const float n = (float)(hsh & 63u) - 32.f;
    out[(size_t)y * w + x] = (uint16_t)fminf(4095.f, fmaxf(0.f, v + n));
}

struct Tuner {
    const flowroi_config *cfg;
    int streams, steps;
    bool half;
    TileTable best;
    std::string device;
    std::string err;

    struct Run {
        flowroi_ctx *ctx = nullptr;
        uint16_t *frames = nullptr;
        int w = 0, h = 0, t = 0;
        ~Run()
        {
            if (ctx) flowroi_destroy(ctx);
            if (frames) cudaFree(frames);
        }
    };

    bool setup(Run &r, int w, int h)
    {
        flowroi_config c2 = *cfg;
        c2.flags = (cfg->flags | FLOWROI_MANUAL) & ~(unsigned)(FLOWROI_PLAIN | FLOWROI_KEEP_INTERMEDIATES | FLOWROI_TEST_EXPIRE_TMA |
                                                             FLOWROI_TEST_EXPIRE_LOOP);
        c2.tile_table = nullptr;
        c2.max_batch_frames = std::max(cfg->max_batch_frames, streams);
        c2.codestream_bpp = 0.f;
        if (flowroi_create(&c2, &r.ctx) != FLOWROI_OK) {
            err = std::string("flowroi_create: ") + flowroi_last_error(nullptr);
            return false;
        }
        r.w = w;
        r.h = h;
        if (cudaMalloc(&r.frames, (size_t)streams * w * h * sizeof(uint16_t)) != cudaSuccess) {
            err = "cudaMalloc of the synthetic frames failed";
            return false;
        }
        return apply(r) && flowroi_set_profiling(r.ctx, 2) == FLOWROI_OK && advance(r, 2);
    }

    bool apply(Run &r)
    {
        const std::string j = tiles_json(best, nullptr);
        if (flowroi_set_tiles(r.ctx, j.c_str()) != FLOWROI_OK) {
            err = std::string("flowroi_set_tiles: ") + flowroi_last_error(r.ctx);
            return false;
        }
        return true;
    }

    // n steps: the next frame of every stream, one batch each.
    bool advance(Run &r, int n)
    {
        for (int k = 0; k < n; k++, r.t++) {
            for (int s = 0; s < streams; s++)
                k_tune_frame<<<dim3((r.w + 255) / 256, r.h), 256>>>(r.frames + (size_t)s * r.w * r.h, r.w, r.h, r.t, s);
            if (cudaDeviceSynchronize() != cudaSuccess) {
                err = "synthetic frame generation failed";
                return false;
            }
            for (int s = 0; s < streams; s++) {
                flowroi_frame f;
                std::memset(&f, 0, sizeof f);
                f.struct_size = sizeof f;
                f.width = r.w;
                f.height = r.h;
                f.dtype = FLOWROI_U16;
                f.bit_depth = 12;
                f.frame_idx = r.t;
                f.data = r.frames + (size_t)s * r.w * r.h;
                f.data_on_device = 1;
                if (flowroi_submit_frame(r.ctx, 1000 + s, &f) != FLOWROI_OK) {
                    err = std::string("flowroi_submit_frame: ") + flowroi_last_error(r.ctx);
                    return false;
                }
            }
            if (flowroi_flush(r.ctx, 120000) != FLOWROI_OK) {
                err = std::string("flowroi_flush: ") + flowroi_last_error(r.ctx);
                return false;
            }
        }
        return true;
    }

    // Device time (ms, summed over `steps` steps) of the kernels named in
    // `names` (level < 0: every level).
    bool measure(Run &r, const std::vector<std::pair<const char *, int>> &names, double &ms)
    {
        if (!apply(r) || flowroi_set_profiling(r.ctx, 2) != FLOWROI_OK || !advance(r, steps)) return false;
        std::vector<flowroi_kernel_time> kt(512);
        const int n = flowroi_get_kernel_times(r.ctx, kt.data(), (int)kt.size());
        if (n < 0) {
            err = std::string("flowroi_get_kernel_times: ") + flowroi_last_error(r.ctx);
            return false;
        }
        ms = 0.0;
        for (int i = 0; i < std::min(n, (int)kt.size()); i++)
            for (auto &nm : names)
                if (!std::strcmp(kt[i].name, nm.first) && (nm.second < 0 || kt[i].level == nm.second)) ms += kt[i].total_ms;
        return true;
    }

    // Tries every candidate of one tunable (set(v) writes it into `best`):
    // kRounds interleaved rounds over the candidates, each candidate's
    // steps after one untimed step on its shapes, and a candidate's time
    // the least over the rounds, so that a clock still ramping during one
    // candidate's turn does not decide.
    static constexpr int kRounds = 2;
    template <class Set>
    bool search(Run &r, const std::vector<int> &cands, const std::vector<std::pair<const char *, int>> &names, Set set)
    {
        if (cands.size() < 2) {
            if (!cands.empty()) set(cands[0]);
            return true;
        }
        std::vector<double> t(cands.size(), 1e300);
        for (int round = 0; round < kRounds; round++)
            for (size_t i = 0; i < cands.size(); i++) {
                set(cands[i]);
                double ms = 0.0;
                if (!apply(r) || !advance(r, 1) || !measure(r, names, ms)) return false;
                t[i] = std::min(t[i], ms);
            }
        set(cands[std::min_element(t.begin(), t.end()) - t.begin()]);
        return true;
    }

    bool per_frame(int w, int h)
    {
        Run r;
        if (!setup(r, w, h)) return false;
        const int c = width_class(w), sh = half ? 1 : 0;
        for (int l = 1; l <= cfg->dwt_levels; l++) {
            const int bh = h >> l;
            std::vector<int> cands;
            // fine steps: the unit count against the resident warps decides
            // how full the last wave of units is
            for (int v : {8, 10, 12, 14, 16, 18, 20, 22, 24, 28, 32, 40, 48, 64})
                if (v <= std::max(8, bh)) cands.push_back(v);
            if (!search(r, cands, {{"dwt", l}}, [&](int v) { best.dwt_seg[sh][c][l - 1] = v; })) return false;
        }
        if (!search(r, {8, 16, 32, 64}, {{"saliency", -1}}, [&](int v) { best.saliency_rows[sh][c] = v; })) return false;
        return true;
    }

    bool per_context(int w, int h)
    {
        Run r;
        if (!setup(r, w, h)) return false;
        const int sh = half ? 1 : 0;
        if (!search(r, {5, 6}, {{"dwt", -1}}, [&](int v) { best.dwt_variant[sh] = v; })) return false;
        if (!search(r, {4, 8, 16, 32}, {{"update", -1}}, [&](int v) { best.update_rows[sh] = v; })) return false;
        const int occ[TK_COUNT] = {occupancy_expand(half, cfg->poly_n_half),
                                   occupancy_update(half, best.update_rows[sh] ? best.update_rows[sh] : kUpdRows),
                                   occupancy_window(half, cfg->win_r), occupancy_mask_kernels(),
                                   occupancy_dwt(cfg->wavelet, best.dwt_variant[sh] ? best.dwt_variant[sh] : 5)};
        const std::vector<std::pair<const char *, int>> names[TK_COUNT] = {
            {{"expand", -1}}, {{"update", -1}}, {{"window", -1}}, {{"saliency", -1}, {"select_pass", -1}, {"morph", -1}}, {{"dwt", -1}}};
        for (int k = 0; k < TK_COUNT; k++) {
            std::vector<int> cands;
            for (int v : {occ[k], occ[k] - 1, occ[k] / 2})
                if (v >= 1 && std::find(cands.begin(), cands.end(), v) == cands.end()) cands.push_back(v);
            if (!search(r, cands, names[k], [&](int v) { best.blocks_per_sm[sh][k] = v; })) return false;
        }
        return true;
    }
};

}  // namespace
}  // namespace flowroi

using namespace flowroi;

extern "C" int flowroi_tiles_check(const char *json, char *err, uint64_t err_cap)
{
    TileTable t;
    tiles_clear(t);
    std::string e;
    const bool ok = tiles_parse(json, t, e);
    if (err && err_cap > 0) snprintf(err, (size_t)err_cap, "%s", ok ? "" : e.c_str());
    return ok ? FLOWROI_OK : FLOWROI_EINVAL;
}

extern "C" int flowroi_autotune(const flowroi_config *cfg, int nsizes, const int *widths, const int *heights, int streams,
                                int steps, char *out, uint64_t out_cap, uint64_t *out_len)
{
    if (!cfg || cfg->struct_size != sizeof(flowroi_config) || nsizes < 1 || nsizes > 16 || !widths || !heights || !out_len)
        return FLOWROI_EINVAL;
    if (streams < 1 || streams > kMaxBatch || steps < 1 || steps > 100) return FLOWROI_EINVAL;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return FLOWROI_EDEVICE;
    Tuner tu;
    tu.cfg = cfg;
    tu.streams = streams;
    tu.steps = steps;
    tu.half = cfg->precision == FLOWROI_FP16;
    tiles_clear(tu.best);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, cfg->device) == cudaSuccess) tu.device = prop.name;
    int big = 0;
    for (int i = 0; i < nsizes; i++) {
        if (widths[i] < 16 || heights[i] < 16) return FLOWROI_EINVAL;
        if ((int64_t)widths[i] * heights[i] > (int64_t)widths[big] * heights[big]) big = i;
    }
    // per-context shapes first (on the largest frames), then every size's own
    bool ok = tu.per_context(widths[big], heights[big]);
    for (int i = 0; ok && i < nsizes; i++) ok = tu.per_frame(widths[i], heights[i]);
    if (!ok) {
        fprintf(stderr, "flowroi_autotune: %s\n", tu.err.c_str());
        return FLOWROI_EDEVICE;
    }
    const std::string j = tiles_json(tu.best, tu.device.c_str());
    *out_len = j.size();
    if (!out || out_cap < j.size() + 1) return FLOWROI_ERANGE;
    std::memcpy(out, j.c_str(), j.size() + 1);
    return FLOWROI_OK;
}
