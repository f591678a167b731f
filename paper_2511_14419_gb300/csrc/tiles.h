// Tile table: the launch and tile shapes the kernels run with, per frame
// width class and storage type, and the search that chooses them
// (flowroi_autotune, tiles.cu).  Host code only.
//
// Per-frame entries are read into each frame's descriptor, so one captured
// graph serves a batch of mixed sizes with every frame on its own class's
// shapes; per-context entries (persistent grid sizes, the DWT's register
// budget) are fixed when the context's graphs are captured.
#pragma once

#include <string>

#include "common.cuh"

namespace flowroi {

constexpr int kWClasses = 6;  // frame widths up to 256, 512, 1024, 2048, 4096, and wider

// Width class of a frame width (level 0), and the class's nominal width.
int width_class(int w);
int class_width(int c);

// Persistent kernel families whose grid size (blocks per SM) is tunable.
enum TileKernel { TK_EXPAND = 0, TK_UPDATE, TK_WINDOW, TK_MASK, TK_DWT, TK_COUNT };
const char *tile_kernel_name(int k);

struct TileTable {
    // per frame [storage: 0 fp32, 1 fp16][width class]; 0 = built-in default
    int dwt_seg[2][kWClasses][kMaxLevels];  // DWT band rows per warp unit, per level (index level-1)
    int saliency_rows[2][kWClasses];        // rows of a k_saliency tile (a multiple of kSalSub)
    // per context [storage]; 0 = built-in default
    int blocks_per_sm[2][TK_COUNT];         // persistent grid = min(this, occupancy) x SMs
    int dwt_variant[2];                     // DWT register budget: 5 or 6 resident blocks per SM
    int update_rows[2];                     // rows of a k_update tile: 4, 8, 16 or 32 (taken 4 at a time)
};

void tiles_clear(TileTable &t);
// Parses a table (JSON text, format "flowroi-tiles-1") into t (entries
// override what t holds).  false with a message on a malformed table.
bool tiles_parse(const char *json, TileTable &t, std::string &err);
// The table as JSON: every non-default entry.
std::string tiles_json(const TileTable &t, const char *device_name);

// The values a frame runs with (defaults filled in).
int tiles_dwt_seg(const TileTable &t, bool half, int W, int level, int bw, int bh);
int tiles_saliency_strips(const TileTable &t, bool half, int W);

}  // namespace flowroi
