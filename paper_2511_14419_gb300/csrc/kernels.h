// Host-side launchers of the FlowRoI kernels (one translation unit per
// kernel family).  `grid` is the number of blocks; every kernel walks its
// tiles with a grid-stride loop, so any grid >= 1 is correct.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace flowroi {

void launch_expand(const BatchDesc *bd, const MethodConsts &mc, int level, bool half, int grid, cudaStream_t s);
// rows: rows of a tile (kUpdRows x 1, 2, 4 or 8), taken kUpdRows at a time
void launch_update(const BatchDesc *bd, const MethodConsts &mc, int level, int iter, int src, bool half, int rows,
                   int grid, cudaStream_t s);
void launch_window(const BatchDesc *bd, const MethodConsts &mc, int level, int dst, bool half, int grid, cudaStream_t s);
void launch_frame_init(const BatchDesc *bd, int grid, cudaStream_t s);
void launch_saliency(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s);
void launch_select_pass(const BatchDesc *bd, int pass, int grid, cudaStream_t s);
void launch_select_find(const BatchDesc *bd, const MethodConsts &mc, int pass, int grid, cudaStream_t s);
void launch_morph(const BatchDesc *bd, const MethodConsts &mc, int grid, cudaStream_t s);
// variant: the register budget's resident blocks per SM (5 or 6)
void launch_dwt(const BatchDesc *bd, const MethodConsts &mc, int level, int grid, int variant, cudaStream_t s);
// DWT work units (one warp each) of a level whose bands are bw x bh, with
// seg band rows per unit; blocks needed for `units` (at most the persistent grid).
int dwt_units(int bw, int bh, int seg);
int dwt_default_seg(int bw, int bh);  // band rows per unit when no tile table entry applies
int dwt_grid(int units, int persistent_blocks);
// Registration to the predecessor: steps 0-7 (level-image sum, row and
// column FFTs, cross-power spectrum, inverse FFTs, peak, drift).
void launch_register(const BatchDesc *bd, const MethodConsts &mc, bool half, int step, int grid, cudaStream_t s);
int occupancy_register();
int register_max_log();  // padded FFT sizes up to 2^this
int register_cols();     // columns per block of the column FFTs
int register_unit();     // elements per block-unit of the element-wise steps
// Adjacent-factor merge of per-frame masks (entries with n_adj > 0).
void launch_merge(const BatchDesc *bd, int grid, cudaStream_t s);
// Removal of small connected components of the final mask: steps 0-3
// (local labels, border unions, areas, filter), one launch each.
void launch_cc(const BatchDesc *bd, const MethodConsts &mc, int step, int grid, cudaStream_t s);
// Optional denoising of the flow input (level-0 tiles of the expansion).
void launch_denoise(const BatchDesc *bd, const MethodConsts &mc, bool half, int grid, cudaStream_t s);

// Resident blocks per SM (also sets any shared-memory attribute the kernel
// needs; call once per device before the first launch).
int occupancy_expand(bool half, int n_half);
int occupancy_update(bool half, int rows);
// TMA box of the window kernel: it starts xo elements left of a tile, bw wide, eh rows.
int window_box(bool half, int win_r, int *xo, int *bw, int *eh);
int occupancy_window(bool half, int win_r);
int occupancy_mask_kernels();
int occupancy_dwt(int wavelet, int variant);
int occupancy_denoise(bool half, int radius);
int occupancy_cc();

bool flow_radius_supported(int r);
bool morph_radius_supported(int r);
bool denoise_radius_supported(int r);

// Embedded block coding of coefficient planes into frame containers
// (k_ebcot.cu); CsFrame, CsJob and the coder's constants are in common.cuh.
int ebcot_codeblocks(int w, int h, int levels);
// chains: some frame carries its contexts from pass to pass; passes: some
// frame resets them at every pass (each launches its own MQ state stage).
void launch_ebcot(const CsJob *job_dev, int nframes, int ncb, bool chains, bool passes, cudaStream_t s);
// The same with fixed (persistent, grid-stride) grids, for captured graphs.
void launch_ebcot_persistent(const CsJob *job_dev, int grid_t1, int grid_mq, int grid_copy, bool reset, cudaStream_t s);
int occupancy_t1();

// 9/7 quantisation steps (host, double precision); see flowroi_quant_steps.
int quant_steps(int levels, int bit_depth, double delta_base, float *delta, int *eps, int *mu, double *gain);

}  // namespace flowroi
