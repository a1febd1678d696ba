/* rts_grid.h - C ABI of the GB300 gridder (librtspeel.so).
 *
 * Section 6 of Edgar et al. (arXiv:1003.5575), "Acceleration of the Gridder":
 * the gridder interpolates the visibilities scattered over the u-v plane onto
 * a regular grid before the imager's FFT by convolving each visibility with a
 * compact gridding convolution function (GCF) that vanishes beyond r_max,
 *   V_grid(u, v) = sum_i f_i(r) * V_i delta(u - u_i, v - v_i),
 * and its CUDA implementation is a gather over visibilities sorted into bins
 * of B x B pixels (B >= r_max; the paper uses 24 x 24 bins for r_max = 12):
 * each pixel only visits the visibilities of its own bin and the eight
 * neighbouring bins, found through first/last tables of the sorted list, and
 * the threads of a block share them through shared memory.
 *
 * Conventions (reading R18 of the design notes): pixel (x, y) has its centre
 * at integer coordinates x, y in [0, n_pix); a visibility at pixel
 * coordinates (x_i, y_i) (floats, the caller's u, v scaled by the cell size
 * and offset to the grid centre) adds f(r) V_i to every pixel centre at
 * distance r < r_max; f is radial, the linear interpolation of a table of
 * n_tab samples at r_k = k r_max / (n_tab - 1) (the same f for every
 * visibility, as the paper's spheroidal function); visibilities outside
 * [0, n_pix) in either coordinate are not gridded.  Each visibility carries
 * n_pol complex values, each gridded into its own plane.  Sums are FP32 in a
 * fixed order (bins row by row, the sorted order inside a bin), so the grid
 * is bitwise reproducible.
 *
 * Ownership: the caller owns every pointer it passes ("d_" device, "h_"
 * host); the handle owns its workspace (sorted copies of up to max_vis
 * visibilities, bin tables) and frees it in rts_grid_destroy.  Calls are
 * asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Errors: RTS_OK (0) or a negative code of rts_peel.h; the text is available
 * from rts_grid_last_error.  Invalid arguments are rejected on the host.
 */
#ifndef RTS_GRID_H
#define RTS_GRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rts_grid_t rts_grid_t;

typedef struct rts_grid_config {
  int32_t n_pix;        /* grid side in pixels (square grid), 1 .. 16384 */
  int32_t bin;          /* bin side in pixels, r_max <= bin <= 40, and
                           ceil(n_pix / bin)^2 <= 8192 bins */
  double r_max;         /* support radius of the GCF in pixels, > 0 */
  const double* gcf;    /* host [n_tab] radial GCF samples at r_k = k r_max/(n_tab - 1); copied */
  int32_t n_tab;        /* 2 .. 4096 */
  int32_t n_pol;        /* complex values per visibility, 1 .. 4 */
  int32_t max_vis;      /* largest n_vis any call passes, >= 1 */
} rts_grid_config;

/* Validate cfg, allocate the workspace on the current device and copy the GCF
 * table.  On success *out is a new handle.  RTS_EINVAL (cfg), RTS_ENOMEM,
 * RTS_ECUDA; *out is then NULL and the message is available from
 * rts_grid_last_error(NULL). */
int rts_grid_init(const rts_grid_config* cfg, rts_grid_t** out);

/* Grid n_vis visibilities.
 *   d_xy    device float [n_vis][2] pixel coordinates (x, y), 8-byte aligned
 *   d_vis   device complex64 [n_vis][n_pol], 8-byte aligned
 *   n_vis   0 .. max_vis
 *   d_grid  device complex64 [n_pol][n_pix][n_pix]; every pixel is overwritten
 * Sorts the visibilities by bin (stable counting sort: counts per chunk of
 * 1024, a scan, a stable scatter) and gathers each bin's pixels from the 3 x 3
 * neighbouring bins.  RTS_EINVAL for bad arguments, RTS_ECUDA for a failed launch. */
int rts_grid_run(rts_grid_t* g, const void* d_xy, const void* d_vis, int32_t n_vis, void* d_grid,
                 void* stream);

/* Device time of the last rts_grid_run, split into the sort (count, scan,
 * scatter) and the gather, in ms (waits for the events).  Either pointer may
 * be NULL.  RTS_EINVAL for a NULL handle or before the first run. */
int rts_grid_last_ms(rts_grid_t* g, double* ms_sort, double* ms_gather);

/* Text of the last error on this handle (NULL: of the last failed init). */
const char* rts_grid_last_error(const rts_grid_t* g);

void rts_grid_destroy(rts_grid_t* g);

#ifdef __cplusplus
}
#endif
#endif
