// Gridder (Section 6): V_grid(x, y) = sum_i f(r_i) V_i over the visibilities
// with r_i = |(x, y) - (x_i, y_i)| < r_max, the pixel centres at integer
// coordinates and f a radial gridding convolution function given as a table
// (linear interpolation between samples r_k = k r_max / (n_tab - 1)).
//
// The paper's CUDA gridder is a gather over binned visibilities: the grid is
// cut into bins of B x B pixels (B >= r_max), the visibilities are sorted by
// bin with first/last tables, and the threads of one block (a patch of pixels
// inside one bin) share the visibilities of the bin and its eight neighbours
// through shared memory.  Here:
//   k_grid_sort_pass<false>  one warp per chunk of kGridChunk visibilities
//                   counts its visibilities per bin (shared-memory counters)
//   k_grid_bin_totals, k_grid_scan_bins, k_grid_offsets
//                   exclusive scan in (bin, chunk) order over the [chunk][bin]
//                   count table: each chunk's first slot in each bin, and
//                   each bin's first and last
//   k_grid_sort_pass<true>   the same warps place their visibilities, stably:
//                   a lane's rank among the lanes with the same bin
//                   (__match_any_sync) plus the chunk's running count for it
//   k_grid_gather   one CTA per bin, one 8 x 8 pixel tile per warp (2 pixels
//                   per lane); each warp walks the 9 bins' visibilities in a
//                   fixed order straight from the (L2-resident) sorted list,
//                   32 at a time: every lane tests one against the tile's
//                   box, and only the hits (a ballot) cost per-pixel work.
//                   The paper staged the visibilities in shared memory for
//                   the whole block; here that staging made every warp wait
//                   for the busiest one at each stage.  Every pixel's sum is
//                   deterministic and every pixel is written exactly once
//                   (no atomics, no memset).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rts {

constexpr int kGridChunk = 1024;      // visibilities per counting warp
constexpr int kGridWarps = 4;         // counting warps per CTA
constexpr int kGridMaxBins = 8192;    // shared-memory counters per warp
constexpr int kGridPix = 2;           // pixels per gather thread
constexpr int kGridTile = 8;          // gather warp tile: 8 x 8 pixels (kGridPix = 2 per lane)
constexpr int kGridMaxBin = 40;       // at most 5 x 5 tiles (800 threads) per bin
constexpr int kGridMaxPol = 4;

// bin of a visibility, or -1 outside [0, n_pix)^2 (NaN compares false)
__device__ __forceinline__ int grid_bin(float2 p, int n_pix, int bin, int nbx) {
  if (!(p.x >= 0.f && p.x < (float)n_pix && p.y >= 0.f && p.y < (float)n_pix)) return -1;
  return ((int)p.y / bin) * nbx + (int)p.x / bin;
}

struct GridSortArgs {
  const float2* xy;         // [n_vis] pixel coordinates
  const float2* vis;        // [n_vis][n_pol]
  int n_vis, n_pol, n_pix, bin, nbx, n_bins, n_chunks;
  int* counts;              // [n_chunks][n_bins] visibilities of chunk in bin, then exclusive offsets
  int* bin_start;           // [n_bins + 1]
  float2* sxy;              // [n_vis] sorted positions
  float2* svis;             // [n_vis][n_pol] sorted values
};

// Warp w of the CTA walks chunk blockIdx.x * kGridWarps + w, 32 visibilities
// at a time; SCATTER places them, else it counts them.
template <bool SCATTER>
__global__ void __launch_bounds__(kGridWarps * 32) k_grid_sort_pass(GridSortArgs a) {
  extern __shared__ int s_cnt[];                       // [kGridWarps][n_bins]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = blockIdx.x * kGridWarps + warp;
  int* cnt = s_cnt + (size_t)warp * a.n_bins;
  for (int b = lane; b < a.n_bins; b += 32)
    cnt[b] = (SCATTER && chunk < a.n_chunks) ? a.counts[(size_t)chunk * a.n_bins + b] : 0;
  __syncwarp();
  if (chunk < a.n_chunks) {
    const int i0 = chunk * kGridChunk, i1 = min(a.n_vis, i0 + kGridChunk);
    const unsigned lt = (1u << lane) - 1u;
    int bins[kGridChunk / 32];                        // this lane's bins, all loads issued first
    #pragma unroll
    for (int j = 0; j < kGridChunk / 32; ++j) {
      const int i = i0 + 32 * j + lane;
      bins[j] = i < i1 ? grid_bin(a.xy[i], a.n_pix, a.bin, a.nbx) : -1;
    }
    #pragma unroll
    for (int j = 0; j < kGridChunk / 32; ++j) {
      const int i = i0 + 32 * j + lane;
      const int b = bins[j];
      const unsigned same = __match_any_sync(0xffffffffu, b);
      const int rank = __popc(same & lt);
      const bool leader = rank == 0;
      int dest = 0;
      if (b >= 0) dest = cnt[b] + rank;
      __syncwarp();
      if (b >= 0 && leader) cnt[b] += __popc(same);
      __syncwarp();
      if (SCATTER && b >= 0) {
        a.sxy[dest] = a.xy[i];
        for (int p = 0; p < a.n_pol; ++p) a.svis[(size_t)dest * a.n_pol + p] = a.vis[(size_t)i * a.n_pol + p];
      }
    }
  }
  __syncwarp();
  if (!SCATTER && chunk < a.n_chunks)
    for (int b = lane; b < a.n_bins; b += 32) a.counts[(size_t)chunk * a.n_bins + b] = cnt[b];
}

// Exclusive scan of counts in (bin, chunk) order, in three steps:
//   k_grid_bin_totals  one thread per bin sums its counts over the chunks
//                      (the [chunk][bin] rows are read coalesced)
//   k_grid_scan_bins   one CTA scans the bin totals into bin_start
//   k_grid_offsets     one thread per bin turns its counts into each chunk's
//                      first slot, chunk by chunk
__global__ void __launch_bounds__(256) k_grid_bin_totals(GridSortArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.n_bins) return;
  int s = 0;
  #pragma unroll 8
  for (int c = 0; c < a.n_chunks; ++c) s += a.counts[(size_t)c * a.n_bins + b];
  a.bin_start[b] = s;                               // total for now; start after the scan
}

__global__ void __launch_bounds__(1024) k_grid_scan_bins(GridSortArgs a) {
  __shared__ int s_tot[1024];
  const int per = (a.n_bins + 1023) / 1024;
  const int b0 = min(a.n_bins, (int)threadIdx.x * per), b1 = min(a.n_bins, b0 + per);
  int s = 0;
  for (int b = b0; b < b1; ++b) s += a.bin_start[b];
  s_tot[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {              // inclusive Hillis-Steele scan
    const int v = threadIdx.x >= o ? s_tot[threadIdx.x - o] : 0;
    __syncthreads();
    s_tot[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s_tot[threadIdx.x] - s;
  for (int b = b0; b < b1; ++b) {
    const int t = a.bin_start[b];
    a.bin_start[b] = run;
    run += t;
  }
  if (threadIdx.x == 1023) a.bin_start[a.n_bins] = s_tot[1023];
}

__global__ void __launch_bounds__(256) k_grid_offsets(GridSortArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.n_bins) return;
  int run = a.bin_start[b];
  for (int c = 0; c < a.n_chunks; ++c) {
    const size_t j = (size_t)c * a.n_bins + b;
    const int k = a.counts[j];
    a.counts[j] = run;
    run += k;
  }
}

struct GridGatherArgs {
  const float2* sxy;
  const float2* svis;
  const int* bin_start;     // [n_bins + 1]
  const float* gcf;         // [n_tab] (copied to shared memory, one extra sample repeated)
  int n_tab, n_pol, n_pix, bin, nbx, nby;
  float r_max, r2max, tab_scale;   // tab_scale = (n_tab - 1) / r_max
  float2* grid;             // [n_pol][n_pix][n_pix]
};

template <int NPOL>
__global__ void __launch_bounds__(1024, 1) k_grid_gather(GridGatherArgs a) {
  extern __shared__ float s_tab[];                  // gcf [n_tab + 1] (last sample repeated)
  const int bx = blockIdx.x % a.nbx, by = blockIdx.x / a.nbx;
  for (int k = threadIdx.x; k <= a.n_tab; k += blockDim.x) s_tab[k] = a.gcf[min(k, a.n_tab - 1)];
  __syncthreads();
  // warp w owns the 8 x 8 tile (w % tpb, w / tpb) of the bin; lane l its pixels
  // (l % 8, l / 8) and (l % 8, l / 8 + 4).  Warps walk the sorted list
  // independently (it is L2-resident), so no warp waits for another.
  const int tpb = (a.bin + kGridTile - 1) / kGridTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tx = (warp % tpb) * kGridTile, ty = (warp / tpb) * kGridTile;     // tile origin in the bin
  const float x0 = (float)(bx * a.bin + tx), y0 = (float)(by * a.bin + ty);
  int px[kGridPix], py[kGridPix];
  bool live[kGridPix];
  float acc[kGridPix][2 * NPOL];
  #pragma unroll
  for (int u = 0; u < kGridPix; ++u) {
    const int ix = tx + (lane & 7), iy = ty + (lane >> 3) + 4 * u;            // pixel in the bin
    px[u] = bx * a.bin + ix;
    py[u] = by * a.bin + iy;
    live[u] = ix < a.bin && iy < a.bin && px[u] < a.n_pix && py[u] < a.n_pix;
    #pragma unroll
    for (int k = 0; k < 2 * NPOL; ++k) acc[u][k] = 0.f;
  }
  const float ext = (float)(kGridTile - 1);
  for (int ny = max(0, by - 1); ny <= min(a.nby - 1, by + 1); ++ny)
    for (int nx = max(0, bx - 1); nx <= min(a.nbx - 1, bx + 1); ++nx) {
      const int nb = ny * a.nbx + nx;
      const int v0 = a.bin_start[nb], v1 = a.bin_start[nb + 1];
      for (int k0 = v0; k0 < v1; k0 += 32) {
        // lane l tests visibility k0 + l against the warp's tile box; the warp
        // then walks the hits in increasing order
        float2 q = make_float2(0.f, 0.f);
        bool hit = false;
        if (k0 + lane < v1) {
          q = __ldg(a.sxy + k0 + lane);
          const float ex = fmaxf(fmaxf(x0 - q.x, q.x - (x0 + ext)), 0.f);
          const float ey = fmaxf(fmaxf(y0 - q.y, q.y - (y0 + ext)), 0.f);
          hit = fmaf(ex, ex, ey * ey) < a.r2max;
        }
        unsigned hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
          const int j = __ffs(hits) - 1;
          hits &= hits - 1;
          const float2 p = make_float2(__shfl_sync(0xffffffffu, q.x, j), __shfl_sync(0xffffffffu, q.y, j));
          const float2* vk = a.svis + (size_t)(k0 + j) * NPOL;
          float2 v[NPOL];
          #pragma unroll
          for (int pp = 0; pp < NPOL; ++pp) v[pp] = __ldg(vk + pp);
          #pragma unroll
          for (int u = 0; u < kGridPix; ++u) {
            const float dx = (float)px[u] - p.x, dy = (float)py[u] - p.y;
            const float d2 = fmaf(dx, dx, dy * dy);
            if (live[u] && d2 < a.r2max) {
              const float sidx = (d2 > 0.f ? d2 * rsqrtf(d2) : 0.f) * a.tab_scale;
              const int t = min((int)sidx, a.n_tab - 1);
              const float w = sidx - (float)t;
              const float f = fmaf(w, s_tab[t + 1] - s_tab[t], s_tab[t]);
              #pragma unroll
              for (int pp = 0; pp < NPOL; ++pp) {
                acc[u][2 * pp] = fmaf(f, v[pp].x, acc[u][2 * pp]);
                acc[u][2 * pp + 1] = fmaf(f, v[pp].y, acc[u][2 * pp + 1]);
              }
            }
          }
        }
      }
    }
  const size_t plane = (size_t)a.n_pix * a.n_pix;
  #pragma unroll
  for (int u = 0; u < kGridPix; ++u)
    if (live[u])
      #pragma unroll
      for (int pp = 0; pp < NPOL; ++pp)
        a.grid[pp * plane + (size_t)py[u] * a.n_pix + px[u]] = make_float2(acc[u][2 * pp], acc[u][2 * pp + 1]);
}

}  // namespace rts
