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
//   k_grid_scan     exclusive scan over (bin, chunk): each chunk's first slot
//                   in each bin, and each bin's first and last
//   k_grid_sort_pass<true>   the same warps place their visibilities, stably:
//                   a lane's rank among the lanes with the same bin
//                   (__match_any_sync) plus the chunk's running count for it
//   k_grid_gather   one CTA per bin, kGridPix pixels per thread; the 9 bins'
//                   visibilities staged through shared memory in a fixed
//                   order, so every pixel's sum is deterministic and every
//                   pixel is written exactly once (no atomics, no memset).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rts {

constexpr int kGridChunk = 1024;      // visibilities per counting warp
constexpr int kGridWarps = 4;         // counting warps per CTA
constexpr int kGridMaxBins = 8192;    // shared-memory counters per warp
constexpr int kGridPix = 2;           // pixels per gather thread
constexpr int kGridMaxPol = 4;
constexpr int kGridStage = 256;       // visibilities staged per gather round

// bin of a visibility, or -1 outside [0, n_pix)^2 (NaN compares false)
__device__ __forceinline__ int grid_bin(float2 p, int n_pix, int bin, int nbx) {
  if (!(p.x >= 0.f && p.x < (float)n_pix && p.y >= 0.f && p.y < (float)n_pix)) return -1;
  return ((int)p.y / bin) * nbx + (int)p.x / bin;
}

struct GridSortArgs {
  const float2* xy;         // [n_vis] pixel coordinates
  const float2* vis;        // [n_vis][n_pol]
  int n_vis, n_pol, n_pix, bin, nbx, n_bins, n_chunks;
  int* counts;              // [n_bins][n_chunks] visibilities of chunk in bin, then exclusive offsets
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
    cnt[b] = (SCATTER && chunk < a.n_chunks) ? a.counts[(size_t)b * a.n_chunks + chunk] : 0;
  __syncwarp();
  if (chunk < a.n_chunks) {
    const int i0 = chunk * kGridChunk, i1 = min(a.n_vis, i0 + kGridChunk);
    const unsigned lt = (1u << lane) - 1u;
    for (int base = i0; base < i1; base += 32) {
      const int i = base + lane;
      const int b = i < i1 ? grid_bin(a.xy[i], a.n_pix, a.bin, a.nbx) : -1;
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
    for (int b = lane; b < a.n_bins; b += 32) a.counts[(size_t)b * a.n_chunks + chunk] = cnt[b];
}

// Exclusive scan of counts in (bin, chunk) order, one CTA of 1024 threads:
// each thread scans a contiguous segment, the segment totals are scanned in
// shared memory, and each bin's first slot lands in bin_start.
__global__ void __launch_bounds__(1024) k_grid_scan(GridSortArgs a) {
  __shared__ int s_tot[1024];
  const int64_t n = (int64_t)a.n_bins * a.n_chunks;
  const int64_t seg = (n + 1023) / 1024;
  const int64_t j0 = min(n, (int64_t)threadIdx.x * seg), j1 = min(n, j0 + seg);
  int s = 0;
  for (int64_t j = j0; j < j1; ++j) s += a.counts[j];
  s_tot[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {              // inclusive Hillis-Steele scan
    const int v = threadIdx.x >= o ? s_tot[threadIdx.x - o] : 0;
    __syncthreads();
    s_tot[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s_tot[threadIdx.x] - s;                 // exclusive start of this segment
  for (int64_t j = j0; j < j1; ++j) {
    const int c = a.counts[j];
    a.counts[j] = run;
    if (j % a.n_chunks == 0) a.bin_start[j / a.n_chunks] = run;
    run += c;
  }
  if (threadIdx.x == 1023) a.bin_start[a.n_bins] = s_tot[1023];
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
  extern __shared__ float4 g_sm[];
  // [kGridStage] positions | [kGridStage][NPOL] values | gcf [n_tab + 1] (last sample repeated)
  float2* s_xy = reinterpret_cast<float2*>(g_sm);
  float2* s_v = s_xy + kGridStage;
  float* s_tab = reinterpret_cast<float*>(s_v + (size_t)kGridStage * NPOL);
  const int bx = blockIdx.x % a.nbx, by = blockIdx.x / a.nbx;
  for (int k = threadIdx.x; k <= a.n_tab; k += blockDim.x) s_tab[k] = a.gcf[min(k, a.n_tab - 1)];
  int px[kGridPix], py[kGridPix];
  bool live[kGridPix];
  float acc[kGridPix][2 * NPOL];
  #pragma unroll
  for (int u = 0; u < kGridPix; ++u) {
    const int q = threadIdx.x + u * blockDim.x;      // pixel of the bin, row major
    px[u] = bx * a.bin + q % a.bin;
    py[u] = by * a.bin + q / a.bin;
    live[u] = q < a.bin * a.bin && px[u] < a.n_pix && py[u] < a.n_pix;
    #pragma unroll
    for (int k = 0; k < 2 * NPOL; ++k) acc[u][k] = 0.f;
  }
  for (int ny = max(0, by - 1); ny <= min(a.nby - 1, by + 1); ++ny)
    for (int nx = max(0, bx - 1); nx <= min(a.nbx - 1, bx + 1); ++nx) {
      const int nb = ny * a.nbx + nx;
      const int v0 = a.bin_start[nb], v1 = a.bin_start[nb + 1];
      for (int s0 = v0; s0 < v1; s0 += kGridStage) {
        const int ns = min(kGridStage, v1 - s0);
        __syncthreads();                            // previous stage consumed (and the table written)
        for (int k = threadIdx.x; k < ns; k += blockDim.x) s_xy[k] = a.sxy[s0 + k];
        for (int k = threadIdx.x; k < ns * NPOL; k += blockDim.x) s_v[k] = a.svis[(size_t)s0 * NPOL + k];
        __syncthreads();
        for (int k = 0; k < ns; ++k) {
          const float2 p = s_xy[k];
          #pragma unroll
          for (int u = 0; u < kGridPix; ++u) {
            const float dx = (float)px[u] - p.x, dy = (float)py[u] - p.y;
            const float d2 = fmaf(dx, dx, dy * dy);
            if (live[u] && d2 < a.r2max) {
              const float sidx = sqrtf(d2) * a.tab_scale;
              const int t = min((int)sidx, a.n_tab - 1);
              const float w = sidx - (float)t;
              const float f = fmaf(w, s_tab[t + 1] - s_tab[t], s_tab[t]);
              #pragma unroll
              for (int pp = 0; pp < NPOL; ++pp) {
                const float2 v = s_v[k * NPOL + pp];
                acc[u][2 * pp] = fmaf(f, v.x, acc[u][2 * pp]);
                acc[u][2 * pp + 1] = fmaf(f, v.y, acc[u][2 * pp + 1]);
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
