// librtspeel: C ABI of the gridder (see include/rts_grid.h, grid_kernels.cuh).
#include "rts_grid.h"
#include "rts_peel.h"

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "grid_kernels.cuh"

using namespace rts;

struct rts_grid_t {
  int n_pix = 0, bin = 0, nbx = 0, n_bins = 0, n_tab = 0, n_pol = 0, max_vis = 0, max_chunks = 0;
  double r_max = 0;
  int device = 0;
  float* d_gcf = nullptr;      // [n_tab]
  int* d_counts = nullptr;     // [n_bins][max_chunks]
  int* d_bin_start = nullptr;  // [n_bins + 1]
  float2* d_sxy = nullptr;     // [max_vis]
  float2* d_svis = nullptr;    // [max_vis][n_pol]
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool ran = false;
  std::string err;
};

namespace {

std::string g_grid_init_err;

int gfail(rts_grid_t* g, int code, const std::string& msg) {
  (g ? g->err : g_grid_init_err) = msg;
  return code;
}

int gcuda(rts_grid_t* g, cudaError_t e, const char* what) {
  return gfail(g, e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define GRID_CUDA(g, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return gcuda((g), e_, #call);     \
  } while (0)

int gather_threads(int bin) {
  const int tpb = (bin + kGridTile - 1) / kGridTile;
  return 32 * tpb * tpb;
}

}  // namespace

extern "C" {

int rts_grid_init(const rts_grid_config* cfg, rts_grid_t** out) {
  g_grid_init_err.clear();
  if (!out) return gfail(nullptr, RTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return gfail(nullptr, RTS_EINVAL, "cfg is NULL");
  if (cfg->n_pix < 1 || cfg->n_pix > 16384) return gfail(nullptr, RTS_EINVAL, "n_pix must be in [1, 16384]");
  if (!(cfg->r_max > 0.0) || !std::isfinite(cfg->r_max)) return gfail(nullptr, RTS_EINVAL, "r_max must be finite and > 0");
  if (cfg->bin < cfg->r_max || cfg->bin > kGridMaxBin)
    return gfail(nullptr, RTS_EINVAL, "bin must satisfy r_max <= bin <= 40");
  const int nbx = (cfg->n_pix + cfg->bin - 1) / cfg->bin;
  if ((int64_t)nbx * nbx > kGridMaxBins) return gfail(nullptr, RTS_EINVAL, "ceil(n_pix / bin)^2 must be <= 8192 bins");
  if (cfg->n_tab < 2 || cfg->n_tab > 4096) return gfail(nullptr, RTS_EINVAL, "n_tab must be in [2, 4096]");
  if (!cfg->gcf) return gfail(nullptr, RTS_EINVAL, "gcf is NULL");
  for (int k = 0; k < cfg->n_tab; ++k)
    if (!std::isfinite(cfg->gcf[k])) return gfail(nullptr, RTS_EINVAL, "gcf has a non-finite sample");
  if (cfg->n_pol < 1 || cfg->n_pol > kGridMaxPol) return gfail(nullptr, RTS_EINVAL, "n_pol must be in [1, 4]");
  if (cfg->max_vis < 1) return gfail(nullptr, RTS_EINVAL, "max_vis must be >= 1");

  rts_grid_t* g = new rts_grid_t();
  g->n_pix = cfg->n_pix; g->bin = cfg->bin; g->nbx = nbx; g->n_bins = nbx * nbx;
  g->n_tab = cfg->n_tab; g->n_pol = cfg->n_pol; g->max_vis = cfg->max_vis; g->r_max = cfg->r_max;
  g->max_chunks = (cfg->max_vis + kGridChunk - 1) / kGridChunk;
  cudaGetDevice(&g->device);
  auto bail = [&](cudaError_t e, const char* what) {
    gcuda(nullptr, e, what);
    rts_grid_destroy(g);
    return e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA;
  };
  cudaError_t e;
  std::vector<float> tab(cfg->gcf, cfg->gcf + cfg->n_tab);
  if ((e = cudaMalloc(&g->d_gcf, sizeof(float) * g->n_tab)) != cudaSuccess) return bail(e, "cudaMalloc(gcf)");
  if ((e = cudaMemcpy(g->d_gcf, tab.data(), sizeof(float) * g->n_tab, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "cudaMemcpy(gcf)");
  if ((e = cudaMalloc(&g->d_counts, sizeof(int) * (size_t)g->n_bins * g->max_chunks)) != cudaSuccess)
    return bail(e, "cudaMalloc(counts)");
  if ((e = cudaMalloc(&g->d_bin_start, sizeof(int) * (size_t)(g->n_bins + 1))) != cudaSuccess)
    return bail(e, "cudaMalloc(bin_start)");
  if ((e = cudaMalloc(&g->d_sxy, sizeof(float2) * (size_t)g->max_vis)) != cudaSuccess) return bail(e, "cudaMalloc(sxy)");
  if ((e = cudaMalloc(&g->d_svis, sizeof(float2) * (size_t)g->max_vis * g->n_pol)) != cudaSuccess)
    return bail(e, "cudaMalloc(svis)");
  for (int k = 0; k < 3; ++k)
    if ((e = cudaEventCreate(&g->ev[k])) != cudaSuccess) return bail(e, "cudaEventCreate");
  const size_t sort_smem = sizeof(int) * (size_t)kGridWarps * g->n_bins;
  if ((e = cudaFuncSetAttribute(k_grid_sort_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sort_smem)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_grid_sort_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sort_smem)) != cudaSuccess)
    return bail(e, "cudaFuncSetAttribute(sort)");
  *out = g;
  return RTS_OK;
}

int rts_grid_run(rts_grid_t* g, const void* d_xy, const void* d_vis, int32_t n_vis, void* d_grid,
                 void* stream) {
  if (!g) return gfail(nullptr, RTS_EINVAL, "handle is NULL");
  if (n_vis < 0 || n_vis > g->max_vis) return gfail(g, RTS_EINVAL, "n_vis must be in [0, max_vis]");
  if (!d_grid || (n_vis > 0 && (!d_xy || !d_vis))) return gfail(g, RTS_EINVAL, "d_xy, d_vis and d_grid are required");
  if ((reinterpret_cast<uintptr_t>(d_xy) | reinterpret_cast<uintptr_t>(d_vis) | reinterpret_cast<uintptr_t>(d_grid)) & 7u)
    return gfail(g, RTS_EINVAL, "d_xy, d_vis and d_grid must be 8-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nbx = g->nbx;
  GRID_CUDA(g, cudaEventRecord(g->ev[0], s));
  const int n_chunks = (n_vis + kGridChunk - 1) / kGridChunk;
  GridSortArgs a;
  a.xy = static_cast<const float2*>(d_xy); a.vis = static_cast<const float2*>(d_vis);
  a.n_vis = n_vis; a.n_pol = g->n_pol; a.n_pix = g->n_pix; a.bin = g->bin; a.nbx = nbx;
  a.n_bins = g->n_bins; a.n_chunks = n_chunks;
  a.counts = g->d_counts; a.bin_start = g->d_bin_start; a.sxy = g->d_sxy; a.svis = g->d_svis;
  if (n_vis == 0) {
    GRID_CUDA(g, cudaMemsetAsync(g->d_bin_start, 0, sizeof(int) * (size_t)(g->n_bins + 1), s));
  } else {
    const size_t sort_smem = sizeof(int) * (size_t)kGridWarps * g->n_bins;
    const unsigned sort_grid = (unsigned)((n_chunks + kGridWarps - 1) / kGridWarps);
    k_grid_sort_pass<false><<<sort_grid, kGridWarps * 32, sort_smem, s>>>(a);
    const unsigned bins_grid = (unsigned)((g->n_bins + 255) / 256);
    k_grid_bin_totals<<<bins_grid, 256, 0, s>>>(a);
    k_grid_scan_bins<<<1, 1024, 0, s>>>(a);
    k_grid_offsets<<<bins_grid, 256, 0, s>>>(a);
    k_grid_sort_pass<true><<<sort_grid, kGridWarps * 32, sort_smem, s>>>(a);
  }
  GRID_CUDA(g, cudaGetLastError());
  GRID_CUDA(g, cudaEventRecord(g->ev[1], s));
  GridGatherArgs b;
  b.sxy = g->d_sxy; b.svis = g->d_svis; b.bin_start = g->d_bin_start; b.gcf = g->d_gcf;
  b.n_tab = g->n_tab; b.n_pol = g->n_pol; b.n_pix = g->n_pix; b.bin = g->bin; b.nbx = nbx; b.nby = nbx;
  b.r_max = (float)g->r_max; b.r2max = (float)(g->r_max * g->r_max);
  b.tab_scale = (float)((g->n_tab - 1) / g->r_max);
  b.grid = static_cast<float2*>(d_grid);
  const size_t gsm = sizeof(float) * (size_t)(g->n_tab + 1);
  const dim3 gg((unsigned)g->n_bins), gb((unsigned)gather_threads(g->bin));
  switch (g->n_pol) {
    case 1: k_grid_gather<1><<<gg, gb, gsm, s>>>(b); break;
    case 2: k_grid_gather<2><<<gg, gb, gsm, s>>>(b); break;
    case 3: k_grid_gather<3><<<gg, gb, gsm, s>>>(b); break;
    default: k_grid_gather<4><<<gg, gb, gsm, s>>>(b); break;
  }
  GRID_CUDA(g, cudaGetLastError());
  GRID_CUDA(g, cudaEventRecord(g->ev[2], s));
  g->ran = true;
  return RTS_OK;
}

int rts_grid_last_ms(rts_grid_t* g, double* ms_sort, double* ms_gather) {
  if (!g) return gfail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!g->ran) return gfail(g, RTS_EINVAL, "no run yet");
  GRID_CUDA(g, cudaEventSynchronize(g->ev[2]));
  float a = 0.f, b = 0.f;
  GRID_CUDA(g, cudaEventElapsedTime(&a, g->ev[0], g->ev[1]));
  GRID_CUDA(g, cudaEventElapsedTime(&b, g->ev[1], g->ev[2]));
  if (ms_sort) *ms_sort = a;
  if (ms_gather) *ms_gather = b;
  return RTS_OK;
}

const char* rts_grid_last_error(const rts_grid_t* g) { return g ? g->err.c_str() : g_grid_init_err.c_str(); }

void rts_grid_destroy(rts_grid_t* g) {
  if (!g) return;
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != g->device) cudaSetDevice(g->device);
  void* ptrs[] = {g->d_gcf, g->d_counts, g->d_bin_start, g->d_sxy, g->d_svis};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 3; ++k)
    if (g->ev[k]) cudaEventDestroy(g->ev[k]);
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  delete g;
}

}  // extern "C"
