// librtspeel: C ABI of the GB300 calibrate-and-peel loop (see include/rts_peel.h).
#include "rts_peel.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "als_kernels.cuh"
#include "block_kernels.cuh"
#include "block_tc05_kernels.cuh"
#include "block_tc_kernels.cuh"
#include "common.cuh"
#include "grad_kernels.cuh"
#include "offset_kernels.cuh"
#include "phase_kernels.cuh"
#include "predict_kernels.cuh"
#include "solve_kernels.cuh"
#include "stream_kernels.cuh"
#include "taylor_kernels.cuh"
#include "taylor_block_kernels.cuh"

using namespace rts;

struct rts_peel_t {
  int n_ant = 0, n_chan = 0, n_time = 0, n_iter = 0, precision = 0, max_sources = 0;
  int per_pass = 1;                // sources per streaming pass (1 or RTS_BLOCK)
  bool block_tc = false;           // blocked passes as TF32 mma.sync (k_block_pass_tc)
  bool block_tc05 = false;           // blocked passes as tcgen05 MMAs (k_block_pass_tc05)
  int* d_perr = nullptr;           // [1] set by a tcgen05 pass whose mbarrier wait ran out
  int64_t n_bl = 0;
  double nu0 = 0, dnu = 0;
  int device = 0;
  int n_sm = 1;                    // multiprocessors of the device (grid sizing)
  size_t elem = 8;                 // bytes per complex element of the cube
  // device workspace, allocated once in rts_peel_init
  double* d_uvw = nullptr;         // [n_time][n_ant][3]
  int2* d_bl_ant = nullptr;        // [n_bl]
  double* d_freq_c = nullptr;      // [n_chan] nu_c / c
  void* d_avg = nullptr;           // [n_bl][4] cube precision
  double2* d_J[2] = {nullptr, nullptr};
  float2* d_Jf[2] = {nullptr, nullptr};
  double* d_norms = nullptr;       // [n_ant][2]
  int* d_flag = nullptr;           // [1]
  int* d_status = nullptr;         // [max_sources]
  double* d_rel = nullptr;         // [max_sources]
  double* d_src = nullptr;         // [max_sources][3]
  void* d_jones_stage = nullptr;   // [max_sources][n_ant][4] cube precision (host-buffer calls)
  GradWorkspace grad;
  // gains Taylor-expanded in frequency (allocated on the first Taylor cadence)
  float2* t_mom = nullptr;         // [3][n_bl][4] channel moments of the averaged source
  double2* t_X[2] = {nullptr, nullptr};   // [n_ant][8] FP64 iterates (G then H)
  float2* t_Xf[2] = {nullptr, nullptr};   // FP32 copies
  double* t_rot_part = nullptr;    // [t_rot_grid][kRotVals] slope-rotation sums per CTA
  unsigned* t_rot_count = nullptr; // [1] CTAs done (zero between launches)
  double* t_rot_step = nullptr;    // [5] the step (k_0..k_3, taken)
  int t_rot_grid = 0;
  // blocked peel workspace (allocated on the first blocked cadence).  The phase
  // and D_jk tables depend on geometry only; a second stream fills a ring of
  // kRing block slots ahead of the main stream (events order the reuse).
  static constexpr int kRing = 4;
  int n_band = 0, band_chan0 = 0;   // the whole band's channel count, this handle's first channel in it
  // a blocked cadence in progress (between rts_peel_shard_begin and the last rts_peel_shard_step)
  struct BlockRun {
    const void* vis = nullptr; void* resid = nullptr; void* jones = nullptr;
    int n_src = 0, b = 0, nb = 0;
    std::vector<double> src;       // host copy of the source list
    cudaStream_t user = nullptr;
    BlockPassArgs a;
    bool active = false;
  } br;
  PhaseAB* b_ph[kRing] = {};       // [n_bl][n_time][BK] phases of a block
  GeoTrig* b_trig[kRing] = {};     // [n_bl][n_time][BK] trigonometry for D_jk
  float2* b_dir[kRing] = {};       // [BK(BK-1)/2 x n_bl] in-block closed-form averages D_jk (dir_index)
  PhaseAB* b_aph = nullptr;        // [n_time][n_ant][BK] antenna phases of the block being prepared
  float2* b_avg = nullptr;         // [BK][n_bl][4] plain averages of a block
  float2* b_model = nullptr;       // [BK][n_bl][4] model matrices of a block
  // persistent block solve (k_block_solve, one cooperative launch per block)
  int solve_kernel = RTS_SOLVE_AUTO;
  bool grad_direct = false;        // adjoint with one sin/cos per sample (RTS_GRAD_DIRECT)
  bool bs_ok = false;              // set up and fits (shared memory, cooperative launch)
  int bs_grid = 0, bs_apc = 0;
  size_t bs_smem = 0;
  unsigned* b_sync = nullptr;      // [2] barrier counter, abort flag
  double* b_part = nullptr;        // [BK][n_ant][4] per-antenna convergence sums of the last sweep
  cudaStream_t b_main = nullptr;   // high-priority stream for passes, corrections and solves
  cudaStream_t b_prep = nullptr;   // low-priority geometry stream
  cudaEvent_t b_ev_in = nullptr;   // caller's stream -> main
  cudaEvent_t b_ev_out = nullptr;  // main -> caller's stream
  cudaEvent_t b_ev_src = nullptr;  // source list uploaded (main -> prep)
  cudaEvent_t b_ev_ready[kRing] = {};   // slot filled (prep -> main)
  cudaEvent_t b_ev_free[kRing] = {};    // slot consumed (main -> prep)
  cudaEvent_t b_ev_done = nullptr; // prep finished (prep -> main)
  // pipelined host-buffer cadences (two slots)
  void* p_cube[2] = {nullptr, nullptr};     // device cubes
  void* p_jones[2] = {nullptr, nullptr};    // device Jones staging [max_sources][n_ant][4]
  int32_t* p_status[2] = {nullptr, nullptr};// device status copies [max_sources]
  cudaStream_t p_in = nullptr, p_comp = nullptr, p_out = nullptr;
  cudaEvent_t p_ev_in[2] = {}, p_ev_comp[2] = {}, p_ev_out[2] = {};
  bool p_busy[2] = {false, false};
  int32_t* p_hstatus[2] = {nullptr, nullptr};
  void* p_hjones[2] = {nullptr, nullptr};       // the caller's Jones buffers, filled at retire
  void* p_jones_pin[2] = {nullptr, nullptr};    // page-locked Jones staging [max_sources][n_ant][4]
  int32_t* p_status_pin[2] = {nullptr, nullptr};// page-locked status staging [max_sources]
  int32_t p_nsrc[2] = {0, 0};
  int p_next = 0;
  // tracing: CUDA events around kernel groups, launch counters
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  int64_t launches[RTS_K_CLASSES] = {};
  std::string err;
};

namespace {

thread_local std::string g_init_err;

int fail(rts_peel_t* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_init_err = msg;
  return code;
}

// device cubes are read and written 16 bytes at a time
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

int cuda_fail(rts_peel_t* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA, m);
}

#define RTS_CUDA(h, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

int check_launch(rts_peel_t* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  return RTS_OK;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

cudaEvent_t next_event(rts_peel_t* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// brackets one kernel (or group of kernels) of class `cls` on stream s
struct Span {
  rts_peel_t* h; int cls; cudaStream_t s; cudaEvent_t a = nullptr;
  Span(rts_peel_t* h_, int cls_, cudaStream_t s_) : h(h_), cls(cls_), s(s_) {
    if (h->timing && (a = next_event(h))) cudaEventRecord(a, s);
  }
  void end(int n_launch) {
    h->launches[cls] += n_launch;
    if (a) {
      cudaEvent_t b = next_event(h);
      if (b) { cudaEventRecord(b, s); h->recs.push_back({cls, a, b}); }
      a = nullptr;
    }
  }
};

int validate_sources(rts_peel_t* h, int32_t n_src, const double* src) {
  if (n_src < 0 || n_src > h->max_sources)
    return fail(h, RTS_EINVAL, "n_src must be in [0, max_sources]");
  if (n_src > 0 && !src) return fail(h, RTS_EINVAL, "source list is NULL");
  for (int k = 0; k < n_src; ++k) {
    const double l = src[3 * k], m = src[3 * k + 1], S = src[3 * k + 2];
    if (!std::isfinite(l) || !std::isfinite(m) || !std::isfinite(S))
      return fail(h, RTS_EINVAL, "source " + std::to_string(k) + " has a non-finite l, m or S");
    if (!(l * l + m * m < 1.0))
      return fail(h, RTS_EINVAL, "source " + std::to_string(k) + " is not above the horizon (l^2+m^2 >= 1)");
    if (!(S > 0.0)) return fail(h, RTS_EINVAL, "source " + std::to_string(k) + " has flux S <= 0");
  }
  return RTS_OK;
}

StreamArgs stream_args(rts_peel_t* h, const void* src, void* dst, void* avg) {
  StreamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.src = src; a.dst = dst; a.uvw = h->d_uvw; a.bl_ant = h->d_bl_ant; a.freq_c = h->d_freq_c;
  a.n_ant = h->n_ant; a.n_chan = h->n_chan; a.n_time = h->n_time; a.n_bl = h->n_bl;
  a.nu0_c = h->nu0 / kCLight; a.dnu_c = h->dnu / kCLight;
  a.avg = avg;
  a.inv_n = 1.0 / ((double)h->n_time * h->n_chan);
  return a;
}

// one streaming pass: sub (subtract source) and/or acc (average for source)
int launch_stream(rts_peel_t* h, bool sub, bool acc, const StreamArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)h->n_bl), block(kStreamThreads);
  Span span(h, sub && acc ? RTS_K_SUB_AVERAGE : (sub ? RTS_K_SUBTRACT : RTS_K_AVERAGE), s);
  if (h->precision == RTS_PREC_MIXED) {
    const size_t smem = (size_t)h->n_time * 4 * sizeof(unsigned long long);
    if (sub && acc) k_stream_mixed<true, true><<<grid, block, smem, s>>>(a);
    else if (sub) k_stream_mixed<true, false><<<grid, block, smem, s>>>(a);
    else k_stream_mixed<false, true><<<grid, block, smem, s>>>(a);
  } else {
    const size_t smem = (size_t)h->n_time * 2 * sizeof(double);
    if (sub && acc) k_stream_fp64<true, true><<<grid, block, smem, s>>>(a);
    else if (sub) k_stream_fp64<true, false><<<grid, block, smem, s>>>(a);
    else k_stream_fp64<false, true><<<grid, block, smem, s>>>(a);
  }
  span.end(1);
  return check_launch(h, "streaming kernel launch");
}

// n_iter ALS sweeps on avg; Jones to jones_out (cube precision) and the FP64
// solution left in h->d_J[n_iter & 1]; status/rel to slot `slot`.
int launch_als(rts_peel_t* h, const void* avg, double S, void* jones_out, int slot, cudaStream_t s) {
  Span span(h, RTS_K_SOLVE, s);
  for (int it = 1; it <= h->n_iter; ++it) {
    AlsArgs a;
    a.avg = avg;
    a.J_old = h->d_J[(it - 1) & 1]; a.Jf_old = h->d_Jf[(it - 1) & 1];
    a.J_new = h->d_J[it & 1]; a.Jf_new = h->d_Jf[it & 1];
    a.norms = h->d_norms; a.flag = h->d_flag;
    a.jones_out = it == h->n_iter ? jones_out : nullptr;
    a.n_ant = h->n_ant; a.S = S; a.first = it == 1; a.average = (it % 2) == 0;
    if (h->precision == RTS_PREC_MIXED) k_als_sweep<float><<<als_grid(h->n_ant), kAlsThreads, 0, s>>>(a);
    else k_als_sweep<double><<<als_grid(h->n_ant), kAlsThreads, 0, s>>>(a);
  }
  k_als_finalize<<<1, 256, 0, s>>>(h->d_norms, h->n_ant, h->d_flag, h->d_status + slot, h->d_rel + slot);
  span.end(h->n_iter + 1);
  return check_launch(h, "ALS kernel launch");
}

const double2* als_solution(rts_peel_t* h) { return h->d_J[h->n_iter & 1]; }

int read_status(rts_peel_t* h, int32_t n, int32_t* h_status, cudaStream_t s) {
  RTS_CUDA(h, cudaMemcpyAsync(h_status, h->d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  int perr = 0;
  if (h->d_perr) RTS_CUDA(h, cudaMemcpyAsync(&perr, h->d_perr, sizeof(int), cudaMemcpyDeviceToHost, s));
  RTS_CUDA(h, cudaStreamSynchronize(s));
  if (perr) return fail(h, RTS_ECUDA, "a tensor-core completion wait of the blocked pass timed out");
  for (int k = 0; k < n; ++k)
    if (h_status[k] == kSolveStatusTimeout)
      return fail(h, RTS_ECUDA, "a grid barrier of the block solve timed out at source " + std::to_string(k));
  for (int k = 0; k < n; ++k)
    if (h_status[k] == RTS_ENONFINITE)
      return fail(h, RTS_ENONFINITE, "non-finite value in the solve of source " + std::to_string(k));
  return RTS_OK;
}

size_t block_pass_smem(const rts_peel_t* h) {
  // strip [n_chan][2] float4 | phases 2 x [BK] | FP64 sums [splits][BK][8] (splits*BK = 512)
  return (size_t)h->n_chan * 2 * sizeof(float4) + (size_t)2 * h->per_pass * sizeof(PhaseAB) +
         (size_t)2 * kBlkThreads * 8 * sizeof(double);
}

// geometry of block b (phases, then D_jk) into ring slot b % kRing, on the prep stream
void launch_block_geometry(rts_peel_t* h, int b, int n_src, cudaStream_t ps) {
  const int BK = h->per_pass, s0 = b * BK, nblk = std::min(BK, n_src - s0);
  const int r = b % rts_peel_t::kRing;
  const double* src = h->d_src + 3 * (size_t)s0;
  const unsigned g = 4 * (unsigned)h->n_sm;
  const double nu0_c = h->nu0 / kCLight, dnu_c = h->dnu / kCLight;
  const unsigned grid = (unsigned)h->n_bl;
  PhaseAB* ph = h->b_ph[r];
  GeoTrig* tg = h->b_trig[r];
  float2* Dt = h->b_dir[r];
#define RTS_GEOM(BKV)                                                                                   \
  k_block_ant_phases<BKV><<<g, 256, 0, ps>>>(src, nblk, h->d_uvw, h->n_ant, h->n_time, nu0_c, dnu_c,   \
                                             h->b_aph);                                                 \
  k_block_phases<BKV><<<g, 256, 0, ps>>>(h->b_aph, nblk, h->d_bl_ant, h->n_ant, h->n_time, h->n_band,  \
                                         h->band_chan0, h->n_bl, ph, tg);                               \
  if (nblk > 1)                                                                                          \
    k_block_dirichlet<BKV><<<grid, 256, 0, ps>>>(ph, tg, nblk, Dt, h->n_bl, h->n_time, h->n_band);
  switch (BK) {
    case 8: RTS_GEOM(8) break;
    case 16: RTS_GEOM(16) break;
    case 32: RTS_GEOM(32) break;
    default: RTS_GEOM(64) break;
  }
#undef RTS_GEOM
  h->launches[RTS_K_BLOCK_FIX] += nblk > 1 ? 3 : 2;
}

template <int BK>
int set_block_smem(rts_peel_t* h, int smem) {
  RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass<BK, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass<BK, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass<BK, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return RTS_OK;
}

int setup_block_solve(rts_peel_t* h);

// the tcgen05 pass holds all 512 TMEM columns: at least 116 KB of shared memory
// keeps it at one CTA per SM (a second CTA would wait in its TMEM allocation)
size_t tc05_launch_smem(const rts_peel_t* h) { return std::max<size_t>(tc05_pass_smem(h->n_chan), 116 * 1024); }
size_t tc05_tay_launch_smem(const rts_peel_t* h) {
  return std::max<size_t>(tc05_pass_smem(h->n_chan, true), 116 * 1024);
}

int ensure_block_workspace(rts_peel_t* h) {
  if (h->b_avg) return RTS_OK;
  const int BK = h->per_pass;
  const size_t n_ph = (size_t)h->n_bl * h->n_time * BK;
  for (int r = 0; r < rts_peel_t::kRing; ++r) {
    RTS_CUDA(h, cudaMalloc((void**)&h->b_ph[r], n_ph * sizeof(PhaseAB)));
    RTS_CUDA(h, cudaMalloc((void**)&h->b_trig[r], n_ph * sizeof(GeoTrig)));
    RTS_CUDA(h, cudaMalloc((void**)&h->b_dir[r], (size_t)h->n_bl * (BK * (BK - 1) / 2) * sizeof(float2)));
    RTS_CUDA(h, cudaEventCreateWithFlags(&h->b_ev_ready[r], cudaEventDisableTiming));
    RTS_CUDA(h, cudaEventCreateWithFlags(&h->b_ev_free[r], cudaEventDisableTiming));
  }
  RTS_CUDA(h, cudaMalloc((void**)&h->b_aph, (size_t)h->n_time * h->n_ant * BK * sizeof(PhaseAB)));
  RTS_CUDA(h, cudaMalloc((void**)&h->b_avg, (size_t)BK * h->n_bl * 4 * sizeof(float2)));
  RTS_CUDA(h, cudaMalloc((void**)&h->b_model, (size_t)BK * h->n_bl * 4 * sizeof(float2)));
  int lo_prio = 0, hi_prio = 0;
  RTS_CUDA(h, cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
  RTS_CUDA(h, cudaStreamCreateWithPriority(&h->b_main, cudaStreamNonBlocking, hi_prio));
  RTS_CUDA(h, cudaStreamCreateWithPriority(&h->b_prep, cudaStreamNonBlocking, lo_prio));
  RTS_CUDA(h, cudaEventCreateWithFlags(&h->b_ev_in, cudaEventDisableTiming));
  RTS_CUDA(h, cudaEventCreateWithFlags(&h->b_ev_out, cudaEventDisableTiming));
  RTS_CUDA(h, cudaEventCreateWithFlags(&h->b_ev_src, cudaEventDisableTiming));
  RTS_CUDA(h, cudaEventCreateWithFlags(&h->b_ev_done, cudaEventDisableTiming));
  int rc = setup_block_solve(h);
  if (rc) return rc;
  RTS_CUDA(h, cudaMalloc((void**)&h->d_perr, sizeof(int)));
  RTS_CUDA(h, cudaMemset(h->d_perr, 0, sizeof(int)));
  if (h->block_tc05) {
    const int tsm = (int)tc05_launch_smem(h);
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc05<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm));
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc05<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm));
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc05<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm));
    const int tay = (int)tc05_tay_launch_smem(h);
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc05<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tay));
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc05<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tay));
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc05<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tay));
    return RTS_OK;
  }
  if (h->block_tc) {
    const int tsm = (int)tc_pass_smem(h->n_chan);
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm));
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm));
    RTS_CUDA(h, cudaFuncSetAttribute(k_block_pass_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm));
    return RTS_OK;
  }
  const int smem = (int)block_pass_smem(h);
  switch (BK) {
    case 8: return set_block_smem<8>(h, smem);
    case 16: return set_block_smem<16>(h, smem);
    case 32: return set_block_smem<32>(h, smem);
    default: return set_block_smem<64>(h, smem);
  }
}

// geometry of the persistent block solve: one CTA per SM at most (fewer for
// small arrays), the rows of ceil(n_ant / G) antennas per CTA in shared memory.
// Leaves bs_ok false (the per-sweep launches are used) when the device has no
// cooperative launch or the rows do not fit.
int setup_block_solve(rts_peel_t* h) {
  if (h->solve_kernel != RTS_SOLVE_AUTO) return RTS_OK;
  int coop = 0, n_sm = 0, smem_max = 0;
  RTS_CUDA(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
  RTS_CUDA(h, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device));
  RTS_CUDA(h, cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  if (!coop || n_sm < 1) return RTS_OK;
  const int64_t want = std::max<int64_t>(h->n_ant, (h->n_bl + kSolveThreads - 1) / kSolveThreads);
  const int G = (int)std::min<int64_t>(n_sm, want);
  const int apc = (h->n_ant + G - 1) / G;
  if (apc > kSolveMaxApc || h->per_pass > kCorrMaxJ) return RTS_OK;
  const size_t smem = block_solve_smem(h->n_ant, apc);
  cudaFuncAttributes fa;
  RTS_CUDA(h, cudaFuncGetAttributes(&fa, k_block_solve));
  if (smem + fa.sharedSizeBytes + 1024 > (size_t)smem_max) return RTS_OK;
  RTS_CUDA(h, cudaFuncSetAttribute(k_block_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the whole unified memory as shared memory: the smallest carveout that holds one
  // solve CTA leaves no room beside it for the next block's phase and Dirichlet
  // kernels on the prep stream, which then wait for the solve to end
  RTS_CUDA(h, cudaFuncSetAttribute(k_block_solve, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared));
  int occ = 0;
  RTS_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_block_solve, kSolveThreads, smem));
  if (occ < 1) return RTS_OK;
  RTS_CUDA(h, cudaMalloc((void**)&h->b_sync, 2 * sizeof(unsigned)));
  RTS_CUDA(h, cudaMalloc((void**)&h->b_part, (size_t)h->per_pass * h->n_ant * 4 * sizeof(double)));
  h->bs_grid = G;
  h->bs_apc = apc;
  h->bs_smem = smem;
  h->bs_ok = true;
  return RTS_OK;
}

// the solve chain of sources s0 .. s0 + nblk - 1 (corrected averages, ALS,
// model matrices) as one cooperative launch
int launch_block_solve(rts_peel_t* h, int s0, int nblk, const float2* Dt, void* d_jones, cudaStream_t s) {
  Span span(h, RTS_K_SOLVE, s);
  BlockSolveArgs a;
  a.Ablk = h->b_avg; a.Dtab = Dt;
  a.src = h->d_src; a.s0 = s0; a.n_blk = nblk;
  a.bl_ant = h->d_bl_ant; a.n_ant = h->n_ant; a.n_bl = h->n_bl; a.n_iter = h->n_iter;
  a.apc = h->bs_apc;
  a.P = static_cast<float2*>(h->d_avg); a.M = h->b_model;
  a.Jf[0] = h->d_Jf[0]; a.Jf[1] = h->d_Jf[1];
  a.part = h->b_part; a.status = h->d_status; a.rel = h->d_rel;
  a.jones = static_cast<float2*>(d_jones);
  a.sync = h->b_sync;
  RTS_CUDA(h, cudaMemsetAsync(h->b_sync, 0, 2 * sizeof(unsigned), s));
  void* args[] = {&a};
  RTS_CUDA(h, cudaLaunchCooperativeKernel((const void*)k_block_solve, dim3(h->bs_grid), dim3(kSolveThreads), args,
                                          h->bs_smem, s));
  span.end(1);
  return check_launch(h, "block solve launch");
}

template <int BK>
void block_pass_t(bool sub, bool acc, const BlockPassArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  if (sub && acc) k_block_pass<BK, true, true><<<grid, kBlkThreads, smem, s>>>(a);
  else if (sub) k_block_pass<BK, true, false><<<grid, kBlkThreads, smem, s>>>(a);
  else k_block_pass<BK, false, true><<<grid, kBlkThreads, smem, s>>>(a);
}

int launch_block_pass(rts_peel_t* h, bool sub, bool acc, const BlockPassArgs& a, cudaStream_t s) {
  Span span(h, RTS_K_BLOCK_PASS, s);
  const unsigned grid = (unsigned)h->n_bl;
  if (h->block_tc05) {
    const size_t tsm = tc05_launch_smem(h);
    // up to kTc5BaselinesPerCta baselines a CTA, keeping at least 8 waves of CTAs
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kTc5BaselinesPerCta, h->n_bl / (8 * h->n_sm)));
    const unsigned g5 = (unsigned)((h->n_bl + nb - 1) / nb);
    if (sub && acc) k_block_pass_tc05<true, true><<<g5, kTc5Threads, tsm, s>>>(a, h->per_pass, nb, h->d_perr);
    else if (sub) k_block_pass_tc05<true, false><<<g5, kTc5Threads, tsm, s>>>(a, h->per_pass, nb, h->d_perr);
    else k_block_pass_tc05<false, true><<<g5, kTc5Threads, tsm, s>>>(a, h->per_pass, nb, h->d_perr);
    span.end(1);
    return check_launch(h, "block pass launch");
  }
  if (h->block_tc) {
    const size_t tsm = tc_pass_smem(h->n_chan);
    if (sub && acc) k_block_pass_tc<true, true><<<grid, kTcThreads, tsm, s>>>(a, h->per_pass);
    else if (sub) k_block_pass_tc<true, false><<<grid, kTcThreads, tsm, s>>>(a, h->per_pass);
    else k_block_pass_tc<false, true><<<grid, kTcThreads, tsm, s>>>(a, h->per_pass);
    span.end(1);
    return check_launch(h, "block pass launch");
  }
  const size_t smem = block_pass_smem(h);
  switch (h->per_pass) {
    case 8: block_pass_t<8>(sub, acc, a, grid, smem, s); break;
    case 16: block_pass_t<16>(sub, acc, a, grid, smem, s); break;
    case 32: block_pass_t<32>(sub, acc, a, grid, smem, s); break;
    default: block_pass_t<64>(sub, acc, a, grid, smem, s); break;
  }
  span.end(1);
  return check_launch(h, "block pass launch");
}

// The blocked cadence: one HBM pass per block of BK sources (see block_kernels.cuh).
// Main stream: passes, in-block corrections, solves.  Prep stream: the
// geometry tables of the blocks, up to kRing blocks ahead.  The cadence runs as
// blocked_begin (the first pass: block 0's averages), blocked_block for every
// block (its solve, then the pass that subtracts it and averages the next
// block) and blocked_end; rts_peel_cadence runs them back to back, the
// channel-shard calls return to the caller before each solve so that the
// averages of all shards can be summed.
int blocked_begin(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src, const double* h_src,
                  void* d_jones, cudaStream_t user) {
  int rc = ensure_block_workspace(h);
  if (rc) return rc;
  constexpr int R = rts_peel_t::kRing;
  const int BK = h->per_pass;
  rts_peel_t::BlockRun& br = h->br;
  br = rts_peel_t::BlockRun();
  br.vis = d_vis; br.resid = d_resid; br.jones = d_jones; br.n_src = n_src;
  br.src.assign(h_src, h_src + 3 * (size_t)n_src);
  br.nb = (n_src + BK - 1) / BK;
  br.b = 0;
  br.user = user;
  // work on the library's high-priority stream, ordered after the caller's stream
  cudaStream_t s = h->b_main;
  RTS_CUDA(h, cudaEventRecord(h->b_ev_in, user));
  RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_in, 0));
  RTS_CUDA(h, cudaMemsetAsync(h->d_perr, 0, sizeof(int), s));      // the pass's wait-timeout flag
  RTS_CUDA(h, cudaMemcpyAsync(h->d_src, br.src.data(), sizeof(double) * 3 * n_src, cudaMemcpyHostToDevice, s));
  RTS_CUDA(h, cudaEventRecord(h->b_ev_src, s));
  RTS_CUDA(h, cudaStreamWaitEvent(h->b_prep, h->b_ev_src, 0));
  for (int b = 0; b < std::min(br.nb, R); ++b) {
    launch_block_geometry(h, b, n_src, h->b_prep);
    RTS_CUDA(h, cudaEventRecord(h->b_ev_ready[b % R], h->b_prep));
  }
  BlockPassArgs& a = br.a;
  std::memset(&a, 0, sizeof(a));
  a.n_ant = h->n_ant; a.n_chan = h->n_chan; a.n_time = h->n_time; a.n_bl = h->n_bl;
  a.inv_n = 1.0 / ((double)h->n_time * h->n_band);     // the whole band's samples: shards' averages add up
  a.M_sub = h->b_model; a.avg = h->b_avg;
  // first pass: plain averages of block 0 from the input
  RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_ready[0], 0));
  a.src = static_cast<const float4*>(d_vis);
  a.n_acc = std::min(BK, (int)n_src); a.ph_acc = h->b_ph[0];
  rc = launch_block_pass(h, false, true, a, s);
  if (rc) return rc;
  br.active = true;
  return RTS_OK;
}

// block br.b: its solve from the (summed) averages in b_avg, then the pass that
// subtracts it and averages block br.b + 1
int blocked_block(rts_peel_t* h) {
  constexpr int R = rts_peel_t::kRing;
  rts_peel_t::BlockRun& br = h->br;
  const int BK = h->per_pass, b = br.b;
  const int n_src = br.n_src, s0 = b * BK, nblk = std::min(BK, n_src - s0);
  const double* h_src = br.src.data();
  cudaStream_t s = h->b_main;
  const size_t jstride = (size_t)h->n_ant * 4 * h->elem;
  const unsigned bl_grid = (unsigned)((h->n_bl + 255) / 256);
  const float2* Dt = h->b_dir[b % R];
  int rc;
  if (h->bs_ok) {
    rc = launch_block_solve(h, s0, nblk, Dt, br.jones, s);
    if (rc) return rc;
  }
  for (int q = 0; q < nblk && !h->bs_ok; ++q) {
    const int k = s0 + q;
    {
      Span span(h, RTS_K_BLOCK_FIX, s);
      if (q > 0)
        k_block_model<<<bl_grid, 256, 0, s>>>(als_solution(h), h_src[3 * (k - 1) + 2], h->d_bl_ant, h->n_bl,
                                               h->b_model + (size_t)(q - 1) * h->n_bl * 4);
      k_block_correct<<<bl_grid, 256, 0, s>>>(h->b_avg, q, h->b_model, Dt, h->n_bl,
                                              static_cast<float2*>(h->d_avg));
      span.end(q > 0 ? 2 : 1);
    }
    rc = launch_als(h, h->d_avg, h_src[3 * k + 2], static_cast<char*>(br.jones) + k * jstride, k, s);
    if (rc) return rc;
  }
  if (!h->bs_ok) {
    Span span(h, RTS_K_BLOCK_FIX, s);
    k_block_model<<<bl_grid, 256, 0, s>>>(als_solution(h), h_src[3 * (s0 + nblk - 1) + 2], h->d_bl_ant,
                                           h->n_bl, h->b_model + (size_t)(nblk - 1) * h->n_bl * 4);
    span.end(1);
  }
  // subtract block b (input -> residual on the first block), average block b+1
  BlockPassArgs& a = br.a;
  const bool more = b + 1 < br.nb;
  if (more) RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_ready[(b + 1) % R], 0));
  a.src = static_cast<const float4*>(b == 0 ? br.vis : br.resid);
  a.dst = static_cast<float4*>(br.resid);
  a.n_sub = nblk; a.ph_sub = h->b_ph[b % R];
  a.n_acc = more ? std::min(BK, n_src - s0 - BK) : 0;
  a.ph_acc = h->b_ph[(b + 1) % R];
  rc = launch_block_pass(h, true, more, a, s);
  if (rc) return rc;
  // slot b is free once that pass has run: the prep stream may fill it with block b + R
  RTS_CUDA(h, cudaEventRecord(h->b_ev_free[b % R], s));
  if (b + R < br.nb) {
    RTS_CUDA(h, cudaStreamWaitEvent(h->b_prep, h->b_ev_free[b % R], 0));
    launch_block_geometry(h, b + R, n_src, h->b_prep);
    RTS_CUDA(h, cudaEventRecord(h->b_ev_ready[b % R], h->b_prep));
  }
  ++br.b;
  return RTS_OK;
}

// the caller's stream waits for the library's (outputs or partial averages ready)
int blocked_to_user(rts_peel_t* h) {
  RTS_CUDA(h, cudaEventRecord(h->b_ev_out, h->b_main));
  RTS_CUDA(h, cudaStreamWaitEvent(h->br.user, h->b_ev_out, 0));
  return RTS_OK;
}

int blocked_end(rts_peel_t* h, int32_t* h_status) {
  rts_peel_t::BlockRun& br = h->br;
  br.active = false;
  RTS_CUDA(h, cudaEventRecord(h->b_ev_done, h->b_prep));
  RTS_CUDA(h, cudaStreamWaitEvent(h->b_main, h->b_ev_done, 0));
  int rc = blocked_to_user(h);
  if (rc) return rc;
  rc = check_launch(h, "block geometry launch");
  if (rc) return rc;
  if (h_status) return read_status(h, br.n_src, h_status, br.user);
  return RTS_OK;
}

int peel_blocked(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src,
                 const double* h_src, void* d_jones, int32_t* h_status, cudaStream_t s) {
  int rc = blocked_begin(h, d_vis, d_resid, n_src, h_src, d_jones, s);
  while (rc == RTS_OK && h->br.b < h->br.nb) rc = blocked_block(h);
  if (rc) {
    h->br.active = false;
    return rc;
  }
  return blocked_end(h, h_status);
}

int peel_device(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src,
                const double* h_src, void* d_jones, int32_t* h_status, cudaStream_t s) {
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  if (n_src == 0) {
    if (d_resid != d_vis) RTS_CUDA(h, cudaMemcpyAsync(d_resid, d_vis, cube, cudaMemcpyDeviceToDevice, s));
    return RTS_OK;
  }
  if (h->per_pass > 1) return peel_blocked(h, d_vis, d_resid, n_src, h_src, d_jones, h_status, s);
  const size_t jstride = (size_t)h->n_ant * 4 * h->elem;
  StreamArgs a = stream_args(h, d_vis, d_resid, h->d_avg);
  a.acc = make_dir(h_src[0], h_src[1], h_src[2]);
  int rc = launch_stream(h, false, true, a, s);
  if (rc) return rc;
  for (int k = 0; k < n_src; ++k) {
    rc = launch_als(h, h->d_avg, h_src[3 * k + 2], static_cast<char*>(d_jones) + k * jstride, k, s);
    if (rc) return rc;
    StreamArgs b = stream_args(h, k == 0 ? d_vis : d_resid, d_resid, h->d_avg);
    b.sub = make_dir(h_src[3 * k], h_src[3 * k + 1], h_src[3 * k + 2]);
    b.Jsub = als_solution(h);
    const bool more = k + 1 < n_src;
    if (more) b.acc = make_dir(h_src[3 * (k + 1)], h_src[3 * (k + 1) + 1], h_src[3 * (k + 1) + 2]);
    rc = launch_stream(h, true, more, b, s);
    if (rc) return rc;
  }
  if (h_status) return read_status(h, n_src, h_status, s);
  return RTS_OK;
}

// ---- gains Taylor-expanded in frequency (taylor_kernels.cuh) -------------------

// allocates whatever is still missing (a failed call leaves the rest for the next)
int taylor_setup(rts_peel_t* h) {
  if (!h->t_mom) RTS_CUDA(h, cudaMalloc(&h->t_mom, (size_t)3 * h->n_bl * 4 * sizeof(float2)));
  for (int k = 0; k < 2; ++k) {
    if (!h->t_X[k]) RTS_CUDA(h, cudaMalloc(&h->t_X[k], (size_t)h->n_ant * 8 * sizeof(double2)));
    if (!h->t_Xf[k]) RTS_CUDA(h, cudaMalloc(&h->t_Xf[k], (size_t)h->n_ant * 8 * sizeof(float2)));
  }
  h->t_rot_grid = (int)std::max<int64_t>(1, std::min<int64_t>(kRotMaxGrid, (h->n_bl + kRotThreads - 1) / kRotThreads));
  if (!h->t_rot_part) RTS_CUDA(h, cudaMalloc(&h->t_rot_part, (size_t)h->t_rot_grid * kRotVals * sizeof(double)));
  if (!h->t_rot_step) RTS_CUDA(h, cudaMalloc(&h->t_rot_step, 5 * sizeof(double)));
  if (!h->t_rot_count) {
    RTS_CUDA(h, cudaMalloc(&h->t_rot_count, sizeof(unsigned)));
    RTS_CUDA(h, cudaMemset(h->t_rot_count, 0, sizeof(unsigned)));
  }
  return RTS_OK;
}

// x_c = x0 + c dx, the channel's offset from the band centre in band widths
void taylor_axis(const rts_peel_t* h, float* x0, float* dx, double (&mu)[5]) {
  const int n = h->n_chan;
  for (int k = 0; k < 5; ++k) mu[k] = 0.0;
  for (int c = 0; c < n; ++c) {
    const double x = (c - 0.5 * (n - 1)) / n;
    double xp = 1.0;
    for (int k = 0; k < 5; ++k) { mu[k] += xp; xp *= x; }
  }
  for (int k = 0; k < 5; ++k) mu[k] /= n;
  *x0 = (float)(-0.5 * (n - 1) / n);
  *dx = (float)(1.0 / n);
}

int launch_stream_taylor(rts_peel_t* h, bool sub, bool acc, const TaylorStreamArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)h->n_bl), block(kStreamThreads);
  const size_t smem = (size_t)h->n_time * 4 * sizeof(unsigned long long);
  Span span(h, sub && acc ? RTS_K_SUB_AVERAGE : (sub ? RTS_K_SUBTRACT : RTS_K_AVERAGE), s);
  if (sub && acc) k_stream_taylor<true, true><<<grid, block, smem, s>>>(a);
  else if (sub) k_stream_taylor<true, false><<<grid, block, smem, s>>>(a);
  else k_stream_taylor<false, true><<<grid, block, smem, s>>>(a);
  span.end(1);
  return check_launch(h, "Taylor streaming kernel launch");
}

// n_iter Taylor sweeps on h->t_mom; G, H of the last sweep to gain_out / slope_out,
// the FP64 solution left in h->t_X[n_iter & 1]; status/rel to slot `slot`
int launch_als_taylor(rts_peel_t* h, double S, float2* gain_out, float2* slope_out, int slot,
                      cudaStream_t s) {
  float x0, dx;
  double mu[5];
  taylor_axis(h, &x0, &dx, mu);
  Span span(h, RTS_K_SOLVE, s);
  for (int it = 1; it <= h->n_iter; ++it) {
    TaylorAlsArgs a;
    a.mom = h->t_mom;
    a.X_old = h->t_X[(it - 1) & 1]; a.Xf_old = h->t_Xf[(it - 1) & 1];
    a.X_new = h->t_X[it & 1]; a.Xf_new = h->t_Xf[it & 1];
    a.norms = h->d_norms; a.flag = h->d_flag;
    a.gain_out = it == h->n_iter ? gain_out : nullptr;
    a.slope_out = it == h->n_iter ? slope_out : nullptr;
    a.n_ant = h->n_ant; a.n_bl = h->n_bl; a.S = S;
    for (int k = 0; k < 5; ++k) a.mu[k] = mu[k];
    a.first = it == 1; a.average = (it % 2) == 0;
    k_als_taylor_sweep<<<(unsigned)h->n_ant, kAlsThreads, 0, s>>>(a);
    if (it >= 2 && h->n_chan >= 3) {         // the common slope-rotation step (three channels or more)
      TaylorRotArgs r;
      r.mom = h->t_mom; r.Xf = h->t_Xf[it & 1]; r.bl_ant = h->d_bl_ant; r.n_bl = h->n_bl;
      r.S = (float)S; r.mu2 = (float)mu[2]; r.mu3 = (float)mu[3]; r.mu4 = (float)mu[4];
      r.part = h->t_rot_part; r.count = h->t_rot_count; r.step = h->t_rot_step;
      k_taylor_rot_sums<<<(unsigned)h->t_rot_grid, kRotThreads, 0, s>>>(r);
      k_taylor_rot_apply<<<(unsigned)((8 * h->n_ant + 255) / 256), 256, 0, s>>>(
          h->t_rot_step, h->t_X[it & 1], h->t_X[(it - 1) & 1], h->t_Xf[it & 1], h->d_norms, h->d_flag,
          a.gain_out, a.slope_out, h->n_ant);
    }
  }
  k_als_finalize<<<1, 256, 0, s>>>(h->d_norms, h->n_ant, h->d_flag, h->d_status + slot, h->d_rel + slot);
  span.end(h->n_chan >= 3 ? 3 * h->n_iter - 1 : h->n_iter + 1);
  return check_launch(h, "Taylor ALS kernel launch");
}

int peel_taylor(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src, const double* h_src,
                void* d_gain, void* d_slope, int32_t* h_status, cudaStream_t s) {
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  if (n_src == 0) {
    if (d_resid != d_vis) RTS_CUDA(h, cudaMemcpyAsync(d_resid, d_vis, cube, cudaMemcpyDeviceToDevice, s));
    return RTS_OK;
  }
  int rc = taylor_setup(h);
  if (rc) return rc;
  float x0, dx;
  double mu[5];
  taylor_axis(h, &x0, &dx, mu);
  const size_t jstride = (size_t)h->n_ant * 4;
  TaylorStreamArgs a;
  a.s = stream_args(h, d_vis, d_resid, nullptr);
  a.s.acc = make_dir(h_src[0], h_src[1], h_src[2]);
  a.Xsub = nullptr; a.mom = h->t_mom; a.x0 = x0; a.dx = dx;
  rc = launch_stream_taylor(h, false, true, a, s);
  if (rc) return rc;
  for (int k = 0; k < n_src; ++k) {
    rc = launch_als_taylor(h, h_src[3 * k + 2], static_cast<float2*>(d_gain) + k * jstride,
                           static_cast<float2*>(d_slope) + k * jstride, k, s);
    if (rc) return rc;
    TaylorStreamArgs b;
    b.s = stream_args(h, k == 0 ? d_vis : d_resid, d_resid, nullptr);
    b.s.sub = make_dir(h_src[3 * k], h_src[3 * k + 1], h_src[3 * k + 2]);
    b.Xsub = h->t_X[h->n_iter & 1];
    b.mom = h->t_mom; b.x0 = x0; b.dx = dx;
    const bool more = k + 1 < n_src;
    if (more) b.s.acc = make_dir(h_src[3 * (k + 1)], h_src[3 * (k + 1) + 1], h_src[3 * (k + 1) + 2]);
    rc = launch_stream_taylor(h, true, more, b, s);
    if (rc) return rc;
  }
  if (h_status) return read_status(h, n_src, h_status, s);
  return RTS_OK;
}

// ---- gains Taylor-expanded in frequency, blocked (taylor_block_kernels.cuh) ----
// kTayBlk sources per pass through the tcgen05 pass's Taylor form; needs the
// tcgen05 blocked workspace of 64-source blocks (its tables hold a Taylor
// block: phases of 21 <= 32 sources, 210 x 5 <= 2016 D terms, 63 slots)
bool taylor_blocked(const rts_peel_t* h) {
  return h->block_tc05 && h->per_pass == kTc5Src && h->n_band == h->n_chan;
}

// mu_j = mean_c x_c^j, x_c = (c - (N - 1)/2) / N, in FP64 (odd j: zero by symmetry)
TayMu taylor_mu(const rts_peel_t* h) {
  const int n = h->n_chan;
  double acc[kTayMu] = {};
  for (int c = 0; c < n; ++c) {
    const double x = (c - 0.5 * (n - 1)) / n;
    double xp = 1.0;
    for (int j = 0; j < kTayMu; ++j, xp *= x) acc[j] += xp;
  }
  TayMu mu;
  for (int j = 0; j < kTayMu; ++j) mu.mu[j] = (j & 1) ? 0.f : (float)(acc[j] / n);
  return mu;
}

// geometry of Taylor block b (phases with a stride of 32 sources, D^(0..4)) into
// ring slot b % kRing, on the prep stream
void launch_taylor_geometry(rts_peel_t* h, int b, int n_src, cudaStream_t ps) {
  constexpr int BKG = 32;
  const int s0 = b * kTayBlk, nblk = std::min(kTayBlk, n_src - s0);
  const int r = b % rts_peel_t::kRing;
  const unsigned g = 4 * (unsigned)h->n_sm;
  const double nu0_c = h->nu0 / kCLight, dnu_c = h->dnu / kCLight;
  k_block_ant_phases<BKG><<<g, 256, 0, ps>>>(h->d_src + 3 * (size_t)s0, nblk, h->d_uvw, h->n_ant, h->n_time,
                                             nu0_c, dnu_c, h->b_aph);
  k_block_phases<BKG><<<g, 256, 0, ps>>>(h->b_aph, nblk, h->d_bl_ant, h->n_ant, h->n_time, h->n_band,
                                         h->band_chan0, h->n_bl, h->b_ph[r], h->b_trig[r]);
  if (nblk > 1)
    k_block_dirichlet_taylor<BKG><<<(unsigned)h->n_bl, 256, 0, ps>>>(h->b_ph[r], h->b_trig[r], nblk, h->b_dir[r],
                                                                     h->n_bl, h->n_time, h->n_chan, taylor_mu(h));
  h->launches[RTS_K_BLOCK_FIX] += nblk > 1 ? 3 : 2;
}

int launch_taylor_pass(rts_peel_t* h, bool sub, bool acc, const BlockPassArgs& a, cudaStream_t s) {
  Span span(h, RTS_K_BLOCK_PASS, s);
  const unsigned grid = (unsigned)h->n_bl;
  const size_t tsm = tc05_tay_launch_smem(h);
  if (sub && acc) k_block_pass_tc05<true, true, true><<<grid, kTc5Threads, tsm, s>>>(a, 32, 1, h->d_perr);
  else if (sub) k_block_pass_tc05<true, false, true><<<grid, kTc5Threads, tsm, s>>>(a, 32, 1, h->d_perr);
  else k_block_pass_tc05<false, true, true><<<grid, kTc5Threads, tsm, s>>>(a, 32, 1, h->d_perr);
  span.end(1);
  return check_launch(h, "Taylor block pass launch");
}

// The blocked Taylor cadence: a pass subtracts block b's models and takes the
// plain moments of block b + 1; inside a block each source's moments are
// corrected with D^(0..4) (k_taylor_correct), solved by the Taylor ALS, and its
// P0, P1, P2 go to the block's model table (k_taylor_model)
int peel_taylor_blocked(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src, const double* h_src,
                        void* d_gain, void* d_slope, int32_t* h_status, cudaStream_t user) {
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  if (n_src == 0) {
    if (d_resid != d_vis) RTS_CUDA(h, cudaMemcpyAsync(d_resid, d_vis, cube, cudaMemcpyDeviceToDevice, user));
    return RTS_OK;
  }
  constexpr int R = rts_peel_t::kRing;
  const int nb = (n_src + kTayBlk - 1) / kTayBlk;
  const size_t jstride = (size_t)h->n_ant * 4;
  const unsigned bl_grid = (unsigned)((h->n_bl + 255) / 256);
  cudaStream_t s = h->b_main;
  RTS_CUDA(h, cudaEventRecord(h->b_ev_in, user));
  RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_in, 0));
  RTS_CUDA(h, cudaMemsetAsync(h->d_perr, 0, sizeof(int), s));
  std::vector<double> src(h_src, h_src + 3 * (size_t)n_src);
  RTS_CUDA(h, cudaMemcpyAsync(h->d_src, src.data(), sizeof(double) * 3 * n_src, cudaMemcpyHostToDevice, s));
  RTS_CUDA(h, cudaEventRecord(h->b_ev_src, s));
  RTS_CUDA(h, cudaStreamWaitEvent(h->b_prep, h->b_ev_src, 0));
  for (int b = 0; b < std::min(nb, R); ++b) {
    launch_taylor_geometry(h, b, n_src, h->b_prep);
    RTS_CUDA(h, cudaEventRecord(h->b_ev_ready[b % R], h->b_prep));
  }
  float x0, dx;
  double mu[5];
  taylor_axis(h, &x0, &dx, mu);
  BlockPassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_ant = h->n_ant; a.n_chan = h->n_chan; a.n_time = h->n_time; a.n_bl = h->n_bl;
  a.inv_n = 1.0 / ((double)h->n_time * h->n_chan);
  a.M_sub = h->b_model; a.avg = h->b_avg;
  a.tx0 = x0; a.tdx = dx;
  RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_ready[0], 0));
  a.src = static_cast<const float4*>(d_vis);
  a.n_acc = std::min(kTayBlk, (int)n_src); a.ph_acc = h->b_ph[0];
  int rc = launch_taylor_pass(h, false, true, a, s);
  if (rc) return rc;
  for (int b = 0; b < nb; ++b) {
    const int s0 = b * kTayBlk, nblk = std::min(kTayBlk, n_src - s0);
    const float2* Dt = h->b_dir[b % R];
    for (int q = 0; q < nblk; ++q) {
      const int k = s0 + q;
      {
        Span span(h, RTS_K_BLOCK_FIX, s);
        k_taylor_correct<<<bl_grid, 256, 0, s>>>(h->b_avg, q, h->b_model, Dt, h->n_bl, h->t_mom);
        span.end(1);
      }
      rc = launch_als_taylor(h, src[3 * k + 2], static_cast<float2*>(d_gain) + k * jstride,
                             static_cast<float2*>(d_slope) + k * jstride, k, s);
      if (rc) return rc;
      {
        Span span(h, RTS_K_BLOCK_FIX, s);
        k_taylor_model<<<bl_grid, 256, 0, s>>>(h->t_Xf[h->n_iter & 1], (float)src[3 * k + 2], h->d_bl_ant,
                                               h->n_bl, h->b_model + (size_t)(3 * q) * h->n_bl * 4);
        span.end(1);
      }
    }
    const bool more = b + 1 < nb;
    if (more) RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_ready[(b + 1) % R], 0));
    a.src = static_cast<const float4*>(b == 0 ? d_vis : d_resid);
    a.dst = static_cast<float4*>(d_resid);
    a.n_sub = nblk; a.ph_sub = h->b_ph[b % R];
    a.n_acc = more ? std::min(kTayBlk, n_src - s0 - kTayBlk) : 0;
    a.ph_acc = h->b_ph[(b + 1) % R];
    rc = launch_taylor_pass(h, true, more, a, s);
    if (rc) return rc;
    RTS_CUDA(h, cudaEventRecord(h->b_ev_free[b % R], s));
    if (b + R < nb) {
      RTS_CUDA(h, cudaStreamWaitEvent(h->b_prep, h->b_ev_free[b % R], 0));
      launch_taylor_geometry(h, b + R, n_src, h->b_prep);
      RTS_CUDA(h, cudaEventRecord(h->b_ev_ready[b % R], h->b_prep));
    }
  }
  RTS_CUDA(h, cudaEventRecord(h->b_ev_done, h->b_prep));
  RTS_CUDA(h, cudaStreamWaitEvent(s, h->b_ev_done, 0));
  RTS_CUDA(h, cudaEventRecord(h->b_ev_out, s));
  RTS_CUDA(h, cudaStreamWaitEvent(user, h->b_ev_out, 0));
  rc = check_launch(h, "Taylor block geometry launch");
  if (rc) return rc;
  if (h_status) return read_status(h, n_src, h_status, user);
  return RTS_OK;
}

}  // namespace

extern "C" {

int rts_peel_cadence_taylor(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src,
                            const double* h_src, void* d_gain, void* d_slope, int32_t* h_status,
                            void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (h->precision != RTS_PREC_MIXED) return fail(h, RTS_EINVAL, "Taylor gains need an RTS_PREC_MIXED handle");
  if (h->n_band != h->n_chan || h->br.active)
    return fail(h, RTS_EINVAL, "Taylor gains need a handle that holds the whole band and no cadence in progress");
  if (h->n_chan < 2) return fail(h, RTS_EINVAL, "Taylor gains need n_chan >= 2");
  if (!d_vis || !d_resid) return fail(h, RTS_EINVAL, "d_vis and d_resid are required");
  if (misaligned(d_vis) || misaligned(d_resid))
    return fail(h, RTS_EINVAL, "d_vis and d_resid must start on a 16-byte boundary");
  int rc = validate_sources(h, n_src, h_src);
  if (rc) return rc;
  if (n_src > 0 && (!d_gain || !d_slope)) return fail(h, RTS_EINVAL, "d_gain and d_slope are required");
  if (n_src > 0 && (misaligned(d_gain) || misaligned(d_slope)))
    return fail(h, RTS_EINVAL, "d_gain and d_slope must start on a 16-byte boundary");
  if (taylor_blocked(h))
    return peel_taylor_blocked(h, d_vis, d_resid, n_src, h_src, d_gain, d_slope, h_status, as_stream(stream));
  return peel_taylor(h, d_vis, d_resid, n_src, h_src, d_gain, d_slope, h_status, as_stream(stream));
}

int rts_peel_init(const rts_peel_config* cfg, rts_peel_t** out) {
  g_init_err.clear();
  if (!out) return fail(nullptr, RTS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, RTS_EINVAL, "cfg is NULL");
  if (cfg->n_ant < 2 || cfg->n_ant > 8192) return fail(nullptr, RTS_EINVAL, "n_ant must be in [2, 8192]");
  if (cfg->n_chan < 1 || cfg->n_chan > 65536) return fail(nullptr, RTS_EINVAL, "n_chan must be in [1, 65536]");
  if (cfg->n_time < 1 || cfg->n_time > 1024) return fail(nullptr, RTS_EINVAL, "n_time must be in [1, 1024]");
  if (cfg->n_iter < 1 || cfg->n_iter > 10000) return fail(nullptr, RTS_EINVAL, "n_iter must be in [1, 10000]");
  if (cfg->precision != RTS_PREC_MIXED && cfg->precision != RTS_PREC_FP64)
    return fail(nullptr, RTS_EINVAL, "precision must be RTS_PREC_MIXED or RTS_PREC_FP64");
  if (cfg->max_sources < 1 || cfg->max_sources > (1 << 20))
    return fail(nullptr, RTS_EINVAL, "max_sources must be in [1, 2^20]");
  if (!cfg->uvw || !cfg->freq_hz) return fail(nullptr, RTS_EINVAL, "uvw and freq_hz are required");
  const int64_t n_bl = (int64_t)cfg->n_ant * (cfg->n_ant - 1) / 2;
  if ((double)cfg->n_time * cfg->n_chan * n_bl >= 4.0e12)
    return fail(nullptr, RTS_EINVAL, "cube too large");
  const size_t n_uvw = (size_t)cfg->n_time * cfg->n_ant * 3;
  for (size_t i = 0; i < n_uvw; ++i)
    if (!std::isfinite(cfg->uvw[i])) return fail(nullptr, RTS_EINVAL, "uvw has a non-finite value");
  const double* f = cfg->freq_hz;
  const double nu0 = f[0];
  const double dnu = cfg->n_chan > 1 ? (f[cfg->n_chan - 1] - f[0]) / (cfg->n_chan - 1) : 0.0;
  for (int c = 0; c < cfg->n_chan; ++c) {
    if (!std::isfinite(f[c]) || !(f[c] > 0)) return fail(nullptr, RTS_EINVAL, "frequencies must be finite and > 0");
    if (std::fabs(f[c] - (nu0 + c * dnu)) > 1e-9 * std::fabs(f[c]))
      return fail(nullptr, RTS_EINVAL, "channels must be uniformly spaced (nu_c = nu_0 + c dnu)");
  }

  int per_pass = cfg->sources_per_pass;
  if (per_pass == 0) per_pass = cfg->precision == RTS_PREC_MIXED ? RTS_BLOCK : 1;
  if (per_pass != 1 && per_pass != 8 && per_pass != 16 && per_pass != 32 && per_pass != 64)
    return fail(nullptr, RTS_EINVAL, "sources_per_pass must be 0, 1, 8, 16, 32 or 64");
  if (per_pass > 1 && cfg->precision != RTS_PREC_MIXED)
    return fail(nullptr, RTS_EINVAL, "the blocked peel (sources_per_pass = RTS_BLOCK) is RTS_PREC_MIXED only");
  if (per_pass > 1 && (size_t)cfg->n_chan * 32 + 2048 + 32768 > 200 * 1024)
    return fail(nullptr, RTS_EINVAL, "the blocked peel needs n_chan*32 + 34 KB <= 200 KB of shared memory "
                                     "(n_chan <= 5300); use sources_per_pass = 1");
  if (cfg->block_kernel < RTS_BLOCK_AUTO || cfg->block_kernel > RTS_BLOCK_TCGEN05)
    return fail(nullptr, RTS_EINVAL,
                "block_kernel must be RTS_BLOCK_AUTO, RTS_BLOCK_FMA, RTS_BLOCK_TENSOR or RTS_BLOCK_TCGEN05");
  if (cfg->block_kernel == RTS_BLOCK_TENSOR && cfg->n_chan > kTcMaxChan)
    return fail(nullptr, RTS_EINVAL, "the tensor-core blocked pass needs n_chan <= 960");
  if (cfg->block_kernel == RTS_BLOCK_TCGEN05 && cfg->n_chan > kTc5MaxChan)
    return fail(nullptr, RTS_EINVAL, "the tcgen05 blocked pass needs n_chan <= 768");

  const int n_band = cfg->band_n_chan > 0 ? cfg->band_n_chan : cfg->n_chan;
  if (cfg->band_n_chan < 0 || cfg->band_chan0 < 0 || cfg->band_chan0 + cfg->n_chan > n_band ||
      (cfg->band_n_chan == 0 && cfg->band_chan0 != 0))
    return fail(nullptr, RTS_EINVAL, "band_chan0 .. band_chan0 + n_chan - 1 must lie in the band's band_n_chan channels");
  if (n_band != cfg->n_chan && per_pass == 1)
    return fail(nullptr, RTS_EINVAL, "a channel shard (band_n_chan > n_chan) needs the blocked peel "
                                     "(RTS_PREC_MIXED, sources_per_pass > 1)");
  if (cfg->solve_kernel != RTS_SOLVE_AUTO && cfg->solve_kernel != RTS_SOLVE_LAUNCHES)
    return fail(nullptr, RTS_EINVAL, "solve_kernel must be RTS_SOLVE_AUTO or RTS_SOLVE_LAUNCHES");
  if (cfg->grad_kernel != RTS_GRAD_AUTO && cfg->grad_kernel != RTS_GRAD_DIRECT)
    return fail(nullptr, RTS_EINVAL, "grad_kernel must be RTS_GRAD_AUTO or RTS_GRAD_DIRECT");

  rts_peel_t* h = new rts_peel_t();
  h->per_pass = per_pass;
  h->solve_kernel = cfg->solve_kernel;
  h->grad_direct = cfg->grad_kernel == RTS_GRAD_DIRECT;
  {
    int bk = cfg->block_kernel;
    if (bk == RTS_BLOCK_AUTO)
      bk = cfg->n_chan <= kTc5MaxChan ? RTS_BLOCK_TCGEN05 : (cfg->n_chan <= kTcMaxChan ? RTS_BLOCK_TENSOR : RTS_BLOCK_FMA);
    h->block_tc05 = per_pass > 1 && bk == RTS_BLOCK_TCGEN05;
    h->block_tc = per_pass > 1 && bk == RTS_BLOCK_TENSOR;
  }
  h->n_ant = cfg->n_ant; h->n_chan = cfg->n_chan; h->n_time = cfg->n_time;
  h->n_iter = cfg->n_iter; h->precision = cfg->precision; h->max_sources = cfg->max_sources;
  h->n_bl = n_bl; h->nu0 = nu0; h->dnu = dnu;
  h->n_band = n_band; h->band_chan0 = cfg->band_chan0;
  h->elem = cfg->precision == RTS_PREC_MIXED ? sizeof(float2) : sizeof(double2);
  auto bail = [&](cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    int code = e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA;
    rts_peel_destroy(h);
    return fail(nullptr, code, m);
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
    return bail(e, "cudaDeviceGetAttribute");
  std::vector<int2> map((size_t)n_bl);
  {
    int64_t b = 0;
    for (int i = 0; i < h->n_ant; ++i)
      for (int j = i + 1; j < h->n_ant; ++j) map[b++] = make_int2(i, j);
  }
  std::vector<double> fc(h->n_chan);
  for (int c = 0; c < h->n_chan; ++c) fc[c] = f[c] / kCLight;
  const size_t n_cplx_ant = (size_t)h->n_ant * 4;
  struct { void** p; size_t bytes; } allocs[] = {
      {(void**)&h->d_uvw, n_uvw * sizeof(double)},
      {(void**)&h->d_bl_ant, (size_t)n_bl * sizeof(int2)},
      {(void**)&h->d_freq_c, (size_t)h->n_chan * sizeof(double)},
      {(void**)&h->d_avg, (size_t)n_bl * 4 * h->elem},
      {(void**)&h->d_J[0], n_cplx_ant * sizeof(double2)},
      {(void**)&h->d_J[1], n_cplx_ant * sizeof(double2)},
      {(void**)&h->d_Jf[0], n_cplx_ant * sizeof(float2)},
      {(void**)&h->d_Jf[1], n_cplx_ant * sizeof(float2)},
      {(void**)&h->d_norms, (size_t)h->n_ant * 2 * sizeof(double)},
      {(void**)&h->d_flag, sizeof(int)},
      {(void**)&h->d_status, (size_t)h->max_sources * sizeof(int)},
      {(void**)&h->d_rel, (size_t)h->max_sources * sizeof(double)},
      {(void**)&h->d_src, (size_t)h->max_sources * 3 * sizeof(double)},
      {(void**)&h->d_jones_stage, (size_t)h->max_sources * n_cplx_ant * h->elem},
  };
  for (auto& a : allocs)
    if ((e = cudaMalloc(a.p, a.bytes)) != cudaSuccess) return bail(e, "cudaMalloc(workspace)");
  if ((e = cudaMemcpy(h->d_uvw, cfg->uvw, n_uvw * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "copy uvw");
  if ((e = cudaMemcpy(h->d_bl_ant, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "copy baseline map");
  if ((e = cudaMemcpy(h->d_freq_c, fc.data(), fc.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "copy frequencies");
  if ((e = cudaMemset(h->d_flag, 0, sizeof(int))) != cudaSuccess) return bail(e, "clear flag");
  if ((e = cudaMemset(h->d_status, 0, (size_t)h->max_sources * sizeof(int))) != cudaSuccess)
    return bail(e, "clear status");
  // the blocked schedule's tables, streams and solve set-up, and the Taylor
  // cadence's moments and iterates, are allocated here too (the paper's Section 5
  // advice), so a cadence allocates nothing
  int rc = RTS_OK;
  if (h->per_pass > 1) rc = ensure_block_workspace(h);
  if (rc == RTS_OK && h->precision == RTS_PREC_MIXED) rc = taylor_setup(h);
  if (rc != RTS_OK) {
    const std::string m = h->err;
    rts_peel_destroy(h);
    return fail(nullptr, rc, m);
  }
  *out = h;
  return RTS_OK;
}

int rts_peel_set_uvw(rts_peel_t* h, const double* h_uvw, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!h_uvw) return fail(h, RTS_EINVAL, "uvw is NULL");
  const size_t n = (size_t)h->n_time * h->n_ant * 3;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(h_uvw[i])) return fail(h, RTS_EINVAL, "uvw has a non-finite value");
  RTS_CUDA(h, cudaMemcpyAsync(h->d_uvw, h_uvw, n * sizeof(double), cudaMemcpyHostToDevice, as_stream(stream)));
  RTS_CUDA(h, cudaStreamSynchronize(as_stream(stream)));
  return RTS_OK;
}

namespace {
int not_a_shard(rts_peel_t* h) {
  if (h->n_band != h->n_chan)
    return fail(h, RTS_EINVAL, "this handle holds a channel shard of a wider band: use the rts_peel_shard_* calls");
  if (h->br.active) return fail(h, RTS_EINVAL, "a channel-shard cadence is in progress on this handle");
  return RTS_OK;
}
}  // namespace

int rts_peel_cadence(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src,
                     const double* h_src, void* d_jones, int32_t* h_status, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (int rc0 = not_a_shard(h)) return rc0;
  if (!d_vis || !d_resid) return fail(h, RTS_EINVAL, "d_vis and d_resid are required");
  if (misaligned(d_vis) || misaligned(d_resid))
    return fail(h, RTS_EINVAL, "d_vis and d_resid must start on a 16-byte boundary");
  int rc = validate_sources(h, n_src, h_src);
  if (rc) return rc;
  if (n_src > 0 && !d_jones) return fail(h, RTS_EINVAL, "d_jones is NULL");
  if (n_src > 0 && misaligned(d_jones)) return fail(h, RTS_EINVAL, "d_jones must start on a 16-byte boundary");
  return peel_device(h, d_vis, d_resid, n_src, h_src, d_jones, h_status, as_stream(stream));
}

int rts_peel_shard_begin(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src, const double* h_src,
                         void* d_jones, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (h->per_pass == 1) return fail(h, RTS_EINVAL, "channel-shard cadences need the blocked peel (sources_per_pass > 1)");
  if (h->br.active) return fail(h, RTS_EINVAL, "a channel-shard cadence is already in progress on this handle");
  if (!d_vis || !d_resid) return fail(h, RTS_EINVAL, "d_vis and d_resid are required");
  if (misaligned(d_vis) || misaligned(d_resid))
    return fail(h, RTS_EINVAL, "d_vis and d_resid must start on a 16-byte boundary");
  int rc = validate_sources(h, n_src, h_src);
  if (rc) return rc;
  if (n_src < 1) return fail(h, RTS_EINVAL, "a channel-shard cadence needs n_src >= 1");
  if (!d_jones) return fail(h, RTS_EINVAL, "d_jones is NULL");
  if (misaligned(d_jones)) return fail(h, RTS_EINVAL, "d_jones must start on a 16-byte boundary");
  rc = blocked_begin(h, d_vis, d_resid, n_src, h_src, d_jones, as_stream(stream));
  if (rc) {
    h->br.active = false;
    return rc;
  }
  return blocked_to_user(h);
}

int rts_peel_shard_partials(rts_peel_t* h, float** d_partial, int64_t* n_float) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!d_partial || !n_float) return fail(h, RTS_EINVAL, "d_partial and n_float are required");
  if (!h->br.active) return fail(h, RTS_EINVAL, "no channel-shard cadence is in progress");
  const int nblk = std::min(h->per_pass, h->br.n_src - h->br.b * h->per_pass);
  *d_partial = reinterpret_cast<float*>(h->b_avg);
  *n_float = (int64_t)nblk * h->n_bl * 8;
  return RTS_OK;
}

int rts_peel_shard_step(rts_peel_t* h, int32_t* h_status, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!h->br.active) return fail(h, RTS_EINVAL, "no channel-shard cadence is in progress");
  if (as_stream(stream) != h->br.user)
    return fail(h, RTS_EINVAL, "rts_peel_shard_step must use the stream of rts_peel_shard_begin");
  // the library's stream waits for the caller's exchange of the partial averages
  RTS_CUDA(h, cudaEventRecord(h->b_ev_in, h->br.user));
  RTS_CUDA(h, cudaStreamWaitEvent(h->b_main, h->b_ev_in, 0));
  int rc = blocked_block(h);
  if (rc) {
    h->br.active = false;
    return rc;
  }
  if (h->br.b < h->br.nb) {
    rc = blocked_to_user(h);
    return rc ? rc : 1;
  }
  return blocked_end(h, h_status);
}

int rts_peel_cadence_host(rts_peel_t* h, const void* h_vis, void* h_resid, int32_t n_src,
                          const double* h_src, void* h_jones, int32_t* h_status,
                          void* d_work, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (int rc0 = not_a_shard(h)) return rc0;
  if (!h_vis || !h_resid || !d_work) return fail(h, RTS_EINVAL, "h_vis, h_resid and d_work are required");
  int rc = validate_sources(h, n_src, h_src);
  if (rc) return rc;
  if (n_src > 0 && !h_jones) return fail(h, RTS_EINVAL, "h_jones is NULL");
  cudaStream_t s = as_stream(stream);
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  RTS_CUDA(h, cudaMemcpyAsync(d_work, h_vis, cube, cudaMemcpyHostToDevice, s));
  rc = peel_device(h, d_work, d_work, n_src, h_src, h->d_jones_stage, nullptr, s);
  if (rc) return rc;
  RTS_CUDA(h, cudaMemcpyAsync(h_resid, d_work, cube, cudaMemcpyDeviceToHost, s));
  if (n_src > 0)
    RTS_CUDA(h, cudaMemcpyAsync(h_jones, h->d_jones_stage, (size_t)n_src * h->n_ant * 4 * h->elem,
                                cudaMemcpyDeviceToHost, s));
  if (h_status && n_src > 0) return read_status(h, n_src, h_status, s);
  RTS_CUDA(h, cudaStreamSynchronize(s));
  return RTS_OK;
}

namespace {

int pipeline_setup(rts_peel_t* h) {
  if (h->p_cube[0]) return RTS_OK;
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  for (int k = 0; k < 2; ++k) {
    RTS_CUDA(h, cudaMalloc(&h->p_cube[k], cube));
    RTS_CUDA(h, cudaMalloc(&h->p_jones[k], (size_t)h->max_sources * h->n_ant * 4 * h->elem));
    RTS_CUDA(h, cudaMalloc((void**)&h->p_status[k], (size_t)h->max_sources * sizeof(int32_t)));
    // Jones and statuses go out through page-locked staging: a copy to pageable
    // memory would make the submit wait for its own cadence
    RTS_CUDA(h, cudaHostAlloc(&h->p_jones_pin[k], (size_t)h->max_sources * h->n_ant * 4 * h->elem,
                              cudaHostAllocDefault));
    RTS_CUDA(h, cudaHostAlloc((void**)&h->p_status_pin[k], (size_t)h->max_sources * sizeof(int32_t),
                              cudaHostAllocDefault));
    RTS_CUDA(h, cudaEventCreateWithFlags(&h->p_ev_in[k], cudaEventDisableTiming));
    RTS_CUDA(h, cudaEventCreateWithFlags(&h->p_ev_comp[k], cudaEventDisableTiming));
    RTS_CUDA(h, cudaEventCreateWithFlags(&h->p_ev_out[k], cudaEventDisableTiming));
  }
  RTS_CUDA(h, cudaStreamCreateWithFlags(&h->p_in, cudaStreamNonBlocking));
  RTS_CUDA(h, cudaStreamCreateWithFlags(&h->p_comp, cudaStreamNonBlocking));
  RTS_CUDA(h, cudaStreamCreateWithFlags(&h->p_out, cudaStreamNonBlocking));
  return RTS_OK;
}

// wait for slot k's cadence, hand its Jones matrices and statuses to the
// caller's buffers; RTS_ENONFINITE if one of its sources failed
int pipeline_retire(rts_peel_t* h, int k) {
  if (!h->p_busy[k]) return RTS_OK;
  RTS_CUDA(h, cudaEventSynchronize(h->p_ev_out[k]));
  h->p_busy[k] = false;
  const int n = h->p_nsrc[k];
  if (n > 0 && h->p_hjones[k])
    std::memcpy(h->p_hjones[k], h->p_jones_pin[k], (size_t)n * h->n_ant * 4 * h->elem);
  if (n > 0 && h->p_hstatus[k]) std::memcpy(h->p_hstatus[k], h->p_status_pin[k], sizeof(int32_t) * n);
  for (int i = 0; i < n; ++i)
    if (h->p_status_pin[k][i] == RTS_ENONFINITE)
      return fail(h, RTS_ENONFINITE, "non-finite value in the solve of source " + std::to_string(i));
  return RTS_OK;
}

}  // namespace

int rts_peel_pipeline_submit(rts_peel_t* h, const void* h_vis, void* h_resid, int32_t n_src,
                             const double* h_src, void* h_jones, int32_t* h_status) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (int rc0 = not_a_shard(h)) return rc0;
  if (!h_vis || !h_resid) return fail(h, RTS_EINVAL, "h_vis and h_resid are required");
  int rc = validate_sources(h, n_src, h_src);
  if (rc) return rc;
  if (n_src > 0 && !h_jones) return fail(h, RTS_EINVAL, "h_jones is NULL");
  rc = pipeline_setup(h);
  if (rc) return rc;
  const int k = h->p_next;
  rc = pipeline_retire(h, k);                       // the slot's previous cadence
  if (rc) return rc;
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  RTS_CUDA(h, cudaMemcpyAsync(h->p_cube[k], h_vis, cube, cudaMemcpyHostToDevice, h->p_in));
  RTS_CUDA(h, cudaEventRecord(h->p_ev_in[k], h->p_in));
  RTS_CUDA(h, cudaStreamWaitEvent(h->p_comp, h->p_ev_in[k], 0));
  rc = peel_device(h, h->p_cube[k], h->p_cube[k], n_src, h_src, h->p_jones[k], nullptr, h->p_comp);
  if (rc) return rc;
  if (n_src > 0)
    RTS_CUDA(h, cudaMemcpyAsync(h->p_status[k], h->d_status, sizeof(int32_t) * n_src,
                                cudaMemcpyDeviceToDevice, h->p_comp));
  RTS_CUDA(h, cudaEventRecord(h->p_ev_comp[k], h->p_comp));
  RTS_CUDA(h, cudaStreamWaitEvent(h->p_out, h->p_ev_comp[k], 0));
  RTS_CUDA(h, cudaMemcpyAsync(h_resid, h->p_cube[k], cube, cudaMemcpyDeviceToHost, h->p_out));
  if (n_src > 0) {
    RTS_CUDA(h, cudaMemcpyAsync(h->p_jones_pin[k], h->p_jones[k], (size_t)n_src * h->n_ant * 4 * h->elem,
                                cudaMemcpyDeviceToHost, h->p_out));
    RTS_CUDA(h, cudaMemcpyAsync(h->p_status_pin[k], h->p_status[k], sizeof(int32_t) * n_src,
                                cudaMemcpyDeviceToHost, h->p_out));
  }
  RTS_CUDA(h, cudaEventRecord(h->p_ev_out[k], h->p_out));
  // the next cadence's copy-in may not overwrite this slot until its copy-out is done;
  // the next slot's copy-in only needs that slot's previous copy-out (checked at submit)
  h->p_busy[k] = true;
  h->p_hstatus[k] = h_status;
  h->p_hjones[k] = h_jones;
  h->p_nsrc[k] = n_src;
  h->p_next = 1 - k;
  return RTS_OK;
}

int rts_peel_pipeline_wait(rts_peel_t* h) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  int worst = RTS_OK;
  for (int i = 0; i < 2; ++i) {
    const int k = (h->p_next + i) & 1;             // oldest first
    int rc = pipeline_retire(h, k);
    if (rc && !worst) worst = rc;
  }
  return worst;
}

int rts_peel_predict(rts_peel_t* h, void* d_vis, int32_t n_src, const double* h_src,
                     const void* d_jones, int32_t accumulate, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!d_vis) return fail(h, RTS_EINVAL, "d_vis is NULL");
  if (misaligned(d_vis)) return fail(h, RTS_EINVAL, "d_vis must start on a 16-byte boundary");
  int rc = validate_sources(h, n_src, h_src);
  if (rc) return rc;
  if (n_src > 0 && !d_jones) return fail(h, RTS_EINVAL, "d_jones is NULL");
  cudaStream_t s = as_stream(stream);
  const size_t cube = (size_t)h->n_time * h->n_bl * h->n_chan * 4 * h->elem;
  if (n_src == 0) {
    if (!accumulate) RTS_CUDA(h, cudaMemsetAsync(d_vis, 0, cube, s));
    return RTS_OK;
  }
  RTS_CUDA(h, cudaMemcpyAsync(h->d_src, h_src, sizeof(double) * 3 * n_src, cudaMemcpyHostToDevice, s));
  const size_t per_src = (size_t)h->n_time * (h->precision == RTS_PREC_MIXED ? 16 : 8);
  int chunk = (int)std::min<size_t>(kPredictChunk, std::max<size_t>(1, 40960 / per_src));
  for (int k0 = 0; k0 < n_src; k0 += chunk) {
    PredictArgs a;
    a.vis = d_vis; a.uvw = h->d_uvw; a.bl_ant = h->d_bl_ant; a.freq_c = h->d_freq_c;
    a.src = h->d_src + 3 * k0;
    a.jones = static_cast<const char*>(d_jones) + (size_t)k0 * h->n_ant * 4 * h->elem;
    a.n_src = std::min(chunk, n_src - k0);
    a.n_ant = h->n_ant; a.n_chan = h->n_chan; a.n_time = h->n_time; a.n_bl = h->n_bl;
    a.nu0_c = h->nu0 / kCLight; a.dnu_c = h->dnu / kCLight;
    a.accumulate = (k0 > 0 || accumulate) ? 1 : 0;
    const size_t smem = per_src * a.n_src;
    Span span(h, RTS_K_PREDICT, s);
    if (h->precision == RTS_PREC_MIXED) k_predict_mixed<<<(unsigned)h->n_bl, kStreamThreads, smem, s>>>(a);
    else k_predict_fp64<<<(unsigned)h->n_bl, kStreamThreads, smem, s>>>(a);
    span.end(1);
    rc = check_launch(h, "predict kernel launch");
    if (rc) return rc;
  }
  return RTS_OK;
}

int rts_peel_rotate_average(rts_peel_t* h, const void* d_vis, double l, double m, void* d_avg,
                            void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!d_vis || !d_avg) return fail(h, RTS_EINVAL, "d_vis and d_avg are required");
  if (misaligned(d_vis) || misaligned(d_avg))
    return fail(h, RTS_EINVAL, "d_vis and d_avg must start on a 16-byte boundary");
  if (!std::isfinite(l) || !std::isfinite(m) || !(l * l + m * m < 1.0))
    return fail(h, RTS_EINVAL, "direction must be finite with l^2 + m^2 < 1");
  StreamArgs a = stream_args(h, d_vis, nullptr, d_avg);
  a.acc = make_dir(l, m, 1.0);
  return launch_stream(h, false, true, a, as_stream(stream));
}

int rts_peel_solve(rts_peel_t* h, const void* d_avg, double S, void* d_jones, int32_t* h_status,
                   void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!d_avg || !d_jones) return fail(h, RTS_EINVAL, "d_avg and d_jones are required");
  if (misaligned(d_avg) || misaligned(d_jones))
    return fail(h, RTS_EINVAL, "d_avg and d_jones must start on a 16-byte boundary");
  if (!std::isfinite(S) || !(S > 0.0)) return fail(h, RTS_EINVAL, "S must be finite and > 0");
  cudaStream_t s = as_stream(stream);
  int rc = launch_als(h, d_avg, S, d_jones, 0, s);
  if (rc) return rc;
  if (h_status) return read_status(h, 1, h_status, s);
  return RTS_OK;
}

int rts_peel_grad(rts_peel_t* h, const void* d_vis, int32_t n_src, const void* d_jones,
                  const double* d_src, double* d_loss, void* d_gJ, double* d_gsrc, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!d_vis || !d_loss) return fail(h, RTS_EINVAL, "d_vis and d_loss are required");
  if (misaligned(d_vis)) return fail(h, RTS_EINVAL, "d_vis must start on a 16-byte boundary");
  if (n_src < 0 || n_src > h->max_sources) return fail(h, RTS_EINVAL, "n_src must be in [0, max_sources]");
  if (n_src > 0 && (!d_jones || !d_src)) return fail(h, RTS_EINVAL, "d_jones and d_src are required");
  cudaStream_t s = as_stream(stream);
  const bool mixed = h->precision == RTS_PREC_MIXED;
  int rc = grad_prepare(h->grad, n_src, d_src, h->n_bl, h->max_sources, s, h->err);
  if (rc) return rc;
  {
    Span span(h, RTS_K_GRAD, s);
    rc = grad_sweep(h->grad, mixed, d_vis, n_src, d_jones, h->d_uvw, h->d_bl_ant, h->d_freq_c,
                    h->n_ant, h->n_chan, h->n_time, h->n_bl, h->nu0 / kCLight, h->dnu / kCLight, s,
                    h->err, nullptr, h->grad_direct);
    span.end(1);
    if (rc) return rc;
  }
  Span span(h, RTS_K_GRAD_REDUCE, s);
  int nl = 0;
  rc = grad_reduce(h->grad, mixed, n_src, d_jones, d_loss, d_gJ, d_gsrc, h->n_ant, h->n_bl, s, h->err, &nl);
  span.end(nl);
  return rc;
}

int rts_peel_offsets(rts_peel_t* h, const void* d_vis, int32_t n_src, const void* d_jones,
                     const double* d_src, double alpha, double nu_ref_hz, double* d_out,
                     double* d_offsets, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (n_src < 0 || n_src > h->max_sources) return fail(h, RTS_EINVAL, "n_src must be in [0, max_sources]");
  if (!std::isfinite(alpha)) return fail(h, RTS_EINVAL, "alpha must be finite");
  if (alpha != 0.0 && !(nu_ref_hz > 0.0 && std::isfinite(nu_ref_hz)))
    return fail(h, RTS_EINVAL, "nu_ref_hz must be positive and finite when alpha != 0");
  if (n_src == 0) return RTS_OK;
  if (!d_vis || !d_jones || !d_src || !d_out || !d_offsets)
    return fail(h, RTS_EINVAL, "d_vis, d_jones, d_src, d_out and d_offsets are required");
  if (misaligned(d_vis)) return fail(h, RTS_EINVAL, "d_vis must start on a 16-byte boundary");
  cudaStream_t s = as_stream(stream);
  const bool mixed = h->precision == RTS_PREC_MIXED;
  int rc = grad_prepare(h->grad, n_src, d_src, h->n_bl, h->max_sources, s, h->err);
  if (rc) return rc;
  const double* wtab = h->d_freq_c;              // alpha = 0: w_c = nu_c / c
  if (alpha != 0.0) {
    if (!h->grad.wchan) RTS_CUDA(h, cudaMalloc(&h->grad.wchan, (size_t)h->n_chan * sizeof(double)));
    Span span(h, RTS_K_OFFSETS, s);
    k_offset_weights<<<(h->n_chan + 255) / 256, 256, 0, s>>>(h->d_freq_c, h->n_chan, alpha,
                                                             nu_ref_hz / kCLight, h->grad.wchan);
    span.end(1);
    wtab = h->grad.wchan;
  }
  {
    Span span(h, RTS_K_GRAD, s);
    rc = grad_sweep(h->grad, mixed, d_vis, n_src, d_jones, h->d_uvw, h->d_bl_ant, h->d_freq_c,
                    h->n_ant, h->n_chan, h->n_time, h->n_bl, h->nu0 / kCLight, h->dnu / kCLight, s,
                    h->err, alpha != 0.0 ? wtab : nullptr, h->grad_direct);
    span.end(1);
    if (rc) return rc;
  }
  Span span(h, RTS_K_OFFSETS, s);
  if (mixed)
    k_offset_normal<float><<<n_src, kOffThreads, 0, s>>>(d_jones, h->grad.dir, h->d_uvw, h->d_bl_ant,
                                                         wtab, h->grad.gsc, h->grad.loss_bl,
                                                         h->n_ant, h->n_chan, h->n_time, h->n_bl,
                                                         d_out, d_offsets);
  else
    k_offset_normal<double><<<n_src, kOffThreads, 0, s>>>(d_jones, h->grad.dir, h->d_uvw, h->d_bl_ant,
                                                          wtab, h->grad.gsc, h->grad.loss_bl,
                                                          h->n_ant, h->n_chan, h->n_time, h->n_bl,
                                                          d_out, d_offsets);
  RTS_CUDA(h, cudaGetLastError());
  span.end(1);
  return RTS_OK;
}

int rts_offsets_solve(const double* d_out, int32_t n_src, double* d_offsets, void* stream) {
  if (n_src < 0) return fail(nullptr, RTS_EINVAL, "n_src must be >= 0");
  if (n_src == 0) return RTS_OK;
  if (!d_out || !d_offsets) return fail(nullptr, RTS_EINVAL, "d_out and d_offsets are required");
  k_offset_solve<<<(n_src + 127) / 128, 128, 0, as_stream(stream)>>>(d_out, n_src, d_offsets);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, RTS_ECUDA, std::string("offset solve launch: ") + cudaGetErrorString(e));
  return RTS_OK;
}

int rts_peel_timing(rts_peel_t* h, int32_t enable) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (enable) {
    h->recs.clear();
    h->ev_used = 0;
    for (auto& n : h->launches) n = 0;
  }
  h->timing = enable != 0;
  return RTS_OK;
}

int rts_peel_timing_read(rts_peel_t* h, double* ms, int64_t* groups, int64_t* launches) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  double acc[RTS_K_CLASSES] = {};
  int64_t cnt[RTS_K_CLASSES] = {};
  for (const auto& r : h->recs) {
    RTS_CUDA(h, cudaEventSynchronize(r.b));
    float t = 0.f;
    RTS_CUDA(h, cudaEventElapsedTime(&t, r.a, r.b));
    acc[r.cls] += t;
    cnt[r.cls] += 1;
  }
  for (int c = 0; c < RTS_K_CLASSES; ++c) {
    if (ms) ms[c] = acc[c];
    if (groups) groups[c] = cnt[c];
    if (launches) launches[c] = h->launches[c];
  }
  return RTS_OK;
}

int rts_host_alloc(uint64_t bytes, void** out) {
  if (!out) return RTS_EINVAL;
  *out = nullptr;
  cudaError_t e = cudaHostAlloc(out, (size_t)bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    g_init_err = std::string("cudaHostAlloc: ") + cudaGetErrorString(e);
    *out = nullptr;
    return e == cudaErrorMemoryAllocation ? RTS_ENOMEM : RTS_ECUDA;
  }
  return RTS_OK;
}

int rts_host_free(void* p) {
  if (!p) return RTS_OK;
  return cudaFreeHost(p) == cudaSuccess ? RTS_OK : RTS_ECUDA;
}

int rts_peel_kernels(const rts_peel_t* h, int32_t* block_kernel, int32_t* solve_kernel) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (block_kernel)
    *block_kernel = h->per_pass == 1 ? 0 : (h->block_tc05 ? RTS_BLOCK_TCGEN05 : (h->block_tc ? RTS_BLOCK_TENSOR : RTS_BLOCK_FMA));
  if (solve_kernel)
    *solve_kernel = h->b_avg ? (h->bs_ok ? RTS_SOLVE_AUTO : RTS_SOLVE_LAUNCHES) : h->solve_kernel;
  return RTS_OK;
}

int rts_peel_rel(rts_peel_t* h, int32_t n_src, double* h_rel, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (n_src < 0 || n_src > h->max_sources) return fail(h, RTS_EINVAL, "n_src must be in [0, max_sources]");
  if (n_src == 0) return RTS_OK;
  if (!h_rel) return fail(h, RTS_EINVAL, "h_rel is NULL");
  cudaStream_t s = as_stream(stream);
  RTS_CUDA(h, cudaMemcpyAsync(h_rel, h->d_rel, sizeof(double) * n_src, cudaMemcpyDeviceToHost, s));
  RTS_CUDA(h, cudaStreamSynchronize(s));
  return RTS_OK;
}

int rts_peel_phases(rts_peel_t* h, double l, double m, int32_t n_pair, const int32_t* d_tb, int32_t form,
                    double* d_phase, void* stream) {
  if (!h) return fail(nullptr, RTS_EINVAL, "handle is NULL");
  if (!std::isfinite(l) || !std::isfinite(m) || !(l * l + m * m < 1.0))
    return fail(h, RTS_EINVAL, "direction must be finite with l^2 + m^2 < 1");
  if (n_pair < 0) return fail(h, RTS_EINVAL, "n_pair must be >= 0");
  if (form < 0 || form > 2) return fail(h, RTS_EINVAL, "form must be 0, 1 or 2");
  if (n_pair == 0) return RTS_OK;
  if (!d_tb || !d_phase) return fail(h, RTS_EINVAL, "d_tb and d_phase are required");
  const int64_t n = (int64_t)n_pair * h->n_chan;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)h->n_sm * 16);
  k_phase_table<<<grid, 256, 0, as_stream(stream)>>>(h->d_uvw, h->d_bl_ant, h->n_ant, h->n_chan, h->n_time, h->n_bl,
                                                      make_dir(l, m, 1.0), h->nu0 / kCLight, h->dnu / kCLight,
                                                      n_pair, d_tb, form, d_phase);
  return check_launch(h, "phase table launch");
}

const char* rts_peel_last_error(const rts_peel_t* h) {
  return h ? h->err.c_str() : g_init_err.c_str();
}

void rts_peel_destroy(rts_peel_t* h) {
  if (!h) return;
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != h->device) cudaSetDevice(h->device);
  void* ptrs[] = {h->d_uvw, h->d_bl_ant, h->d_freq_c, h->d_avg, h->d_J[0], h->d_J[1], h->d_Jf[0],
                  h->d_Jf[1], h->d_norms, h->d_flag, h->d_status, h->d_rel, h->d_src, h->d_jones_stage,
                  h->b_avg, h->b_aph, h->b_model, h->b_sync, h->b_part, h->d_perr, h->t_mom, h->t_X[0],
                  h->t_X[1], h->t_Xf[0], h->t_Xf[1], h->t_rot_part, h->t_rot_count, h->t_rot_step};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int r = 0; r < rts_peel_t::kRing; ++r) {
    if (h->b_ph[r]) cudaFree(h->b_ph[r]);
    if (h->b_trig[r]) cudaFree(h->b_trig[r]);
    if (h->b_dir[r]) cudaFree(h->b_dir[r]);
    if (h->b_ev_ready[r]) cudaEventDestroy(h->b_ev_ready[r]);
    if (h->b_ev_free[r]) cudaEventDestroy(h->b_ev_free[r]);
  }
  if (h->b_ev_src) cudaEventDestroy(h->b_ev_src);
  if (h->b_ev_done) cudaEventDestroy(h->b_ev_done);
  if (h->b_prep) cudaStreamDestroy(h->b_prep);
  if (h->b_main) cudaStreamDestroy(h->b_main);
  if (h->b_ev_in) cudaEventDestroy(h->b_ev_in);
  if (h->b_ev_out) cudaEventDestroy(h->b_ev_out);
  grad_free(h->grad);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    if (h->p_cube[k]) cudaFree(h->p_cube[k]);
    if (h->p_jones[k]) cudaFree(h->p_jones[k]);
    if (h->p_status[k]) cudaFree(h->p_status[k]);
    if (h->p_jones_pin[k]) cudaFreeHost(h->p_jones_pin[k]);
    if (h->p_status_pin[k]) cudaFreeHost(h->p_status_pin[k]);
    if (h->p_ev_in[k]) cudaEventDestroy(h->p_ev_in[k]);
    if (h->p_ev_comp[k]) cudaEventDestroy(h->p_ev_comp[k]);
    if (h->p_ev_out[k]) cudaEventDestroy(h->p_ev_out[k]);
  }
  if (h->p_in) cudaStreamDestroy(h->p_in);
  if (h->p_comp) cudaStreamDestroy(h->p_comp);
  if (h->p_out) cudaStreamDestroy(h->p_out);
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  delete h;
}

}  // extern "C"

namespace {

// FP64 FMA throughput probe: 8 independent chains per thread, so the FP64
// pipe, not the dependency latency, limits the rate; the result is stored so
// the loop is kept.
constexpr int kF64Chains = 8;
__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double seed, double* out) {
  double x[kF64Chains];
  #pragma unroll
  for (int c = 0; c < kF64Chains; ++c) x[c] = seed + 1e-3 * (threadIdx.x + c);
  const double a = 0.999999, b = 1e-7;
  for (int i = 0; i < iters; ++i)
    #pragma unroll
    for (int c = 0; c < kF64Chains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
  #pragma unroll
  for (int c = 0; c < kF64Chains; ++c) s += x[c];
  if (s == 12345.678) out[0] = s;                    // practically never: keeps the work
}

}  // namespace

extern "C" {

int rts_fp64_rate(double* h_tflops) {
  g_init_err.clear();
  if (!h_tflops) return fail(nullptr, RTS_EINVAL, "h_tflops is NULL");
  int dev = 0, n_sm = 0;
  RTS_CUDA(nullptr, cudaGetDevice(&dev));
  RTS_CUDA(nullptr, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  double* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RTS_CUDA(nullptr, cudaMalloc(&d_out, sizeof(double)));
  auto done = [&](int rc) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_out);
    return rc;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return done(fail(nullptr, RTS_ECUDA, "cudaEventCreate"));
  const int iters = 1 << 14, blocks = 8 * n_sm;
  k_fp64_rate<<<blocks, 256>>>(iters / 16, 1.0, d_out);    // warm-up
  cudaEventRecord(e0);
  k_fp64_rate<<<blocks, 256>>>(iters, 1.0, d_out);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return done(fail(nullptr, RTS_ECUDA, std::string("FP64 rate probe: ") + cudaGetErrorString(e)));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double flops = 2.0 * kF64Chains * (double)iters * blocks * 256;
  *h_tflops = flops / (ms * 1e-3) / 1e12;
  return done(RTS_OK);
}

int rts_barrier_selftest(int32_t n_cta, int32_t missing, int32_t rounds, int32_t* h_completed) {
  g_init_err.clear();
  if (!h_completed) return fail(nullptr, RTS_EINVAL, "h_completed is NULL");
  if (n_cta < 1 || n_cta > 1024 || missing < 0 || missing > 1 || rounds < 1 || rounds > 10000)
    return fail(nullptr, RTS_EINVAL, "rts_barrier_selftest: n_cta in [1, 1024], missing in [0, 1], rounds in [1, 10000]");
  int dev = 0, coop = 0, n_sm = 0, occ = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_barrier_selftest, 128, 0)) != cudaSuccess)
    return cuda_fail(nullptr, e, "device query");
  if (!coop || n_cta > n_sm * occ) return fail(nullptr, RTS_EINVAL, "rts_barrier_selftest: n_cta above the co-resident limit");
  unsigned* sync = nullptr;
  int* ok = nullptr;
  if ((e = cudaMalloc((void**)&sync, 2 * sizeof(unsigned))) != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc");
  if ((e = cudaMalloc((void**)&ok, n_cta * sizeof(int))) != cudaSuccess) {
    cudaFree(sync);
    return cuda_fail(nullptr, e, "cudaMalloc");
  }
  std::vector<int> h_ok(n_cta, 0);
  int r = missing;
  void* args[] = {&sync, &rounds, &r, &ok};
  if ((e = cudaMemset(sync, 0, 2 * sizeof(unsigned))) == cudaSuccess &&
      (e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(n_cta), dim3(128), args, 0, 0)) ==
          cudaSuccess &&
      (e = cudaDeviceSynchronize()) == cudaSuccess)
    e = cudaMemcpy(h_ok.data(), ok, n_cta * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(sync);
  cudaFree(ok);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "barrier self-test");
  int done = 0;
  for (int v : h_ok) done += v != 0;
  *h_completed = done;
  return RTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free solve.  Its scratch (Jones iterates, their FP32 copies, the
// per-antenna norms and the status words) lives in one file-scope device
// array, sized for RTS_NOALLOC_MAX_ANT antennas and held by every device that
// loads this library until the process exits.  Host code cannot use the
// array's name as a device address, so each device's address is looked up
// once with cudaGetSymbolAddress (on the first call made on that device).

namespace {

struct NoallocScratch {
  double2 J[2][RTS_NOALLOC_MAX_ANT * 4];
  float2 Jf[2][RTS_NOALLOC_MAX_ANT * 4];
  double norms[RTS_NOALLOC_MAX_ANT * 2];
  double rel;
  int flag;
  int status;
};

__device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoallocScratch* g_noalloc_addr[kNoallocMaxDevices] = {};

}  // namespace

extern "C" int rts_peel_solve_noalloc(const void* d_avg, int32_t n_ant, double S, int32_t n_iter,
                                      int32_t precision, void* d_jones, int32_t* h_status,
                                      void* stream) {
  g_init_err.clear();
  if (!d_avg || !d_jones) return fail(nullptr, RTS_EINVAL, "d_avg and d_jones are required");
  if (misaligned(d_avg) || misaligned(d_jones))
    return fail(nullptr, RTS_EINVAL, "d_avg and d_jones must start on a 16-byte boundary");
  if (n_ant < 2 || n_ant > RTS_NOALLOC_MAX_ANT)
    return fail(nullptr, RTS_EINVAL, "rts_peel_solve_noalloc: n_ant must be in [2, " +
                                         std::to_string(RTS_NOALLOC_MAX_ANT) + "] (static scratch limit)");
  if (n_iter < 1 || n_iter > 10000) return fail(nullptr, RTS_EINVAL, "n_iter must be in [1, 10000]");
  if (precision != RTS_PREC_MIXED && precision != RTS_PREC_FP64)
    return fail(nullptr, RTS_EINVAL, "precision must be RTS_PREC_MIXED or RTS_PREC_FP64");
  if (!std::isfinite(S) || !(S > 0.0)) return fail(nullptr, RTS_EINVAL, "S must be finite and > 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(nullptr, RTS_EINVAL, "device ordinal too large");
  NoallocScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(scratch)");
      g_noalloc_addr[dev] = static_cast<NoallocScratch*>(ptr);
    }
    sc = g_noalloc_addr[dev];
  }
  cudaStream_t s = as_stream(stream);
  // the flag must start at zero; the rest is written before it is read
  e = cudaMemsetAsync(&sc->flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "clear scratch flag");
  for (int it = 1; it <= n_iter; ++it) {
    AlsArgs a;
    a.avg = d_avg;
    a.J_old = sc->J[(it - 1) & 1]; a.Jf_old = sc->Jf[(it - 1) & 1];
    a.J_new = sc->J[it & 1]; a.Jf_new = sc->Jf[it & 1];
    a.norms = sc->norms; a.flag = &sc->flag;
    a.jones_out = it == n_iter ? d_jones : nullptr;
    a.n_ant = n_ant; a.S = S; a.first = it == 1; a.average = (it % 2) == 0;
    if (precision == RTS_PREC_MIXED) k_als_sweep<float><<<als_grid(n_ant), kAlsThreads, 0, s>>>(a);
    else k_als_sweep<double><<<als_grid(n_ant), kAlsThreads, 0, s>>>(a);
  }
  k_als_finalize<<<1, 256, 0, s>>>(sc->norms, n_ant, &sc->flag, &sc->status, &sc->rel);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "ALS kernel launch (no-alloc)");
  if (h_status) {
    e = cudaMemcpyAsync(h_status, &sc->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "read status (no-alloc)");
    if (*h_status == RTS_ENONFINITE) return fail(nullptr, RTS_ENONFINITE, "non-finite value in the solve");
  }
  return RTS_OK;
}
