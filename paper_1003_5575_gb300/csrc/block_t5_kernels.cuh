// Blocked peel pass on the 5th-generation tensor cores (tcgen05.mma, TMEM
// accumulators): the same pass as k_block_pass / k_block_pass_tc (subtract
// the solved sources of block b, average the directions of block b+1).
//
// The phasors factor per 16-channel tile q as in block_tc_kernels.cuh,
//   P_k(16 q + r) = T1_k[q] T2_k[r],
// which turns both contractions of a (baseline, time step) into GEMMs whose
// small factor depends on T2 only:
//
//   subtraction  O[(q,e), (pout,r)] = sum_(k,pin) W[(q,e), (k,pin)] B2[(k,pin), (pout,r)]
//     W = conj(T1_k[q]) M_k(e) as (re, im) pairs along K (A operand, written to
//     TMEM by the threads), B2 the real form of conj(T2): rows (r, 0) = (T2r, T2i),
//     rows (r, 1) = (-T2i, T2r) per source (B operand in shared memory);
//     M = 4 nq rows in tiles of 128, N = 32, K = 128;  R(16 q + r, e) -= O.
//   average      D[(pout,k), (q,e)] = sum_(pin,r) A2[(pout,k), (pin,r)] R[(q,e), (pin,r)]
//     A2 the real form of T2 (rows (0, k) = (T2r, -T2i), rows (1, k) = (T2i, T2r)),
//     R the new residual split along K into (re, im) x 16 channels (B operand,
//     written by the subtraction's epilogue); M = 128, N = 4 nq, K = 32;
//     then A_k(e) += sum_q T1_k[q] G_k(q, e), G = D(0,k) + i D(1,k), in FP32 on
//     the CUDA cores (compensated sums across time steps).
//
// TF32 keeps 11 significand bits, so every operand is split x = hi + lo (both
// TF32) and each product is three MMAs, lo*hi + hi*lo + hi*hi (the lo*lo term
// is below 2^-22 relative).  The tensor cores' FP32 accumulation does not round
// to nearest, so its error grows with the number of MMAs chained into one
// accumulator: the subtraction keeps one accumulator per group of 8 sources
// (a chain of 6 MMAs, cross terms first) and the average one for the hi*hi
// terms and one for the cross terms; the epilogues add them in FP32 with
// round-to-nearest.
//
// One CTA (16 warps, 1 per SM: ~217 KB of shared memory, all 512 TMEM columns)
// per baseline, looping over time steps; one lane in each of several warps
// issues the MMAs of its accumulators and commits them to an mbarrier that
// warp 0 waits on (bounded polls: a wait that runs out sets *err and the pass
// reports an error instead of hanging).
// Limits: at most 64 sources per role, n_chan <= kT5MaxChan.
#pragma once
#include "block_tc_kernels.cuh"
#include "tc05.cuh"

namespace rts {

constexpr int kT5Threads = 512;
constexpr int kT5Src = 64;                  // sources per role
constexpr int kT5MaxChan = 768;             // shared memory limit
// TMEM columns.  Subtraction: W hi [0, 128), lo [128, 256); 8 accumulators of
// 32 columns at [256, 512).  Average (after the subtraction has finished with
// all of them): hi*hi accumulator [0, 4 nq4), cross-term accumulator
// [256, 256 + 4 nq4).
constexpr uint32_t kT5ColW = 0;
constexpr uint32_t kT5ColO = 256;
constexpr uint32_t kT5ColDm = 0;
constexpr uint32_t kT5ColDx = 256;
constexpr uint32_t kT5Cols = 512;
constexpr uint32_t kT5MaxPolls = 1u << 17;  // mbarrier polls (each up to 20 us) before giving up

// shared-memory layout (byte offsets) for nq4 = 16-channel tiles rounded up to 4
struct T5Smem {
  int strip, bavg_hi, bavg_lo, bsub_hi, bsub_lo, aavg_hi, aavg_lo, t1, mtab, ph, red, bar, total;
  __host__ __device__ explicit T5Smem(int nq4) {
    int o = 0;
    strip = o;   o += 2 * nq4 * 16 * 8 * 4;      // two FP32 strips [16 nq4][4 pol][2]
    bavg_hi = o; o += 4 * nq4 * 32 * 4;          // residual split, [4 nq4 rows][32 K]
    bavg_lo = o; o += 4 * nq4 * 32 * 4;
    bsub_hi = o; o += 32 * 128 * 4;              // real form of conj(T2), [32 rows][128 K]
    bsub_lo = o; o += 32 * 128 * 4;
    aavg_hi = o; o += 128 * 32 * 4;              // real form of T2, [128 rows][32 K]
    aavg_lo = o; o += 128 * 32 * 4;
    t1 = o;      o += 128 * (nq4 + 1) * 8;       // T1 [source][nq4 + 1] float2
    mtab = o;    o += 64 * 4 * 8;                // model matrices [64][4] float2
    ph = o;      o += 128 * 16;                  // phases of the time step
    red = o;     o += 64 * 8 * 8;                // FP64 partial averages of the imaginary rows
    bar = o;     o += 32;                        // two mbarriers + TMEM address
    total = o;
  }
};

inline int t5_nq4(int n_chan) { return (((n_chan + 15) >> 4) + 3) & ~3; }
inline size_t t5_pass_smem(int n_chan) { return (size_t)T5Smem(t5_nq4(n_chan)).total; }

// strip rows are XOR-swizzled within groups of 4 channels by the tile index, so
// the subtraction epilogue (8 tiles x 4 pols per warp) reads conflict-free
__device__ __forceinline__ int t5_swz(int c) { return c ^ ((c >> 4) & 3); }

// TF32 rounding (to nearest, ties away from zero: the result of cvt.rna.tf32.f32
// for finite x below the FP32 maximum) with two integer operations: add half of
// the dropped 13-bit unit to the magnitude bits and clear them.  A conversion
// instruction per value was a large share of this pass on GB300.
__device__ __forceinline__ uint32_t t5_tf32(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

// x = hi + lo with hi the TF32 rounding of x and lo the exact remainder; the
// MMA reads lo truncated to TF32 (error below 2^-21 |x|)
__device__ __forceinline__ float2 t5_split(float x) {
  const float hi = __uint_as_float(t5_tf32(x));
  return make_float2(hi, x - hi);
}

// stored operand tables: hi and lo both rounded to TF32
__device__ __forceinline__ float2 t5_split_store(float x) {
  const float hi = __uint_as_float(t5_tf32(x));
  return make_float2(hi, __uint_as_float(t5_tf32(x - hi)));
}

template <bool SUB, bool ACC>
__global__ void __launch_bounds__(kT5Threads, 1) k_block_pass_t5(BlockPassArgs a, int bk, int* err) {
  using namespace tc05;
  const int nq = (a.n_chan + 15) >> 4, nq4 = (nq + 3) & ~3, n16 = 16 * nq4, P = nq4 + 1;
  const T5Smem L(nq4);
  extern __shared__ __align__(1024) unsigned char t5_smem[];
  float* strip0 = reinterpret_cast<float*>(t5_smem + L.strip);
  unsigned char* bavg_hi = t5_smem + L.bavg_hi;
  unsigned char* bavg_lo = t5_smem + L.bavg_lo;
  unsigned char* bsub_hi = t5_smem + L.bsub_hi;
  unsigned char* bsub_lo = t5_smem + L.bsub_lo;
  unsigned char* aavg_hi = t5_smem + L.aavg_hi;
  unsigned char* aavg_lo = t5_smem + L.aavg_lo;
  float2* t1 = reinterpret_cast<float2*>(t5_smem + L.t1);
  float2* mtab = reinterpret_cast<float2*>(t5_smem + L.mtab);
  PhaseAB* ph = reinterpret_cast<PhaseAB*>(t5_smem + L.ph);
  double* red = reinterpret_cast<double*>(t5_smem + L.red);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(t5_smem + L.bar);     // [0] subtraction, [1] average
  uint32_t* tslot = reinterpret_cast<uint32_t*>(t5_smem + L.bar + 16);

  const int64_t bl = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quarter = warp & 3;
  const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;

  if (warp == 0) tmem_alloc(tslot, kT5Cols);
  if (tid == 0) {
    mbar_init(&mbar[0], 8);                   // the subtraction's 8 issuing warps commit to it
    mbar_init(&mbar[1], 2);                   // the average's 2 issuing warps
  }
  // padding channels of both strips stay zero (the copies never write them)
  for (int i = tid; i < (n16 - a.n_chan) * 8; i += kT5Threads) {
    const int c = a.n_chan + (i >> 3), j = i & 7;
    strip0[t5_swz(c) * 8 + j] = 0.f;
    strip0[(n16 + t5_swz(c)) * 8 + j] = 0.f;
  }
  if (SUB)
    for (int i = tid; i < kT5Src * 4; i += kT5Threads) {
      const int s = i >> 2, e = i & 3;
      mtab[i] = s < a.n_sub ? a.M_sub[((size_t)s * a.n_bl + bl) * 4 + e] : make_float2(0.f, 0.f);
    }
  auto prefetch = [&](int t, int buf) {
    const float4* gsrc = a.src + ((size_t)t * a.n_bl + bl) * a.n_chan * 2;
    float4* sdst = reinterpret_cast<float4*>(strip0 + (size_t)buf * n16 * 8);
    for (int i = tid; i < a.n_chan * 2; i += kT5Threads) cp_async16(sdst + t5_swz(i >> 1) * 2 + (i & 1), gsrc + i);
  };
  prefetch(0, 0);
  cp_async_commit();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  // average accumulators (warps 0..3, row m = 32 quarter + lane = (pout, k)):
  // compensated FP32 sums of the real and imaginary contributions per pol
  float ks[8], kc[8];
  #pragma unroll
  for (int i = 0; i < 8; ++i) ks[i] = kc[i] = 0.f;
  uint32_t par_sub = 0, par_avg = 0;
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  const int ntile = (4 * nq4 + 127) / 128;
  // operand descriptors (fixed addresses; the k-step offset is added per MMA)
  const uint64_t dsub_hi = desc_kmajor(smem_u32(bsub_hi), 128, 4096), dsub_lo = desc_kmajor(smem_u32(bsub_lo), 128, 4096);
  const uint64_t da_hi = desc_kmajor(smem_u32(aavg_hi), 128, 1024), da_lo = desc_kmajor(smem_u32(aavg_lo), 128, 1024);
  const uint64_t db_hi = desc_kmajor(smem_u32(bavg_hi), 128, 1024), db_lo = desc_kmajor(smem_u32(bavg_lo), 128, 1024);

  // T1_k[q] = exp(2 pi i (A + 16 q B)) of 64 sources from s0: thread (s, q0)
  // steps q by 8 with an exact 64-bit phase increment
  auto t1_fill = [&](int s0) {
    const int s = s0 + (tid & 63);
    const PhaseAB p = ph[s];
    const unsigned long long step = 128ull * p.b;
    unsigned long long x = p.a + (unsigned long long)(16 * (tid >> 6)) * p.b;
    for (int q = tid >> 6; q < nq4; q += 8, x += step) t1[s * P + q] = phasor_hw(x);
  };
  // the average's A operand, the real form of T2
  auto aavg_fill = [&]() {
    if (tid < 256) {
      // real form of T2 for the average: thread (k, i) makes T2 of source 64 + k
      // at offsets 4i .. 4i+3 and writes 16 bytes of rows k ((T2r), (-T2i)) and
      // 64 + k ((T2i), (T2r)) at K = 4i and 16 + 4i.  Lanes: k & 7 = lane & 7.
      const int k = (tid & 7) + 8 * (tid >> 5), i = (tid >> 3) & 3;
      float2 zr[4], zi[4], zn[4];
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 z = phasor_hw((unsigned long long)(4 * i + u) * ph[kT5Src + k].b);
        zr[u] = t5_split_store(z.x); zi[u] = t5_split_store(z.y); zn[u] = t5_split_store(-z.y);
      }
      const int o0 = kmaj_byte(k, 4 * i, 32), o1 = kmaj_byte(k, 16 + 4 * i, 32);
      const int o2 = kmaj_byte(64 + k, 4 * i, 32), o3 = kmaj_byte(64 + k, 16 + 4 * i, 32);
      *reinterpret_cast<float4*>(aavg_hi + o0) = make_float4(zr[0].x, zr[1].x, zr[2].x, zr[3].x);
      *reinterpret_cast<float4*>(aavg_lo + o0) = make_float4(zr[0].y, zr[1].y, zr[2].y, zr[3].y);
      *reinterpret_cast<float4*>(aavg_hi + o1) = make_float4(zn[0].x, zn[1].x, zn[2].x, zn[3].x);
      *reinterpret_cast<float4*>(aavg_lo + o1) = make_float4(zn[0].y, zn[1].y, zn[2].y, zn[3].y);
      *reinterpret_cast<float4*>(aavg_hi + o2) = make_float4(zi[0].x, zi[1].x, zi[2].x, zi[3].x);
      *reinterpret_cast<float4*>(aavg_lo + o2) = make_float4(zi[0].y, zi[1].y, zi[2].y, zi[3].y);
      *reinterpret_cast<float4*>(aavg_hi + o3) = make_float4(zr[0].x, zr[1].x, zr[2].x, zr[3].x);
      *reinterpret_cast<float4*>(aavg_lo + o3) = make_float4(zr[0].y, zr[1].y, zr[2].y, zr[3].y);
    }
  };

  // the subtraction's B operand, the real form of conj(T2): thread (r, j) makes
  // T2 of sources 2j, 2j+1 at offset r and writes 16 bytes (K = 4j .. 4j+3) of
  // rows 2r (T2r, T2i per source) and 2r+1 (-T2i, T2r).  Lanes: r & 3 = lane & 3,
  // j & 7 = lane >> 2; the row written first alternates with j, so each store
  // instruction covers 8 row residues x 4 core matrices (no extra conflicts).
  auto bsub_fill = [&]() {
    const int r = (tid & 3) + 4 * (tid >> 7), j = (tid >> 2) & 31;
    const float2 z0 = phasor_hw((unsigned long long)r * ph[2 * j].b);
    const float2 z1 = phasor_hw((unsigned long long)r * ph[2 * j + 1].b);
    const float2 a0 = t5_split_store(z0.x), a1 = t5_split_store(z0.y), a2 = t5_split_store(z1.x), a3 = t5_split_store(z1.y);
    const float2 n1 = t5_split_store(-z0.y), n3 = t5_split_store(-z1.y);
    #pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int pout = u ^ (j & 1);
      const int o = kmaj_byte(2 * r + pout, 4 * j, 128);
      const float4 h = pout ? make_float4(n1.x, a0.x, n3.x, a2.x) : make_float4(a0.x, a1.x, a2.x, a3.x);
      const float4 l = pout ? make_float4(n1.y, a0.y, n3.y, a2.y) : make_float4(a0.y, a1.y, a2.y, a3.y);
      *reinterpret_cast<float4*>(bsub_hi + o) = h;
      *reinterpret_cast<float4*>(bsub_lo + o) = l;
    }
  };
  // one thread issues the MMAs; warp 0 (converged) waits for their commit
  auto mma_wait = [&](uint64_t* bar, uint32_t parity) {
    if (warp == 0) {
      if (!mbar_wait(bar, parity, kT5MaxPolls) && lane == 0) s_bad = 1;
      fence_before_sync();
    }
    __syncthreads();
    fence_after_sync();
  };
  auto load_ph = [&](int t, bool sub) {     // 64 threads: the phases of one role at time t
    const int base = sub ? 0 : kT5Src;
    if (tid >= base && tid < base + kT5Src) {
      const int k = tid - base;
      PhaseAB p;
      p.a = 0; p.b = 0;
      if (sub ? (SUB && k < a.n_sub) : (ACC && k < a.n_acc))
        p = (sub ? a.ph_sub : a.ph_acc)[((size_t)bl * a.n_time + t) * bk + k];
      ph[tid] = p;
    }
  };
  auto sub_tables = [&]() {                 // T1 of the subtracted sources and the subtraction's B operand
    t1_fill(0);
    bsub_fill();
  };
  const int ncg = (4 * nq4 + 47) / 48;      // column groups of the average with data

  // tables of the first time step's subtraction
  if (SUB) {
    load_ph(0, true);
    __syncthreads();
    sub_tables();
  }
  for (int t = 0; t < a.n_time; ++t) {
    const int buf = t & 1;
    if (ACC) load_ph(t, false);
    if (t + 1 < a.n_time) prefetch(t + 1, buf ^ 1);
    cp_async_commit();
    cp_async_wait1();                         // this step's strip has landed
    fence_smem_async();
    __syncthreads();                          // strip, phases and the subtraction's tables ready
    const float* strip = strip0 + (size_t)buf * n16 * 8;
    if (!SUB) {                               // first pass: the average's tables now
      t1_fill(kT5Src);
      aavg_fill();
      fence_smem_async();
      __syncthreads();
    }

    if (SUB) {
      float2* dst = reinterpret_cast<float2*>(a.dst + ((size_t)t * a.n_bl + bl) * a.n_chan * 2);
      for (int T = 0; T < ntile; ++T) {
        const int rows = min(128, 4 * nq4 - 128 * T);
        // W of this tile -> TMEM: warp (quarter, kq) writes rows 32 quarter + lane,
        // sources 16 kq .. 16 kq + 15 (columns 32 kq .. 32 kq + 31, hi and lo)
        if (32 * quarter < rows) {
          const int n = 128 * T + 32 * quarter + lane, q = n >> 2, e = n & 3, kq = warp >> 2;
          #pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t rh[16], rl[16];
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int k = 16 * kq + 8 * h + j;
              const float2 w = t1[k * P + q], m = mtab[4 * k + e];
              const float wr = fmaf(w.x, m.x, w.y * m.y), wi = fmaf(w.x, m.y, -w.y * m.x);
              const uint32_t hr = t5_tf32(wr), hi = t5_tf32(wi);
              rh[2 * j] = hr;
              rh[2 * j + 1] = hi;
              rl[2 * j] = __float_as_uint(wr - __uint_as_float(hr));       // the MMA truncates lo to TF32
              rl[2 * j + 1] = __float_as_uint(wi - __uint_as_float(hi));
            }
            const uint32_t col = kT5ColW + 32 * kq + 16 * h;
            tmem_st16(tmem + lane_base + col, rh);
            tmem_st16(tmem + lane_base + col + 128, rl);
          }
          tmem_wait_st();
        }
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (warp < 8 && lane == 0) {
          // warp g issues accumulator g: sources 8g .. 8g+7 (k-steps 2g, 2g+1),
          // lo(W) hi(B2), hi(W) lo(B2), then hi(W) hi(B2); k-step s adds 256 s
          // bytes (16 s in the descriptor's address field).  Eight issuers keep
          // any one warp's delay short; each commits to the same mbarrier.
          const uint32_t id = idesc_tf32(128, 32);
          const int g = warp;
          const uint32_t d = tmem + kT5ColO + 32 * g;
          #pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint32_t acol = tmem + kT5ColW + (pass == 0 ? 128 : 0);
            const uint64_t bd = pass == 1 ? dsub_lo : dsub_hi;
            #pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int s = 2 * g + u;
              mma_ts(d, acol + 8 * s, bd + 16 * s, id, (pass | u) != 0);
            }
          }
          commit(&mbar[0]);
        }
        if (ACC && T == 0) {                  // overlaps the subtraction MMAs of tile 0
          t1_fill(kT5Src);
          aavg_fill();
          fence_smem_async();
        }
        mma_wait(&mbar[0], par_sub);          // subtraction MMAs of this tile complete
        par_sub ^= 1;
        // epilogue: residual = strip - O, to HBM, and split into the average's B
        // operand.  Warp (quarter, j) takes rows 32 quarter + lane of the tile and
        // channels 16 q + 4 j .. 16 q + 4 j + 3 (columns 8 j .. 8 j + 7 of each
        // accumulator: (re, im) of 4 channels)
        if (32 * quarter < rows) {
          const int n = 128 * T + 32 * quarter + lane, q = n >> 2, e = n & 3, j = warp >> 2;
          float o[8];
          #pragma unroll
          for (int i = 0; i < 8; ++i) o[i] = 0.f;
          float v[8][8];
          #pragma unroll
          for (int g = 0; g < 8; ++g) tmem_ld8(tmem + lane_base + kT5ColO + 32 * g + 8 * j, v[g]);
          tmem_wait_ld();
          #pragma unroll
          for (int g = 0; g < 8; ++g)
            #pragma unroll
            for (int i = 0; i < 8; ++i) o[i] += v[g][i];
          float xr[4], xi[4];
          #pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = 16 * q + 4 * j + u;
            const float2 sv = *reinterpret_cast<const float2*>(strip + t5_swz(c) * 8 + 2 * e);
            const float2 x = make_float2(sv.x - o[2 * u], sv.y - o[2 * u + 1]);
            const bool live = c < a.n_chan;
            if (live) __stcs(dst + (size_t)c * 4 + e, x);
            xr[u] = live ? x.x : 0.f;
            xi[u] = live ? x.y : 0.f;
          }
          if (ACC) {
            float2 s0 = t5_split(xr[0]), s1 = t5_split(xr[1]), s2 = t5_split(xr[2]), s3 = t5_split(xr[3]);
            const float4 hr = make_float4(s0.x, s1.x, s2.x, s3.x), lr = make_float4(s0.y, s1.y, s2.y, s3.y);
            s0 = t5_split(xi[0]); s1 = t5_split(xi[1]); s2 = t5_split(xi[2]); s3 = t5_split(xi[3]);
            const float4 hi4 = make_float4(s0.x, s1.x, s2.x, s3.x), li4 = make_float4(s0.y, s1.y, s2.y, s3.y);
            const int ore = kmaj_byte(n, 4 * j, 32), oim = kmaj_byte(n, 16 + 4 * j, 32);
            *reinterpret_cast<float4*>(bavg_hi + ore) = hr;
            *reinterpret_cast<float4*>(bavg_lo + ore) = lr;
            *reinterpret_cast<float4*>(bavg_hi + oim) = hi4;
            *reinterpret_cast<float4*>(bavg_lo + oim) = li4;
          }
        }
        fence_before_sync();
        __syncthreads();                      // W columns free for the next tile
        fence_after_sync();
      }
    } else if (ACC) {
      // first pass: the average's B operand straight from the strip
      for (int i = tid; i < 4 * nq4 * 8; i += kT5Threads) {
        // lanes: row residue n & 7 = lane & 7, so a warp's 16-byte stores spread over all banks
        const int n = (i & 7) + 8 * (i >> 6), j = (i >> 3) & 7, q = n >> 2, e = n & 3, pin = j >> 2, r0 = 4 * (j & 3);
        float x[4];
        #pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = strip[t5_swz(16 * q + r0 + u) * 8 + 2 * e + pin];
        const float2 s0 = t5_split(x[0]), s1 = t5_split(x[1]), s2 = t5_split(x[2]), s3 = t5_split(x[3]);
        const int o = kmaj_byte(n, 16 * pin + r0, 32);
        *reinterpret_cast<float4*>(bavg_hi + o) = make_float4(s0.x, s1.x, s2.x, s3.x);
        *reinterpret_cast<float4*>(bavg_lo + o) = make_float4(s0.y, s1.y, s2.y, s3.y);
      }
    }

    if (ACC) {
      fence_smem_async();
      fence_before_sync();
      __syncthreads();                        // residual split complete
      fence_after_sync();
      if (warp >= 14 && lane == 0) {
        // warp 14: hi(A2) hi(R) into the main accumulator; warp 15: lo(A2) hi(R)
        // and hi(A2) lo(R) into the cross-term accumulator
        const uint32_t id = idesc_tf32(128, 4 * nq4);
        if (warp == 14) {
          #pragma unroll
          for (int s = 0; s < 4; ++s) mma_ss(tmem + kT5ColDm, da_hi + 16 * s, db_hi + 16 * s, id, s != 0);
        } else {
          #pragma unroll
          for (int s = 0; s < 4; ++s) mma_ss(tmem + kT5ColDx, da_lo + 16 * s, db_hi + 16 * s, id, s != 0);
          #pragma unroll
          for (int s = 0; s < 4; ++s) mma_ss(tmem + kT5ColDx, da_hi + 16 * s, db_lo + 16 * s, id, 1);
        }
        commit(&mbar[1]);
      }
      if (SUB && t + 1 < a.n_time) {          // next step's subtraction tables, beside the average MMAs
        load_ph(t + 1, true);
        __syncthreads();
        sub_tables();
      }
      mma_wait(&mbar[1], par_avg);            // average MMAs complete
      par_avg ^= 1;
      // epilogue: warp (quarter, cg) takes rows m = 32 quarter + lane = (pout, k)
      // and tiles q = 12 cg .. 12 cg + 11; G = main + cross, then the T1-weighted
      // sums, whose column-group parts meet in shared memory (in the average's
      // B operand space, free once its MMAs are complete: ncg x 4 KB <= nq4 KB)
      {
        const int m = 32 * quarter + lane, pout = m >> 6, k = m & 63, cg = warp >> 2;
        const float2* t1k = t1 + (size_t)(kT5Src + k) * P;
        float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
        const int c_end = min(48 * cg + 48, 4 * nq4);
        for (int c0 = 48 * cg; c0 < c_end; c0 += 16) {
          float gm[16], gx[16];
          tmem_ld16(tmem + lane_base + kT5ColDm + c0, gm);
          tmem_ld16(tmem + lane_base + kT5ColDx + c0, gx);
          tmem_wait_ld();
          #pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float2 w = t1k[(c0 >> 2) + qq];
            const float wr = pout ? -w.y : w.x, wi = pout ? w.x : w.y;
            #pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float g = gm[4 * qq + e] + gx[4 * qq + e];
              sr[e] = fmaf(wr, g, sr[e]);
              si[e] = fmaf(wi, g, si[e]);
            }
          }
        }
        float* part = reinterpret_cast<float*>(bavg_hi);     // [ncg][8][128 m]
        if (cg < ncg)
          #pragma unroll
          for (int e = 0; e < 4; ++e) {
            part[(cg * 8 + 2 * e) * 128 + m] = sr[e];
            part[(cg * 8 + 2 * e + 1) * 128 + m] = si[e];
          }
      }
      __syncthreads();
      if (warp < 4) {
        const int m = 32 * quarter + lane;
        const float* part = reinterpret_cast<const float*>(bavg_hi);
        // compensated accumulation across time steps of the parts (fixed order)
        #pragma unroll
        for (int i = 0; i < 8; ++i) {
          float x = part[i * 128 + m];
          for (int c = 1; c < ncg; ++c) x += part[(c * 8 + i) * 128 + m];
          const float y = x - kc[i];
          const float tt = ks[i] + y;
          kc[i] = (tt - ks[i]) - y;
          ks[i] = tt;
        }
      }
    } else if (SUB && t + 1 < a.n_time) {    // last pass: next step's subtraction tables
      load_ph(t + 1, true);
      __syncthreads();
      sub_tables();
    }
    fence_smem_async();
    fence_before_sync();
    __syncthreads();                          // tables, operands and accumulators ready for the next step
    fence_after_sync();
    if (s_bad) break;                         // a wait ran out: stop (reported through *err)
  }

  if (ACC) {
    const int m = 32 * quarter + lane, pout = m >> 6, k = m & 63;
    if (warp < 4 && pout == 1)
      #pragma unroll
      for (int i = 0; i < 8; ++i) red[k * 8 + i] = (double)ks[i] - (double)kc[i];
    __syncthreads();
    if (warp < 4 && pout == 0 && k < a.n_acc)
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        const double re = ((double)ks[2 * e] - (double)kc[2 * e]) + red[k * 8 + 2 * e];
        const double im = ((double)ks[2 * e + 1] - (double)kc[2 * e + 1]) + red[k * 8 + 2 * e + 1];
        a.avg[((size_t)k * a.n_bl + bl) * 4 + e] = make_float2((float)(re * a.inv_n), (float)(im * a.inv_n));
      }
  }
  if (tid == 0 && s_bad) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, kT5Cols);
}

}  // namespace rts
