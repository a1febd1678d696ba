// Blocked peel pass on the 5th-generation tensor cores, transposed form: the
// same pass as k_block_pass (subtract the solved sources of block b from one
// (baseline, time step) strip of channels, average the directions of block b+1),
// with both contractions as tcgen05.mma kind::tf32 GEMMs whose operands the
// CUDA cores form in O(sources x 16) or O(sources x channels / 16) work.
//
// The phasor of source k at channel c = 16 q + r factors as
//   P_k(c) = T1_k[q] T2_k[r],  T1_k[q] = e^{2 pi i (A_k + 16 q B_k)},  T2_k[r] = e^{2 pi i r B_k}.
//
// subtraction  R(16 q + r, e) -= sum_k [M_k(e) conj(T2_k[r])] conj(T1_k[q])
//   GEMM D_s[m, q] = sum_K A_s[m, K] B_s[q, K], M = 128 rows m = 8 r + 2 e + o
//   (o: real or imaginary part of the output), K = 128 = (source k, re/im),
//   N = NQ (the 16-channel tiles, rounded up to 16).  A_s = the real form of
//   a_k(r, e) = M_k(e) conj(T2_k[r]) (rows o = 0: (a_re, -a_im), o = 1:
//   (a_im, a_re)), written by the threads into TMEM; B_s = conj(T1) as
//   (re, im) pairs along K in shared memory.  One 128-row tile whatever the
//   channel count, and 64 x 16 x 4 operand products per step.
// average      A_k(e) += sum_r T2_k[r] H_k(r, e),  H_k(r, e) = sum_q T1_k[q] R(16 q + r, e)
//   GEMM D_a[m', n] = sum_K' A_a[m', K'] B_a[n, K'], M = 128 rows m' = 2 k + o,
//   K' = 2 NQ = (re/im i, q) at i NQ + q, N = 64 columns n = 4 r + e.  A_a =
//   the real form of T1 (row o = 0: t_re at i = 0, -t_im at i = 1; row o = 1:
//   t_im, t_re) in TMEM; B_a = the new residual, written by the subtraction's
//   epilogue in shared memory (4 consecutive tiles of one part per 16-byte
//   store).  The 16-term T2 contraction of H runs on the CUDA cores (32 FMAs a
//   thread) beside the next step's subtraction MMAs, summed over time steps
//   with compensation.
//
// TF32 keeps 11 significand bits, so every operand is split x = hi + lo and
// each product takes three MMAs, hi*hi + lo*hi + hi*lo.  The tensor cores'
// FP32 accumulation does not round to nearest, so the hi*hi products go to
// accumulators of 4 k-steps each and the (2^-11 smaller) cross terms to one
// more; the epilogues add them in FP32 with round-to-nearest.
//
// One CTA of 16 warps per baseline (1 per SM: ~170 KB of shared memory, all 512
// TMEM columns), looping over the time steps.  The strip of a time step
// arrives by a bulk asynchronous copy one step ahead and the residual leaves
// by one, so the CUDA cores move no visibility data to or from HBM.  A step:
//   P1  subtraction MMAs   | beside them: the previous step's T2 contraction,
//                            T1 and T2 of the averaged sources
//   P2  subtraction epilogue (residual into the strip and B_a), A_a into TMEM
//   P3  average MMAs       | beside them: the residual's store, the next
//                            step's B_s and T2 of the subtracted sources
//   P4  the average's accumulators into registers, the next step's A_s into TMEM
// Four more warps issue the MMAs, one accumulator each: an issuing thread
// stalls while its MMAs are accepted (a few tens of cycles each), so the 16
// compute warps, which meet at a named barrier of their own, never wait for
// it; operands-ready and MMAs-done mbarriers hand each phase between them.  Every wait is bounded
// (a wait that runs out sets *err and stops the pass, which the status read
// reports, after the copies in flight have been waited for and TMEM is freed).
// Limits: at most 64 sources per role, n_chan <= kTc5MaxChan.
//
// Gains Taylor-expanded in frequency (TAY): a source's model on a baseline is
// (P0 + x_c P1 + x_c^2 P2) e^{-2 pi i phi} and its averages are the three
// moments mean x_c^n R e^{+2 pi i phi}.  With x_c = u_q + v_r (u_q = x_0 + 16 q dx,
// v_r = r dx) the same two GEMMs carry them when each source takes three of
// the 64 operand slots, s = 3 k + m (21 sources per block):
//   subtraction  slot (k, m): A_s = [sum_{n >= m} C(n, m) v_r^{n-m} P_n] conj(T2_k[r])
//                             B_s = u_q^m conj(T1_k[q])
//   average      slot (k, m): A_a rows = u_q^m T1_k[q] (real form), so the GEMM gives
//                             H_km(r, e) = sum_q u_q^m T1_k[q] R(16 q + r, e), and
//                M_kn = sum_{m <= n} C(n, m) sum_r v_r^{n-m} T2_k[r] H_km(r, e).
// The CUDA cores form the coefficient table once per CTA, the u_q^m weights
// beside the phasors, and three v_r-weighted T2 sums per slot.
#pragma once
#include "block_kernels.cuh"
#include "tc05.cuh"

namespace rts {

constexpr int kTc5Compute = 512;             // 16 compute warps (4 per TMEM lane quarter)
constexpr int kTc5Issuers = 4;               // and 4 warps whose lane 0 issues one accumulator's MMAs
constexpr int kTc5Threads = kTc5Compute + 32 * kTc5Issuers;
constexpr int kTc5Src = 64;                  // sources per role
constexpr int kTc5BaselinesPerCta = 16;     // baselines a CTA peels one after another (not Taylor):
                                             // its set-up and first operands are paid once for them
constexpr int kTc5MaxChan = 768;             // NQ <= 48: 5 NQ accumulator columns beside A_s
constexpr uint32_t kTc5MaxPolls = 1u << 17;  // mbarrier polls (each up to 20 us) before giving up
constexpr int kTc5T2Row = 17;                // T2 table row stride (float2): conflict-free column reads
// TMEM columns.  Subtraction: accumulators g = 0..3 at g NQ (< 192), A_s lo at
// [192, 320), A_s hi at [384, 512).  Average: accumulators g < NQ / 16 at 64 g
// (< 192), A_a hi at [192, 192 + 2 NQ), lo after it (< 384).  So the next step's
// A_s hi can be written while the average's MMAs run, and its lo once they are
// done, beside the reads of the average's accumulators.
constexpr uint32_t kTc5ColAcc = 0;
constexpr uint32_t kTc5ColALo = 192;         // A_s lo; A_a (hi then lo)
constexpr uint32_t kTc5ColAHi = 384;         // A_s hi
constexpr uint32_t kTc5Cols = 512;

// shared-memory layout (byte offsets) for NQ 16-channel tiles (16, 32 or 48)
constexpr int kTayBlk = 21;                  // Taylor sources per block: 3 slots each
constexpr int kTayOut = 6 * kTayBlk;         // v_r-weighted T2 sums per block (6 per source)

struct Tc05Smem {
  int strip, bs_hi, bs_lo, ba_hi, ba_lo, t2s, t2a, mtab, ph, bar, cf, total;
  __host__ __device__ explicit Tc05Smem(int NQ, bool tay = false) {
    int o = 0;
    strip = o; o += 2 * 16 * NQ * 32;            // two strips [16 NQ channels][4 pol][re, im]
    bs_hi = o; o += NQ * 128 * 4;                // B_s [NQ rows][128 K], K-major
    bs_lo = o; o += NQ * 128 * 4;
    ba_hi = o; o += 64 * 2 * NQ * 4;             // B_a [64 rows][2 NQ K], K-major
    ba_lo = o; o += 64 * 2 * NQ * 4;
    t2s = o;   o += kTc5Src * kTc5T2Row * 8;       // T2 of the subtracted sources [64][17] float2
    t2a = o;   o += kTc5Src * kTc5T2Row * 8;       // T2 of the averaged sources
    mtab = o;  o += kTc5Src * 4 * 8;              // model matrices [64][4] float2
    ph = o;    o += 2 * 2 * kTc5Src * 16;         // phases of two time steps [2][sub 64, avg 64]
    bar = o;   o += 80;                          // mbarriers (sub done, avg done, strip 0, strip 1, sub
                                                 // operands ready, avg operands ready, phases 0, phases 1),
                                                 // TMEM address
    cf = o;    o += tay ? kTc5Src * 16 * 4 * 8 : 0;  // Taylor A_s coefficients [64 slots][16 r][4 e] float2
    total = o;
  }
};

inline int tc05_nq(int n_chan) { return (((n_chan + 15) >> 4) + 15) & ~15; }
inline size_t tc05_pass_smem(int n_chan, bool tay = false) { return (size_t)Tc05Smem(tc05_nq(n_chan), tay).total; }

// TF32 rounding (to nearest, ties away from zero, as cvt.rna.tf32.f32 for
// finite x below the FP32 maximum) by two integer operations
__device__ __forceinline__ uint32_t tc05_tf32(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
// x = hi + lo, hi the TF32 rounding of x, lo the exact remainder (the MMA reads
// lo truncated to TF32: error below 2^-21 |x|)
__device__ __forceinline__ float2 tc05_split(float x) {
  const float hi = __uint_as_float(tc05_tf32(x));
  return make_float2(hi, x - hi);
}

template <bool SUB, bool ACC, bool TAY = false>
__global__ void __launch_bounds__(kTc5Threads, 1) k_block_pass_tc05(BlockPassArgs a, int bk, int nb, int* err) {
  using namespace tc05;
  const int nq = (a.n_chan + 15) >> 4;
  const int NQ = (nq + 15) & ~15;           // 16, 32 or 48
  const int QW = NQ >> 2;                   // tiles per column-group warp: 4, 8 or 12
  const int nmain_a = NQ >> 4;              // the average's hi*hi accumulators: 1, 2 or 3
  const int n16 = 16 * NQ;
  const uint32_t strip_bytes = (uint32_t)a.n_chan * 32u;
  const Tc05Smem L(NQ, TAY);
  extern __shared__ __align__(1024) unsigned char tc05_smem[];
  float* strip0 = reinterpret_cast<float*>(tc05_smem + L.strip);
  unsigned char* bs_hi = tc05_smem + L.bs_hi;
  unsigned char* bs_lo = tc05_smem + L.bs_lo;
  unsigned char* ba_hi = tc05_smem + L.ba_hi;
  unsigned char* ba_lo = tc05_smem + L.ba_lo;
  float2* t2s = reinterpret_cast<float2*>(tc05_smem + L.t2s);
  float2* t2a = reinterpret_cast<float2*>(tc05_smem + L.t2a);
  float2* mtab = reinterpret_cast<float2*>(tc05_smem + L.mtab);
  PhaseAB* ph = reinterpret_cast<PhaseAB*>(tc05_smem + L.ph);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc05_smem + L.bar);      // see Tc05Smem::bar
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc05_smem + L.bar + 64);
  float2* cf = reinterpret_cast<float2*>(tc05_smem + L.cf);             // Taylor only
  // [4 cg][64 slots][8] (Taylor: [4 cg][128 sums][8], B_a hi and lo): B_a is free in P4
  constexpr int kPartRows = TAY ? 2 * kTc5Src : kTc5Src;
  float* part = reinterpret_cast<float*>(ba_hi);
  // slot -> source, and the slot's power m of u_q (Taylor: slot 3 k + m)
  auto src_of = [](int s) { return TAY ? s / 3 : s; };
  auto pow_of = [](int s) { return TAY ? s % 3 : 0; };
  // u_q^m, u_q = x_0 + 16 q dx the offset of tile q's channel 0 from the band centre
  auto upow = [&](int q, int m) {
    const float u = fmaf((float)(16 * q), a.tdx, a.tx0);
    return m == 0 ? 1.f : (m == 1 ? u : u * u);
  };

  // baselines bl0 .. bl0 + nbl - 1, their time steps one after another: step g
  // is time g % n_time of baseline bl0 + g / n_time
  const int64_t bl0 = (int64_t)blockIdx.x * nb;
  const int nbl = TAY ? 1 : (int)min((int64_t)nb, a.n_bl - bl0), n_steps = TAY ? a.n_time : nbl * a.n_time;
  auto bl_of = [&](int g) { return bl0 + g / a.n_time; };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qtr = warp & 3, cg = warp >> 2;
  const uint32_t lane_base = (uint32_t)(32 * qtr) << 16;

  if (warp == 0) tmem_alloc(tslot, kTc5Cols);
  if (tid == 0) {
    mbar_init(&mbar[0], kTc5Issuers);        // subtraction MMAs done: one commit per issuer
    mbar_init(&mbar[1], nmain_a);           // average MMAs done: one commit per accumulator
    for (int i = 2; i < 8; ++i) mbar_init(&mbar[i], 1);   // each completed by one arrival
  }
  const bool compute = tid < kTc5Compute;
  // padding channels of both strips stay zero (the copies never write them)
  for (int i = tid; compute && i < (n16 - a.n_chan) * 8; i += kTc5Compute) {
    strip0[a.n_chan * 8 + i] = 0.f;
    strip0[(n16 + a.n_chan) * 8 + i] = 0.f;
  }
  const int n_sub_slots = TAY ? 3 * a.n_sub : a.n_sub;
  if (SUB)
    for (int i = tid; compute && i < kTc5Src * 4; i += kTc5Compute) {
      const int s = i >> 2, e = i & 3;
      mtab[i] = s < n_sub_slots ? a.M_sub[((size_t)s * a.n_bl + bl0) * 4 + e] : make_float2(0.f, 0.f);
    }
  if (SUB && TAY) {
    // the Taylor subtraction's A_s coefficients, slot (k, m), channel offset r:
    // sum_{n >= m} C(n, m) v_r^{n-m} P_n, v_r = r dx (from the model table mtab)
    __syncthreads();
    for (int i = tid; compute && i < kTc5Src * 64; i += kTc5Compute) {
      const int s = i >> 6, r = (i >> 2) & 15, e = i & 3, k = s / 3, m = s - 3 * k;
      float2 c = make_float2(0.f, 0.f);
      if (k < a.n_sub) {
        const float v = (float)r * a.tdx;
        const float2 p2 = mtab[4 * (3 * k + 2) + e];
        if (m == 2) {
          c = p2;
        } else if (m == 1) {
          const float2 p1 = mtab[4 * (3 * k + 1) + e];
          c = make_float2(fmaf(2.f * v, p2.x, p1.x), fmaf(2.f * v, p2.y, p1.y));
        } else {
          const float2 p1 = mtab[4 * (3 * k + 1) + e], p0 = mtab[4 * (3 * k) + e];
          c = make_float2(fmaf(v, fmaf(v, p2.x, p1.x), p0.x), fmaf(v, fmaf(v, p2.y, p1.y), p0.y));
        }
      }
      cf[i] = c;
    }
  }
  // phases of sources beyond bk stay zero (the copies bring bk per role)
  for (int i = tid; compute && i < 4 * kTc5Src; i += kTc5Compute) {
    ph[i].a = 0;
    ph[i].b = 0;
  }
  fence_smem_async();                      // the zero fills precede the bulk copies into the same words
  // a pass in which some CTA's wait already ran out does no more work
  __shared__ int s_bad;
  if (tid == 0) s_bad = *reinterpret_cast<volatile int*>(err);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  const uint64_t dbs_hi = desc_kmajor(smem_u32(bs_hi), 128, 4096), dbs_lo = desc_kmajor(smem_u32(bs_lo), 128, 4096);
  const uint64_t dba_hi = desc_kmajor(smem_u32(ba_hi), 128, 64 * NQ), dba_lo = desc_kmajor(smem_u32(ba_lo), 128, 64 * NQ);

  // strip of step g -> buffer g & 1 (thread 0)
  auto issue_load = [&](int g) {
    const int b = g & 1, t = g % a.n_time;
    mbar_expect_tx(&mbar[2 + b], strip_bytes);
    bulk_load(strip0 + (size_t)b * n16 * 8, a.src + ((size_t)t * a.n_bl + bl_of(g)) * a.n_chan * 2, strip_bytes,
              &mbar[2 + b]);
  };
  // the phases of both roles at step g -> ring slot g & 1 (thread 0): one bulk
  // copy of bk entries per role, completing on mbarrier 6 + (g & 1)
  auto issue_ph = [&](int g) {
    const int b = g & 1;
    const uint32_t bytes = (uint32_t)bk * sizeof(PhaseAB);
    mbar_expect_tx(&mbar[6 + b], (SUB ? bytes : 0u) + (ACC ? bytes : 0u));
    const size_t at = ((size_t)bl_of(g) * a.n_time + g % a.n_time) * bk;
    if (SUB) bulk_load(ph + 2 * kTc5Src * b, a.ph_sub + at, bytes, &mbar[6 + b]);
    if (ACC) bulk_load(ph + 2 * kTc5Src * b + kTc5Src, a.ph_acc + at, bytes, &mbar[6 + b]);
  };
  // T2_k[r] of one role from its phases p[64]: [64][kTc5T2Row]
  auto t2_fill = [&](float2* t2, const PhaseAB* p) {
    for (int i = tid; i < kTc5Src * 16; i += kTc5Compute) {
      const int k = i >> 4, r = i & 15;
      t2[k * kTc5T2Row + r] = phasor_hw((unsigned long long)r * p[src_of(k)].b);
    }
  };
  // B_s = conj(T1_k[q]) of the subtracted sources: thread (q & 7 = lane & 7,
  // k = (lane >> 3) + 4 warp) steps q by 8 with an exact 64-bit phase increment;
  // its 8-byte (re, im) stores cover 16 distinct slots of each 128-byte line
  auto bs_fill = [&](const PhaseAB* ps) {
    const int ql = tid & 7, k = ((tid >> 3) & 3) + 4 * warp, m = pow_of(k);
    const PhaseAB p = ps[src_of(k)];
    const unsigned long long step = 128ull * p.b;
    unsigned long long x = p.a + (unsigned long long)(16 * ql) * p.b;
    for (int q = ql; q < NQ; q += 8, x += step) {
      float2 z = phasor_hw(x);
      if (TAY) {
        const float w = upow(q, m);
        z = make_float2(z.x * w, z.y * w);
      }
      const float hr = __uint_as_float(tc05_tf32(z.x)), hi = __uint_as_float(tc05_tf32(-z.y));
      const int o = kmaj_byte(q, 2 * k, 128);
      *reinterpret_cast<float2*>(bs_hi + o) = make_float2(hr, hi);
      *reinterpret_cast<float2*>(bs_lo + o) = make_float2(__uint_as_float(tc05_tf32(z.x - hr)),
                                                          __uint_as_float(tc05_tf32(-z.y - hi)));
    }
  };
  // A_s of warp (qtr, cg): rows m = 32 qtr + lane = 8 r + 2 e + o, sources
  // 16 cg .. 16 cg + 15 (columns 32 cg .. 32 cg + 31): the hi parts go to TMEM
  // here, the lo parts stay in lo[] for as_store_lo
  auto as_store_hi = [&](uint32_t (&lo)[32]) {
    const int r = 4 * qtr + (lane >> 3), e = (lane >> 1) & 3, o = lane & 1;
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t vh[16];
      #pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = 16 * cg + 8 * h + j;
        const float2 m = TAY ? cf[(k * 16 + r) * 4 + e] : mtab[4 * k + e], z = t2s[k * kTc5T2Row + r];
        const float ar = fmaf(m.x, z.x, m.y * z.y), ai = fmaf(m.y, z.x, -m.x * z.y);   // m conj(z)
        const float v0 = o ? ai : ar, v1 = o ? ar : -ai;
        const uint32_t h0 = tc05_tf32(v0), h1 = tc05_tf32(v1);
        vh[2 * j] = h0;
        vh[2 * j + 1] = h1;
        lo[16 * h + 2 * j] = __float_as_uint(v0 - __uint_as_float(h0));
        lo[16 * h + 2 * j + 1] = __float_as_uint(v1 - __uint_as_float(h1));
      }
      tmem_st16(tmem + lane_base + kTc5ColAHi + 32 * cg + 16 * h, vh);
    }
  };
  auto as_store_lo = [&](const uint32_t (&lo)[32]) {
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t vl[16];
      #pragma unroll
      for (int i = 0; i < 16; ++i) vl[i] = lo[16 * h + i];
      tmem_st16(tmem + lane_base + kTc5ColALo + 32 * cg + 16 * h, vl);
    }
  };
  // T1_k[q] of the averaged source k = 16 qtr + lane / 2 for the warp's tiles
  // q = cg QW .. cg QW + QW - 1: the lane pair (o = 0, 1) computes even and odd
  // tiles and exchanges them
  auto aa_compute = [&](float2 (&t1v)[12], const PhaseAB* pa) {
    const int k = 16 * qtr + (lane >> 1), o = lane & 1, q0 = cg * QW, m = pow_of(k);
    const PhaseAB p = pa[src_of(k)];
    const unsigned long long step = 32ull * p.b;
    unsigned long long x = p.a + (unsigned long long)(16 * (q0 + o)) * p.b;
    #pragma unroll
    for (int jj = 0; jj < 6; ++jj) {
      float2 mine = make_float2(0.f, 0.f);
      if (2 * jj < QW) {
        mine = phasor_hw(x);
        if (TAY) {
          const float w = upow(q0 + 2 * jj + o, m);
          mine = make_float2(mine.x * w, mine.y * w);
        }
        x += step;
      }
      const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, mine.x, 1), __shfl_xor_sync(0xffffffffu, mine.y, 1));
      t1v[2 * jj] = o ? other : mine;
      t1v[2 * jj + 1] = o ? mine : other;
    }
  };
  // A_a -> TMEM: rows m' = 2 k + o, columns i NQ + q of the warp's tiles
  auto aa_store = [&](const float2 (&t1v)[12]) {
    const int o = lane & 1, q0 = cg * QW;
    #pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      if (4 * ch < QW) {
        uint32_t h0[4], l0[4], h1[4], l1[4];
        #pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 t = t1v[4 * ch + u];
          const float v0 = o ? t.y : t.x, v1 = o ? t.x : -t.y;     // i = 0, i = 1
          h0[u] = tc05_tf32(v0);
          h1[u] = tc05_tf32(v1);
          l0[u] = __float_as_uint(v0 - __uint_as_float(h0[u]));
          l1[u] = __float_as_uint(v1 - __uint_as_float(h1[u]));
        }
        const uint32_t col = kTc5ColALo + q0 + 4 * ch;
        tmem_st4(tmem + lane_base + col, h0);
        tmem_st4(tmem + lane_base + NQ + col, h1);
        tmem_st4(tmem + lane_base + 2 * NQ + col, l0);
        tmem_st4(tmem + lane_base + 3 * NQ + col, l1);
      }
    }
  };
  // residual values x[u] = R(16 (q + u) + r, e).o, u = 0..3, into B_a at
  // (n = 4 r + e, K' = o NQ + q + u): one 16-byte store each for hi and lo
  auto ba_put4 = [&](int n, int q, int o, const float (&x)[4]) {
    float4 h, l;
    float2 s2 = tc05_split(x[0]); h.x = s2.x; l.x = s2.y;
    s2 = tc05_split(x[1]); h.y = s2.x; l.y = s2.y;
    s2 = tc05_split(x[2]); h.z = s2.x; l.z = s2.y;
    s2 = tc05_split(x[3]); h.w = s2.x; l.w = s2.y;
    const int off = kmaj_byte(n, o * NQ + q, 2 * NQ);
    *reinterpret_cast<float4*>(ba_hi + off) = h;
    *reinterpret_cast<float4*>(ba_lo + off) = l;
  };
  // subtraction epilogue: warp (qtr, cg), rows m = 8 r + 2 e + o of lane, tiles
  // q = cg QW .. ; the strip word (16 q + r) 8 + 2 e + o of the 32 lanes is 32
  // consecutive words (conflict-free)
  auto sub_epilogue = [&](float* strip) {
    const int r = 4 * qtr + (lane >> 3), e = (lane >> 1) & 3, o = lane & 1, n = 4 * r + e, q0 = cg * QW;
    const uint32_t base = tmem + lane_base + kTc5ColAcc + q0;
    #pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      if (4 * ch < QW) {
        float v[4][4];
        #pragma unroll
        for (int g = 0; g < 4; ++g) tmem_ld4(base + g * NQ + 4 * ch, v[g]);
        tmem_wait_ld();
        float x[4];
        #pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = 16 * (q0 + 4 * ch + u) + r;
          const float d = ((v[0][u] + v[1][u]) + v[2][u]) + v[3][u];
          x[u] = 0.f;
          if (c < a.n_chan) {
            float* sp = strip + c * 8 + 2 * e + o;
            x[u] = *sp - d;
            *sp = x[u];
          }
        }
        if (ACC) ba_put4(n, q0 + 4 * ch, o, x);
      }
    }
  };
  // first pass: B_a straight from the strip
  auto ba_from_strip = [&](const float* strip) {
    const int r = 4 * qtr + (lane >> 3), e = (lane >> 1) & 3, o = lane & 1, n = 4 * r + e, q0 = cg * QW;
    for (int j = 0; j < QW; j += 4) {
      float x[4];
      #pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = strip[(16 * (q0 + j + u) + r) * 8 + 2 * e + o];
      ba_put4(n, q0 + j, o, x);
    }
  };
  // the T2 contraction of one step's H (rows m' = 2 k + o of lane, columns
  // n = 4 r + e of r = 4 cg .. 4 cg + 3): o = 0 holds Re H (A += T2 Re H), o = 1
  // Im H (A += i T2 Im H); the lane pair's sums meet by a shuffle and the four
  // column groups' in part[cg][k]
  auto avg_contract_plain = [&](const float (&H)[16]) {
    const int k = 16 * qtr + (lane >> 1), o = lane & 1;
    float pr[4] = {0.f, 0.f, 0.f, 0.f}, pi[4] = {0.f, 0.f, 0.f, 0.f};
    #pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const float2 z = t2a[k * kTc5T2Row + 4 * cg + rr];
      const float wr = o ? -z.y : z.x, wi = o ? z.x : z.y;
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        pr[e] = fmaf(wr, H[4 * rr + e], pr[e]);
        pi[e] = fmaf(wi, H[4 * rr + e], pi[e]);
      }
    }
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      pr[e] += __shfl_xor_sync(0xffffffffu, pr[e], 1);
      pi[e] += __shfl_xor_sync(0xffffffffu, pi[e], 1);
    }
    if (o == 0) {
      float4* dst = reinterpret_cast<float4*>(part + (cg * kPartRows + k) * 8);
      dst[0] = make_float4(pr[0], pi[0], pr[1], pi[1]);
      dst[1] = make_float4(pr[2], pi[2], pr[3], pi[3]);
    }
  };
  // Taylor: slot s = 3 k + m gives Q_{k,m,d}(e) = sum_r v_r^d T2_k[r] H_km(r, e) for
  // d = 0 .. 2 - m, sum index 6 k + {0, 3, 5}[m] + d (the moments combine them at the end)
  auto avg_contract_tay = [&](const float (&H)[16]) {
    const int s = 16 * qtr + (lane >> 1), o = lane & 1, k = s / 3, m = s - 3 * k;
    float pr[3][4], pi[3][4];
    #pragma unroll
    for (int d = 0; d < 3; ++d)
      #pragma unroll
      for (int e = 0; e < 4; ++e) { pr[d][e] = 0.f; pi[d][e] = 0.f; }
    #pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const float2 z = t2a[s * kTc5T2Row + 4 * cg + rr];
      const float v = (float)(4 * cg + rr) * a.tdx;
      float wr = o ? -z.y : z.x, wi = o ? z.x : z.y;
      #pragma unroll
      for (int d = 0; d < 3; ++d) {
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          pr[d][e] = fmaf(wr, H[4 * rr + e], pr[d][e]);
          pi[d][e] = fmaf(wi, H[4 * rr + e], pi[d][e]);
        }
        wr *= v;
        wi *= v;
      }
    }
    #pragma unroll
    for (int d = 0; d < 3; ++d)
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        pr[d][e] += __shfl_xor_sync(0xffffffffu, pr[d][e], 1);
        pi[d][e] += __shfl_xor_sync(0xffffffffu, pi[d][e], 1);
      }
    if (o == 0) {
      const int base = 6 * k + (m == 0 ? 0 : (m == 1 ? 3 : 5));
      #pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (m + d <= 2 && base + d < kTayOut) {
          float4* dst = reinterpret_cast<float4*>(part + (cg * kPartRows + base + d) * 8);
          dst[0] = make_float4(pr[d][0], pi[d][0], pr[d][1], pi[d][1]);
          dst[1] = make_float4(pr[d][2], pi[d][2], pr[d][3], pi[d][3]);
        }
      }
    }
  };
  auto avg_contract = [&](const float (&H)[16]) {
    if (TAY) avg_contract_tay(H);
    else avg_contract_plain(H);
  };
  // compensated accumulation of the four column groups' sums (fixed order):
  // compute thread tid owns value i = tid & 7 of row k = tid >> 3 (Taylor: and
  // of row k + 64)
  float ks[2] = {0.f, 0.f}, kc[2] = {0.f, 0.f};
  auto avg_accumulate = [&]() {
    #pragma unroll
    for (int u = 0; u < (TAY ? 2 : 1); ++u) {
      const int k = (tid >> 3) + 64 * u, i = tid & 7;
      if (TAY && k >= kTayOut) continue;
      float x = part[k * 8 + i];
      #pragma unroll
      for (int c = 1; c < 4; ++c) x += part[(c * kPartRows + k) * 8 + i];
      const float y = x - kc[u];
      const float tt = ks[u] + y;
      kc[u] = (tt - ks[u]) - y;
      ks[u] = tt;
    }
  };
  // a baseline's averages out, the sums reset for the next (not Taylor: one
  // baseline per CTA there)
  auto flush_avg = [&](int64_t blf) {
    const int k = tid >> 3, i = tid & 7;     // value i = (re, im) of pol i / 2
    if (k < a.n_acc)
      reinterpret_cast<float*>(a.avg)[((size_t)k * a.n_bl + blf) * 8 + i] =
          (float)(((double)ks[0] - (double)kc[0]) * a.inv_n);
    ks[0] = 0.f;
    kc[0] = 0.f;
  };

  // the 16 compute warps' own barrier (the MMA-issuing warp is not in it)
  auto csync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(kTc5Compute) : "memory"); };
  // a bounded mbarrier wait that also gives up once another thread has raised s_bad
  auto wait_or_bad = [&](uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kTc5MaxPolls / 64; ++it) {
      if (mbar_wait(bar, parity, 64, 20000)) return true;
      if (*reinterpret_cast<volatile int*>(&s_bad)) return false;
    }
    return false;
  };

  if (!compute) {
    // ---- the MMA-issuing warps: lane 0 of warp 16 + g issues accumulator g's
    // MMAs (a thread's MMAs are accepted one at a time, so one thread issuing
    // them all leaves the tensor core half idle).  Each accumulator takes the
    // cross terms (lo*hi, hi*lo) of its 4 k-steps first, then their hi*hi
    // products
    const int g = warp - kTc5Compute / 32;
    if (lane == 0) {
      uint32_t p_sub = 0, p_avg = 0;
      const uint32_t id_s = idesc_tf32(128, NQ), id_a = idesc_tf32(128, 64);
      for (int t = 0; t < n_steps; ++t) {
        if (SUB) {
          if (!wait_or_bad(&mbar[4], p_sub)) break;
          p_sub ^= 1;
          fence_after_sync();
          #pragma unroll
          for (int j = 0; j < 12; ++j) {
            const int s = 4 * g + (j & 3);
            const uint32_t acol = tmem + (j < 4 ? kTc5ColALo : kTc5ColAHi) + 8 * s;   // lo(A) for j < 4, else hi(A)
            const uint64_t bd = (j >= 4 && j < 8 ? dbs_lo : dbs_hi) + 16 * s;
            mma_ts(tmem + kTc5ColAcc + g * NQ, acol, bd, id_s, j != 0);
          }
          commit(&mbar[0]);
        }
        if (ACC && g < nmain_a) {
          if (!wait_or_bad(&mbar[5], p_avg)) break;
          p_avg ^= 1;
          fence_after_sync();
          #pragma unroll
          for (int j = 0; j < 12; ++j) {
            const int s = 4 * g + (j & 3);
            const uint32_t acol = tmem + kTc5ColALo + (j < 4 ? 2 * NQ : 0) + 8 * s;
            const uint64_t bd = (j >= 4 && j < 8 ? dba_lo : dba_hi) + 16 * s;
            mma_ts(tmem + kTc5ColAcc + 64 * g, acol, bd, id_a, j != 0);
          }
          commit(&mbar[1]);
        }
      }
    }
  } else {
    // ---- the compute warps
    float H[16];                             // the average's H of the last step, this thread's columns
    uint32_t par_sub = 0, par_avg = 0;
    // thread 0: strip loads issued into / landed in buffers 0 and 1 (uses of each mbarrier)
    int issued0 = 0, issued1 = 0, landed0 = 0, landed1 = 0;
    auto ph_slot = [&](int t) { return ph + 2 * kTc5Src * (t & 1); };   // [sub 64][avg 64]
    auto wait_ph = [&](int t) { return wait_or_bad(&mbar[6 + (t & 1)], (uint32_t)(t >> 1) & 1u); };

    if (tid == 0) {
      issue_ph(0);
      issue_load(0);
      issued0 = 1;
    }
    uint32_t as_lo[32];                      // the next step's A_s lo, between C3 and C4
    if (SUB) {                               // the first step's subtraction operands
      if (!wait_ph(0)) s_bad = 1;
      bs_fill(ph_slot(0));
      t2_fill(t2s, ph_slot(0));
      csync();
      as_store_hi(as_lo);
      as_store_lo(as_lo);
      tmem_wait_st();
      fence_smem_async();
      fence_before_sync();
      csync();
      if (tid == 0 && !s_bad) mbar_arrive(&mbar[4]);
    }

    int tt_run = 0;                          // the time step of step t
    int64_t bl_run = bl0;                    // and its baseline (Taylor: step t is time t of bl0)
    for (int t = 0; t < n_steps && !s_bad;
         ++t, tt_run = (TAY || tt_run + 1 == a.n_time) ? 0 : tt_run + 1, bl_run += (!TAY && tt_run == 0)) {
      const int tt = TAY ? t : tt_run;
      const int64_t bl = TAY ? bl0 : bl_run;
      const int buf = t & 1;
      const bool bl_last = !TAY && tt == a.n_time - 1 && t + 1 < n_steps;   // another baseline follows
      float* strip = strip0 + (size_t)buf * n16 * 8;
      // ---- C1 (beside the subtraction MMAs): the next step's strip and
      // phases, the previous step's T2 contraction, T1 and T2 of the averaged
      // sources
      if (tid == 0 && t + 1 < n_steps) {
        if (SUB && t >= 1) bulk_wait_read();   // the residual store of step t - 1 has left buffer (t + 1) & 1
        issue_ph(t + 1);
        issue_load(t + 1);
        if ((t + 1) & 1) ++issued1;
        else ++issued0;
      }
      // the next baseline's model matrices into mtab (free since the previous
      // step formed this step's A_s) by asynchronous copies, before this step
      // forms the next step's A_s in C3
      if (SUB && bl_last && tid < kTc5Src * 4 && (tid >> 2) < n_sub_slots) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(mtab + tid);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa),
                     "l"(a.M_sub + ((size_t)(tid >> 2) * a.n_bl + bl + 1) * 4 + (tid & 3)) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      float2 t1v[12];
      if (ACC) {
        if (t > 0) avg_contract(H);          // the previous step's H with its T2 (still in t2a)
        if (!wait_ph(t)) s_bad = 1;
        csync();                             // parts written; t2a free
        if (t > 0) avg_accumulate();
        if (!TAY && tt == 0 && t > 0) flush_avg(bl - 1);   // the previous baseline is complete
        aa_compute(t1v, ph_slot(t) + kTc5Src);
        t2_fill(t2a, ph_slot(t) + kTc5Src);
      }
      // this step's strip has landed; the subtraction MMAs are complete
      {
        bool ok = wait_or_bad(&mbar[2 + buf], (uint32_t)(t >> 1) & 1u);
        if (ok && tid == 0) {
          if (buf) landed1 = (t >> 1) + 1;
          else landed0 = (t >> 1) + 1;
        }
        if (ok && SUB) ok = wait_or_bad(&mbar[0], par_sub);
        if (!ok) s_bad = 1;
      }
      if (SUB) par_sub ^= 1;
      fence_after_sync();
      csync();
      if (s_bad) break;
      // ---- C2: residual into the strip and B_a; A_a into TMEM (A_s is done with)
      if (SUB) sub_epilogue(strip);
      else if (ACC) ba_from_strip(strip);
      if (ACC) {
        aa_store(t1v);
        tmem_wait_st();
      }
      fence_smem_async();
      fence_before_sync();
      csync();
      if (ACC && tid == 0) mbar_arrive(&mbar[5]);
      if (SUB && tid == 0) {
        bulk_store(a.dst + ((size_t)tt * a.n_bl + bl) * a.n_chan * 2, strip, strip_bytes);
        bulk_commit();
      }
      // ---- C3 (beside the average MMAs): the next step's subtraction tables
      // and A_s hi (its TMEM columns are free of the average)
      const bool next_sub = SUB && t + 1 < n_steps;
      if (next_sub) {
        if (!wait_ph(t + 1)) s_bad = 1;
        bs_fill(ph_slot(t + 1));
        t2_fill(t2s, ph_slot(t + 1));
        if (bl_last) asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's model copy
        csync();
        as_store_hi(as_lo);
      }
      // ---- C4: the average's accumulators into registers (H = the sum of its
      // accumulators); the next step's A_s lo into the columns A_a has left
      if (ACC) {
        if (!wait_or_bad(&mbar[1], par_avg)) s_bad = 1;
        par_avg ^= 1;
        fence_after_sync();
        const uint32_t base = tmem + lane_base + kTc5ColAcc + 16 * cg;
        tmem_ld16(base, H);
        #pragma unroll
        for (int g = 1; g < 3; ++g) {
          if (g < nmain_a) {
            float h[16];
            tmem_ld16(base + 64 * g, h);
            tmem_wait_ld();
            #pragma unroll
            for (int i = 0; i < 16; ++i) H[i] += h[i];
          }
        }
        tmem_wait_ld();
      }
      if (next_sub) as_store_lo(as_lo);
      tmem_wait_st();
      fence_smem_async();
      fence_before_sync();
      csync();                               // accumulators read by every warp; the next A_s and B_s ready
      fence_after_sync();
      if (next_sub && !s_bad && tid == 0) mbar_arrive(&mbar[4]);
      if (s_bad) break;
    }

    if (ACC && !s_bad) {                     // the last step's contraction
      avg_contract(H);
      csync();
      avg_accumulate();
    }
    if (ACC && !s_bad && !TAY) flush_avg(bl0 + nbl - 1);
    if (ACC && !s_bad && TAY) {
      // the moments M_kn = sum_{m <= n} C(n, m) Q_{k,m,n-m} from the compensated sums
      // (the coefficient table is no longer read: its words hold them)
      float* qs = reinterpret_cast<float*>(cf);  // [128][8][2]: sum, compensation
      #pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = (tid >> 3) + 64 * u, i = tid & 7;
        if (k < kTayOut) {
          qs[(k * 8 + i) * 2] = ks[u];
          qs[(k * 8 + i) * 2 + 1] = kc[u];
        }
      }
      csync();
      const int s = tid >> 3, i = tid & 7, k = s / 3, n = s - 3 * k;
      if (k < a.n_acc) {
        auto val = [&](int j) {
          const int w = ((6 * k + j) * 8 + i) * 2;
          return (double)qs[w] - (double)qs[w + 1];
        };
        const double V = n == 0 ? val(0) : (n == 1 ? val(1) + val(3) : val(2) + 2.0 * val(4) + val(5));
        reinterpret_cast<float*>(a.avg)[((size_t)s * a.n_bl + bl0) * 8 + i] = (float)(V * a.inv_n);
      }
    }
    if (tid == 0) {
      // a load still in flight after a failed wait must land before the CTA's
      // shared memory goes away (bounded); stores are waited for unconditionally
      for (int u = landed0; u < issued0; ++u)
        if (!mbar_wait(&mbar[2], (uint32_t)u & 1u, kTc5MaxPolls)) break;
      for (int u = landed1; u < issued1; ++u)
        if (!mbar_wait(&mbar[3], (uint32_t)u & 1u, kTc5MaxPolls)) break;
      bulk_wait_all();
      if (s_bad) atomicExch(err, 1);
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, kTc5Cols);
}

}  // namespace rts
