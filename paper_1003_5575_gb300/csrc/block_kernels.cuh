// Blocked peel: the same per-source results as the one-source-per-pass loop,
// with one HBM pass per block of BK sources.
//
// The average of source k over the residual left by all earlier sources is
//   A_k = mean_{t,c} (V - sum_{j<k} M_j e^{-2 pi i phi_j}) e^{+2 pi i phi_k}
//       = mean_{t,c} R_s e^{+2 pi i phi_k} - sum_{s<=j<k} M_j D_jk,
// where R_s is the residual after the sources before k's block (start s) and
//   D_jk = mean_{t,c} e^{2 pi i (phi_k - phi_j)}
//        = mean_t e^{2 pi i (P_k - P_j)} sin(pi N dB) / (N sin(pi dB)),  dB = B_k - B_j,
// with P = A + (N-1) B / 2 the phase at the band centre (the geometric series
// over N uniform channels; M_j is constant over the cadence).  So one pass over
// the cube subtracts the BK sources of block b and averages the BK
// directions of block b+1; inside a block the averages are corrected with
// D_jk, which needs no pass over the cube.
#pragma once
#include "stream_kernels.cuh"

namespace rts {

constexpr int kBlkMax = 64;               // largest block (sources per pass)
constexpr int kBlkThreads = 256;          // threads of a pass CTA = block size x channel ranges
constexpr int kBlkPairsMax = kBlkMax * (kBlkMax - 1) / 2;

struct __align__(16) PhaseAB { unsigned long long a, b; };   // Q0.64 A (channel 0) and B (step)

// Per (baseline, time, source) trigonometry for the closed-form D_jk, with B
// taken as its signed value (|B| < 1/2):
//   u = exp(2 pi i P), P = A + (N-1) B / 2 (band-centre phase)
//   (sn, cn) = (sin, cos)(pi N B)
struct __align__(16) GeoTrig { float2 u; float sn, cn; };

struct BlockPassArgs {
  const float4* src;        // cube read (input or residual)
  float4* dst;              // residual written (may equal src); unused when n_sub == 0
  const double* uvw;
  const int2* bl_ant;
  int n_ant, n_chan, n_time;
  int64_t n_bl;
  double nu0_c, dnu_c;
  int n_sub;                // sources subtracted in this pass (block b), 0..BK
  const float2* M_sub;      // [BK][n_bl][4] their model matrices S J_i J_j^H
  const PhaseAB* ph_sub;    // [n_bl][n_time][BK] their phases (written by the previous pass)
  int n_acc;                // sources averaged in this pass (block b+1), 0..BK
  const PhaseAB* ph_acc;    // [n_bl][n_time][BK] their phases (precomputed)
  float2* avg;              // [BK][n_bl][4] plain averages of R_s in their directions
  double inv_n;
  float tx0, tdx;           // gains Taylor-expanded in frequency: x_c = tx0 + c tdx (tcgen05 pass only)
};

// a Q0.64 phase read as a signed fraction of a turn, x 2^-64, in FP32: the high
// word exactly (scaled by 2^-32) plus the low word (scaled by 2^-64)
__device__ __forceinline__ float q64_signed_to_float(unsigned long long x) {
  const int hi = (int)(x >> 32);
  const unsigned lo = (unsigned)x;
  return fmaf((float)hi, 2.3283064365386963e-10f, (float)lo * 5.42101086242752217e-20f);
}

// exp(+2 pi i phi) from a Q0.64 phase, using its high word (truncation error
// below 2^-32 turns)
__device__ inline float2 phasor_hw(unsigned long long ph) {
  constexpr float kRadPerUnit = kTwoM32F * kTwoPiF;      // 2 pi / 2^32
  float s, c;
  __sincosf((float)(int)(ph >> 32) * kRadPerUnit, &s, &c);
  return make_float2(c, s);
}

// exp(2 pi i x) for a Q0.64 phase x: the top 24 bits through sincospif, the
// remaining bits (0 <= r < 2^-24 turns) by the first-order rotation 1 + 2 pi i r
// (second-order term below 1e-13).  32-bit integer conversions only (64-bit
// integer-to-float conversions are slow on this GPU).
__device__ inline float2 phasor_q64_fine(unsigned long long x) {
  const int xh = (int)(x >> 32);
  const float hi = (float)(xh >> 8) * 5.9604644775390625e-08f;                           // 2^-24
  const float lo = fmaf((float)(xh & 0xff), 2.3283064365386963e-10f,                     // 2^-32
                        (float)(unsigned)x * 5.42101086242752217e-20f);                 // 2^-64
  float sn, cs;
  sincospif(2.0f * hi, &sn, &cs);
  const float w = 6.28318530717958647692f * lo;
  return make_float2(cs - sn * w, sn + cs * w);
}

constexpr int kSubCh = 3;     // channels a thread keeps in registers while subtracting
template <int BK, bool SUB, bool ACC>
__global__ void __launch_bounds__(kBlkThreads, 3) k_block_pass(BlockPassArgs a) {
  constexpr int kHalf = BK / 2;                   // averaging: two sources per thread
  constexpr int kSplits = kBlkThreads / kHalf;    // channel ranges per source pair
  extern __shared__ __align__(16) unsigned char b_smem[];
  float4* sR = reinterpret_cast<float4*>(b_smem);                       // [n_chan][2]
  PhaseAB* sPs = reinterpret_cast<PhaseAB*>(sR + (size_t)a.n_chan * 2);  // [BK] at the current time
  PhaseAB* sPa = sPs + BK;                                               // [BK] at the current time
  __shared__ float2 sM[BK][4];       // model matrix entries (re, im)
  __shared__ float2 sMs[BK][4];      // the same with re and im swapped
  // FP64 running sums of the averages, one slot per (channel range, source):
  // [kSplits][BK][8] doubles (32 KB) after the strip and the phase tables
  double (*sRed)[BK][8] = reinterpret_cast<double (*)[BK][8]>(sPa + BK);

  const int64_t bl = blockIdx.x;
  const int tid = threadIdx.x;
  if (SUB) {
    for (int q = tid; q < a.n_sub * 4; q += kBlkThreads) {
      const int k = q >> 2, e = q & 3;
      const float2 m = a.M_sub[((size_t)k * a.n_bl + bl) * 4 + e];
      sM[k][e] = m;
      sMs[k][e] = make_float2(m.y, m.x);
    }
  }
  // averaging role: sources k0 = tid % kHalf and k0 + kHalf over channels [c_beg, c_end)
  const int k0 = tid % kHalf, split = tid / kHalf;
  const bool has0 = k0 < a.n_acc, has1 = k0 + kHalf < a.n_acc;
  const int chunk = (a.n_chan + kSplits - 1) / kSplits;
  const int c_beg = min(a.n_chan, split * chunk), c_end = min(a.n_chan, c_beg + chunk);
  if (ACC) {
    #pragma unroll
    for (int e = 0; e < 8; ++e) { sRed[split][k0][e] = 0.0; sRed[split][k0 + kHalf][e] = 0.0; }
  }

  for (int t = 0; t < a.n_time; ++t) {
    __syncthreads();                                   // previous strip consumed; tables ready
    const size_t base = ((size_t)t * a.n_bl + bl) * a.n_chan * 2;
    for (int q = tid; q < a.n_chan * 2; q += kBlkThreads) sR[q] = __ldcs(a.src + base + q);
    if (SUB && tid < a.n_sub) sPs[tid] = a.ph_sub[((size_t)bl * a.n_time + t) * BK + tid];
    if (ACC && tid >= BK && tid - BK < a.n_acc) sPa[tid - BK] = a.ph_acc[((size_t)bl * a.n_time + t) * BK + tid - BK];
    __syncthreads();
    if (SUB) {
      // channels c0, c0 + 256, c0 + 512 in registers; sources in the inner loop.
      // x_e -= M_e conj(ph) as two packed FMAs per entry:
      //   x_e += M_e * (-pr, -pr);  x_e += swap(M_e) * (-pi, +pi)
      for (int c0 = tid; c0 < a.n_chan; c0 += kBlkThreads * kSubCh) {
        float2 x[kSubCh][4];
        #pragma unroll
        for (int u = 0; u < kSubCh; ++u) {
          const int c = c0 + u * kBlkThreads;
          if (c < a.n_chan) {
            const float4 v0 = sR[2 * c], v1 = sR[2 * c + 1];
            x[u][0] = make_float2(v0.x, v0.y); x[u][1] = make_float2(v0.z, v0.w);
            x[u][2] = make_float2(v1.x, v1.y); x[u][3] = make_float2(v1.z, v1.w);
          }
        }
        for (int j = 0; j < a.n_sub; ++j) {
          const PhaseAB p = sPs[j];
          float2 M[4], Ms[4];
          #pragma unroll
          for (int e = 0; e < 4; ++e) { M[e] = sM[j][e]; Ms[e] = sMs[j][e]; }
          unsigned long long phase = p.a + (unsigned long long)c0 * p.b;
          const unsigned long long dstep = p.b * (unsigned long long)kBlkThreads;
          #pragma unroll
          for (int u = 0; u < kSubCh; ++u, phase += dstep) {
            if (c0 + u * kBlkThreads < a.n_chan) {
              const float2 ph = phasor_hw(phase);
              const float2 nr = make_float2(-ph.x, -ph.x), si = make_float2(-ph.y, ph.y);
              #pragma unroll
              for (int e = 0; e < 4; ++e) x[u][e] = ffma2(Ms[e], si, ffma2(M[e], nr, x[u][e]));
            }
          }
        }
        #pragma unroll
        for (int u = 0; u < kSubCh; ++u) {
          const int c = c0 + u * kBlkThreads;
          if (c < a.n_chan) {
            const float4 v0 = make_float4(x[u][0].x, x[u][0].y, x[u][1].x, x[u][1].y);
            const float4 v1 = make_float4(x[u][2].x, x[u][2].y, x[u][3].x, x[u][3].y);
            sR[2 * c] = v0; sR[2 * c + 1] = v1;
            __stcs(a.dst + base + 2 * c, v0);
            __stcs(a.dst + base + 2 * c + 1, v1);
          }
        }
      }
      __syncthreads();
    }
    if (ACC && has0 && c_beg < c_end) {
      // exact fixed-point phase per channel (a recurrence ph *= exp(2 pi i B) would
      // carry the step's rounding coherently across channels).  Packed sums
      // P_e = sum x_e pr and Q_e = sum x_e pi give  acc_e = (P.x - Q.y, P.y + Q.x).
      const PhaseAB p0 = sPa[k0];
      const PhaseAB p1 = has1 ? sPa[k0 + kHalf] : p0;
      float2 P0[4], Q0[4], P1[4], Q1[4];
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        P0[e] = make_float2(0.f, 0.f); Q0[e] = P0[e]; P1[e] = P0[e]; Q1[e] = P0[e];
      }
      unsigned long long ph0 = p0.a + (unsigned long long)c_beg * p0.b;
      unsigned long long ph1 = p1.a + (unsigned long long)c_beg * p1.b;
      for (int c = c_beg; c < c_end; ++c, ph0 += p0.b, ph1 += p1.b) {
        const float4 v0 = sR[2 * c], v1 = sR[2 * c + 1];
        const float2 xs[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                              make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
        const float2 e0 = phasor_hw(ph0), e1 = phasor_hw(ph1);
        const float2 r0 = make_float2(e0.x, e0.x), i0 = make_float2(e0.y, e0.y);
        const float2 r1 = make_float2(e1.x, e1.x), i1 = make_float2(e1.y, e1.y);
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          P0[e] = ffma2(xs[e], r0, P0[e]); Q0[e] = ffma2(xs[e], i0, Q0[e]);
          P1[e] = ffma2(xs[e], r1, P1[e]); Q1[e] = ffma2(xs[e], i1, Q1[e]);
        }
      }
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        sRed[split][k0][2 * e] += (double)(P0[e].x - Q0[e].y);
        sRed[split][k0][2 * e + 1] += (double)(P0[e].y + Q0[e].x);
        if (has1) {
          sRed[split][k0 + kHalf][2 * e] += (double)(P1[e].x - Q1[e].y);
          sRed[split][k0 + kHalf][2 * e + 1] += (double)(P1[e].y + Q1[e].x);
        }
      }
    }
  }
  if (ACC) {
    __syncthreads();
    for (int q = tid; q < a.n_acc * 4; q += kBlkThreads) {
      const int k = q >> 2, e = q & 3;
      double re = 0.0, im = 0.0;
      #pragma unroll
      for (int s = 0; s < kSplits; ++s) { re += sRed[s][k][2 * e]; im += sRed[s][k][2 * e + 1]; }
      a.avg[((size_t)k * a.n_bl + bl) * 4 + e] = make_float2((float)(re * a.inv_n), (float)(im * a.inv_n));
    }
  }
}

// ---------------------------------------------------------------------------
// D_jk for every pair j < k of one block, per baseline:  Dtab[dir_index(n_bl, bl, j, k)]

// Phase of the band-centre term of the pair: dA + (N-1) dB / 2 modulo one turn,
// exactly, with dB taken as the signed representative in [-1/2, 1/2).  The
// closed form e^{i pi (N-1) x} sin(pi N x) / (N sin(pi x)) is periodic in x with
// period one, so any representative works as long as the ratio below uses the
// same one.
__device__ inline unsigned long long pair_mid_phase(unsigned long long dA, long long dB, int n_chan) {
  const long long f = n_chan - 1;
  const unsigned long long lo = (unsigned long long)f * (unsigned long long)dB;   // wraps mod 2^64
  const unsigned long long hi = (unsigned long long)__mul64hi(f, dB);             // signed high word
  return dA + ((hi << 63) | (lo >> 1));                                           // 128-bit value / 2
}

// ---------------------------------------------------------------------------
// geometry of one block (no visibility data): Q0.64 phases of its sources,
//   ph[bl][t][k] = (frac(tau nu_0 / c), frac(tau dnu / c)).
// The array's baselines are antenna pairs with (u, v, w)_ij = uvw_i - uvw_j, so
// tau_ij = tau_i - tau_j with the antenna delay tau_i = u_i l + v_i m + w_i (n - 1),
// and the Q0.64 phases of a baseline are the differences of its antennas'
// phases modulo one turn (2^64: exact integer arithmetic).  The FP64 work is
// per (time, antenna, source) instead of per (time, baseline, source); the
// result differs from the per-baseline FP64 evaluation by the rounding of the
// antenna products (~1e-16 of tau nu / c, below 1e-12 turns).

// aph[t][i][k] = (frac(tau_i nu_0 / c), frac(tau_i dnu / c)) for the block's sources
template <int BK>
__global__ void __launch_bounds__(256) k_block_ant_phases(const double* __restrict__ src, int n_blk,
                                                         const double* __restrict__ uvw, int n_ant, int n_time,
                                                         double nu0_c, double dnu_c, PhaseAB* __restrict__ aph) {
  const int64_t n = (int64_t)n_time * n_ant * BK;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % BK);
    const int64_t ti = q / BK;                  // t * n_ant + i
    PhaseAB p;
    p.a = 0; p.b = 0;
    if (k < n_blk) {
      const double l = src[3 * k], m = src[3 * k + 1];
      const double r2 = l * l + m * m;
      const double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
      const double* x = uvw + ti * 3;
      const double tau = x[0] * l + x[1] * m + x[2] * nm1;
      p.a = frac_q64(tau * nu0_c);
      p.b = frac_q64(tau * dnu_c);
    }
    aph[q] = p;
  }
}

// ph: the phases of this handle's first channel; trig: the band-centre phasor
// and sin/cos(pi N B) of the whole band of n_band channels, whose channel c0 is
// this handle's first (A_band = A - c0 B, exactly)
template <int BK>
__global__ void __launch_bounds__(256) k_block_phases(const PhaseAB* __restrict__ aph, int n_blk,
                                                     const int2* __restrict__ bl_ant, int n_ant,
                                                     int n_time, int n_chan, int c0, int64_t n_bl,
                                                     PhaseAB* __restrict__ ph, GeoTrig* __restrict__ trig) {
  const int64_t n = n_bl * n_time * BK;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % BK);
    if (k >= n_blk) continue;
    const int64_t r = q / BK;
    const int t = (int)(r % n_time);
    const int64_t bl = r / n_time;
    const int2 ij = bl_ant[bl];
    const PhaseAB pi = aph[((int64_t)t * n_ant + ij.x) * BK + k], pj = aph[((int64_t)t * n_ant + ij.y) * BK + k];
    PhaseAB p;
    p.a = pi.a - pj.a;                          // modulo 2^64
    p.b = pi.b - pj.b;
    ph[q] = p;
    GeoTrig g;
    const long long bs = (long long)p.b;                           // signed B
    g.u = phasor_q64_fine(pair_mid_phase(p.a - (unsigned long long)c0 * p.b, bs, n_chan));
    // pi N B: N B = hi + lo 2^-64 = (hi + [lo_s < 0]) + lo_s 2^-64 with lo_s in [-1/2, 1/2)
    const long long nn = n_chan;
    const unsigned long long lo = (unsigned long long)nn * (unsigned long long)bs;
    const long long hi = __mul64hi(nn, bs);
    const long long los = (long long)lo;
    float sn, cn;
    sincospif(q64_signed_to_float((unsigned long long)los), &sn, &cn);
    if ((hi + (los < 0 ? 1 : 0)) & 1) { sn = -sn; cn = -cn; }
    g.sn = sn; g.cn = cn;
    trig[q] = g;
  }
}

// Layout of a block's closed-form averages D_jk (j < k): by target source k,
// then baseline, then j, so the terms of source k's correction for a run of
// consecutive baselines are one contiguous stretch of memory
__host__ __device__ inline int64_t dir_index(int64_t n_bl, int64_t bl, int j, int k) {
  return n_bl * (k * (k - 1) / 2) + bl * k + j;
}

// sin(z) / z by its Taylor series to z^12 (first omitted term z^14/15!, below
// 5e-10 for |z| <= pi/2)
__device__ inline float sinc_series(float z) {
  const float z2 = z * z;
  return 1.0f + z2 * (-1.0f / 6 + z2 * (1.0f / 120 + z2 * (-1.0f / 5040 + z2 * (1.0f / 362880
         + z2 * (-1.0f / 39916800 + z2 * (1.0f / 6227020800.0f))))));
}

// sin(N th) / (N sin th) for |N th| <= pi/2
__device__ inline float ratio_series(float z, float th) { return sinc_series(z) / sinc_series(th); }

template <int BK>
__global__ void __launch_bounds__(256) k_block_dirichlet(const PhaseAB* __restrict__ ph,
                                                        const GeoTrig* __restrict__ trig, int n_blk,
                                                        float2* __restrict__ Dtab, int64_t n_bl,
                                                        int n_time, int n_chan) {
  constexpr int kPairs = BK * (BK - 1) / 2;
  constexpr int kU = (kPairs + 255) / 256;
  __shared__ GeoTrig sG[16][BK];               // times handled in chunks of 16
  __shared__ unsigned long long sB[16][BK];
  __shared__ float sBf[16][BK];                // signed B in turns (FP32)
  const int64_t bl = blockIdx.x;
  const int n_pairs = n_blk * (n_blk - 1) / 2;
  const float fN = (float)n_chan;
  int pj[kU], pk[kU];
  float dre[kU], dim[kU];
  #pragma unroll
  for (int u = 0; u < kU; ++u) {
    dre[u] = 0.f; dim[u] = 0.f;
    const int pr = threadIdx.x + 256 * u;              // pr = k(k-1)/2 + j, j < k
    int k = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)pr)) * 0.5f);
    while (k > 1 && k * (k - 1) / 2 > pr) --k;
    while ((k + 1) * k / 2 <= pr) ++k;
    pk[u] = k; pj[u] = pr - k * (k - 1) / 2;
  }
  for (int t0 = 0; t0 < n_time; t0 += 16) {
    const int nt = min(16, n_time - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < nt * n_blk; q += blockDim.x) {
      const int t = q / n_blk, k = q - t * n_blk;
      const size_t at = ((size_t)bl * n_time + t0 + t) * BK + k;
      sG[t][k] = trig[at];
      const unsigned long long b = ph[at].b;
      sB[t][k] = b;
      sBf[t][k] = q64_signed_to_float(b);
    }
    __syncthreads();
    #pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (threadIdx.x + 256 * u < n_pairs) {
        const int j = pj[u], k = pk[u];
        for (int t = 0; t < nt; ++t) {
          const GeoTrig gk = sG[t][k], gj = sG[t][j];
          // band-centre phase difference: u_k conj(u_j)
          const float er = gk.u.x * gj.u.x + gk.u.y * gj.u.y;
          const float ei = gk.u.y * gj.u.x - gk.u.x * gj.u.y;
          // ratio sin(pi N x) / (N sin(pi x)) at x = B_k - B_j (signed values)
          // the exact 64-bit difference, converted through 32-bit halves (64-bit
          // integer-to-float conversions are slow on this GPU)
          const float xw = q64_signed_to_float(sB[t][k] - sB[t][j]);
          const float xs = sBf[t][k] - sBf[t][j];
          // near pairs (|N x| < 1/2): series in the exact x; others: the numerator
          // by angle difference, the denominator N sin(pi x) from the exact x (an
          // angle difference there would cancel).  When the signed difference
          // wraps (|x| >= 1/2), sin(pi x) = -sin(pi x_wrapped).
          // branch-free (lanes of a warp mix near and far pairs): r = s(z) / sinc(th)
          // with z = N th, s(z) = sin(z) / z from the series (near) or from the
          // exact numerator (far, sign flipped when the difference wraps)
          const bool wrap = fabsf(xs) >= 0.5f;
          const float th = 3.14159265358979f * xw, z = fN * th;
          const bool near = !wrap && fabsf(fN * xw) < 0.5f;
          const float num = gk.sn * gj.cn - gk.cn * gj.sn;
          const float s_far = __fdividef(wrap ? -num : num, near ? 1.0f : z);
          const float s_z = near ? sinc_series(z) : s_far;
          const float r = __fdividef(s_z, sinc_series(th));
          dre[u] += r * er;
          dim[u] += r * ei;
        }
      }
    }
  }
  const float inv_t = 1.0f / (float)n_time;
  #pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int pr = threadIdx.x + 256 * u;
    if (pr < n_pairs) Dtab[dir_index(n_bl, bl, pj[u], pk[u])] = make_float2(dre[u] * inv_t, dim[u] * inv_t);
  }
}

// ---------------------------------------------------------------------------
// per source: model matrices of the previous source, then the corrected average
//   avg_k = A_k - sum_{j<k in block} M_j D_jk        (one thread per baseline)

__global__ void __launch_bounds__(256) k_block_model(const double2* __restrict__ J, double S,
                                                    const int2* __restrict__ bl_ant, int64_t n_bl,
                                                    float2* __restrict__ M_out) {
  const int64_t bl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (bl >= n_bl) return;
  const int2 ij = bl_ant[bl];
  float2 M[4];
  model_matrix_f(J, 0, ij.x, ij.y, S, M);
  #pragma unroll
  for (int e = 0; e < 4; ++e) M_out[bl * 4 + e] = M[e];
}

__global__ void __launch_bounds__(256) k_block_correct(const float2* __restrict__ Ablk, int q,
                                                      const float2* __restrict__ Mblk,
                                                      const float2* __restrict__ Dtab,
                                                      int64_t n_bl, float2* __restrict__ avg_out) {
  const int64_t bl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (bl >= n_bl) return;
  float2 v[4];
  #pragma unroll
  for (int e = 0; e < 4; ++e) v[e] = Ablk[((size_t)q * n_bl + bl) * 4 + e];
  const float2* D = Dtab + dir_index(n_bl, bl, 0, q);
  for (int j = 0; j < q; ++j) {
    const float2 d = D[j];
    #pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = csub(v[e], cmul(Mblk[((size_t)j * n_bl + bl) * 4 + e], d));
  }
  #pragma unroll
  for (int e = 0; e < 4; ++e) avg_out[bl * 4 + e] = v[e];
}

}  // namespace rts
