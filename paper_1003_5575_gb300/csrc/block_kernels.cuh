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
  const double* src_acc;    // device [n_acc][3] (l, m, S)
  PhaseAB* ph_acc;          // [n_bl][n_time][BK] their phases (written here)
  float2* avg;              // [BK][n_bl][4] plain averages of R_s in their directions
  double inv_n;
};

// exp(+2 pi i phi) from a Q0.64 phase, using its high word (truncation error
// below 2^-32 turns)
__device__ inline float2 phasor_hw(unsigned long long ph) {
  return phasor_f((float)(int)(ph >> 32) * kTwoM32F);
}

constexpr int kSubCh = 3;     // channels a thread keeps in registers while subtracting

template <int BK, bool SUB, bool ACC>
__global__ void __launch_bounds__(kBlkThreads, 2) k_block_pass(BlockPassArgs a) {
  constexpr int kHalf = BK / 2;                   // averaging: two sources per thread
  constexpr int kSplits = kBlkThreads / kHalf;    // channel ranges per source pair
  extern __shared__ __align__(16) unsigned char b_smem[];
  float4* sR = reinterpret_cast<float4*>(b_smem);                       // [n_chan][2]
  PhaseAB* sPs = reinterpret_cast<PhaseAB*>(sR + (size_t)a.n_chan * 2);  // [n_time][BK]
  PhaseAB* sPa = sPs + (size_t)a.n_time * BK;                            // [n_time][BK]
  __shared__ float4 sM[BK][2];
  __shared__ double sRed[kSplits][BK][8];

  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  const int tid = threadIdx.x;
  if (SUB) {
    const float4* Mg = reinterpret_cast<const float4*>(a.M_sub);
    for (int q = tid; q < a.n_sub * 2; q += kBlkThreads) {
      const int k = q >> 1, h = q & 1;
      sM[k][h] = Mg[((size_t)k * a.n_bl + bl) * 2 + h];
    }
    for (int q = tid; q < a.n_time * a.n_sub; q += kBlkThreads) {
      const int t = q / a.n_sub, k = q - t * a.n_sub;
      sPs[t * BK + k] = a.ph_sub[((size_t)bl * a.n_time + t) * BK + k];
    }
  }
  if (ACC) {
    for (int q = tid; q < a.n_time * a.n_acc; q += kBlkThreads) {
      const int t = q / a.n_acc, k = q - t * a.n_acc;
      SrcDir d;
      d.l = a.src_acc[3 * k]; d.m = a.src_acc[3 * k + 1]; d.S = a.src_acc[3 * k + 2];
      const double r2 = d.l * d.l + d.m * d.m;
      d.nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
      const double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, d);
      PhaseAB p;
      p.a = frac_q64(tau * a.nu0_c);
      p.b = frac_q64(tau * a.dnu_c);
      sPa[t * BK + k] = p;
      a.ph_acc[((size_t)bl * a.n_time + t) * BK + k] = p;
    }
  }
  // averaging role: sources k0 = tid % kHalf and k0 + kHalf over channels [c_beg, c_end)
  const int k0 = tid % kHalf, split = tid / kHalf;
  const bool has0 = k0 < a.n_acc, has1 = k0 + kHalf < a.n_acc;
  const int chunk = (a.n_chan + kSplits - 1) / kSplits;
  const int c_beg = min(a.n_chan, split * chunk), c_end = min(a.n_chan, c_beg + chunk);
  double accd[16];
  #pragma unroll
  for (int e = 0; e < 16; ++e) accd[e] = 0.0;

  for (int t = 0; t < a.n_time; ++t) {
    __syncthreads();                                   // previous strip consumed; tables ready
    const size_t base = ((size_t)t * a.n_bl + bl) * a.n_chan * 2;
    for (int q = tid; q < a.n_chan * 2; q += kBlkThreads) sR[q] = __ldcs(a.src + base + q);
    __syncthreads();
    if (SUB) {
      // channels c0, c0 + 256, c0 + 512 in registers; sources in the inner loop
      for (int c0 = tid; c0 < a.n_chan; c0 += kBlkThreads * kSubCh) {
        float4 x0[kSubCh], x1[kSubCh];
        #pragma unroll
        for (int u = 0; u < kSubCh; ++u) {
          const int c = c0 + u * kBlkThreads;
          if (c < a.n_chan) { x0[u] = sR[2 * c]; x1[u] = sR[2 * c + 1]; }
        }
        for (int j = 0; j < a.n_sub; ++j) {
          const PhaseAB p = sPs[t * BK + j];
          const float4 m01 = sM[j][0], m23 = sM[j][1];
          const float2 M[4] = {make_float2(m01.x, m01.y), make_float2(m01.z, m01.w),
                               make_float2(m23.x, m23.y), make_float2(m23.z, m23.w)};
          unsigned long long phase = p.a + (unsigned long long)c0 * p.b;
          const unsigned long long dstep = p.b * (unsigned long long)kBlkThreads;
          #pragma unroll
          for (int u = 0; u < kSubCh; ++u, phase += dstep)
            if (c0 + u * kBlkThreads < a.n_chan) sub_model(x0[u], x1[u], M, phasor_hw(phase));
        }
        #pragma unroll
        for (int u = 0; u < kSubCh; ++u) {
          const int c = c0 + u * kBlkThreads;
          if (c < a.n_chan) {
            sR[2 * c] = x0[u]; sR[2 * c + 1] = x1[u];
            __stcs(a.dst + base + 2 * c, x0[u]);
            __stcs(a.dst + base + 2 * c + 1, x1[u]);
          }
        }
      }
      __syncthreads();
    }
    if (ACC && has0 && c_beg < c_end) {
      // exact fixed-point phase per channel (a recurrence ph *= exp(2 pi i B) would
      // carry the step's rounding coherently across channels)
      const PhaseAB p0 = sPa[t * BK + k0];
      const PhaseAB p1 = has1 ? sPa[t * BK + k0 + kHalf] : p0;
      float acc0[8], acc1[8];
      #pragma unroll
      for (int e = 0; e < 8; ++e) { acc0[e] = 0.f; acc1[e] = 0.f; }
      unsigned long long ph0 = p0.a + (unsigned long long)c_beg * p0.b;
      unsigned long long ph1 = p1.a + (unsigned long long)c_beg * p1.b;
      for (int c = c_beg; c < c_end; ++c, ph0 += p0.b, ph1 += p1.b) {
        const float4 r0 = sR[2 * c], r1 = sR[2 * c + 1];
        acc_rot(acc0, r0, r1, phasor_hw(ph0));
        acc_rot(acc1, r0, r1, phasor_hw(ph1));
      }
      #pragma unroll
      for (int e = 0; e < 8; ++e) { accd[e] += (double)acc0[e]; accd[8 + e] += (double)acc1[e]; }
    }
  }
  if (ACC) {
    #pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (has0) sRed[split][k0][e] = accd[e];
      if (has1) sRed[split][k0 + kHalf][e] = accd[8 + e];
    }
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
// D_jk for every pair j < k of one block, per baseline:  Dtab[bl][k(k-1)/2 + j]

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

// sin(pi N x) / (N sin(pi x)) for x = dB (signed Q0.64 turns, |x| < 1/2); 1 at x = 0
__device__ inline float dirichlet_ratio(long long x, int n_chan) {
  if (x == 0) return 1.0f;
  const float xf = (float)x * 5.42101086242752217e-20f;            // 2^-64
  const float s1 = sinpif(xf);
  // N x = hi * 2^64 + lo (two's complement).  With g = lo as a signed Q0.64
  // value in [-1/2, 1/2): N x = (hi + [g < 0]) + g, so
  // sin(pi N x) = (-1)^(hi + [g < 0]) sin(pi g), and g stays accurate in FP32.
  const long long n = n_chan;
  const unsigned long long lo = (unsigned long long)n * (unsigned long long)x;   // wraps mod 2^64
  const long long hi = __mul64hi(n, x);
  const long long g = (long long)lo;
  const float gf = (float)g * 5.42101086242752217e-20f;
  float s2 = sinpif(gf);
  if ((hi + (g < 0 ? 1 : 0)) & 1) s2 = -s2;
  return s2 / ((float)n_chan * s1);
}

// exp(2 pi i x) for a Q0.64 phase x: the top 24 bits through sincospif, the
// remaining bits (|r| < 2^-25 turns) by the first-order rotation 1 + 2 pi i r
__device__ inline float2 phasor_q64_fine(unsigned long long x) {
  const long long sx = (long long)x;
  const float hi = __ll2float_rn(sx) * 5.42101086242752217e-20f;          // 2^-64
  const long long back = __float2ll_rn(hi * 1.8446744073709551616e19f);   // exact
  const float lo = (float)(sx - back) * 5.42101086242752217e-20f;
  float sn, cs;
  sincospif(2.0f * hi, &sn, &cs);
  const float w = 6.28318530717958647692f * lo;
  return make_float2(cs - sn * w, sn + cs * w);
}

template <int BK>
__global__ void __launch_bounds__(256) k_block_dirichlet(const PhaseAB* __restrict__ ph, int n_blk,
                                                        float2* __restrict__ Dtab, int64_t n_bl,
                                                        int n_time, int n_chan) {
  constexpr int kPairs = BK * (BK - 1) / 2;
  constexpr int kU = (kPairs + 255) / 256;
  __shared__ PhaseAB sP[16][BK];               // times handled in chunks of 16
  const int64_t bl = blockIdx.x;
  const int n_pairs = n_blk * (n_blk - 1) / 2;
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
      sP[t][k] = ph[((size_t)bl * n_time + t0 + t) * BK + k];
    }
    __syncthreads();
    #pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (threadIdx.x + 256 * u < n_pairs) {
        const int j = pj[u], k = pk[u];
        for (int t = 0; t < nt; ++t) {
          const long long dB = (long long)(sP[t][k].b - sP[t][j].b);
          const unsigned long long mid = pair_mid_phase(sP[t][k].a - sP[t][j].a, dB, n_chan);
          const float r = dirichlet_ratio(dB, n_chan);
          const float2 e = phasor_q64_fine(mid);
          dre[u] += r * e.x;
          dim[u] += r * e.y;
        }
      }
    }
  }
  const float inv_t = 1.0f / (float)n_time;
  #pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int pr = threadIdx.x + 256 * u;
    if (pr < n_pairs) Dtab[(size_t)bl * kPairs + pr] = make_float2(dre[u] * inv_t, dim[u] * inv_t);
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
                                                      const float2* __restrict__ Dtab, int n_pairs,
                                                      int64_t n_bl, float2* __restrict__ avg_out) {
  const int64_t bl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (bl >= n_bl) return;
  float2 v[4];
  #pragma unroll
  for (int e = 0; e < 4; ++e) v[e] = Ablk[((size_t)q * n_bl + bl) * 4 + e];
  const float2* D = Dtab + (size_t)bl * n_pairs + q * (q - 1) / 2;
  for (int j = 0; j < q; ++j) {
    const float2 d = D[j];
    #pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = csub(v[e], cmul(Mblk[((size_t)j * n_bl + bl) * 4 + e], d));
  }
  #pragma unroll
  for (int e = 0; e < 4; ++e) avg_out[bl * 4 + e] = v[e];
}

}  // namespace rts
