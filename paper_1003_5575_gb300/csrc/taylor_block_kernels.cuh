// Gains Taylor-expanded in frequency in the blocked schedule (Section 3.1; the
// constant-gain blocked schedule is in block_kernels.cuh).
//
// Source k's three moments over the residual left by every earlier source are
//   M_kn = mean_{t,c} x_c^n (R_s - sum_{j<k} sum_m x_c^m P_jm e^{-2 pi i phi_j}) e^{+2 pi i phi_k}
//        = mean_{t,c} x_c^n R_s e^{+2 pi i phi_k} - sum_{s<=j<k} sum_m P_jm D^(n+m)_jk,
//   D^(p)_jk = mean_{t,c} x_c^p e^{2 pi i (phi_k - phi_j)},  p = 0 .. 4,
// R_s the residual after the sources before k's block.  So one pass over the
// cube subtracts a block's Taylor models and takes the plain moments of the
// next block (k_block_pass_tc05<.., .., true>), and inside a block the moments
// are corrected with D^(p), which needs no pass over the cube.
//
// D^(p) in closed form.  With uniform channels, x_c = y / N (y = c - (N-1)/2),
// B = B_k - B_j and z = pi N B:
//   mean_c x_c^p e^{2 pi i (A + c B)} = e^{2 pi i (A + (N-1) B / 2)} G_p,
//   G_p = mean_y (y/N)^p e^{2 i (y/N) z} = (-i/2)^p f^(p)(z),  f(z) = sin z / (N sin(z/N)),
// the band-centre phasor being the one the constant-gain D_jk uses.  For
// |z| < 2 the power series of e^{2 i (y/N) z} about z = 0 gives
//   G_p = sum_m (2 i z)^m / m! mu_{p+m},  mu_j = mean_c x_c^j  (zero for odd j),
// whose terms fall below 1e-11 by m = 17; elsewhere the derivatives follow from
// f w = sin z, w = N sin(z / N), differentiated p times (Leibniz):
//   f^(p) = (sin^(p) z - sum_{j<p} C(p, j) f^(j) w^(p-j)) / w,  |w| >= about 2.
// The 64-bit phase difference is exact, so sin/cos(z) and sin/cos(z / N) are
// taken from exact turns.  When the signed difference of the two sources'
// signed steps leaves [-1/2, 1/2) the wrapped value B' = B -+ 1 is used and
// G_p(B) = (-1)^(N-1) G_p(B') (the half-integer y of an even N).
#pragma once
#include "block_kernels.cuh"
#include "block_tc05_kernels.cuh"
#include "taylor_kernels.cuh"

namespace rts {

constexpr int kTayPairs = kTayBlk * (kTayBlk - 1) / 2;   // pairs j < k of one Taylor block
constexpr int kTayMu = 22;                              // mu_0 .. mu_21
constexpr int kTaySeriesM = 17;                         // highest power of 2z in the series

struct TayMu { float mu[kTayMu]; };                     // mu_j = mean_c x_c^j of the band

// h_p = (-i)^-p G_p = f^(p)(z) / 2^p, p = 0 .. 4 (real).  z = pi N B' in FP32,
// (sz, cz) = sin/cos z and (sth, cth) = sin/cos (z / N) from exact turns.
__device__ inline void taylor_dirichlet(float z, float sz, float cz, float sth, float cth, float fN,
                                        const TayMu& mu, float (&h)[5]) {
  if (fabsf(z) < 2.f) {
    // h_p = sum_{m + p even} (-1)^((m + p) / 2) (2 z)^m / m! mu_{p+m}
    float am[kTaySeriesM + 1];
    am[0] = 1.f;
    const float t = 2.f * z;
    #pragma unroll
    for (int m = 1; m <= kTaySeriesM; ++m) am[m] = am[m - 1] * t * (1.f / (float)m);
    #pragma unroll
    for (int p = 0; p < 5; ++p) {
      float acc = 0.f;
      #pragma unroll
      for (int m = kTaySeriesM; m >= 0; --m) {
        if (((m + p) & 1) || p + m >= kTayMu) continue;
        const float term = am[m] * mu.mu[p + m];
        acc += (((m + p) >> 1) & 1) ? -term : term;
      }
      h[p] = acc;
    }
  } else {
    const float w = fN * sth, iw = 1.f / w;
    const float w1 = cth, w2 = -sth / fN, w3 = -cth / (fN * fN), w4 = sth / (fN * fN * fN);
    const float f0 = sz * iw;
    const float f1 = (cz - f0 * w1) * iw;
    const float f2 = (-sz - 2.f * f1 * w1 - f0 * w2) * iw;
    const float f3 = (-cz - 3.f * f2 * w1 - 3.f * f1 * w2 - f0 * w3) * iw;
    const float f4 = (sz - 4.f * f3 * w1 - 6.f * f2 * w2 - 4.f * f1 * w3 - f0 * w4) * iw;
    h[0] = f0; h[1] = 0.5f * f1; h[2] = 0.25f * f2; h[3] = 0.125f * f3; h[4] = 0.0625f * f4;
  }
}

// sin/cos(pi n x) for a signed Q0.64 x (x 2^-64) and an integer n: n x = hi + f
// exactly (f in [-1/2, 1/2)), sin(pi (hi + f)) = (-1)^hi sin(pi f)
__device__ inline void sincospi_scaled(long long x, long long n, float* s, float* c) {
  const unsigned long long lo = (unsigned long long)n * (unsigned long long)x;
  const long long hi = __mul64hi(n, x);
  const long long los = (long long)lo;
  sincospif(q64_signed_to_float((unsigned long long)los), s, c);
  if ((hi + (los < 0 ? 1 : 0)) & 1) { *s = -*s; *c = -*c; }
}

// D^(p)_jk for every pair j < k of a Taylor block, per baseline (one CTA each):
//   Dt[bl][k(k-1)/2 + j][p], p = 0 .. 4
template <int BK>
__global__ void __launch_bounds__(256) k_block_dirichlet_taylor(const PhaseAB* __restrict__ ph,
                                                               const GeoTrig* __restrict__ trig, int n_blk,
                                                               float2* __restrict__ Dt, int64_t n_bl,
                                                               int n_time, int n_chan, TayMu mu) {
  static_assert(BK >= kTayBlk, "a Taylor block's phases need BK >= 21 entries");
  __shared__ float2 sU[16][kTayBlk];               // band-centre phasors, times in chunks of 16
  __shared__ long long sB[16][kTayBlk];            // signed steps B (Q0.64)
  const int64_t bl = blockIdx.x;
  const int n_pairs = n_blk * (n_blk - 1) / 2;
  const int pr = threadIdx.x;
  int k = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)pr)) * 0.5f);
  while (k > 1 && k * (k - 1) / 2 > pr) --k;
  while ((k + 1) * k / 2 <= pr) ++k;
  const int j = pr - k * (k - 1) / 2;
  const float fN = (float)n_chan;
  const bool even = (n_chan & 1) == 0;
  float2 D[5];
  #pragma unroll
  for (int p = 0; p < 5; ++p) D[p] = make_float2(0.f, 0.f);
  for (int t0 = 0; t0 < n_time; t0 += 16) {
    const int nt = min(16, n_time - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < nt * n_blk; q += blockDim.x) {
      const int t = q / n_blk, s = q - t * n_blk;
      const size_t at = ((size_t)bl * n_time + t0 + t) * BK + s;
      sU[t][s] = trig[at].u;
      sB[t][s] = (long long)ph[at].b;
    }
    __syncthreads();
    if (pr < n_pairs) {
      for (int t = 0; t < nt; ++t) {
        const float2 uk = sU[t][k], uj = sU[t][j];
        float er = uk.x * uj.x + uk.y * uj.y;      // u_k conj(u_j)
        float ei = uk.y * uj.x - uk.x * uj.y;
        const long long bk = sB[t][k], bj = sB[t][j];
        const long long d = (long long)((unsigned long long)bk - (unsigned long long)bj);   // wrapped B'
        const bool wrap = ((bk ^ bj) & (bk ^ d)) < 0;
        if (wrap && even) { er = -er; ei = -ei; }
        float sz, cz, sth, cth;
        sincospi_scaled(d, n_chan, &sz, &cz);
        sincospi_scaled(d, 1, &sth, &cth);
        const float z = 3.14159265358979f * fN * q64_signed_to_float((unsigned long long)d);
        float h[5];
        taylor_dirichlet(z, sz, cz, sth, cth, fN, mu, h);
        // G_p = (-i)^p h_p
        D[0].x += er * h[0];  D[0].y += ei * h[0];
        D[1].x += ei * h[1];  D[1].y -= er * h[1];
        D[2].x -= er * h[2];  D[2].y -= ei * h[2];
        D[3].x -= ei * h[3];  D[3].y += er * h[3];
        D[4].x += er * h[4];  D[4].y += ei * h[4];
      }
    }
  }
  if (pr < n_pairs) {
    const float inv_t = 1.0f / (float)n_time;
    float2* o = Dt + ((size_t)bl * kTayPairs + pr) * 5;
    #pragma unroll
    for (int p = 0; p < 5; ++p) o[p] = make_float2(D[p].x * inv_t, D[p].y * inv_t);
  }
}

// corrected moments of source q of a Taylor block (one thread per baseline):
//   mom[n][bl] = Ablk[3q + n][bl] - sum_{j<q} sum_m P[3j + m][bl] D^(n+m)_jq
__global__ void __launch_bounds__(256) k_taylor_correct(const float2* __restrict__ Ablk, int q,
                                                       const float2* __restrict__ P,
                                                       const float2* __restrict__ Dt, int64_t n_bl,
                                                       float2* __restrict__ mom) {
  const int64_t bl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (bl >= n_bl) return;
  float2 v[3][4];
  #pragma unroll
  for (int n = 0; n < 3; ++n)
    #pragma unroll
    for (int e = 0; e < 4; ++e) v[n][e] = Ablk[((size_t)(3 * q + n) * n_bl + bl) * 4 + e];
  const float2* D = Dt + ((size_t)bl * kTayPairs + q * (q - 1) / 2) * 5;
  for (int j = 0; j < q; ++j) {
    float2 d[5];
    #pragma unroll
    for (int p = 0; p < 5; ++p) d[p] = D[5 * j + p];
    #pragma unroll
    for (int m = 0; m < 3; ++m) {
      float2 Pm[4];
      #pragma unroll
      for (int e = 0; e < 4; ++e) Pm[e] = P[((size_t)(3 * j + m) * n_bl + bl) * 4 + e];
      #pragma unroll
      for (int n = 0; n < 3; ++n)
        #pragma unroll
        for (int e = 0; e < 4; ++e) v[n][e] = csub(v[n][e], cmul(Pm[e], d[n + m]));
    }
  }
  #pragma unroll
  for (int n = 0; n < 3; ++n)
    #pragma unroll
    for (int e = 0; e < 4; ++e) mom[((size_t)n * n_bl + bl) * 4 + e] = v[n][e];
}

// P0, P1, P2 of a solved Taylor source into slots 3q .. 3q + 2 of the block's
// model table, P[n][bl][4], in FP32 from the FP32 copy of its iterate Xf =
// [G H] [n_ant][8] (one thread per baseline; the table is FP32)
__global__ void __launch_bounds__(256) k_taylor_model(const float2* __restrict__ Xf, float S,
                                                     const int2* __restrict__ bl_ant, int64_t n_bl,
                                                     float2* __restrict__ P) {
  const int64_t bl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (bl >= n_bl) return;
  const int2 ij = bl_ant[bl];
  float2 Gi[4], Hi[4], Gj[4], Hj[4];
  #pragma unroll
  for (int e = 0; e < 4; ++e) {
    Gi[e] = Xf[(size_t)ij.x * 8 + e]; Hi[e] = Xf[(size_t)ij.x * 8 + 4 + e];
    Gj[e] = Xf[(size_t)ij.y * 8 + e]; Hj[e] = Xf[(size_t)ij.y * 8 + 4 + e];
  }
  // (A B^H)[r][c] = sum_k A[r][k] conj(B[c][k])
  auto ent = [](const float2 (&A)[4], const float2 (&B)[4], int r, int c) {
    return cadd(cmulc(A[2 * r], B[2 * c]), cmulc(A[2 * r + 1], B[2 * c + 1]));
  };
  #pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int r = e >> 1, c = e & 1;
    const float2 p0 = ent(Gi, Gj, r, c), p1 = cadd(ent(Gi, Hj, r, c), ent(Hi, Gj, r, c)), p2 = ent(Hi, Hj, r, c);
    P[((size_t)0 * n_bl + bl) * 4 + e] = make_float2(S * p0.x, S * p0.y);
    P[((size_t)1 * n_bl + bl) * 4 + e] = make_float2(S * p1.x, S * p1.y);
    P[((size_t)2 * n_bl + bl) * 4 + e] = make_float2(S * p2.x, S * p2.y);
  }
}

}  // namespace rts
