// Model prediction: vis (+)= sum over a chunk of sources of
// S_k J_i J_j^H exp(-2 pi i phi_k), one CTA per baseline.  The FP32 sums over
// sources are Kahan-compensated, so a 1000-source prediction stays within a
// few ulp of the exact sum.
#pragma once
#include "stream_kernels.cuh"
#include "kahan.cuh"

namespace rts {


constexpr int kPredictChunk = 32;

struct PredictArgs {
  void* vis;
  const double* uvw;
  const int2* bl_ant;
  const double* freq_c;
  const double* src;         // device [n_src][3] (l, m, S) of this chunk
  const void* jones;         // device [n_src][n_ant][4] (cube precision) of this chunk
  int n_src;                 // <= kPredictChunk
  int n_ant, n_chan, n_time;
  int64_t n_bl;
  double nu0_c, dnu_c;
  int accumulate;
};

__device__ inline SrcDir dev_dir(const double* s) {
  SrcDir d; d.l = s[0]; d.m = s[1]; d.S = s[2];
  double r2 = d.l * d.l + d.m * d.m;
  d.nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
  return d;
}

__global__ void __launch_bounds__(kStreamThreads) k_predict_mixed(PredictArgs a) {
  extern __shared__ unsigned long long s_ab[];      // [n_time][n_src][2]
  __shared__ float2 s_M[kPredictChunk][4];    // -S_k J_i J_j^H
  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  for (int q = threadIdx.x; q < a.n_time * a.n_src; q += blockDim.x) {
    const int t = q / a.n_src, k = q - t * a.n_src;
    SrcDir d = dev_dir(a.src + 3 * k);
    double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, d);
    s_ab[2 * q] = frac_q64(tau * a.nu0_c);
    s_ab[2 * q + 1] = frac_q64(tau * a.dnu_c);
  }
  for (int k = threadIdx.x; k < a.n_src; k += blockDim.x) {
    const float2* J = static_cast<const float2*>(a.jones) + (size_t)k * a.n_ant * 4;
    M22<double2> Ji, Jj;
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      float2 p = J[(size_t)ij.x * 4 + e], q = J[(size_t)ij.y * 4 + e];
      Ji.e[e] = make_double2(p.x, p.y); Jj.e[e] = make_double2(q.x, q.y);
    }
    M22<double2> P = mmul_h(Ji, Jj);
    const double S = a.src[3 * k + 2];
    #pragma unroll
    for (int e = 0; e < 4; ++e) s_M[k][e] = make_float2((float)(-S * P.e[e].x), (float)(-S * P.e[e].y));
  }
  __syncthreads();
  float4* vis = static_cast<float4*>(a.vis);
  const int n_s = a.n_time * a.n_chan;
  TCWalk w;
  w.init(threadIdx.x, a.n_chan);
  for (int s = threadIdx.x; s < n_s; s += kStreamThreads, w.next()) {
    const size_t idx = (((size_t)w.t * a.n_bl + bl) * a.n_chan + w.c) * 2;
    float sum[8], comp[8];
    if (a.accumulate) {
      const float4 x0 = vis[idx], x1 = vis[idx + 1];
      sum[0] = x0.x; sum[1] = x0.y; sum[2] = x0.z; sum[3] = x0.w;
      sum[4] = x1.x; sum[5] = x1.y; sum[6] = x1.z; sum[7] = x1.w;
    } else {
      #pragma unroll
      for (int e = 0; e < 8; ++e) sum[e] = 0.f;
    }
    #pragma unroll
    for (int e = 0; e < 8; ++e) comp[e] = 0.f;
    for (int k = 0; k < a.n_src; ++k) {
      const unsigned long long A = s_ab[2 * (w.t * a.n_src + k)];
      const unsigned long long B = s_ab[2 * (w.t * a.n_src + k) + 1];
      const float2 ph = phasor_f(q64_to_turns(A + (unsigned long long)w.c * B));
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        // term = M exp(-2 pi i phi) = M conj(ph); s_M holds -M
        const float2 nm = s_M[k][e];
        const float tr = -(nm.x * ph.x + nm.y * ph.y);
        const float ti = -(nm.y * ph.x - nm.x * ph.y);
        kahan_add(sum[2 * e], comp[2 * e], tr);
        kahan_add(sum[2 * e + 1], comp[2 * e + 1], ti);
      }
    }
    vis[idx] = make_float4(sum[0], sum[1], sum[2], sum[3]);
    vis[idx + 1] = make_float4(sum[4], sum[5], sum[6], sum[7]);
  }
}

__global__ void __launch_bounds__(kStreamThreads) k_predict_fp64(PredictArgs a) {
  extern __shared__ double s_tau64[];               // [n_time][n_src]
  __shared__ double2 s_M64[kPredictChunk][4];
  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  for (int q = threadIdx.x; q < a.n_time * a.n_src; q += blockDim.x) {
    const int t = q / a.n_src, k = q - t * a.n_src;
    SrcDir d = dev_dir(a.src + 3 * k);
    s_tau64[q] = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, d);
  }
  for (int k = threadIdx.x; k < a.n_src; k += blockDim.x) {
    const double2* J = static_cast<const double2*>(a.jones) + (size_t)k * a.n_ant * 4;
    M22<double2> Ji, Jj;
    #pragma unroll
    for (int e = 0; e < 4; ++e) { Ji.e[e] = J[(size_t)ij.x * 4 + e]; Jj.e[e] = J[(size_t)ij.y * 4 + e]; }
    M22<double2> P = mmul_h(Ji, Jj);
    const double S = a.src[3 * k + 2];
    #pragma unroll
    for (int e = 0; e < 4; ++e) s_M64[k][e] = make_double2(S * P.e[e].x, S * P.e[e].y);
  }
  __syncthreads();
  double2* vis = static_cast<double2*>(a.vis);
  const int n_s = a.n_time * a.n_chan;
  TCWalk w;
  w.init(threadIdx.x, a.n_chan);
  for (int s = threadIdx.x; s < n_s; s += kStreamThreads, w.next()) {
    const size_t idx = (((size_t)w.t * a.n_bl + bl) * a.n_chan + w.c) * 4;
    double2 x[4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) x[e] = a.accumulate ? vis[idx + e] : make_double2(0.0, 0.0);
    for (int k = 0; k < a.n_src; ++k) {
      double2 ph = phasor_d(s_tau64[w.t * a.n_src + k] * a.freq_c[w.c]);
      #pragma unroll
      for (int e = 0; e < 4; ++e) x[e] = cadd(x[e], cmulc(s_M64[k][e], ph));
    }
    #pragma unroll
    for (int e = 0; e < 4; ++e) vis[idx + e] = x[e];
  }
}

}  // namespace rts
