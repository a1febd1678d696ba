// Streaming kernels over the visibility cube vis[t][bl][c][4]:
//   rotate + average      (the average step of one source)
//   subtract + average    (subtract source k, average for source k+1, one pass)
//   subtract              (last source)
// One CTA per baseline: its N_t strips of N_c contiguous visibilities are read
// with coalesced 16-byte loads (consecutive threads = consecutive channels) and
// its average is reduced in the CTA (warp shuffles, FP64 across warps), so no
// atomics and a deterministic result.
#pragma once
#include "common.cuh"

namespace rts {

constexpr int kStreamThreads = 256;
constexpr int kStreamBatch = 4;   // visibilities in flight per thread

struct StreamArgs {
  const void* src;          // cube read
  void* dst;                // cube written (may equal src)
  const double* uvw;        // [n_time][n_ant][3]
  const int2* bl_ant;       // [n_bl] (i, j)
  const double* freq_c;     // [n_chan] nu_c / c_light (per metre), FP64 path only
  int n_ant, n_chan, n_time;
  int64_t n_bl;
  double nu0_c, dnu_c;      // nu_0 / c and dnu / c (per metre)
  SrcDir sub;               // source subtracted
  const double2* Jsub;      // its FP64 Jones [n_ant][4]
  SrcDir acc;               // source averaged
  void* avg;                // [n_bl][4] complex (cube precision)
  double inv_n;             // 1 / (n_time n_chan)
};

// ---------------------------------------------------------------------------
// reductions

template <int N>
__device__ inline void block_sum_f32_to_f64(float (&v)[N], double* s_red /* [32][N] */,
                                            double (&out)[N]) {
  #pragma unroll
  for (int k = 0; k < N; ++k)
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    #pragma unroll
    for (int k = 0; k < N; ++k) s_red[warp * N + k] = (double)v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    #pragma unroll
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += s_red[w * N + k];
      out[k] = s;
    }
  }
}

template <int N>
__device__ inline void block_sum_f64(double (&v)[N], double* s_red, double (&out)[N]) {
  #pragma unroll
  for (int k = 0; k < N; ++k)
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    #pragma unroll
    for (int k = 0; k < N; ++k) s_red[warp * N + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    #pragma unroll
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += s_red[w * N + k];
      out[k] = s;
    }
  }
}

// (t, c) walk of one thread: s = t*n_chan + c advanced by kStreamThreads
struct TCWalk {
  int t, c, dt, dc, n_chan;
  __device__ inline void init(int s0, int n_chan_) {
    n_chan = n_chan_;
    t = s0 / n_chan; c = s0 - t * n_chan;
    dt = kStreamThreads / n_chan; dc = kStreamThreads - dt * n_chan;
  }
  __device__ inline void next() {
    c += dc; t += dt;
    if (c >= n_chan) { c -= n_chan; ++t; }
  }
};

// ---------------------------------------------------------------------------
// mixed precision: complex64 cube, Q0.64 phases, FP32 arithmetic

// x -= M * exp(-2 pi i phi)  on the 4 complex of one visibility
__device__ inline void sub_model(float4& x0, float4& x1, const float2 (&M)[4], float2 ph) {
  // ph = exp(+2 pi i phi); model term M * conj(ph)
  x0.x -= M[0].x * ph.x + M[0].y * ph.y;  x0.y -= M[0].y * ph.x - M[0].x * ph.y;
  x0.z -= M[1].x * ph.x + M[1].y * ph.y;  x0.w -= M[1].y * ph.x - M[1].x * ph.y;
  x1.x -= M[2].x * ph.x + M[2].y * ph.y;  x1.y -= M[2].y * ph.x - M[2].x * ph.y;
  x1.z -= M[3].x * ph.x + M[3].y * ph.y;  x1.w -= M[3].y * ph.x - M[3].x * ph.y;
}
// acc += x * exp(+2 pi i phi)
__device__ inline void acc_rot(float (&a)[8], const float4& x0, const float4& x1, float2 ph) {
  a[0] += x0.x * ph.x - x0.y * ph.y;  a[1] += x0.x * ph.y + x0.y * ph.x;
  a[2] += x0.z * ph.x - x0.w * ph.y;  a[3] += x0.z * ph.y + x0.w * ph.x;
  a[4] += x1.x * ph.x - x1.y * ph.y;  a[5] += x1.x * ph.y + x1.y * ph.x;
  a[6] += x1.z * ph.x - x1.w * ph.y;  a[7] += x1.z * ph.y + x1.w * ph.x;
}

__device__ inline void model_matrix_f(const double2* __restrict__ J, int n_ant, int i, int j,
                                      double S, float2 (&M)[4]) {
  M22<double2> Ji, Jj;
  #pragma unroll
  for (int e = 0; e < 4; ++e) { Ji.e[e] = J[(size_t)i * 4 + e]; Jj.e[e] = J[(size_t)j * 4 + e]; }
  M22<double2> P = mmul_h(Ji, Jj);
  #pragma unroll
  for (int e = 0; e < 4; ++e) M[e] = make_float2((float)(S * P.e[e].x), (float)(S * P.e[e].y));
}

template <bool SUB, bool ACC>
__global__ void __launch_bounds__(kStreamThreads, 3) k_stream_mixed(StreamArgs a) {
  extern __shared__ unsigned long long s_ph[];   // [n_time][4]: A_sub B_sub A_acc B_acc
  __shared__ float2 s_M[4];
  __shared__ double s_red[(kStreamThreads / 32) * 8];
  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  for (int t = threadIdx.x; t < a.n_time; t += blockDim.x) {
    if (SUB) {
      double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, a.sub);
      s_ph[4 * t + 0] = frac_q64(tau * a.nu0_c);
      s_ph[4 * t + 1] = frac_q64(tau * a.dnu_c);
    }
    if (ACC) {
      double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, a.acc);
      s_ph[4 * t + 2] = frac_q64(tau * a.nu0_c);
      s_ph[4 * t + 3] = frac_q64(tau * a.dnu_c);
    }
  }
  if (SUB && threadIdx.x == 0) {
    float2 M[4];
    model_matrix_f(a.Jsub, a.n_ant, ij.x, ij.y, a.sub.S, M);
    #pragma unroll
    for (int e = 0; e < 4; ++e) s_M[e] = M[e];
  }
  __syncthreads();
  float2 M[4];
  if (SUB) {
    #pragma unroll
    for (int e = 0; e < 4; ++e) M[e] = s_M[e];
  }
  float acc[8];
  #pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;

  const float4* src = static_cast<const float4*>(a.src);   // may alias dst (in place)
  float4* dst = static_cast<float4*>(a.dst);
  const int n_s = a.n_time * a.n_chan;
  TCWalk w;
  w.init(threadIdx.x, a.n_chan);
  for (int s0 = threadIdx.x; s0 < n_s; s0 += kStreamBatch * kStreamThreads) {
    float4 x0[kStreamBatch], x1[kStreamBatch];
    int tt[kStreamBatch], cc[kStreamBatch];
    size_t idx[kStreamBatch];
    #pragma unroll
    for (int u = 0; u < kStreamBatch; ++u) {
      tt[u] = w.t; cc[u] = w.c;
      idx[u] = (((size_t)w.t * a.n_bl + bl) * a.n_chan + w.c) * 2;
      if (s0 + u * kStreamThreads < n_s) {
        x0[u] = __ldcs(src + idx[u]);
        x1[u] = __ldcs(src + idx[u] + 1);
      }
      w.next();
    }
    #pragma unroll
    for (int u = 0; u < kStreamBatch; ++u) {
      if (s0 + u * kStreamThreads < n_s) {
        if (SUB) {
          const unsigned long long A = s_ph[4 * tt[u]], B = s_ph[4 * tt[u] + 1];
          float2 ph = phasor_f(q64_to_turns(A + (unsigned long long)cc[u] * B));
          sub_model(x0[u], x1[u], M, ph);
          __stcs(dst + idx[u], x0[u]);
          __stcs(dst + idx[u] + 1, x1[u]);
        }
        if (ACC) {
          const unsigned long long A = s_ph[4 * tt[u] + 2], B = s_ph[4 * tt[u] + 3];
          float2 ph = phasor_f(q64_to_turns(A + (unsigned long long)cc[u] * B));
          acc_rot(acc, x0[u], x1[u], ph);
        }
      }
    }
  }
  if (ACC) {
    double tot[8];
    block_sum_f32_to_f64<8>(acc, s_red, tot);
    if (threadIdx.x == 0) {
      float4* out = static_cast<float4*>(a.avg) + bl * 2;
      out[0] = make_float4((float)(tot[0] * a.inv_n), (float)(tot[1] * a.inv_n),
                           (float)(tot[2] * a.inv_n), (float)(tot[3] * a.inv_n));
      out[1] = make_float4((float)(tot[4] * a.inv_n), (float)(tot[5] * a.inv_n),
                           (float)(tot[6] * a.inv_n), (float)(tot[7] * a.inv_n));
    }
  }
}

// ---------------------------------------------------------------------------
// plain FP64: complex128 cube, per-sample FP64 phase tau * nu_c / c, FP64 sincospi

template <bool SUB, bool ACC>
__global__ void __launch_bounds__(kStreamThreads) k_stream_fp64(StreamArgs a) {
  extern __shared__ double s_tau[];   // [n_time][2]: tau_sub, tau_acc
  __shared__ double2 s_M[4];
  __shared__ double s_red[(kStreamThreads / 32) * 8];
  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  for (int t = threadIdx.x; t < a.n_time; t += blockDim.x) {
    if (SUB) s_tau[2 * t] = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, a.sub);
    if (ACC) s_tau[2 * t + 1] = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, a.acc);
  }
  if (SUB && threadIdx.x == 0) {
    M22<double2> Ji, Jj;
    #pragma unroll
    for (int e = 0; e < 4; ++e) { Ji.e[e] = a.Jsub[(size_t)ij.x * 4 + e]; Jj.e[e] = a.Jsub[(size_t)ij.y * 4 + e]; }
    M22<double2> P = mmul_h(Ji, Jj);
    #pragma unroll
    for (int e = 0; e < 4; ++e) s_M[e] = make_double2(a.sub.S * P.e[e].x, a.sub.S * P.e[e].y);
  }
  __syncthreads();
  double2 M[4];
  if (SUB) {
    #pragma unroll
    for (int e = 0; e < 4; ++e) M[e] = s_M[e];
  }
  double acc[8];
  #pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  const double2* src = static_cast<const double2*>(a.src);
  double2* dst = static_cast<double2*>(a.dst);
  const int n_s = a.n_time * a.n_chan;
  TCWalk w;
  w.init(threadIdx.x, a.n_chan);
  for (int s = threadIdx.x; s < n_s; s += kStreamThreads, w.next()) {
    const size_t idx = (((size_t)w.t * a.n_bl + bl) * a.n_chan + w.c) * 4;
    double2 x[4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) x[e] = src[idx + e];
    if (SUB) {
      double2 ph = phasor_d(s_tau[2 * w.t] * a.freq_c[w.c]);     // exp(+2 pi i phi)
      #pragma unroll
      for (int e = 0; e < 4; ++e) { x[e] = csub(x[e], cmulc(M[e], ph)); dst[idx + e] = x[e]; }
    }
    if (ACC) {
      double2 ph = phasor_d(s_tau[2 * w.t + 1] * a.freq_c[w.c]);
      #pragma unroll
      for (int e = 0; e < 4; ++e) {
        double2 r = cmul(x[e], ph);
        acc[2 * e] += r.x; acc[2 * e + 1] += r.y;
      }
    }
  }
  if (ACC) {
    double tot[8];
    block_sum_f64<8>(acc, s_red, tot);
    if (threadIdx.x == 0) {
      double2* out = static_cast<double2*>(a.avg) + bl * 4;
      #pragma unroll
      for (int e = 0; e < 4; ++e) out[e] = make_double2(tot[2 * e] * a.inv_n, tot[2 * e + 1] * a.inv_n);
    }
  }
}

}  // namespace rts
