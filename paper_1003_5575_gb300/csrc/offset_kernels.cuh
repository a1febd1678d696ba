// Ionospheric position offsets of the peeled sources (Section 3: besides its
// Jones matrices, each calibrator yields a shift of its apparent position;
// Section 3.1: the fit needs six numbers per source and is described by two,
// the ionosphere's response is a known function of frequency, and workers hand
// their numbers to a master that builds the solution).
//
// Shift model: at channel c source k sits at (l, m) + s_c (dl, dm),
// s_c = (nu_ref/nu_c)^alpha (alpha = 2: refraction ~ lambda^2).  One
// Gauss-Newton step of the loss at dl = dm = 0 with the phase derivative
// d phi/d(dl) = a_l w_c,  a_l = u - w l/n,  a_m = v - w m/n,  w_c = s_c nu_c/c:
//
//   H_pq = 2 (2 pi)^2 sum_{t,bl,c} a_p a_q w_c^2 ||M_k||_F^2,  M_k = S_k J_i J_j^H,
//   g = (dL/d dl, dL/d dm)  (adjoint sweep with the weight table w_c),
//   (dl, dm) = -H^-1 g,  or (0, 0) where det H <= 0.
//
// The six numbers (H_ll, H_lm, H_mm, g_l, g_m, L) are sums over channels, so
// channel groups on different GPUs add them (one all-reduce) before the solve.
// H factorises: H_pq = 2 (2 pi)^2 (sum_c w_c^2) sum_bl ||M_k||_F^2 sum_t a_p a_q.
// One CTA per source, threads over baselines, FP64 throughout; the
// per-baseline gradient terms and losses left by the adjoint sweep are summed
// in the same CTA.
#pragma once
#include "grad_kernels.cuh"

namespace rts {

constexpr int kOffThreads = 256;

// w_c = (nu_ref/nu_c)^alpha nu_c/c from freq_c = nu_c/c and nu_ref_c = nu_ref/c
__global__ void k_offset_weights(const double* __restrict__ freq_c, int n_chan, double alpha,
                                 double nu_ref_c, double* __restrict__ w) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_chan) w[c] = pow(nu_ref_c / freq_c[c], alpha) * freq_c[c];
}

// (dl, dm) = -H^-1 g from one source's six numbers; (0, 0) where det H <= 0
__device__ inline void offset_step(const double* o, double* d) {
  const double hll = o[0], hlm = o[1], hmm = o[2], gl = o[3], gm = o[4];
  const double det = hll * hmm - hlm * hlm;
  d[0] = det > 0.0 ? -(hmm * gl - hlm * gm) / det : 0.0;
  d[1] = det > 0.0 ? -(hll * gm - hlm * gl) / det : 0.0;
}

__global__ void k_offset_solve(const double* __restrict__ out, int n_src, double* __restrict__ offsets) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_src) offset_step(out + 6 * (size_t)k, offsets + 2 * (size_t)k);
}

template <typename T>
__global__ void __launch_bounds__(kOffThreads)
k_offset_normal(const void* __restrict__ jones, const DirQ* __restrict__ dir,
                const double* __restrict__ uvw, const int2* __restrict__ bl_ant,
                const double* __restrict__ wchan, const double* __restrict__ gsc,
                const double* __restrict__ loss_bl, int n_ant, int n_chan, int n_time,
                int64_t n_bl, double* __restrict__ out, double* __restrict__ offsets) {
  constexpr int kW = 7;   // hll, hlm, hmm, g_l, g_m, loss, sum_c w_c^2
  __shared__ double s[kW][kOffThreads];
  const int k = blockIdx.x;
  const DirQ d = dir[k];
  const double n = 1.0 + d.z;
  const double lz = d.x / n, mz = d.y / n, S = d.w;
  double acc[kW] = {};
  for (int64_t bl = threadIdx.x; bl < n_bl; bl += kOffThreads) {
    const int2 ij = bl_ant[bl];
    const size_t bi = ((size_t)k * n_ant + ij.x) * 4, bj = ((size_t)k * n_ant + ij.y) * 4;
    double ar[4], ai[4], br[4], bi_[4];
    for (int e = 0; e < 4; ++e) {
      const auto a = load_j<T>(jones, bi + e), b = load_j<T>(jones, bj + e);
      ar[e] = a.x; ai[e] = a.y; br[e] = b.x; bi_[e] = b.y;
    }
    // ||J_i J_j^H||_F^2, entry (r, q) = sum_e Ji[r][e] conj(Jj[q][e])
    double mm = 0.0;
    for (int r = 0; r < 2; ++r)
      for (int q = 0; q < 2; ++q) {
        double re = 0.0, im = 0.0;
        for (int e = 0; e < 2; ++e) {
          const double xr = ar[2 * r + e], xi = ai[2 * r + e];
          const double yr = br[2 * q + e], yi = -bi_[2 * q + e];
          re += xr * yr - xi * yi;
          im += xr * yi + xi * yr;
        }
        mm += re * re + im * im;
      }
    mm *= S * S;
    double sll = 0.0, slm = 0.0, smm = 0.0;
    for (int t = 0; t < n_time; ++t) {
      const double* p = uvw + ((size_t)t * n_ant + ij.x) * 3;
      const double* q = uvw + ((size_t)t * n_ant + ij.y) * 3;
      const double u = p[0] - q[0], v = p[1] - q[1], w = p[2] - q[2];
      const double al = u - w * lz, am = v - w * mz;
      sll += al * al; slm += al * am; smm += am * am;
    }
    acc[0] += mm * sll; acc[1] += mm * slm; acc[2] += mm * smm;
    const double* g = gsc + ((size_t)k * n_bl + bl) * 3;
    acc[3] += g[0]; acc[4] += g[1];
    acc[5] += loss_bl[bl];
  }
  for (int c = threadIdx.x; c < n_chan; c += kOffThreads) acc[6] += wchan[c] * wchan[c];
  for (int w = 0; w < kW; ++w) s[w][threadIdx.x] = acc[w];
  __syncthreads();
  for (int o = kOffThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int w = 0; w < kW; ++w) s[w][threadIdx.x] += s[w][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double two_pi = 6.283185307179586476925286766559;
    const double f = 2.0 * two_pi * two_pi * s[6][0];
    const double hll = f * s[0][0], hlm = f * s[1][0], hmm = f * s[2][0];
    const double gl = s[3][0], gm = s[4][0];
    double* o = out + 6 * (size_t)k;
    o[0] = hll; o[1] = hlm; o[2] = hmm; o[3] = gl; o[4] = gm; o[5] = s[5][0];
    offset_step(o, offsets + 2 * (size_t)k);
  }
}

}  // namespace rts
