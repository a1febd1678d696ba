// Alternating least squares for one source's per-antenna Jones matrices.
//
// For antenna p, with Z_pq = S J_q^H (unpolarised source, B = S I):
//   A_p = sum_{q != p} V_pq Z_pq^H = S sum_q V_pq J_q
//   C_p = sum_{q != p} Z_pq Z_pq^H = S^2 sum_q J_q^H J_q
//   J_p <- A_p C_p^-1 = (sum_q V_pq J_q)(sum_q J_q^H J_q)^-1 / S
// V_qp = V_pq^H for q < p (one triangle is stored).  Jacobi sweep: every p
// uses the previous iterate; every second sweep is averaged with it.
//
// One CTA of kAlsThreads threads per antenna p; thread t takes q = t, t+128,
// ... and issues all of its loads before any arithmetic.  Mixed precision: the
// products and each thread's partial sum (<= ceil(n_ant/128) terms) are FP32;
// the sum across threads is FP64 (a reduce-scatter butterfly inside each warp,
// 16 FP64 adds per lane for the 12 sums, then the warps combined in shared
// memory), and the 2x2 solve is FP64.  The FP64 path does all of it in FP64.
#pragma once
#include "common.cuh"

namespace rts {

constexpr int kAlsThreads = 128;
constexpr int kAlsPerThread = 4;     // q terms whose loads are issued together
inline unsigned als_grid(int n_ant) { return (unsigned)n_ant; }

struct AlsArgs {
  const void* avg;          // [n_bl][4] complex, cube precision
  const double2* J_old;     // [n_ant][4] FP64 iterate (ignored on the first sweep)
  const float2* Jf_old;     // FP32 copy of J_old (mixed path)
  double2* J_new;
  float2* Jf_new;
  double* norms;            // [n_ant][2] ||J_new - J_old||^2, ||J_new||^2
  int* flag;                // set to 1 on a non-finite value (this source)
  void* jones_out;          // [n_ant][4] cube precision, last sweep only (else NULL)
  int n_ant;
  double S;
  int first, average;
};

template <typename C>
__device__ inline void load_vpq(const C* __restrict__ avg, int n_ant, int p, int q, C (&v)[4]) {
  if (p < q) {
    const C* s = avg + bl_index(n_ant, p, q) * 4;
    #pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = s[e];
  } else {                                   // V_pq = V_qp^H
    const C* s = avg + bl_index(n_ant, q, p) * 4;
    v[0] = cconj(s[0]); v[1] = cconj(s[2]); v[2] = cconj(s[1]); v[3] = cconj(s[3]);
  }
}

// Reduce 16 doubles over the 32 lanes of a warp.  Each level exchanges half of
// the remaining values with the partner lane, so a lane does 8+4+2+1+1 adds;
// afterwards lane L holds the warp total of value index L >> 1.
__device__ inline double warp_reduce_scatter16(double (&v)[16], int lane) {
  #pragma unroll
  for (int o = 16, n = 16; o >= 2; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
    #pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double send = upper ? v[i] : v[i + n / 2];
      const double keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Reduce 16 floats over the 32 lanes of a warp (each level exchanges half of the
// remaining values with the partner lane); afterwards lane L holds the warp
// total of value index L >> 1.
__device__ __forceinline__ float warp_reduce_scatter16f(float (&v)[16], int lane) {
  #pragma unroll
  for (int o = 16, n = 16; o >= 2; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
    #pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float send = upper ? v[i] : v[i + n / 2];
      const float keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <typename T>   // T = float (mixed) or double (FP64)
__global__ void __launch_bounds__(kAlsThreads) k_als_sweep(AlsArgs a) {
  using C = typename cplx_of<T>::type;
  __shared__ double s_red[kAlsThreads / 32][12];
  __shared__ double s_tot[12];
  const int p = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per-thread partials: A (4 complex) and Hermitian C (c00, c11, re c01, im c01)
  T A[8], Cm[4];
  #pragma unroll
  for (int k = 0; k < 8; ++k) A[k] = T(0);
  #pragma unroll
  for (int k = 0; k < 4; ++k) Cm[k] = T(0);
  const C* avg = static_cast<const C*>(a.avg);
  for (int q0 = threadIdx.x; q0 < a.n_ant; q0 += kAlsThreads * kAlsPerThread) {
    C V[kAlsPerThread][4], J[kAlsPerThread][4];
    #pragma unroll
    for (int u = 0; u < kAlsPerThread; ++u) {
      const int q = q0 + u * kAlsThreads;
      if (q < a.n_ant && q != p) {
        load_vpq<C>(avg, a.n_ant, p, q, V[u]);
        if (a.first) {
          J[u][0] = cmk<C>(1, 0); J[u][1] = cmk<C>(0, 0); J[u][2] = cmk<C>(0, 0); J[u][3] = cmk<C>(1, 0);
        } else if constexpr (sizeof(T) == 4) {
          #pragma unroll
          for (int e = 0; e < 4; ++e) { float2 f = a.Jf_old[(size_t)q * 4 + e]; J[u][e] = cmk<C>(f.x, f.y); }
        } else {
          #pragma unroll
          for (int e = 0; e < 4; ++e) { double2 d = a.J_old[(size_t)q * 4 + e]; J[u][e] = cmk<C>(d.x, d.y); }
        }
      } else {
        #pragma unroll
        for (int e = 0; e < 4; ++e) { V[u][e] = cmk<C>(0, 0); J[u][e] = cmk<C>(0, 0); }
      }
    }
    #pragma unroll
    for (int u = 0; u < kAlsPerThread; ++u) {
      const C* Vq = V[u];
      const C* Jq = J[u];
      // A += V J
      C a0 = cadd(cmul(Vq[0], Jq[0]), cmul(Vq[1], Jq[2]));
      C a1 = cadd(cmul(Vq[0], Jq[1]), cmul(Vq[1], Jq[3]));
      C a2 = cadd(cmul(Vq[2], Jq[0]), cmul(Vq[3], Jq[2]));
      C a3 = cadd(cmul(Vq[2], Jq[1]), cmul(Vq[3], Jq[3]));
      A[0] += a0.x; A[1] += a0.y; A[2] += a1.x; A[3] += a1.y;
      A[4] += a2.x; A[5] += a2.y; A[6] += a3.x; A[7] += a3.y;
      // C += J^H J  (c00 = |J00|^2 + |J10|^2, c11 = |J01|^2 + |J11|^2, c01 = conj(J00) J01 + conj(J10) J11)
      Cm[0] += Jq[0].x * Jq[0].x + Jq[0].y * Jq[0].y + Jq[2].x * Jq[2].x + Jq[2].y * Jq[2].y;
      Cm[1] += Jq[1].x * Jq[1].x + Jq[1].y * Jq[1].y + Jq[3].x * Jq[3].x + Jq[3].y * Jq[3].y;
      C c01 = cadd(cconjmul(Jq[0], Jq[1]), cconjmul(Jq[2], Jq[3]));
      Cm[2] += c01.x; Cm[3] += c01.y;
    }
  }
  double v[16];
  #pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (double)A[k];
  #pragma unroll
  for (int k = 0; k < 4; ++k) v[8 + k] = (double)Cm[k];
  #pragma unroll
  for (int k = 12; k < 16; ++k) v[k] = 0.0;
  const double wsum = warp_reduce_scatter16(v, lane);
  if ((lane & 1) == 0 && (lane >> 1) < 12) s_red[warp][lane >> 1] = wsum;
  __syncthreads();
  if (threadIdx.x < 12) {
    double t = 0.0;
    #pragma unroll
    for (int w = 0; w < kAlsThreads / 32; ++w) t += s_red[w][threadIdx.x];
    s_tot[threadIdx.x] = t;
  }
  __syncthreads();
  // the 2x2 solve: lanes 0..3 of warp 0 each produce one entry J_new[e]
  if (threadIdx.x >= 4) return;
  const int e = threadIdx.x, r = e >> 1, c = e & 1;
  // J_p = A C^-1 / S in FP64, C = [c00 c01; conj(c01) c11],
  // C^-1 = [c11 -c01; -conj(c01) c00] / det
  const double c00 = s_tot[8], c11 = s_tot[9];
  const double2 c01 = make_double2(s_tot[10], s_tot[11]);
  const double det = c00 * c11 - (c01.x * c01.x + c01.y * c01.y);   // real, >= 0
  const double sc = 1.0 / (det * a.S);
  // column c of C^-1: (i0c, i1c)
  const double2 i0c = c == 0 ? make_double2(c11 * sc, 0.0) : make_double2(-c01.x * sc, -c01.y * sc);
  const double2 i1c = c == 0 ? make_double2(-c01.x * sc, c01.y * sc) : make_double2(c00 * sc, 0.0);
  // row r of A: (Ar0, Ar1)
  const double2 Ar0 = make_double2(s_tot[4 * r], s_tot[4 * r + 1]);
  const double2 Ar1 = make_double2(s_tot[4 * r + 2], s_tot[4 * r + 3]);
  double2 Jn = cadd(cmul(Ar0, i0c), cmul(Ar1, i1c));
  const double2 Jo = a.first ? make_double2((e == 0 || e == 3) ? 1.0 : 0.0, 0.0)
                             : a.J_old[(size_t)p * 4 + e];
  if (a.average) Jn = make_double2(0.5 * (Jn.x + Jo.x), 0.5 * (Jn.y + Jo.y));
  const double dx = Jn.x - Jo.x, dy = Jn.y - Jo.y;
  double dn = dx * dx + dy * dy;
  double nn = Jn.x * Jn.x + Jn.y * Jn.y;
  int bad = !(isfinite(Jn.x) && isfinite(Jn.y));
  #pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    dn += __shfl_xor_sync(0xfu, dn, o);
    nn += __shfl_xor_sync(0xfu, nn, o);
    bad |= __shfl_xor_sync(0xfu, bad, o);
  }
  a.J_new[(size_t)p * 4 + e] = Jn;
  if constexpr (sizeof(T) == 4) a.Jf_new[(size_t)p * 4 + e] = make_float2((float)Jn.x, (float)Jn.y);
  if (a.jones_out) {
    if constexpr (sizeof(T) == 4) static_cast<float2*>(a.jones_out)[(size_t)p * 4 + e] = make_float2((float)Jn.x, (float)Jn.y);
    else static_cast<double2*>(a.jones_out)[(size_t)p * 4 + e] = Jn;
  }
  if (e == 0) {
    a.norms[2 * p] = dn;
    a.norms[2 * p + 1] = nn;
    if (bad) *a.flag = 1;
  }
}

// status of one source from the last sweep's norms: 0 / 1 / -4 (non-finite)
__global__ void __launch_bounds__(256) k_als_finalize(const double* __restrict__ norms, int n_ant,
                                                      int* __restrict__ flag,
                                                      int* __restrict__ status,
                                                      double* __restrict__ rel_out) {
  __shared__ double s_dn[256], s_nn[256];
  double dn = 0.0, nn = 0.0;
  for (int p = threadIdx.x; p < n_ant; p += 256) { dn += norms[2 * p]; nn += norms[2 * p + 1]; }
  s_dn[threadIdx.x] = dn; s_nn[threadIdx.x] = nn;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) { s_dn[threadIdx.x] += s_dn[threadIdx.x + o]; s_nn[threadIdx.x] += s_nn[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rel = sqrt(s_dn[0] / s_nn[0]);
    int st;
    if (*flag || !isfinite(rel)) st = -4;
    else st = rel > 1e-6 ? 1 : 0;
    *status = st;
    *rel_out = rel;
    *flag = 0;
  }
}

}  // namespace rts
