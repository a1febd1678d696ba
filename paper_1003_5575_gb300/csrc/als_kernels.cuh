// Alternating least squares for one source's per-antenna Jones matrices.
//
// For antenna p, with Z_pq = S J_q^H (unpolarised source, B = S I):
//   A_p = sum_{q != p} V_pq Z_pq^H = S sum_q V_pq J_q
//   C_p = sum_{q != p} Z_pq Z_pq^H = S^2 sum_q J_q^H J_q
//   J_p <- A_p C_p^-1 = (sum_q V_pq J_q)(sum_q J_q^H J_q)^-1 / S
// V_qp = V_pq^H for q < p (one triangle is stored).  Jacobi sweep: every p
// uses the previous iterate; every second sweep is averaged with it.
//
// One CTA per antenna; its threads split the q sum.  Mixed precision: the
// products and each thread's partial sum (<= n_ant/128 terms) are FP32, the
// sum across threads and the 2x2 solve are FP64.  The FP64 path does all of
// it in FP64.
#pragma once
#include "common.cuh"

namespace rts {

constexpr int kAlsThreads = 128;

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

template <typename T>   // T = float (mixed) or double (FP64)
__global__ void __launch_bounds__(kAlsThreads) k_als_sweep(AlsArgs a) {
  using C = typename cplx_of<T>::type;
  __shared__ double s_red[(kAlsThreads / 32) * 12];
  const int p = blockIdx.x;
  // per-thread partials: A (4 complex) and Hermitian C (c00, c11, re c01, im c01)
  T A[8], Cm[4];
  #pragma unroll
  for (int k = 0; k < 8; ++k) A[k] = T(0);
  #pragma unroll
  for (int k = 0; k < 4; ++k) Cm[k] = T(0);
  const C* avg = static_cast<const C*>(a.avg);
  for (int q = threadIdx.x; q < a.n_ant; q += kAlsThreads) {
    if (q == p) continue;
    C V[4];
    load_vpq<C>(avg, a.n_ant, p, q, V);
    C J[4];
    if (a.first) {
      J[0] = cmk<C>(1, 0); J[1] = cmk<C>(0, 0); J[2] = cmk<C>(0, 0); J[3] = cmk<C>(1, 0);
    } else if (sizeof(T) == 4) {
      #pragma unroll
      for (int e = 0; e < 4; ++e) { float2 f = a.Jf_old[(size_t)q * 4 + e]; J[e] = cmk<C>(f.x, f.y); }
    } else {
      #pragma unroll
      for (int e = 0; e < 4; ++e) { double2 d = a.J_old[(size_t)q * 4 + e]; J[e] = cmk<C>(d.x, d.y); }
    }
    // A += V J
    C a0 = cadd(cmul(V[0], J[0]), cmul(V[1], J[2]));
    C a1 = cadd(cmul(V[0], J[1]), cmul(V[1], J[3]));
    C a2 = cadd(cmul(V[2], J[0]), cmul(V[3], J[2]));
    C a3 = cadd(cmul(V[2], J[1]), cmul(V[3], J[3]));
    A[0] += a0.x; A[1] += a0.y; A[2] += a1.x; A[3] += a1.y;
    A[4] += a2.x; A[5] += a2.y; A[6] += a3.x; A[7] += a3.y;
    // C += J^H J  (c00 = |J00|^2 + |J10|^2, c11 = |J01|^2 + |J11|^2, c01 = conj(J00) J01 + conj(J10) J11)
    Cm[0] += J[0].x * J[0].x + J[0].y * J[0].y + J[2].x * J[2].x + J[2].y * J[2].y;
    Cm[1] += J[1].x * J[1].x + J[1].y * J[1].y + J[3].x * J[3].x + J[3].y * J[3].y;
    C c01 = cadd(cconjmul(J[0], J[1]), cconjmul(J[2], J[3]));
    Cm[2] += c01.x; Cm[3] += c01.y;
  }
  double v[12], tot[12];
  #pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (double)A[k];
  #pragma unroll
  for (int k = 0; k < 4; ++k) v[8 + k] = (double)Cm[k];
  #pragma unroll
  for (int k = 0; k < 12; ++k)
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    #pragma unroll
    for (int k = 0; k < 12; ++k) s_red[warp * 12 + k] = v[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  #pragma unroll
  for (int k = 0; k < 12; ++k) {
    double s = 0.0;
    for (int w = 0; w < kAlsThreads / 32; ++w) s += s_red[w * 12 + k];
    tot[k] = s;
  }
  // solve J_p = A C^-1 / S in FP64, C = [c00 c01; conj(c01) c11]
  const double2 A00 = make_double2(tot[0], tot[1]), A01 = make_double2(tot[2], tot[3]);
  const double2 A10 = make_double2(tot[4], tot[5]), A11 = make_double2(tot[6], tot[7]);
  const double c00 = tot[8], c11 = tot[9];
  const double2 c01 = make_double2(tot[10], tot[11]);
  const double det = c00 * c11 - (c01.x * c01.x + c01.y * c01.y);   // real, >= 0
  const double sc = 1.0 / (det * a.S);
  // C^-1 = [c11 -c01; -conj(c01) c00] / det
  const double2 i00 = make_double2(c11 * sc, 0.0), i11 = make_double2(c00 * sc, 0.0);
  const double2 i01 = make_double2(-c01.x * sc, -c01.y * sc);
  const double2 i10 = make_double2(-c01.x * sc, c01.y * sc);
  double2 Jn[4];
  Jn[0] = cadd(cmul(A00, i00), cmul(A01, i10));
  Jn[1] = cadd(cmul(A00, i01), cmul(A01, i11));
  Jn[2] = cadd(cmul(A10, i00), cmul(A11, i10));
  Jn[3] = cadd(cmul(A10, i01), cmul(A11, i11));
  double2 Jo[4];
  if (a.first) {
    Jo[0] = make_double2(1, 0); Jo[1] = make_double2(0, 0); Jo[2] = make_double2(0, 0); Jo[3] = make_double2(1, 0);
  } else {
    #pragma unroll
    for (int e = 0; e < 4; ++e) Jo[e] = a.J_old[(size_t)p * 4 + e];
  }
  if (a.average) {
    #pragma unroll
    for (int e = 0; e < 4; ++e) Jn[e] = make_double2(0.5 * (Jn[e].x + Jo[e].x), 0.5 * (Jn[e].y + Jo[e].y));
  }
  double dn = 0.0, nn = 0.0;
  bool finite = true;
  #pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double dx = Jn[e].x - Jo[e].x, dy = Jn[e].y - Jo[e].y;
    dn += dx * dx + dy * dy;
    nn += Jn[e].x * Jn[e].x + Jn[e].y * Jn[e].y;
    finite = finite && isfinite(Jn[e].x) && isfinite(Jn[e].y);
    a.J_new[(size_t)p * 4 + e] = Jn[e];
    if (sizeof(T) == 4) a.Jf_new[(size_t)p * 4 + e] = make_float2((float)Jn[e].x, (float)Jn[e].y);
  }
  a.norms[2 * p] = dn;
  a.norms[2 * p + 1] = nn;
  if (!finite) *a.flag = 1;
  if (a.jones_out) {
    if (sizeof(T) == 4) {
      float2* o = static_cast<float2*>(a.jones_out) + (size_t)p * 4;
      #pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = make_float2((float)Jn[e].x, (float)Jn[e].y);
    } else {
      double2* o = static_cast<double2*>(a.jones_out) + (size_t)p * 4;
      #pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = Jn[e];
    }
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
