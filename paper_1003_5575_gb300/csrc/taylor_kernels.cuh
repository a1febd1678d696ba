// Gains Taylor-expanded in frequency (Section 3.1: when consecutive channels
// are combined, the unknown tile gain may be Taylor-expanded in frequency).
// First order about the band centre (uniform channels):
//   J_p(c) = G_p + x_c H_p,   x_c = (c - (N_c - 1)/2) / N_c,
// so source k's model on baseline (i, j) at channel c is
//   S (G_i + x_c H_i)(G_j + x_c H_j)^H exp(-2 pi i phi) = (P0 + x_c P1 + x_c^2 P2) exp(-2 pi i phi),
//   P0 = S G_i G_j^H,  P1 = S (G_i H_j^H + H_i G_j^H),  P2 = S H_i H_j^H.
// The least-squares solve over every sample uses the unknown X_p = [G_p H_p]
// (2 x 4) and Z_pq(c) = S [W_q(c); x_c W_q(c)], W_q(c) = (G_q + x_c H_q)^H.
// Because the model depends on c only through x_c, its normal equations
// reduce exactly to three channel moments of the rotated residual per baseline,
//   M_n(bl) = mean_{t,c} x_c^n R exp(+2 pi i phi),  n = 0, 1, 2,
// and five scalar channel moments mu_n = mean_c x_c^n:
//   A_p = S sum_q [M0 G_q + M1 H_q,  M1 G_q + M2 H_q]          (M_n,qp = M_n,pq^H)
//   C_p = S^2 [mu0 K0 + mu1 K1 + mu2 K2,  mu1 K0 + mu2 K1 + mu3 K2;
//              mu1 K0 + mu2 K1 + mu3 K2,  mu2 K0 + mu3 K1 + mu4 K2]
//   K0 = sum_q G_q^H G_q,  K1 = sum_q (G_q^H H_q + H_q^H G_q),  K2 = sum_q H_q^H H_q
//   X_p <- A_p C_p^-1   (Jacobi sweeps from G = I, H = 0, every second averaged).
// One streaming pass per source subtracts source k's model and accumulates the
// moments for source k+1 (as the constant-gain pass does with one average).
#pragma once
#include "als_kernels.cuh"
#include "stream_kernels.cuh"

namespace rts {

struct TaylorStreamArgs {
  StreamArgs s;             // cube, geometry, sources; s.avg unused
  const double2* Xsub;      // [n_ant][8] FP64 G (4) then H (4) of the subtracted source
  float2* mom;              // [3][n_bl][4] moments M0, M1, M2 of the averaged source
  float x0, dx;             // x_c = x0 + c dx
};

// Entry e = 2r + c of model matrix n (P0, P1 or P2) of baseline (i, j) from
// the FP64 Taylor Jones X [n_ant][8] (G then H), one entry per calling thread:
// (A B^H)[r][c] = sum_k A[r][k] conj(B[c][k]).
__device__ inline float2 taylor_model_entry(const double2* __restrict__ X, int i, int j, double S, int n,
                                            int e) {
  const int r = e >> 1, c = e & 1;
  auto ent = [&](const double2* A, const double2* B) {
    return cadd(cmul(A[2 * r], cconj(B[2 * c])), cmul(A[2 * r + 1], cconj(B[2 * c + 1])));
  };
  const double2 *Gi = X + (size_t)i * 8, *Hi = Gi + 4, *Gj = X + (size_t)j * 8, *Hj = Gj + 4;
  double2 v;
  if (n == 0) v = ent(Gi, Gj);
  else if (n == 1) v = cadd(ent(Gi, Hj), ent(Hi, Gj));
  else v = ent(Hi, Hj);
  return make_float2((float)(S * v.x), (float)(S * v.y));
}

template <bool SUB, bool ACC>
__global__ void __launch_bounds__(kStreamThreads, 2) k_stream_taylor(TaylorStreamArgs ta) {
  const StreamArgs& a = ta.s;
  extern __shared__ unsigned long long s_ph[];   // [n_time][4]: A_sub B_sub A_acc B_acc
  __shared__ float2 s_P[3][4];
  __shared__ double s_red[kStreamThreads / 32][32];
  __shared__ double s_tot[24];
  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  for (int t = threadIdx.x; t < a.n_time; t += blockDim.x) {
    if (SUB) {
      const double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, a.sub);
      s_ph[4 * t + 0] = frac_q64(tau * a.nu0_c);
      s_ph[4 * t + 1] = frac_q64(tau * a.dnu_c);
    }
    if (ACC) {
      const double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, a.acc);
      s_ph[4 * t + 2] = frac_q64(tau * a.nu0_c);
      s_ph[4 * t + 3] = frac_q64(tau * a.dnu_c);
    }
  }
  if (SUB && threadIdx.x < 12)
    s_P[threadIdx.x >> 2][threadIdx.x & 3] =
        taylor_model_entry(ta.Xsub, ij.x, ij.y, a.sub.S, threadIdx.x >> 2, threadIdx.x & 3);
  __syncthreads();
  float2 P[3][4];
  if (SUB) {
    #pragma unroll
    for (int n = 0; n < 3; ++n)
      #pragma unroll
      for (int e = 0; e < 4; ++e) P[n][e] = s_P[n][e];
  }
  float acc[24];
  #pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0.f;

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
        const float x = fmaf((float)cc[u], ta.dx, ta.x0);
        if (SUB) {
          const unsigned long long A = s_ph[4 * tt[u]], B = s_ph[4 * tt[u] + 1];
          const float2 ph = phasor_f(q64_to_turns(A + (unsigned long long)cc[u] * B));
          float2 M[4];
          #pragma unroll
          for (int e = 0; e < 4; ++e) {               // P0 + x (P1 + x P2)
            M[e].x = fmaf(x, fmaf(x, P[2][e].x, P[1][e].x), P[0][e].x);
            M[e].y = fmaf(x, fmaf(x, P[2][e].y, P[1][e].y), P[0][e].y);
          }
          sub_model(x0[u], x1[u], M, ph);
          __stcs(dst + idx[u], x0[u]);
          __stcs(dst + idx[u] + 1, x1[u]);
        }
        if (ACC) {
          const unsigned long long A = s_ph[4 * tt[u] + 2], B = s_ph[4 * tt[u] + 3];
          const float2 ph = phasor_f(q64_to_turns(A + (unsigned long long)cc[u] * B));
          float y[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          acc_rot(y, x0[u], x1[u], ph);
          const float x2 = x * x;
          #pragma unroll
          for (int k = 0; k < 8; ++k) {
            acc[k] += y[k];
            acc[8 + k] = fmaf(x, y[k], acc[8 + k]);
            acc[16 + k] = fmaf(x2, y[k], acc[16 + k]);
          }
        }
      }
    }
  }
  if (ACC) {
    // warp totals of the 24 sums (two reduce-scatter rounds), then one thread per
    // sum adds the warps' totals in FP64 in warp order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v[16];
    #pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = acc[k];
    const float w0 = warp_reduce_scatter16f(v, lane);
    #pragma unroll
    for (int k = 0; k < 8; ++k) { v[k] = acc[16 + k]; v[8 + k] = 0.f; }
    const float w1 = warp_reduce_scatter16f(v, lane);
    if ((lane & 1) == 0) {
      s_red[warp][lane >> 1] = (double)w0;
      s_red[warp][16 + (lane >> 1)] = (double)w1;
    }
    __syncthreads();
    if (threadIdx.x < 24) {
      double t = 0.0;
      #pragma unroll
      for (int w2 = 0; w2 < kStreamThreads / 32; ++w2) t += s_red[w2][threadIdx.x];
      s_tot[threadIdx.x] = t * a.inv_n;
    }
    __syncthreads();
    if (threadIdx.x < 6) {           // moment n, half h (two polarisations)
      const int n = threadIdx.x >> 1, hh = threadIdx.x & 1;
      const double* t = s_tot + 8 * n + 4 * hh;
      reinterpret_cast<float4*>(ta.mom + ((size_t)n * a.n_bl + bl) * 4)[hh] =
          make_float4((float)t[0], (float)t[1], (float)t[2], (float)t[3]);
    }
  }
}

struct TaylorAlsArgs {
  const float2* mom;        // [3][n_bl][4]
  const double2* X_old;     // [n_ant][8] FP64 iterate (ignored on the first sweep)
  const float2* Xf_old;     // FP32 copy of X_old
  double2* X_new;
  float2* Xf_new;
  double* norms;            // [n_ant][2]
  int* flag;
  float2* gain_out;         // [n_ant][4] G, last sweep only (else NULL)
  float2* slope_out;        // [n_ant][4] H, last sweep only
  int n_ant;
  int64_t n_bl;
  double S;
  double mu[5];             // mean_c x_c^n
  int first, average;
};

// M_n,pq of one baseline pair (conjugate transpose when q < p)
__device__ inline void load_mom(const float2* __restrict__ mom, int64_t n_bl, int n_ant, int p, int q,
                                int n, float2 (&v)[4]) {
  const float2* base = mom + (size_t)n * n_bl * 4;
  load_vpq<float2>(base, n_ant, p, q, v);
}

// 2x2 complex FP32 helpers on [0 1; 2 3]
__device__ inline void mm_acc(const float2 (&a)[4], const float2 (&b)[4], float (&o)[8]) {   // o += a b
  #pragma unroll
  for (int r = 0; r < 2; ++r)
    #pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float2 x = cadd(cmul(a[2 * r], b[c]), cmul(a[2 * r + 1], b[2 + c]));
      o[2 * (2 * r + c)] += x.x; o[2 * (2 * r + c) + 1] += x.y;
    }
}
__device__ inline void mhm_acc(const float2 (&a)[4], const float2 (&b)[4], float (&o)[8]) {  // o += a^H b
  #pragma unroll
  for (int r = 0; r < 2; ++r)
    #pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float2 x = cadd(cconjmul(a[r], b[c]), cconjmul(a[2 + r], b[2 + c]));
      o[2 * (2 * r + c)] += x.x; o[2 * (2 * r + c) + 1] += x.y;
    }
}

// One entry of X = b C^-1 (b one row of the right-hand sides, col its column)
// for a 4x4 Hermitian positive-definite C = [A E; E^H D] (2x2 blocks), by the
// Schur complement of A:
//   T = A^-1 E,  Sc = D - E^H T,  x_h = (b_r - b_l T) Sc^-1,  x_g = (b_l - x_h E^H) A^-1,
// with the 2x2 inverses in closed form.  C is positive definite exactly when
// A_00 > 0, det A > 0, Sc_00 > 0 and det Sc > 0 (its Cholesky pivots are
// A_00, det A / A_00, Sc_00, det Sc / Sc_00); returns false otherwise.  Each
// lane of a warp takes one entry: an FP64 warp instruction costs 64 times an
// FP32 one on this GPU, and the lanes share the instruction stream.
__device__ inline bool schur_solve4_entry(const double2 (&C)[4][4], const double2 (&b)[4], int col, double2* x) {
  // inverse of the Hermitian [a00 a01; conj(a01) a11]
  auto inv2h = [](double a00, double2 a01, double a11, double2 (&o)[2][2], double* det) {
    *det = a00 * a11 - (a01.x * a01.x + a01.y * a01.y);
    const double id = 1.0 / *det;
    o[0][0] = make_double2(a11 * id, 0.0);
    o[1][1] = make_double2(a00 * id, 0.0);
    o[0][1] = make_double2(-a01.x * id, -a01.y * id);
    o[1][0] = make_double2(-a01.x * id, a01.y * id);
  };
  double2 Ai[2][2], Si[2][2], T[2][2], Sc[2][2];
  double detA, detS;
  inv2h(C[0][0].x, C[0][1], C[1][1].x, Ai, &detA);
  if (!(C[0][0].x > 0.0) || !(detA > 0.0)) return false;
  #pragma unroll
  for (int r = 0; r < 2; ++r)
    #pragma unroll
    for (int c = 0; c < 2; ++c) T[r][c] = cadd(cmul(Ai[r][0], C[0][2 + c]), cmul(Ai[r][1], C[1][2 + c]));
  #pragma unroll
  for (int r = 0; r < 2; ++r)
    #pragma unroll
    for (int c = 0; c < 2; ++c)    // (E^H)[r][k] = conj(E[k][r])
      Sc[r][c] = csub(C[2 + r][2 + c], cadd(cmul(cconj(C[0][2 + r]), T[0][c]), cmul(cconj(C[1][2 + r]), T[1][c])));
  inv2h(Sc[0][0].x, Sc[0][1], Sc[1][1].x, Si, &detS);
  if (!(Sc[0][0].x > 0.0) || !(detS > 0.0)) return false;
  double2 Rh[2], Xh[2], Rg[2];
  #pragma unroll
  for (int k = 0; k < 2; ++k) Rh[k] = csub(b[2 + k], cadd(cmul(b[0], T[0][k]), cmul(b[1], T[1][k])));
  #pragma unroll
  for (int c = 0; c < 2; ++c) Xh[c] = cadd(cmul(Rh[0], Si[0][c]), cmul(Rh[1], Si[1][c]));
  if (col >= 2) {
    *x = col == 2 ? Xh[0] : Xh[1];           // selects, not an indexed (local-memory) read
    return true;
  }
  #pragma unroll
  for (int k = 0; k < 2; ++k)       // (x_h E^H)[k] = sum_j x_h[j] conj(E[k][j])
    Rg[k] = csub(b[k], cadd(cmul(Xh[0], cconj(C[k][2])), cmul(Xh[1], cconj(C[k][3]))));
  *x = col == 0 ? cadd(cmul(Rg[0], Ai[0][0]), cmul(Rg[1], Ai[1][0])) : cadd(cmul(Rg[0], Ai[0][1]), cmul(Rg[1], Ai[1][1]));
  return true;
}

// One Jacobi sweep for antenna p = blockIdx.x (kAlsThreads threads).
__global__ void __launch_bounds__(kAlsThreads) k_als_taylor_sweep(TaylorAlsArgs a) {
  __shared__ double s_red[kAlsThreads / 32][32];
  __shared__ double s_tot[32];
  const int p = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per-thread partials: A (2x4 complex: left M0 G + M1 H, right M1 G + M2 H),
  // K0 = G^H G, K1 = G^H H + H^H G, K2 = H^H H (full 2x2 complex each)
  float Al[8], Ar[8], K0[8], K1[8], K2[8];
  #pragma unroll
  for (int k = 0; k < 8; ++k) { Al[k] = 0.f; Ar[k] = 0.f; K0[k] = 0.f; K1[k] = 0.f; K2[k] = 0.f; }
  for (int q = threadIdx.x; q < a.n_ant; q += kAlsThreads) {
    if (q == p) continue;
    float2 M0[4], M1[4], M2[4], G[4], H[4];
    load_mom(a.mom, a.n_bl, a.n_ant, p, q, 0, M0);
    load_mom(a.mom, a.n_bl, a.n_ant, p, q, 1, M1);
    load_mom(a.mom, a.n_bl, a.n_ant, p, q, 2, M2);
    if (a.first) {
      G[0] = make_float2(1.f, 0.f); G[1] = make_float2(0.f, 0.f); G[2] = make_float2(0.f, 0.f);
      G[3] = make_float2(1.f, 0.f);
      #pragma unroll
      for (int e = 0; e < 4; ++e) H[e] = make_float2(0.f, 0.f);
    } else {
      #pragma unroll
      for (int e = 0; e < 4; ++e) { G[e] = a.Xf_old[(size_t)q * 8 + e]; H[e] = a.Xf_old[(size_t)q * 8 + 4 + e]; }
    }
    mm_acc(M0, G, Al); mm_acc(M1, H, Al);
    mm_acc(M1, G, Ar); mm_acc(M2, H, Ar);
    mhm_acc(G, G, K0);
    mhm_acc(G, H, K1); mhm_acc(H, G, K1);
    mhm_acc(H, H, K2);
  }
  // sums across the CTA, 40 values: FP32 within each warp (three reduce-scatter
  // rounds of 16), FP64 across the warps (an FP64 warp instruction costs 64
  // times an FP32 one here, so the lane sums stay FP32)
  float v[16];
  #pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = Al[k]; v[8 + k] = Ar[k]; }
  const float w0 = warp_reduce_scatter16f(v, lane);
  #pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = K0[k]; v[8 + k] = K1[k]; }
  const float w1 = warp_reduce_scatter16f(v, lane);
  #pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = K2[k]; v[8 + k] = 0.f; }
  const float w2 = warp_reduce_scatter16f(v, lane);
  __shared__ double s_red2[kAlsThreads / 32][8];
  if ((lane & 1) == 0) {
    s_red[warp][lane >> 1] = (double)w0;            // 0..15: A left, A right
    s_red[warp][16 + (lane >> 1)] = (double)w1;     // 16..31: K0, K1
    if ((lane >> 1) < 8) s_red2[warp][lane >> 1] = (double)w2;   // K2
  }
  __syncthreads();
  __shared__ double s_k2[8];
  if (threadIdx.x < 32) {
    double t = 0.0;
    #pragma unroll
    for (int w = 0; w < kAlsThreads / 32; ++w) t += s_red[w][threadIdx.x];
    s_tot[threadIdx.x] = t;
  } else if (threadIdx.x < 40) {
    double t = 0.0;
    #pragma unroll
    for (int w = 0; w < kAlsThreads / 32; ++w) t += s_red2[w][threadIdx.x - 32];
    s_k2[threadIdx.x - 32] = t;
  }
  __syncthreads();
  // the normal matrix C (16 lanes, one entry each) and the right-hand sides
  // B = S [A_l A_r] (8 lanes) in FP64, then lane e < 8 solves for entry e of X
  __shared__ double2 s_C[16], s_B[8];
  if (threadIdx.x < 24) {
    auto cm = [&](const double* b, int e) { return make_double2(b[2 * e], b[2 * e + 1]); };
    const double S = a.S;
    const int t = threadIdx.x;
    if (t < 16) {
      // block (bi, bj) = S^2 (mu[bi+bj] K0 + mu[bi+bj+1] K1 + mu[bi+bj+2] K2)
      const int R = t >> 2, Cc = t & 3, bi = R >> 1, bj = Cc >> 1, e = 2 * (R & 1) + (Cc & 1);
      const double S2 = S * S, c0 = S2 * a.mu[bi + bj], c1 = S2 * a.mu[bi + bj + 1], c2 = S2 * a.mu[bi + bj + 2];
      const double2 x0 = cm(s_tot + 16, e), x1 = cm(s_tot + 24, e), x2 = cm(s_k2, e);
      s_C[t] = make_double2(c0 * x0.x + c1 * x1.x + c2 * x2.x, c0 * x0.y + c1 * x1.y + c2 * x2.y);
    } else {
      const int j = t - 16, r = j >> 2, c4 = j & 3;     // B[r][c4]: A_l entry 2r + c4, A_r entry 2r + c4 - 2
      const double2 v = c4 < 2 ? cm(s_tot, 2 * r + c4) : cm(s_tot + 8, 2 * r + c4 - 2);
      s_B[j] = make_double2(S * v.x, S * v.y);
    }
  }
  __syncthreads();
  if (threadIdx.x >= 8) return;
  const int e = threadIdx.x;
  // lane e: G entry (e >> 1, e & 1) for e < 4, H entry ((e - 4) >> 1, e & 1) for e >= 4
  const int row = (e & 3) >> 1, col = e < 4 ? (e & 1) : 2 + (e & 1);
  double2 C[4][4], brow[4];
  #pragma unroll
  for (int i = 0; i < 16; ++i) C[i >> 2][i & 3] = s_C[i];
  #pragma unroll
  for (int c = 0; c < 4; ++c) brow[c] = s_B[4 * row + c];
  double2 Xn;
  if (!schur_solve4_entry(C, brow, col, &Xn)) Xn = make_double2(NAN, NAN);
  double2 Xo;
  if (a.first) Xo = make_double2((e == 0 || e == 3) ? 1.0 : 0.0, 0.0);
  else Xo = a.X_old[(size_t)p * 8 + e];
  if (a.average) Xn = make_double2(0.5 * (Xn.x + Xo.x), 0.5 * (Xn.y + Xo.y));
  const double dx = Xn.x - Xo.x, dy = Xn.y - Xo.y;
  double dn = dx * dx + dy * dy;
  double nn = Xn.x * Xn.x + Xn.y * Xn.y;
  int bad = !(isfinite(Xn.x) && isfinite(Xn.y));
  #pragma unroll
  for (int o = 1; o <= 4; o <<= 1) {
    dn += __shfl_xor_sync(0xffu, dn, o);
    nn += __shfl_xor_sync(0xffu, nn, o);
    bad |= __shfl_xor_sync(0xffu, bad, o);
  }
  a.X_new[(size_t)p * 8 + e] = Xn;
  a.Xf_new[(size_t)p * 8 + e] = make_float2((float)Xn.x, (float)Xn.y);
  if (a.gain_out) {
    float2* o = e < 4 ? a.gain_out + (size_t)p * 4 + e : a.slope_out + (size_t)p * 4 + (e - 4);
    *o = make_float2((float)Xn.x, (float)Xn.y);
  }
  if (e == 0) {
    a.norms[2 * p] = dn;
    a.norms[2 * p + 1] = nn;
    if (bad) *a.flag = 1;
  }
}

// ---- the common slope rotation (reading R27) ------------------------------------
// Rotating every slope by the same Hermitian K, H_p -> H_p + i G_p K, changes
// the model only at second order in x_c, so the Jacobi sweeps barely move the
// iterate along it.  After each sweep from the second on: one Newton step from
// K = 0 on the cost along that direction, K = sum_a k_a B_a over
// B = [1 0; 0 0], [0 0; 0 1], [0 1; 1 0], [0 -i; i 0].  From the moments, per
// baseline (p, q), with rho = M2 - S (mu2 P0 + mu3 P1 + mu4 P2) the
// x_c^2-weighted mean residual, F_a = G_p B_a G_q^H and
// D_a = i (G_p B_a H_q^H - H_p B_a G_q^H) (<X, Y> = tr X^H Y):
//   g_a  = -2 S sum Re<rho, D_a>
//   h_ab =  2 S^2 mu4 sum Re<D_a, D_b> - 2 S sum Re<rho, G_p (B_a B_b + B_b B_a) G_q^H>,
// B_a B_b + B_b B_a being 2 B_0, 2 B_1, 2 I, 2 I on the diagonal, B_2 at (0, 2)
// and (1, 2), B_3 at (0, 3) and (1, 3), 0 at (0, 1) and (2, 3).  The sums over
// all samples carry a common factor (the sample count) that drops out of
// k = -h^-1 g (solved by 2x2 blocks).  The step is taken when every Cholesky
// pivot of h exceeds 1e-6 of its largest diagonal entry, and only with three channels or more (with
// two, x_c^2 is the same at both and G absorbs the change along K).

constexpr int kRotVals = 18;   // per baseline: Re<rho,F_a> (4), Re<rho,D_a> (4), Re<D_a,D_b> a <= b (10)

struct TaylorRotArgs {
  const float2* mom;        // [3][n_bl][4] moments (M2 is used)
  const float2* Xf;         // [n_ant][8] FP32 iterate after the sweep (G then H)
  const int2* bl_ant;
  int64_t n_bl;
  float S, mu2, mu3, mu4;
  double* part;             // [gridDim.x][kRotVals] per-CTA sums
  unsigned* count;          // CTAs done (zero between launches: the last CTA resets it)
  double* step;             // [5]: k_0 .. k_3, then 1 when the step is taken, else 0
};

// X B_a Y^H, a = 0..3, from the outer products O_kl[r][c] = X[r][k] conj(Y[c][l]):
// O_00, O_11, O_01 + O_10, i (O_10 - O_01)
__device__ inline void basis_products(const float2 (&X)[4], const float2 (&Y)[4], float2 (&out)[4][4]) {
  #pragma unroll
  for (int r = 0; r < 2; ++r)
    #pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int e = 2 * r + c;
      const float2 o00 = cmulc(X[2 * r], Y[2 * c]), o11 = cmulc(X[2 * r + 1], Y[2 * c + 1]);
      const float2 o01 = cmulc(X[2 * r], Y[2 * c + 1]), o10 = cmulc(X[2 * r + 1], Y[2 * c]);
      out[0][e] = o00;
      out[1][e] = o11;
      out[2][e] = cadd(o01, o10);
      out[3][e] = make_float2(o01.y - o10.y, o10.x - o01.x);
    }
}

__device__ inline float re_inner(const float2 (&a)[4], const float2 (&b)[4]) {
  float s = 0.f;
  #pragma unroll
  for (int e = 0; e < 4; ++e) s += a[e].x * b[e].x + a[e].y * b[e].y;
  return s;
}

constexpr int kRotThreads = 512;
constexpr int kRotMaxGrid = 256;   // CTAs (one baseline a thread at 512 antennas): the last one
                                   // sums at most 16 partials per lane

__global__ void __launch_bounds__(kRotThreads) k_taylor_rot_sums(TaylorRotArgs a) {
  __shared__ float s_w[kRotThreads / 32][kRotVals];
  __shared__ double s_tot[kRotVals];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float acc[kRotVals];
  #pragma unroll
  for (int i = 0; i < kRotVals; ++i) acc[i] = 0.f;
  for (int64_t bl = blockIdx.x * (int64_t)blockDim.x + tid; bl < a.n_bl; bl += (int64_t)gridDim.x * blockDim.x) {
    const int2 ij = a.bl_ant[bl];
    float2 Gp[4], Hp[4], Gq[4], Hq[4], M2[4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      Gp[e] = a.Xf[(size_t)ij.x * 8 + e]; Hp[e] = a.Xf[(size_t)ij.x * 8 + 4 + e];
      Gq[e] = a.Xf[(size_t)ij.y * 8 + e]; Hq[e] = a.Xf[(size_t)ij.y * 8 + 4 + e];
      M2[e] = a.mom[((size_t)2 * a.n_bl + bl) * 4 + e];
    }
    float2 F[4][4], DA[4][4], DB[4][4];
    basis_products(Gp, Gq, F);
    basis_products(Gp, Hq, DA);
    basis_products(Hp, Gq, DB);
    float2 rho[4], D[4][4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = e >> 1, c = e & 1;
      const float2 P0 = cadd(F[0][e], F[1][e]);
      const float2 P1 = cadd(cadd(DA[0][e], DA[1][e]), cadd(DB[0][e], DB[1][e]));
      const float2 P2 = cadd(cmulc(Hp[2 * r], Hq[2 * c]), cmulc(Hp[2 * r + 1], Hq[2 * c + 1]));
      rho[e] = make_float2(M2[e].x - a.S * (a.mu2 * P0.x + a.mu3 * P1.x + a.mu4 * P2.x),
                           M2[e].y - a.S * (a.mu2 * P0.y + a.mu3 * P1.y + a.mu4 * P2.y));
      #pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float2 d = csub(DA[b][e], DB[b][e]);
        D[b][e] = make_float2(-d.y, d.x);                  // i (G_p B H_q^H - H_p B G_q^H)
      }
    }
    #pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[b] += re_inner(rho, F[b]);
      acc[4 + b] += re_inner(rho, D[b]);
    }
    int k = 8;
    #pragma unroll
    for (int b0 = 0; b0 < 4; ++b0)
      #pragma unroll
      for (int b1 = b0; b1 < 4; ++b1) acc[k++] += re_inner(D[b0], D[b1]);
  }
  // sums in trees: FP32 within each warp (an FP64 warp instruction costs 64
  // times an FP32 one here), FP64 over the CTA's 16 warps (16 lanes per value)
  // and, in the last CTA, over the grid's partials (16 lanes per value, up to
  // 16 partials each)
  #pragma unroll
  for (int i = 0; i < kRotVals; ++i) {
    float v = acc[i];
    #pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[warp][i] = v;
  }
  __syncthreads();
  if (tid < 16 * kRotVals) {                 // warps 0 .. 8, two values each
    const int i = tid >> 4, w = tid & 15;
    double v = (double)s_w[w][i];
    #pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (w == 0) a.part[(size_t)blockIdx.x * kRotVals + i] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(a.count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < 16 * kRotVals) {
    const int i = tid >> 4, w = tid & 15;
    double v = 0.0;
    for (unsigned b = w; b < gridDim.x; b += 16) v += __ldcg(a.part + (size_t)b * kRotVals + i);
    #pragma unroll
    for (int o = 8; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (w == 0) s_tot[i] = v;
  }
  __syncthreads();
  if (tid != 0) return;
  *a.count = 0u;
  const double S = a.S, r0 = s_tot[0], r1 = s_tot[1], r2 = s_tot[2], r3 = s_tot[3];
  const double c4 = 2.0 * S * S * (double)a.mu4, c2 = 2.0 * S;
  // h = [hA hE; hE^T hD] (2x2 blocks), r = -g
  const double* dd = s_tot + 8;              // (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
  const double h00 = c4 * dd[0] - c2 * 2.0 * r0, h01 = c4 * dd[1], h11 = c4 * dd[4] - c2 * 2.0 * r1;
  const double h02 = c4 * dd[2] - c2 * r2, h03 = c4 * dd[3] - c2 * r3;
  const double h12 = c4 * dd[5] - c2 * r2, h13 = c4 * dd[6] - c2 * r3;
  const double h22 = c4 * dd[7] - c2 * 2.0 * (r0 + r1), h23 = c4 * dd[8], h33 = c4 * dd[9] - c2 * 2.0 * (r0 + r1);
  double rv[4];
  #pragma unroll
  for (int b = 0; b < 4; ++b) rv[b] = 2.0 * S * s_tot[4 + b];          // -g_b
  // Cholesky pivots by the Schur complement of the leading block: h00,
  // det A / h00, Sc00, det Sc / Sc00, each against 1e-6 of the largest diagonal
  const double dmax = fmax(fmax(h00, h11), fmax(h22, h33));
  const double detA = h00 * h11 - h01 * h01, idA = 1.0 / detA;
  const double A00 = h11 * idA, A01 = -h01 * idA, A11 = h00 * idA;  // A^-1
  const double T00 = A00 * h02 + A01 * h12, T01 = A00 * h03 + A01 * h13;   // T = A^-1 E
  const double T10 = A01 * h02 + A11 * h12, T11 = A01 * h03 + A11 * h13;
  const double S00 = h22 - (h02 * T00 + h12 * T10), S01 = h23 - (h02 * T01 + h12 * T11);
  const double S11 = h33 - (h03 * T01 + h13 * T11);
  const double detS = S00 * S11 - S01 * S01;
  const double tol = 1e-6 * dmax;
  const bool ok = dmax > 0.0 && h00 > tol && detA > tol * h00 && S00 > tol && detS > tol * S00;
  double k0 = 0.0, k1 = 0.0, k2 = 0.0, k3 = 0.0;
  if (ok) {
    const double idS = 1.0 / detS;
    // k_2 = Sc^-1 (r_2 - T^T r_1), k_1 = A^-1 (r_1 - E k_2)
    const double u0 = rv[2] - (T00 * rv[0] + T10 * rv[1]), u1 = rv[3] - (T01 * rv[0] + T11 * rv[1]);
    k2 = (S11 * u0 - S01 * u1) * idS;
    k3 = (S00 * u1 - S01 * u0) * idS;
    const double w0 = rv[0] - (h02 * k2 + h03 * k3), w1 = rv[1] - (h12 * k2 + h13 * k3);
    k0 = A00 * w0 + A01 * w1;
    k1 = A01 * w0 + A11 * w1;
  }
  a.step[0] = k0; a.step[1] = k1; a.step[2] = k2; a.step[3] = k3;
  a.step[4] = ok ? 1.0 : 0.0;
}

// H_p += i G_p K for every antenna (FP64 iterate and its FP32 copy), then the
// convergence norms of the rotated iterate against the previous one; the
// last sweep's G and H to gain_out / slope_out.  8 threads per antenna.
__global__ void __launch_bounds__(256) k_taylor_rot_apply(const double* __restrict__ step, double2* X_new,
                                                         const double2* __restrict__ X_old, float2* Xf_new,
                                                         double* norms, int* flag, float2* gain_out,
                                                         float2* slope_out, int n_ant) {
  if (step[4] == 0.0) return;                // no step: the sweep's iterate, norms and outputs stand
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = t >> 3, e = t & 7;
  const bool live = p < n_ant;
  double2 Xn = make_double2(0.0, 0.0), Xo = Xn;
  if (live) {
    Xn = X_new[(size_t)p * 8 + e];
    Xo = X_old[(size_t)p * 8 + e];
    if (e >= 4) {
      const int r = (e - 4) >> 1, c = e & 1;
      // K = [k0, k2 - i k3; k2 + i k3, k1], column c
      const double2 K0c = c == 0 ? make_double2(step[0], 0.0) : make_double2(step[2], -step[3]);
      const double2 K1c = c == 0 ? make_double2(step[2], step[3]) : make_double2(step[1], 0.0);
      const double2 gk = cadd(cmul(X_new[(size_t)p * 8 + 2 * r], K0c), cmul(X_new[(size_t)p * 8 + 2 * r + 1], K1c));
      Xn = make_double2(Xn.x - gk.y, Xn.y + gk.x);
      X_new[(size_t)p * 8 + e] = Xn;
      Xf_new[(size_t)p * 8 + e] = make_float2((float)Xn.x, (float)Xn.y);
    }
  }
  const double dx = Xn.x - Xo.x, dy = Xn.y - Xo.y;
  double dn = dx * dx + dy * dy, nn = Xn.x * Xn.x + Xn.y * Xn.y;
  int bad = live && !(isfinite(Xn.x) && isfinite(Xn.y));
  #pragma unroll
  for (int o = 1; o <= 4; o <<= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    nn += __shfl_xor_sync(0xffffffffu, nn, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (!live) return;
  if (e == 0) {
    norms[2 * p] = dn;
    norms[2 * p + 1] = nn;
    if (bad) *flag = 1;
  }
  if (gain_out && e >= 4) slope_out[(size_t)p * 4 + (e - 4)] = make_float2((float)Xn.x, (float)Xn.y);
}

}  // namespace rts
