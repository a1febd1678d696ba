// Adjoint of the multi-source predict step.
//
//   R = V - sum_k M_k exp(-2 pi i phi_k),  M_k = S_k J_i J_j^H,  L = sum ||R||_F^2
//   G_k  = sum_{t,c} R exp(+2 pi i phi_k)
//   H^l_k = sum_{t,c} R exp(+2 pi i phi_k) dphi_k/dl,  dphi/dl = (u - w l/n) nu_c / c
//   (H^m_k likewise with v, m)
//   dL/dJ_i += -2 S G J_j,  dL/dJ_j += -2 S G^H J_i    (dL/dRe + i dL/dIm)
//   dL/dS   += -2 Re tr(G^H J_i J_j^H)
//   dL/dl   += -4 pi Im tr(H^lH M),  dL/dm likewise.
//
// Kernel 1, one CTA per (baseline, chunk of sources): for each time and
// channel tile it forms R for every channel of the tile in shared memory
// (all K sources subtracted, phasors computed, never stored) and adds |R|^2 to
// the loss; then threads = (source, channel group) accumulate
// H0 = sum_c R e^{+i phi} and H1 = sum_c c R e^{+i phi}, from which
// G += H0 and H^l += (u - w l/n)(nu_0/c H0 + dnu/c H1).  Per (source,
// baseline) it stores G and the three scalar contributions (FP64).
// With WEIGHTED the channel weight of the position derivative is a table
// (d phi/d shift = a_p wchan[c], used by the offset fit's frequency law) and
// H^l = (u - w l/n) sum_c wchan[c] R e^{+i phi}.
// Kernels 2-4 reduce those per antenna / per source / for the loss in a fixed
// order, so the result is deterministic (no atomics).
#pragma once
#include <string>
#include <type_traits>

#include "common.cuh"
#include "kahan.cuh"

namespace rts {

constexpr int kGradThreads = 512;
constexpr int kGradTile = 512;        // channels per shared-memory tile
constexpr int kGradChunk = 512;       // sources per CTA in the backward phase
constexpr size_t kGradMaxSmem = 227 * 1024;

struct __align__(16) DirQ { double x, y, z, w; };   // (l, m, n - 1, S) of one source

struct GradWorkspace {
  int cap_src = 0;
  int64_t n_bl = 0;
  double2* G = nullptr;     // [K][n_bl][4]
  double* gsc = nullptr;    // [K][n_bl][3] (dl, dm, dS contributions)
  double* loss_bl = nullptr;// [n_bl]
  DirQ* dir = nullptr;   // [K] (l, m, nm1, S)
  double* wchan = nullptr;  // [n_chan] per-channel weight of the position derivative (offsets)
};

struct GradArgs {
  const void* vis;
  const void* jones;        // [K][n_ant][4] cube precision
  const DirQ* dir;       // [K] (l, m, n-1, S)
  const double* uvw;
  const int2* bl_ant;
  const double* freq_c;
  const double* wchan;      // WEIGHTED: d phi / d(shift) = a_p wchan[c]; else a_p nu_c / c
  double2* G;
  double* gsc;
  double* loss_bl;
  int n_src, n_ant, n_chan, n_time;
  int64_t n_bl;
  double nu0_c, dnu_c;
};

__global__ void k_grad_dirs(const double* __restrict__ src, int n, DirQ* __restrict__ dir) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    double l = src[3 * k], m = src[3 * k + 1], S = src[3 * k + 2];
    double r2 = l * l + m * m;
    dir[k] = DirQ{l, m, -r2 / (1.0 + sqrt(1.0 - r2)), S};
  }
}

template <typename T>
__device__ inline typename cplx_of<T>::type load_j(const void* jones, size_t idx) {
  using C = typename cplx_of<T>::type;
  return static_cast<const C*>(jones)[idx];
}

// exp(+2 pi i phi) for channel c of source k at the current time
template <bool MIXED>
__device__ inline typename cplx_of<typename std::conditional<MIXED, float, double>::type>::type
grad_phasor(unsigned long long A, unsigned long long B, double tau, const double* freq_c, int c) {
  if constexpr (MIXED) {
    return phasor_f(q64_to_turns(A + (unsigned long long)c * B));
  } else {
    return phasor_d(tau * freq_c[c]);
  }
}

// per (source k, baseline bl): G, and the (dl, dm, dS) contributions
//   dL/dl = -4 pi S Im tr(H^lH J_i J_j^H), dL/dm likewise, dL/dS = -2 Re tr(G^H J_i J_j^H)
template <typename T>
__device__ inline void grad_store(const GradArgs& a, int k, int64_t bl, int2 ij, const double (&G)[8],
                                  const double (&Hl)[8], const double (&Hm)[8]) {
  using C = typename cplx_of<T>::type;
  M22<double2> Ji, Jj, Gm, Hlm, Hmm;
  #pragma unroll
  for (int e = 0; e < 4; ++e) {
    C p = load_j<T>(a.jones, ((size_t)k * a.n_ant + ij.x) * 4 + e);
    C q = load_j<T>(a.jones, ((size_t)k * a.n_ant + ij.y) * 4 + e);
    Ji.e[e] = make_double2(p.x, p.y); Jj.e[e] = make_double2(q.x, q.y);
    Gm.e[e] = make_double2(G[2 * e], G[2 * e + 1]);
    Hlm.e[e] = make_double2(Hl[2 * e], Hl[2 * e + 1]);
    Hmm.e[e] = make_double2(Hm[2 * e], Hm[2 * e + 1]);
    a.G[((size_t)k * a.n_bl + bl) * 4 + e] = Gm.e[e];
  }
  const double S = a.dir[k].w;
  M22<double2> P = mmul_h(Ji, Jj);                 // J_i J_j^H
  // tr(X^H Y) = sum_e conj(X_e) Y_e
  double2 tG = make_double2(0, 0), tl = make_double2(0, 0), tm = make_double2(0, 0);
  #pragma unroll
  for (int e = 0; e < 4; ++e) {
    tG = cadd(tG, cconjmul(Gm.e[e], P.e[e]));
    tl = cadd(tl, cconjmul(Hlm.e[e], P.e[e]));
    tm = cadd(tm, cconjmul(Hmm.e[e], P.e[e]));
  }
  const double four_pi = 12.566370614359172953850573533118;
  double* o = a.gsc + ((size_t)k * a.n_bl + bl) * 3;
  o[0] = -four_pi * S * tl.y;
  o[1] = -four_pi * S * tm.y;
  o[2] = -2.0 * tG.x;
}

template <bool MIXED, bool WEIGHTED>
__global__ void __launch_bounds__(kGradThreads) k_grad_sweep(GradArgs a) {
  using T = typename std::conditional<MIXED, float, double>::type;
  using C = typename cplx_of<T>::type;
  extern __shared__ __align__(16) unsigned char g_smem[];
  // layout (16-byte aligned pieces first):
  //   R tile [kGradTile][4] C | M [K][4] C | part [threads][16] T | A, B [K] u64 | tau [K] double
  C* sR = reinterpret_cast<C*>(g_smem);
  C* sM = sR + kGradTile * 4;
  T* sPart = reinterpret_cast<T*>(sM + (size_t)a.n_src * 4);
  unsigned long long* sA = reinterpret_cast<unsigned long long*>(sPart + (size_t)kGradThreads * 16);
  unsigned long long* sB = sA + a.n_src;
  double* sTau = reinterpret_cast<double*>(sB + a.n_src);
  __shared__ double s_uvw[3];
  __shared__ double s_loss[kGradThreads / 32];

  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  const int k0 = blockIdx.y * kGradChunk;
  const int kc = max(1, min(kGradChunk, a.n_src - k0));   // sources of this CTA's backward phase
  const int groups = max(1, kGradThreads / kc);
  const int my_k = threadIdx.x % kc, my_g = threadIdx.x / kc;
  const bool bw = my_g < groups && k0 + my_k < a.n_src;

  // model matrices of all sources on this baseline
  for (int k = threadIdx.x; k < a.n_src; k += blockDim.x) {
    M22<double2> Ji, Jj;
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      C p = load_j<T>(a.jones, ((size_t)k * a.n_ant + ij.x) * 4 + e);
      C q = load_j<T>(a.jones, ((size_t)k * a.n_ant + ij.y) * 4 + e);
      Ji.e[e] = make_double2(p.x, p.y); Jj.e[e] = make_double2(q.x, q.y);
    }
    M22<double2> P = mmul_h(Ji, Jj);
    const double S = a.dir[k].w;
    #pragma unroll
    for (int e = 0; e < 4; ++e) sM[(size_t)k * 4 + e] = cmk<C>(S * P.e[e].x, S * P.e[e].y);
  }
  double G[8], Hl[8], Hm[8];
  #pragma unroll
  for (int e = 0; e < 8; ++e) { G[e] = 0.0; Hl[e] = 0.0; Hm[e] = 0.0; }
  double loss = 0.0;
  double lk_n = 0.0, mk_n = 0.0;
  if (bw) {
    const DirQ d = a.dir[k0 + my_k];
    const double n = 1.0 + d.z;
    lk_n = d.x / n; mk_n = d.y / n;
  }

  for (int t = 0; t < a.n_time; ++t) {
    __syncthreads();                              // previous users of sA/sB/sTau/s_uvw done
    for (int k = threadIdx.x; k < a.n_src; k += blockDim.x) {
      SrcDir d; d.l = a.dir[k].x; d.m = a.dir[k].y; d.nm1 = a.dir[k].z; d.S = a.dir[k].w;
      double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, d);
      sTau[k] = tau;
      if (MIXED) { sA[k] = frac_q64(tau * a.nu0_c); sB[k] = frac_q64(tau * a.dnu_c); }
    }
    if (threadIdx.x < 3)
      s_uvw[threadIdx.x] = a.uvw[((size_t)t * a.n_ant + ij.x) * 3 + threadIdx.x] -
                           a.uvw[((size_t)t * a.n_ant + ij.y) * 3 + threadIdx.x];
    for (int c0 = 0; c0 < a.n_chan; c0 += kGradTile) {
      const int nc = min(kGradTile, a.n_chan - c0);
      __syncthreads();                            // tables ready; previous tile consumed
      // forward: R for each channel of the tile
      for (int cl = threadIdx.x; cl < nc; cl += blockDim.x) {
        const int c = c0 + cl;
        const C* v = static_cast<const C*>(a.vis) + (((size_t)t * a.n_bl + bl) * a.n_chan + c) * 4;
        C r[4];
        #pragma unroll
        for (int e = 0; e < 4; ++e) r[e] = v[e];
        for (int k = 0; k < a.n_src; ++k) {
          C ph = grad_phasor<MIXED>(sA[k], sB[k], sTau[k], a.freq_c, c);
          #pragma unroll
          for (int e = 0; e < 4; ++e) r[e] = csub(r[e], cmulc(sM[(size_t)k * 4 + e], ph));
        }
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          sR[cl * 4 + e] = r[e];
          loss += (double)r[e].x * r[e].x + (double)r[e].y * r[e].y;
        }
      }
      __syncthreads();
      // backward: partial H0, H1 over this thread's channel group
      if (bw) {
        const int k = k0 + my_k;
        T h0[8], h1[8];
        #pragma unroll
        for (int e = 0; e < 8; ++e) { h0[e] = T(0); h1[e] = T(0); }
        for (int cl = my_g; cl < nc; cl += groups) {
          const int c = c0 + cl;
          C ph = grad_phasor<MIXED>(sA[k], sB[k], sTau[k], a.freq_c, c);
          const T cw = WEIGHTED ? (T)a.wchan[c] : (T)c;
          #pragma unroll
          for (int e = 0; e < 4; ++e) {
            C x = cmul(sR[cl * 4 + e], ph);
            h0[2 * e] += x.x; h0[2 * e + 1] += x.y;
            h1[2 * e] += cw * x.x; h1[2 * e + 1] += cw * x.y;
          }
        }
        T* part = sPart + (size_t)threadIdx.x * 16;
        #pragma unroll
        for (int e = 0; e < 8; ++e) { part[e] = h0[e]; part[8 + e] = h1[e]; }
      }
      __syncthreads();
      if (bw && my_g == 0) {
        double H0[8], H1[8];
        #pragma unroll
        for (int e = 0; e < 8; ++e) { H0[e] = 0.0; H1[e] = 0.0; }
        for (int g = 0; g < groups; ++g) {
          const T* part = sPart + (size_t)(g * kc + my_k) * 16;
          #pragma unroll
          for (int e = 0; e < 8; ++e) { H0[e] += (double)part[e]; H1[e] += (double)part[8 + e]; }
        }
        const double wl = s_uvw[0] - s_uvw[2] * lk_n;
        const double wm = s_uvw[1] - s_uvw[2] * mk_n;
        #pragma unroll
        for (int e = 0; e < 8; ++e) {
          const double hn = WEIGHTED ? H1[e] : a.nu0_c * H0[e] + a.dnu_c * H1[e];
          G[e] += H0[e];
          Hl[e] += wl * hn;
          Hm[e] += wm * hn;
        }
      }
    }
  }
  // loss of this baseline (chunk 0 only)
  if (blockIdx.y == 0) {
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = loss;
  }
  __syncthreads();
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kGradThreads / 32; ++w) s += s_loss[w];
    a.loss_bl[bl] = s;
  }
  if (bw && my_g == 0) grad_store<T>(a, k0 + my_k, bl, ij, G, Hl, Hm);
}

// exp(+2 pi i x) of a Q0.64 phase x rounded to Q0.32 (the hardware sin/cos,
// as the per-sample sweep uses for every sample)
__device__ inline float2 grad_phasor_tab(unsigned long long ph) { return phasor_f(q64_to_turns(ph)); }

// The FP32 adjoint with factorised phasors.  Within a tile of kGfTile channels
// starting at c0, channel c = c0 + 16 q + r has
//   exp(+2 pi i phi_k(c)) = T1_k[q] T2_k[r],
//   T1_k[q] = exp(2 pi i (A_k + (c0 + 16 q) B_k)),  T2_k[r] = exp(2 pi i r B_k)
// (A_k, B_k the Q0.64 phase at channel 0 and its per-channel step), so both
// halves of the sweep multiply table entries instead of evaluating sin/cos:
//   forward   R(c) = V(c) - sum_k M_k conj(T1_k[q] T2_k[r])   (thread = channel)
//   backward  sum_c R(c) P_k(c) = sum_q T1_k[q] s_q,  s_q = sum_r R(16q + r) T2_k[r]
//             sum_c c R(c) P_k(c) = sum_q T1_k[q] [(c0 + 16q - 1) s_q + a_q]
//             with a_q = sum_r (r + 1) x_r, x_r = R(16q + r) T2_k[r], built as
//             the running sum of the suffix sums while r runs down from 15
//             (thread = (source, group of q)).
// Tables are [q or r][kp] with kp = 1 (mod 16): the forward's 16 distinct r of
// a warp and the backward's consecutive sources fall on distinct banks.  The
// per-(source, baseline) outputs are those of k_grad_sweep.
constexpr int kGfThreads = 384;
constexpr int kGfTile = 384;          // channels per tile: one per thread in the forward
constexpr int kGfNq = kGfTile / 16;
constexpr int kGfChunk = kGfThreads;  // sources per CTA in the backward

__host__ __device__ inline int grad_fac_kp(int n_src) { return ((n_src + 15) / 16) * 16 + 1; }

inline size_t grad_fac_smem_bytes(int n_src) {
  const size_t kp = (size_t)grad_fac_kp(n_src);
  return (size_t)kGfTile * 4 * sizeof(float2)           // R
         + (size_t)n_src * 4 * sizeof(float2)            // M
         + (size_t)kGfThreads * 16 * sizeof(float)        // backward partials
         + (size_t)(kGfNq + 16) * kp * sizeof(float2)     // T1, T2
         + (size_t)n_src * 2 * sizeof(unsigned long long) // A, B
         + (size_t)kGfTile * sizeof(float);               // channel weights of the tile
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kGfThreads, 1) k_grad_sweep_fac(GradArgs a) {
  extern __shared__ __align__(16) unsigned char g_smem[];
  const int K = a.n_src;
  const int kp = grad_fac_kp(K);
  float2* sR = reinterpret_cast<float2*>(g_smem);                  // [kGfTile][4]
  float2* sM = sR + kGfTile * 4;                                   // [K][4]
  float* sPart = reinterpret_cast<float*>(sM + (size_t)K * 4);     // [16][threads]
  float2* sT1 = reinterpret_cast<float2*>(sPart + (size_t)kGfThreads * 16);   // [kGfNq][kp]
  float2* sT2 = sT1 + (size_t)kGfNq * kp;                          // [16][kp]
  unsigned long long* sA = reinterpret_cast<unsigned long long*>(sT2 + (size_t)16 * kp);
  unsigned long long* sB = sA + K;
  float* sW = reinterpret_cast<float*>(sB + K);                    // [kGfTile]
  __shared__ double s_uvw[3];
  __shared__ double s_loss[kGfThreads / 32];

  const int tid = threadIdx.x;
  const int64_t bl = blockIdx.x;
  const int2 ij = a.bl_ant[bl];
  const int k0 = blockIdx.y * kGfChunk;
  const int kc = max(1, min(kGfChunk, K - k0));            // sources of this CTA's backward phase
  const int groups = max(1, min(kGfNq, kGfThreads / kc));
  const int my_k = tid % kc, my_g = tid / kc;
  const bool bw = my_g < groups && k0 + my_k < K;
  const int kb = k0 + my_k;                                 // source of the backward item
  const int qa = my_g * kGfNq / groups, qb = (my_g + 1) * kGfNq / groups;

  for (int k = tid; k < K; k += kGfThreads) {
    M22<double2> Ji, Jj;
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      float2 p = load_j<float>(a.jones, ((size_t)k * a.n_ant + ij.x) * 4 + e);
      float2 q = load_j<float>(a.jones, ((size_t)k * a.n_ant + ij.y) * 4 + e);
      Ji.e[e] = make_double2(p.x, p.y); Jj.e[e] = make_double2(q.x, q.y);
    }
    M22<double2> P = mmul_h(Ji, Jj);
    const double S = a.dir[k].w;
    #pragma unroll
    for (int e = 0; e < 4; ++e) sM[(size_t)k * 4 + e] = make_float2((float)(S * P.e[e].x), (float)(S * P.e[e].y));
  }
  // per-(source, baseline) sums over tiles, compensated FP32 (the FP64 pipe
  // is far slower than FP32 on this part; 2 x n_time terms per sum)
  float G[8], Hl[8], Hm[8], Gc[8], Hlc[8], Hmc[8];
  #pragma unroll
  for (int e = 0; e < 8; ++e) { G[e] = Hl[e] = Hm[e] = Gc[e] = Hlc[e] = Hmc[e] = 0.f; }
  double loss = 0.0;
  double lk_n = 0.0, mk_n = 0.0;
  if (bw) {
    const DirQ d = a.dir[kb];
    const double n = 1.0 + d.z;
    lk_n = d.x / n; mk_n = d.y / n;
  }

  for (int t = 0; t < a.n_time; ++t) {
    __syncthreads();                              // previous users of sA/sB/sT2/s_uvw done
    for (int k = tid; k < K; k += kGfThreads) {
      SrcDir d; d.l = a.dir[k].x; d.m = a.dir[k].y; d.nm1 = a.dir[k].z; d.S = a.dir[k].w;
      const double tau = delay_m(a.uvw, a.n_ant, t, ij.x, ij.y, d);
      sA[k] = frac_q64(tau * a.nu0_c); sB[k] = frac_q64(tau * a.dnu_c);
    }
    if (tid < 3)
      s_uvw[tid] = a.uvw[((size_t)t * a.n_ant + ij.x) * 3 + tid] - a.uvw[((size_t)t * a.n_ant + ij.y) * 3 + tid];
    __syncthreads();
    for (int k = tid; k < K; k += kGfThreads) {
      const unsigned long long b = sB[k];
      #pragma unroll 4
      for (int r = 0; r < 16; ++r) sT2[(size_t)r * kp + k] = grad_phasor_tab((unsigned long long)r * b);
    }
    for (int c0 = 0; c0 < a.n_chan; c0 += kGfTile) {
      const int nc = min(kGfTile, a.n_chan - c0);
      const int nq = (nc + 15) / 16;
      for (int k = tid; k < K; k += kGfThreads) {
        const unsigned long long b = sB[k], a0 = sA[k] + (unsigned long long)c0 * b;
        #pragma unroll 4
        for (int q = 0; q < nq; ++q) sT1[(size_t)q * kp + k] = grad_phasor_tab(a0 + (unsigned long long)(16 * q) * b);
      }
      if (WEIGHTED)
        for (int i = tid; i < nc; i += kGfThreads) sW[i] = (float)a.wchan[c0 + i];
      __syncthreads();
      // forward: R at channel c0 + tid, all sources subtracted
      if (tid < nc) {
        const int q = tid >> 4, r = tid & 15;
        const float4* v = reinterpret_cast<const float4*>(
            static_cast<const float2*>(a.vis) + (((size_t)t * a.n_bl + bl) * a.n_chan + c0 + tid) * 4);
        const float4 v0 = v[0], v1 = v[1];
        float ax[4] = {v0.x, v0.z, v1.x, v1.z}, ay[4] = {v0.y, v0.w, v1.y, v1.w};
        const float2* t1p = sT1 + (size_t)q * kp;
        const float2* t2p = sT2 + (size_t)r * kp;
        #pragma unroll 4
        for (int k = 0; k < K; ++k) {
          const float2 t1 = t1p[k], t2 = t2p[k];
          const float px = fmaf(t1.x, t2.x, -t1.y * t2.y);
          const float py = fmaf(t1.x, t2.y, t1.y * t2.x);
          const float4 m01 = reinterpret_cast<const float4*>(sM)[2 * k];
          const float4 m23 = reinterpret_cast<const float4*>(sM)[2 * k + 1];
          const float mx[4] = {m01.x, m01.z, m23.x, m23.z}, my[4] = {m01.y, m01.w, m23.y, m23.w};
          #pragma unroll
          for (int e = 0; e < 4; ++e) {          // R -= M conj(P)
            ax[e] = fmaf(-mx[e], px, fmaf(-my[e], py, ax[e]));
            ay[e] = fmaf(-my[e], px, fmaf(mx[e], py, ay[e]));
          }
        }
        float4* o = reinterpret_cast<float4*>(sR + (size_t)tid * 4);
        o[0] = make_float4(ax[0], ay[0], ax[1], ay[1]);
        o[1] = make_float4(ax[2], ay[2], ax[3], ay[3]);
        float l2 = 0.f;
        #pragma unroll
        for (int e = 0; e < 4; ++e) l2 = fmaf(ax[e], ax[e], fmaf(ay[e], ay[e], l2));
        loss += (double)l2;
      }
      __syncthreads();
      // backward: this thread's source over its q groups
      if (bw) {
        float y0[8], y1[8];
        #pragma unroll
        for (int e = 0; e < 8; ++e) { y0[e] = 0.f; y1[e] = 0.f; }
        for (int q = qa; q < min(qb, nq); ++q) {
          const int rv = min(16, nc - 16 * q);
          float s0[8], s1[8];
          #pragma unroll
          for (int e = 0; e < 8; ++e) { s0[e] = 0.f; s1[e] = 0.f; }
          auto step = [&](int r) {
            const int cl = 16 * q + r;
            const float4 ra = reinterpret_cast<const float4*>(sR)[2 * cl];
            const float4 rb = reinterpret_cast<const float4*>(sR)[2 * cl + 1];
            const float rx[4] = {ra.x, ra.z, rb.x, rb.z}, ry[4] = {ra.y, ra.w, rb.y, rb.w};
            const float2 t2 = sT2[(size_t)r * kp + kb];
            if (WEIGHTED) {
              const float w = sW[cl];
              #pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float xr = fmaf(rx[e], t2.x, -ry[e] * t2.y);
                const float xi = fmaf(rx[e], t2.y, ry[e] * t2.x);
                s0[2 * e] += xr; s0[2 * e + 1] += xi;
                s1[2 * e] = fmaf(w, xr, s1[2 * e]); s1[2 * e + 1] = fmaf(w, xi, s1[2 * e + 1]);
              }
            } else {
              #pragma unroll
              for (int e = 0; e < 4; ++e) {
                s0[2 * e] = fmaf(rx[e], t2.x, fmaf(-ry[e], t2.y, s0[2 * e]));
                s0[2 * e + 1] = fmaf(rx[e], t2.y, fmaf(ry[e], t2.x, s0[2 * e + 1]));
              }
              #pragma unroll
              for (int e = 0; e < 8; ++e) s1[e] += s0[e];
            }
          };
          if (rv == 16) {
            #pragma unroll
            for (int r = 15; r >= 0; --r) step(r);
          } else {
            for (int r = rv - 1; r >= 0; --r) step(r);
          }
          const float2 t1 = sT1[(size_t)q * kp + kb];
          const float cw = (float)(c0 + 16 * q - 1);
          #pragma unroll
          for (int e = 0; e < 4; ++e) {
            y0[2 * e] = fmaf(t1.x, s0[2 * e], fmaf(-t1.y, s0[2 * e + 1], y0[2 * e]));
            y0[2 * e + 1] = fmaf(t1.x, s0[2 * e + 1], fmaf(t1.y, s0[2 * e], y0[2 * e + 1]));
            // unweighted: sum_r (c0 + 16q + r) x_r = (c0 + 16q - 1) s0 + sum_r (r + 1) x_r
            const float zr = WEIGHTED ? s1[2 * e] : fmaf(cw, s0[2 * e], s1[2 * e]);
            const float zi = WEIGHTED ? s1[2 * e + 1] : fmaf(cw, s0[2 * e + 1], s1[2 * e + 1]);
            y1[2 * e] = fmaf(t1.x, zr, fmaf(-t1.y, zi, y1[2 * e]));
            y1[2 * e + 1] = fmaf(t1.x, zi, fmaf(t1.y, zr, y1[2 * e + 1]));
          }
        }
        #pragma unroll
        for (int e = 0; e < 8; ++e) {
          sPart[e * kGfThreads + tid] = y0[e];
          sPart[(8 + e) * kGfThreads + tid] = y1[e];
        }
      }
      __syncthreads();
      if (bw && my_g == 0) {
        float H0[8], H1[8];
        #pragma unroll
        for (int e = 0; e < 8; ++e) { H0[e] = 0.f; H1[e] = 0.f; }
        for (int g = 0; g < groups; ++g) {
          const float* part = sPart + g * kc + my_k;
          #pragma unroll
          for (int e = 0; e < 8; ++e) { H0[e] += part[e * kGfThreads]; H1[e] += part[(8 + e) * kGfThreads]; }
        }
        const float wl = (float)(s_uvw[0] - s_uvw[2] * lk_n);
        const float wm = (float)(s_uvw[1] - s_uvw[2] * mk_n);
        const float nu0 = (float)a.nu0_c, dnu = (float)a.dnu_c;
        #pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float hn = WEIGHTED ? H1[e] : fmaf(nu0, H0[e], dnu * H1[e]);
          kahan_add(G[e], Gc[e], H0[e]);
          kahan_add(Hl[e], Hlc[e], wl * hn);
          kahan_add(Hm[e], Hmc[e], wm * hn);
        }
      }
    }
  }
  if (blockIdx.y == 0) {
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0) s_loss[tid >> 5] = loss;
  }
  __syncthreads();
  if (blockIdx.y == 0 && tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kGfThreads / 32; ++w) s += s_loss[w];
    a.loss_bl[bl] = s;
  }
  if (bw && my_g == 0) {
    double Gd[8], Hld[8], Hmd[8];
    #pragma unroll
    for (int e = 0; e < 8; ++e) {
      Gd[e] = (double)G[e] - (double)Gc[e];
      Hld[e] = (double)Hl[e] - (double)Hlc[e];
      Hmd[e] = (double)Hm[e] - (double)Hmc[e];
    }
    grad_store<float>(a, kb, bl, ij, Gd, Hld, Hmd);
  }
}

// dL/dJ for antenna p of source k: -2 S [sum_{q>p} G(pq) J_q + sum_{q<p} G(qp)^H J_q]
template <bool MIXED>
__global__ void __launch_bounds__(128) k_grad_jones(const double2* __restrict__ G,
                                                    const void* __restrict__ jones,
                                                    const DirQ* __restrict__ dir,
                                                    void* __restrict__ gJ, int n_ant, int64_t n_bl) {
  using T = typename std::conditional<MIXED, float, double>::type;
  using C = typename cplx_of<T>::type;
  __shared__ double s_red[4 * 8];
  const int p = blockIdx.x, k = blockIdx.y;
  double acc[8];
  #pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = 0.0;
  const double2* Gk = G + (size_t)k * n_bl * 4;
  for (int q = threadIdx.x; q < n_ant; q += 128) {
    if (q == p) continue;
    double2 g[4];
    if (p < q) {
      const double2* s = Gk + bl_index(n_ant, p, q) * 4;
      g[0] = s[0]; g[1] = s[1]; g[2] = s[2]; g[3] = s[3];
    } else {
      const double2* s = Gk + bl_index(n_ant, q, p) * 4;
      g[0] = cconj(s[0]); g[1] = cconj(s[2]); g[2] = cconj(s[1]); g[3] = cconj(s[3]);
    }
    double2 J[4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      C v = load_j<T>(jones, ((size_t)k * n_ant + q) * 4 + e);
      J[e] = make_double2(v.x, v.y);
    }
    double2 r0 = cadd(cmul(g[0], J[0]), cmul(g[1], J[2]));
    double2 r1 = cadd(cmul(g[0], J[1]), cmul(g[1], J[3]));
    double2 r2 = cadd(cmul(g[2], J[0]), cmul(g[3], J[2]));
    double2 r3 = cadd(cmul(g[2], J[1]), cmul(g[3], J[3]));
    acc[0] += r0.x; acc[1] += r0.y; acc[2] += r1.x; acc[3] += r1.y;
    acc[4] += r2.x; acc[5] += r2.y; acc[6] += r3.x; acc[7] += r3.y;
  }
  #pragma unroll
  for (int e = 0; e < 8; ++e)
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
  if ((threadIdx.x & 31) == 0)
    #pragma unroll
    for (int e = 0; e < 8; ++e) s_red[(threadIdx.x >> 5) * 8 + e] = acc[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    const double f = -2.0 * dir[k].w;
    C* out = static_cast<C*>(gJ) + ((size_t)k * n_ant + p) * 4;
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      double re = 0.0, im = 0.0;
      for (int w = 0; w < 4; ++w) { re += s_red[w * 8 + 2 * e]; im += s_red[w * 8 + 2 * e + 1]; }
      out[e] = cmk<C>(f * re, f * im);
    }
  }
}

// per-source (dl, dm, dS) and the loss, summed over baselines in a fixed order
__global__ void __launch_bounds__(256) k_grad_sum(const double* __restrict__ v, int64_t n, int stride,
                                                  int width, double* __restrict__ out) {
  __shared__ double s[256 * 3];
  const double* base = v + (size_t)blockIdx.x * n * stride;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += 256)
    for (int w = 0; w < width; ++w) acc[w] += base[i * stride + w];
  for (int w = 0; w < width; ++w) s[w * 256 + threadIdx.x] = acc[w];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int w = 0; w < width; ++w) s[w * 256 + threadIdx.x] += s[w * 256 + threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int w = 0; w < width; ++w) out[(size_t)blockIdx.x * width + w] = s[w * 256];
}

inline void grad_free(GradWorkspace& w) {
  if (w.G) cudaFree(w.G);
  if (w.gsc) cudaFree(w.gsc);
  if (w.loss_bl) cudaFree(w.loss_bl);
  if (w.dir) cudaFree(w.dir);
  if (w.wchan) cudaFree(w.wchan);
  w = GradWorkspace();
}

inline int grad_fail(std::string& err, cudaError_t e, const char* what) {
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? -2 : -3;
}

// Allocates its workspace on first use (G and per-baseline terms for up to
// max_src sources: (64 + 24) bytes per source and baseline) and keeps it.
inline int grad_prepare(GradWorkspace& w, int n_src, const double* src, int64_t n_bl, int max_src,
                        cudaStream_t s, std::string& err) {
  cudaError_t e;
  if (!w.loss_bl) {
    w.cap_src = max_src; w.n_bl = n_bl;
    if ((e = cudaMalloc(&w.G, (size_t)max_src * n_bl * 4 * sizeof(double2))) != cudaSuccess ||
        (e = cudaMalloc(&w.gsc, (size_t)max_src * n_bl * 3 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&w.loss_bl, (size_t)n_bl * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&w.dir, (size_t)max_src * sizeof(DirQ))) != cudaSuccess) {
      int rc = grad_fail(err, e, "cudaMalloc(gradient workspace)");
      grad_free(w);
      return rc;
    }
  }
  if (n_src > 0) k_grad_dirs<<<(n_src + 127) / 128, 128, 0, s>>>(src, n_src, w.dir);
  return 0;
}

inline size_t grad_smem_bytes(bool mixed, int n_src) {
  const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
  const size_t tsz = mixed ? sizeof(float) : sizeof(double);
  return (size_t)kGradTile * 4 * esz + (size_t)n_src * (2 * 8 + 8 + 4 * esz) +
         (size_t)kGradThreads * 16 * tsz;
}

// the fused loss + adjoint sweep (one launch)
inline int grad_sweep(GradWorkspace& w, bool mixed, const void* vis, int n_src, const void* jones,
                      const double* uvw, const int2* bl_ant, const double* freq_c, int n_ant,
                      int n_chan, int n_time, int64_t n_bl, double nu0_c, double dnu_c,
                      cudaStream_t s, std::string& err, const double* wchan = nullptr,
                      bool direct = false) {
  cudaError_t e;
  GradArgs a;
  a.vis = vis; a.jones = jones; a.dir = w.dir; a.uvw = uvw; a.bl_ant = bl_ant; a.freq_c = freq_c;
  a.wchan = wchan;
  a.G = w.G; a.gsc = w.gsc; a.loss_bl = w.loss_bl;
  a.n_src = n_src; a.n_ant = n_ant; a.n_chan = n_chan; a.n_time = n_time; a.n_bl = n_bl;
  a.nu0_c = nu0_c; a.dnu_c = dnu_c;
  const size_t smem_fac = grad_fac_smem_bytes(n_src);
  const bool fac = mixed && smem_fac <= kGradMaxSmem && !direct;
  const size_t smem = fac ? smem_fac : grad_smem_bytes(mixed, n_src);
  const int chunk = fac ? kGfChunk : kGradChunk;
  const int chunks = n_src > 0 ? (n_src + chunk - 1) / chunk : 1;
  if (smem > kGradMaxSmem) {
    err = "too many sources for the gradient kernel's shared memory";
    return -1;
  }
  const dim3 grid((unsigned)n_bl, (unsigned)chunks);
  auto launch = [&](auto kernel) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r == cudaSuccess) kernel<<<grid, fac ? kGfThreads : kGradThreads, smem, s>>>(a);
    return r;
  };
  if (fac) e = wchan ? launch(k_grad_sweep_fac<true>) : launch(k_grad_sweep_fac<false>);
  else if (mixed) e = wchan ? launch(k_grad_sweep<true, true>) : launch(k_grad_sweep<true, false>);
  else e = wchan ? launch(k_grad_sweep<false, true>) : launch(k_grad_sweep<false, false>);
  if (e != cudaSuccess) return grad_fail(err, e, "cudaFuncSetAttribute");
  if ((e = cudaGetLastError()) != cudaSuccess) return grad_fail(err, e, "gradient sweep launch");
  return 0;
}

// per-antenna dL/dJ, per-source (dl, dm, dS) and the loss; returns launches made
inline int grad_reduce(GradWorkspace& w, bool mixed, int n_src, const void* jones, double* loss,
                       void* gJ, double* gsrc, int n_ant, int64_t n_bl, cudaStream_t s,
                       std::string& err, int* launches) {
  cudaError_t e;
  int n = 0;
  if (n_src > 0 && gJ) {
    const dim3 gj((unsigned)n_ant, (unsigned)n_src);
    if (mixed) k_grad_jones<true><<<gj, 128, 0, s>>>(w.G, jones, w.dir, gJ, n_ant, n_bl);
    else k_grad_jones<false><<<gj, 128, 0, s>>>(w.G, jones, w.dir, gJ, n_ant, n_bl);
    ++n;
  }
  if (n_src > 0 && gsrc) { k_grad_sum<<<n_src, 256, 0, s>>>(w.gsc, n_bl, 3, 3, gsrc); ++n; }
  k_grad_sum<<<1, 256, 0, s>>>(w.loss_bl, n_bl, 1, 1, loss);
  ++n;
  *launches = n;
  if ((e = cudaGetLastError()) != cudaSuccess) return grad_fail(err, e, "gradient reduction launch");
  return 0;
}

}  // namespace rts
