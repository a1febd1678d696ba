// Blocked peel pass on the tensor cores: the same pass as k_block_pass
// (subtract the solved sources of block b, average the directions of block
// b+1), with both contractions as TF32 MMAs.
//
// Phasors factor per 16-channel tile q: with the fixed-point phases,
//   P_k(16 q + r) = T1_k[q] T2_k[r],  T1_k[q] = exp(2 pi i (A + 16 q B)),
//   T2_k[r] = exp(2 pi i r B),  r = 0..15,
// so for one baseline and time step
//   subtraction  R(16q + r, e) -= sum_k conj(T2_k[r]) W_k(q, e),  W = conj(T1_k[q]) M_k(e)
//   average      A_k(e) += sum_q T1_k[q] G_k(q, e),  G_k(q, e) = sum_r T2_k[r] R(16q + r, e).
// Both inner sums are GEMMs whose A operand is built from T2 alone: the same
// for every tile q, so it is split for TF32 once per time step and read from
// shared memory in fragment order.  Per tile the subtraction forms only its
// small B operand W (8 sources x 4 entries per k-pair, a per-lane factor
// 1 or -i picks the real or imaginary part), and the average only scales the
// 16-channel sums G by T1 in FP32.
//
// Real forms.  Subtraction (m16n8k8, rows = r, k = 8 sources, columns = 2 e +
// part): the k-step on re(T2) takes B = re(W'), the k-step on im(T2) takes
// B = im(W'), W' = W for the real part and -i W for the imaginary part.
// Average: rows g and g + 8 of the A operand are re and im of T2 of source
// 8 m + g, k = 8 channels, B = the residual; G = (c0 - c3, c1 + c2).
//
// TF32 keeps 11 significand bits, so each operand is split x = hi + lo (hi =
// TF32 rounding, lo = the exact remainder) and a product is ahi bhi + ahi blo
// + alo bhi (the alo blo term is below 2^-22 relative): FP32-level accuracy at
// three MMAs per product.  The tensor cores' FP32 accumulation does not round
// to nearest, so its error grows with the length of an accumulation chain:
// every chain here is six MMAs long and starts from zero (cross terms first),
// and the chains are combined with round-to-nearest FP32 arithmetic.
//
// One CTA (16 warps) per baseline, one CTA per SM; the FP32 strip of time
// t + 1 is copied into shared memory (cp.async) while time t is processed.
// The residual's (hi, lo) copy uses an XOR swizzle of its 8 columns so that
// the averaging GEMM's operand loads are free of bank conflicts.
// Limits: at most 64 sources per role, n_chan <= kTcMaxChan (shared memory).
#pragma once
#include "block_kernels.cuh"

namespace rts {

constexpr int kTcThreads = 512;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTcSrc = 64;                      // sources per role (subtracted / averaged)
constexpr int kTcRtMax = 4;                     // 16-channel tiles per warp (subtraction)
constexpr int kTcMaxChan = 960;                 // shared memory limit (fits kTcRtMax)

// dynamic shared memory of k_block_pass_tc for n_chan channels
inline size_t tc_pass_smem(int n_chan) {
  const size_t nq = (size_t)(n_chan + 15) / 16, n16 = 16 * nq;
  return 2 * n16 * 8 * sizeof(float)          // FP32 strip, two buffers
         + n16 * 8 * sizeof(float2)           // (hi, lo) of the residual, swizzled
         + nq * 2 * kTcSrc * sizeof(float2)   // T1
         + 8 * 32 * 4 * sizeof(float4)        // subtraction A fragments (T2), split
         + 8 * 2 * 32 * 2 * sizeof(float4)    // average A fragments (T2), split
         + 8 * 32 * sizeof(float4)            // subtraction model entries, per lane
         + 2 * kTcSrc * sizeof(PhaseAB)       // phases of the time step
         + 2 * kTcSrc * 8 * sizeof(double);   // FP64 averages per channel half
}

// column swizzle of the residual copy: columns 4..7 and 0..3 trade places in
// rows whose bit 1 is set
__device__ __forceinline__ int rhl_index(int c, int col) { return c * 8 + (col ^ (((c >> 1) & 1) << 2)); }

__device__ __forceinline__ unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo exactly; hi is a TF32 value, lo is passed to the MMA as it is
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_rna(x);
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// (hi, lo) with lo also rounded to TF32 (stored operands)
__device__ __forceinline__ float2 split_store(float x) {
  const unsigned hi = tf32_rna(x);
  return make_float2(__uint_as_float(hi), __uint_as_float(tf32_rna(x - __uint_as_float(hi))));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <bool SUB, bool ACC>
__global__ void __launch_bounds__(kTcThreads, 1) k_block_pass_tc(BlockPassArgs a, int bk) {
  const int nq = (a.n_chan + 15) >> 4, n16 = nq << 4;
  extern __shared__ __align__(16) unsigned char tc_smem[];
  float* strip0 = reinterpret_cast<float*>(tc_smem);                    // [2][n16][8]
  float2* rhl = reinterpret_cast<float2*>(strip0 + 2 * n16 * 8);         // [n16][8] swizzled
  float2* t1 = rhl + (size_t)n16 * 8;                                    // [nq][128]
  float4* as_fr = reinterpret_cast<float4*>(t1 + (size_t)nq * 2 * kTcSrc);   // [8 kp][4][32 lanes]
  float4* aa_fr = as_fr + 8 * 32 * 4;                                    // [8 m][2 j][2][32 lanes]
  float4* mq = aa_fr + 8 * 2 * 32 * 2;                                   // [8 kp][32]
  PhaseAB* ph = reinterpret_cast<PhaseAB*>(mq + 8 * 32);                 // [128]
  double* red = reinterpret_cast<double*>(ph + 2 * kTcSrc);              // [2][64][4][2]

  const int64_t bl = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;

  // zero the padding channels of both strip buffers (copies never write them)
  for (int q = a.n_chan * 8 + tid; q < n16 * 8; q += kTcThreads) {
    strip0[q] = 0.f;
    strip0[n16 * 8 + q] = 0.f;
  }
  if (ACC)
    for (int q = tid; q < 2 * kTcSrc * 8; q += kTcThreads) red[q] = 0.0;
  // model entries of the subtraction, per (k-pair, lane): sources 8 kp + tq and
  // 8 kp + tq + 4, entry e = g / 2, times -i for the odd (imaginary) columns
  if (SUB && tid < 8 * 32) {
    const int kp = tid >> 5, ln = tid & 31, gg = ln >> 2, tt = ln & 3;
    const int e = gg >> 1, part = gg & 1;
    float2 mm[2];
    #pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int s = 8 * kp + tt + 4 * u;
      const float2 m = s < a.n_sub ? a.M_sub[((size_t)s * a.n_bl + bl) * 4 + e] : make_float2(0.f, 0.f);
      mm[u] = part ? make_float2(m.y, -m.x) : m;
    }
    mq[kp * 32 + ln] = make_float4(mm[0].x, mm[0].y, mm[1].x, mm[1].y);
  }
  auto prefetch = [&](int t, int buf) {
    const float4* gsrc = a.src + ((size_t)t * a.n_bl + bl) * a.n_chan * 2;
    float4* sdst = reinterpret_cast<float4*>(strip0 + (size_t)buf * n16 * 8);
    for (int q = tid; q < a.n_chan * 2; q += kTcThreads) cp_async16(sdst + q, gsrc + q);
  };
  prefetch(0, 0);
  cp_async_commit();

  const int s_lo = SUB ? 0 : kTcSrc, ncol = (ACC ? 2 * kTcSrc : kTcSrc) - s_lo;   // T1 columns in use
  const int n_t1 = nq * ncol, n_as = SUB ? 8 * 32 : 0, n_aa = ACC ? 8 * 2 * 32 : 0;
  for (int t = 0; t < a.n_time; ++t) {
    const int buf = t & 1;
    if (tid < 2 * kTcSrc) {
      const bool sub = tid < kTcSrc;
      const int k = sub ? tid : tid - kTcSrc;
      PhaseAB p;
      p.a = 0; p.b = 0;
      if (sub ? (SUB && k < a.n_sub) : (ACC && k < a.n_acc))
        p = (sub ? a.ph_sub : a.ph_acc)[((size_t)bl * a.n_time + t) * bk + k];
      ph[tid] = p;
    }
    if (t + 1 < a.n_time) prefetch(t + 1, buf ^ 1);
    cp_async_commit();                       // one group per step (possibly empty)
    __syncthreads();                         // phases ready
    // tables of this time step: T1, and the split T2 operands in fragment order
    for (int it = tid; it < n_t1 + n_as + n_aa; it += kTcThreads) {
      if (it < n_t1) {
        const int s = s_lo + it % ncol, q = it / ncol;
        const PhaseAB p = ph[s];
        t1[q * 2 * kTcSrc + s] = phasor_hw(p.a + (unsigned long long)(16 * q) * p.b);
      } else if (it < n_t1 + n_as) {
        const int j = it - n_t1, kp = j >> 5, ln = j & 31, gg = ln >> 2, tt = ln & 3;
        const unsigned long long b0 = ph[8 * kp + tt].b, b1 = ph[8 * kp + tt + 4].b;
        const float2 p00 = phasor_hw((unsigned long long)gg * b0), p10 = phasor_hw((unsigned long long)(gg + 8) * b0);
        const float2 p01 = phasor_hw((unsigned long long)gg * b1), p11 = phasor_hw((unsigned long long)(gg + 8) * b1);
        const float2 r0 = split_store(p00.x), r1 = split_store(p10.x), r2 = split_store(p01.x), r3 = split_store(p11.x);
        const float2 i0 = split_store(p00.y), i1 = split_store(p10.y), i2 = split_store(p01.y), i3 = split_store(p11.y);
        float4* f = as_fr + kp * 4 * 32 + ln;
        f[0] = make_float4(r0.x, r1.x, r2.x, r3.x);
        f[32] = make_float4(r0.y, r1.y, r2.y, r3.y);
        f[64] = make_float4(i0.x, i1.x, i2.x, i3.x);
        f[96] = make_float4(i0.y, i1.y, i2.y, i3.y);
      } else {
        const int j = it - n_t1 - n_as, m = j >> 6, jj = (j >> 5) & 1, ln = j & 31, gg = ln >> 2, tt = ln & 3;
        const unsigned long long b = ph[kTcSrc + 8 * m + gg].b;
        const float2 p0 = phasor_hw((unsigned long long)(8 * jj + tt) * b);
        const float2 p1 = phasor_hw((unsigned long long)(8 * jj + tt + 4) * b);
        const float2 x0 = split_store(p0.x), x1 = split_store(p0.y), x2 = split_store(p1.x), x3 = split_store(p1.y);
        float4* f = aa_fr + (m * 2 + jj) * 2 * 32 + ln;
        f[0] = make_float4(x0.x, x1.x, x2.x, x3.x);
        f[32] = make_float4(x0.y, x1.y, x2.y, x3.y);
      }
    }
    cp_async_wait1();                        // this step's strip has landed (the next may be in flight)
    __syncthreads();                         // tables and strip ready
    const float* strip = strip0 + (size_t)buf * n16 * 8;

    if (SUB) {
      float D[kTcRtMax][4];
      #pragma unroll
      for (int i = 0; i < kTcRtMax; ++i) D[i][0] = D[i][1] = D[i][2] = D[i][3] = 0.f;
      const int kp_end = (a.n_sub + 7) >> 3;
      for (int kp = 0; kp < kp_end; ++kp) {
        const int s0 = 8 * kp + tq, s1 = s0 + 4;
        const float4* f = as_fr + kp * 4 * 32 + lane;
        const float4 rh = f[0], rl = f[32], ih = f[64], il = f[96];
        const float4 m01 = mq[kp * 32 + lane];
        // W' = conj(T1) M' for every tile of this warp, split; then the six MMAs
        // of each tile, interleaved across tiles (independent chains in flight)
        unsigned bh[kTcRtMax][2], bo[kTcRtMax][2], ch[kTcRtMax][2], co[kTcRtMax][2];
        #pragma unroll
        for (int i = 0; i < kTcRtMax; ++i) {
          const int q = min(warp + kTcWarps * i, nq - 1);
          const float2 w0 = t1[q * 2 * kTcSrc + s0], w1 = t1[q * 2 * kTcSrc + s1];
          const float wr0 = fmaf(w0.x, m01.x, w0.y * m01.y), wi0 = fmaf(w0.x, m01.y, -w0.y * m01.x);
          const float wr1 = fmaf(w1.x, m01.z, w1.y * m01.w), wi1 = fmaf(w1.x, m01.w, -w1.y * m01.z);
          split_tf32(wr0, bh[i][0], bo[i][0]); split_tf32(wr1, bh[i][1], bo[i][1]);
          split_tf32(wi0, ch[i][0], co[i][0]); split_tf32(wi1, ch[i][1], co[i][1]);
        }
        float E[kTcRtMax][4];
        #pragma unroll
        for (int i = 0; i < kTcRtMax; ++i) E[i][0] = E[i][1] = E[i][2] = E[i][3] = 0.f;
        const unsigned Rh[4] = {__float_as_uint(rh.x), __float_as_uint(rh.y), __float_as_uint(rh.z), __float_as_uint(rh.w)};
        const unsigned Rl[4] = {__float_as_uint(rl.x), __float_as_uint(rl.y), __float_as_uint(rl.z), __float_as_uint(rl.w)};
        const unsigned Ih[4] = {__float_as_uint(ih.x), __float_as_uint(ih.y), __float_as_uint(ih.z), __float_as_uint(ih.w)};
        const unsigned Il[4] = {__float_as_uint(il.x), __float_as_uint(il.y), __float_as_uint(il.z), __float_as_uint(il.w)};
#define RTS_TC_ALL(A, B0, B1)                                                        \
        _Pragma("unroll") for (int i = 0; i < kTcRtMax; ++i)                         \
          if (warp + kTcWarps * i < nq) mma_tf32(E[i], A[0], A[1], A[2], A[3], B0, B1);
        RTS_TC_ALL(Rl, bh[i][0], bh[i][1])
        RTS_TC_ALL(Rh, bo[i][0], bo[i][1])
        RTS_TC_ALL(Il, ch[i][0], ch[i][1])
        RTS_TC_ALL(Ih, co[i][0], co[i][1])
        RTS_TC_ALL(Rh, bh[i][0], bh[i][1])
        RTS_TC_ALL(Ih, ch[i][0], ch[i][1])
#undef RTS_TC_ALL
        #pragma unroll
        for (int i = 0; i < kTcRtMax; ++i) {
          D[i][0] += E[i][0]; D[i][1] += E[i][1]; D[i][2] += E[i][2]; D[i][3] += E[i][3];
        }
      }
      // residual = strip - model: to HBM, and split for the averaging GEMM
      float2* dst = reinterpret_cast<float2*>(a.dst + ((size_t)t * a.n_bl + bl) * a.n_chan * 2);
      #pragma unroll
      for (int i = 0; i < kTcRtMax; ++i) {
        const int q = warp + kTcWarps * i;
        if (q < nq) {
          #pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int c = 16 * q + g + 8 * hh;
            const float2 r = *reinterpret_cast<const float2*>(strip + c * 8 + 2 * tq);
            const float2 x = make_float2(r.x - D[i][2 * hh], r.y - D[i][2 * hh + 1]);
            const bool live = c < a.n_chan;
            if (live) __stcs(dst + (size_t)c * 4 + tq, x);
            if (ACC) {   // columns 2 tq and 2 tq + 1 stay adjacent under the swizzle
              const float2 hr = live ? split_store(x.x) : make_float2(0.f, 0.f);
              const float2 hi = live ? split_store(x.y) : make_float2(0.f, 0.f);
              *reinterpret_cast<float4*>(rhl + rhl_index(c, 2 * tq)) = make_float4(hr.x, hr.y, hi.x, hi.y);
            }
          }
        }
      }
    } else {
      for (int q = tid; q < n16 * 8; q += kTcThreads) rhl[rhl_index(q >> 3, q & 7)] = split_store(strip[q]);
    }
    __syncthreads();                         // residual split ready

    if (ACC) {
      const int m = warp & 7, half = warp >> 3;
      if (8 * m < a.n_acc) {
        const float4* f = aa_fr + m * 2 * 2 * 32 + lane;
        const float4 ah0 = f[0], al0 = f[32], ah1 = f[64], al1 = f[96];    // k-steps r = 0..7, 8..15
        const int sc = kTcSrc + 8 * m + g;   // T1 column of this lane's source
        float accr = 0.f, acci = 0.f;
        // tiles q = half, half + 2, ...; two tiles (q, q + 2) in flight per step
        for (int q = half; q < nq; q += 4) {
          const int qb = q + 2 < nq ? q + 2 : q;        // a duplicate tile is computed, not added
          float E[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
          #pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float4 ah = j ? ah1 : ah0, al = j ? al1 : al0;
            const unsigned Ah[4] = {__float_as_uint(ah.x), __float_as_uint(ah.y), __float_as_uint(ah.z), __float_as_uint(ah.w)};
            const unsigned Al[4] = {__float_as_uint(al.x), __float_as_uint(al.y), __float_as_uint(al.z), __float_as_uint(al.w)};
            const int ca = 16 * q + 8 * j + tq, cb = 16 * qb + 8 * j + tq;
            const float2 ya0 = rhl[rhl_index(ca, g)], ya1 = rhl[rhl_index(ca + 4, g)];
            const float2 yb0 = rhl[rhl_index(cb, g)], yb1 = rhl[rhl_index(cb + 4, g)];
            mma_tf32(E[0], Al[0], Al[1], Al[2], Al[3], __float_as_uint(ya0.x), __float_as_uint(ya1.x));
            mma_tf32(E[1], Al[0], Al[1], Al[2], Al[3], __float_as_uint(yb0.x), __float_as_uint(yb1.x));
            mma_tf32(E[0], Ah[0], Ah[1], Ah[2], Ah[3], __float_as_uint(ya0.y), __float_as_uint(ya1.y));
            mma_tf32(E[1], Ah[0], Ah[1], Ah[2], Ah[3], __float_as_uint(yb0.y), __float_as_uint(yb1.y));
            mma_tf32(E[0], Ah[0], Ah[1], Ah[2], Ah[3], __float_as_uint(ya0.x), __float_as_uint(ya1.x));
            mma_tf32(E[1], Ah[0], Ah[1], Ah[2], Ah[3], __float_as_uint(yb0.x), __float_as_uint(yb1.x));
          }
          #pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (u == 1 && qb == q) break;
            const float gr = E[u][0] - E[u][3], gi = E[u][1] + E[u][2];
            const float2 w = t1[(u ? qb : q) * 2 * kTcSrc + sc];
            accr = fmaf(w.x, gr, fmaf(-w.y, gi, accr));
            acci = fmaf(w.x, gi, fmaf(w.y, gr, acci));
          }
        }
        double* r = red + ((size_t)(half * kTcSrc + 8 * m + g) * 4 + tq) * 2;
        r[0] += (double)accr;
        r[1] += (double)acci;
      }
    }
    __syncthreads();                         // tables, phases, split residual free for the next step
  }
  if (ACC) {
    for (int q = tid; q < a.n_acc * 4; q += kTcThreads) {
      const int k = q >> 2, e = q & 3;
      const double re = red[(k * 4 + e) * 2] + red[((kTcSrc + k) * 4 + e) * 2];
      const double im = red[(k * 4 + e) * 2 + 1] + red[((kTcSrc + k) * 4 + e) * 2 + 1];
      a.avg[((size_t)k * a.n_bl + bl) * 4 + e] = make_float2((float)(re * a.inv_n), (float)(im * a.inv_n));
    }
  }
}

}  // namespace rts
