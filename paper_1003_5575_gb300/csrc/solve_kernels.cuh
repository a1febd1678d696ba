// Persistent solve of one block of sources in the blocked peel.
//
// Inside a block the sources are still solved one after another: source q
// needs the model matrices of sources 0..q-1 of its block for its corrected
// average (the closed-form D_jk correction of block_kernels.cuh), and each of
// its n_iter Jacobi ALS sweeps needs every antenna's previous iterate.  Issued
// as separate launches, that chain is n_iter + 2 small kernels per source,
// each a few microseconds of work behind a launch.  Here one cooperative
// launch runs the chain of a whole block: the CTAs stay resident and meet at
// grid-wide barriers, one after each corrected average and one after every
// sweep.
//
// Work split (G CTAs of kSolveThreads threads, G <= number of SMs):
//   per baseline, grid-stride over all threads: the model matrix of source
//     q-1 (FP32, from its solved FP32 Jones matrices) and the corrected average
//     of source q (the sum of k_block_correct, with each M_j recomputed from the
//     solved Jones matrices instead of read back: 8 bytes of HBM per (j, baseline)
//     instead of 40);
//   per antenna: antenna p belongs to CTA p % G (slot p / G).  Its row V_pq,
//     q = 0..n_ant-1 (V_qp = V_pq^H applied while staging, V_pp = 0), is staged
//     in shared memory once per source, and every sweep stages the FP32
//     iterate of all antennas.  Slots go in quads, a quad to W = 16, 8 or 4
//     warps (16 when the CTA has one quad): lane l of warp w of the quad takes
//     slot l >> 3 of the quad and q = (l & 7) + 8 w + 8 W u.  Products and
//     per-lane partial sums are FP32, the W warps' partials of a lane position
//     are added in FP32 in a fixed order, the sum over the 8 lane positions of
//     an antenna is FP64 (the normal-equation accumulation, spread over four
//     warps), and the 2x2 solve, the iterate, its averaging and the
//     convergence norms are FP32 in sweeps 1 .. n_iter-1.  The last sweep
//     solves from the FP64 totals in FP64 and takes the relative change of its
//     FP64 iterate against the FP32 previous one in FP64: the status compares
//     that change with 1e-6, and the FP32 rounding of a solve (a few 1e-7 of
//     each entry) would move it by several per cent near the threshold.
//
// FP64 arithmetic runs at 1/64 of the FP32 rate on GB300, a warp instruction
// costs the same with 4 or 32 lanes active, and each dependent FP64 step
// (conversions included) took ~100 cycles in a sweep: the FP64 part is the
// accumulation only, 3 conversions + 4 additions + 1 conversion per warp in
// four warps on the four sub-partitions.
//
// Barriers spin on a global counter with a time limit: a CTA whose wait runs
// out raises the abort flag, marks the current source's status
// kSolveStatusTimeout and returns, and every other CTA returns at its next
// wait.  The counter and the flag are cleared before each launch.
#pragma once
#include "als_kernels.cuh"
#include "block_kernels.cuh"

namespace rts {

constexpr int kSolveThreads = 512;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr int kSolveBatch = 1;             // q terms per lane per loop iteration (2 spills registers)
constexpr unsigned long long kSolveWaitNs = 2000000000ull;   // 2 s for one barrier wait
constexpr unsigned kSolveMaxSpins = 1u << 24;                // and at most this many polls
constexpr int kSolveStatusTimeout = -3;                      // status value (RTS_ECUDA)

struct BlockSolveArgs {
  const float2* Ablk;      // [BK][n_bl][4] plain averages of the block's directions
  const float2* Dtab;      // [n_bl][n_pairs] closed-form D_jk of the block
  int n_pairs;
  const double* src;       // [n_src][3] (l, m, S), device copy of the source list
  int s0, n_blk;           // first source of the block, sources in it
  const int2* bl_ant;
  int n_ant;
  int64_t n_bl;
  int n_iter;
  int apc;                 // antenna slots per CTA: ceil(n_ant / G)
  float2* avg;             // [n_bl][4] corrected average of the current source
  float2* M;               // [BK][n_bl][4] model matrices of the block (written)
  float2* Jf[2];           // [n_ant][4] FP32 iterates (sweep it writes Jf[it & 1])
  double* part;            // [G][3] per-CTA sums of the last sweep: dn, nn, non-finite
  int* status;             // [n_src] per source: 0, 1 (not converged), -4, kSolveStatusTimeout
  double* rel;             // [n_src] last relative change
  float2* jones;           // [n_src][n_ant][4] solved Jones matrices
  unsigned* sync;          // [2] barrier counter, abort flag (zero at launch)
};

// dynamic shared memory: rows [apc][2][n_ant] float4, iterate [n_ant][4] float2,
// previous iterate of the CTA's antennas [apc][4] float2, per-slot convergence
// sums [apc][3] double, FP64 normal-equation totals of the last sweep [apc][12]
// double, normal-equation totals [apc][12] float
inline size_t block_solve_smem(int n_ant, int apc) {
  return (size_t)apc * n_ant * 4 * sizeof(float2) + (size_t)n_ant * 4 * sizeof(float2) +
         (size_t)apc * 4 * sizeof(float2) + (size_t)apc * 3 * sizeof(double) + (size_t)apc * 12 * sizeof(double) +
         (size_t)apc * 12 * sizeof(float);
}

// J_p = A C^-1 / S, entry e (row r = e >> 1, column c = e & 1), from the 12
// normal-equation totals (A: 8 reals row-major, C: c00, c11, re c01, im c01),
// C = [c00 c01; conj(c01) c11], C^-1 = [c11 -c01; -conj(c01) c00] / det
template <typename T>
__device__ __forceinline__ typename cplx_of<T>::type solve_entry(const T* tot, T S, int e) {
  using C = typename cplx_of<T>::type;
  const int r = e >> 1, c = e & 1;
  const T c00 = tot[8], c11 = tot[9];
  const C c01 = cmk<C>(tot[10], tot[11]);
  const T det = c00 * c11 - (c01.x * c01.x + c01.y * c01.y);
  const T sc = T(1) / (det * S);
  const C i0c = c == 0 ? cmk<C>(c11 * sc, 0) : cmk<C>(-c01.x * sc, -c01.y * sc);
  const C i1c = c == 0 ? cmk<C>(-c01.x * sc, c01.y * sc) : cmk<C>(c00 * sc, 0);
  const C Ar0 = cmk<C>(tot[4 * r], tot[4 * r + 1]);
  const C Ar1 = cmk<C>(tot[4 * r + 2], tot[4 * r + 3]);
  return cadd(cmul(Ar0, i0c), cmul(Ar1, i1c));
}

// Sum 16 doubles over the 8 lanes of a lane group (lanes 8i .. 8i+7): lane j of
// the group ends with the group totals of values 2j and 2j + 1 in v[0], v[1].
__device__ inline void group8_reduce_scatter16(double (&v)[16], int lane) {
  #pragma unroll
  for (int o = 4, n = 16; o >= 1; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
    #pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double send = upper ? v[i] : v[i + n / 2];
      const double keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier number n (1, 2, ...) of a cooperative launch in which
// n_cta CTAs take part.  Returns false when the wait gave up (its own time
// limit, or another CTA's abort).
__device__ bool solve_barrier_n(unsigned* sync, unsigned n, unsigned n_cta, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: this CTA's writes (ordered before by the CTA barrier) are
    // visible to every CTA whose acquire load sees the count
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(sync) : "memory");
    const unsigned target = n * n_cta;
    int ok = 1;
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 0; ld_acquire_u32(sync) < target; ++spin) {
      if ((spin & 31u) == 31u) {
        if (ld_acquire_u32(sync + 1) != 0u) { ok = 0; break; }
        if (global_ns() - t0 > kSolveWaitNs || spin > kSolveMaxSpins) {
          atomicExch(sync + 1, 1u);
          ok = 0;
          break;
        }
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

__device__ __forceinline__ bool solve_barrier(unsigned* sync, unsigned n, int* s_flag) {
  return solve_barrier_n(sync, n, gridDim.x, s_flag);
}

// Failure-detection self-test of the barrier: the CTAs of a cooperative launch
// meet at `rounds` barriers that expect gridDim.x + missing CTAs.  With missing
// = 0 every wait completes; with missing > 0 the first wait cannot complete, a
// CTA's time limit runs out, it raises the abort flag and every CTA returns.
// ok[c] = 1 when every wait of CTA c completed.
__global__ void __launch_bounds__(128) k_barrier_selftest(unsigned* sync, int rounds, int missing, int* ok) {
  __shared__ int s_flag;
  int good = 1;
  for (int r = 1; r <= rounds && good; ++r)
    good = solve_barrier_n(sync, (unsigned)r, gridDim.x + (unsigned)missing, &s_flag);
  if (threadIdx.x == 0) ok[blockIdx.x] = good;
}

// at most 64 registers a thread: half of an SM, so the geometry kernels of later
// blocks (low-priority stream) keep running beside it
// M = S J_i J_j^H in FP32 from a source's solved FP32 Jones matrices J [n_ant][4]
// (M[r][c] = S sum_k J_i[r][k] conj(J_j[c][k])); written once per source during
// the launch, so read through L1
__device__ __forceinline__ void block_model_f(const float2* __restrict__ J, int2 ij, float S, float2 (&M)[4]) {
  const float4* J4 = reinterpret_cast<const float4*>(J);
  const float4 i0 = __ldg(J4 + 2 * ij.x), i1 = __ldg(J4 + 2 * ij.x + 1);
  const float4 j0 = __ldg(J4 + 2 * ij.y), j1 = __ldg(J4 + 2 * ij.y + 1);
  const float2 I00 = make_float2(i0.x, i0.y), I01 = make_float2(i0.z, i0.w);
  const float2 I10 = make_float2(i1.x, i1.y), I11 = make_float2(i1.z, i1.w);
  const float2 J00 = make_float2(j0.x, j0.y), J01 = make_float2(j0.z, j0.w);
  const float2 J10 = make_float2(j1.x, j1.y), J11 = make_float2(j1.z, j1.w);
  const float2 P[4] = {cadd(cmulc(I00, J00), cmulc(I01, J01)), cadd(cmulc(I00, J10), cmulc(I01, J11)),
                       cadd(cmulc(I10, J00), cmulc(I11, J01)), cadd(cmulc(I10, J10), cmulc(I11, J11))};
  #pragma unroll
  for (int e = 0; e < 4; ++e) M[e] = make_float2(S * P[e].x, S * P[e].y);
}

__global__ void __launch_bounds__(kSolveThreads, 2) k_block_solve(BlockSolveArgs a) {
  extern __shared__ __align__(16) unsigned char solve_smem[];
  float2* rows = reinterpret_cast<float2*>(solve_smem);                 // [apc][2][n_ant] float4
  float2* Js = rows + (size_t)a.apc * a.n_ant * 4;                       // [n_ant][4]
  float2* Jold = Js + (size_t)a.n_ant * 4;                               // [apc][4]
  double* s_norm = reinterpret_cast<double*>(Jold + (size_t)a.apc * 4);  // [apc][3]
  double* s_tot64 = s_norm + (size_t)a.apc * 3;                          // [apc][12]
  float* s_tot = reinterpret_cast<float*>(s_tot64 + (size_t)a.apc * 12); // [apc][12]
  __shared__ float s_p32[kSolveWarps][12][32];   // FP32 partials of every lane
  __shared__ int s_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  const int64_t gstride = (int64_t)G * kSolveThreads;
  const int nquad = (a.apc + 3) >> 2;
  // warps per quad: all 16 share the terms when the CTA has one quad (n_ant <= 4 G)
  const int wpq = nquad <= 1 ? 16 : (nquad == 2 ? 8 : 4);
  unsigned nbar = 0;

  for (int q = 0; q <= a.n_blk; ++q) {
    const int k = a.s0 + q;
    // ---- per baseline: model matrix of source q-1, corrected average of source q
    const bool model = q > 0, corr = q < a.n_blk;
    const float Sprev = model ? (float)a.src[3 * (k - 1) + 2] : 0.f;
    // a CTA's threads take consecutive baselines (mostly one first antenna), so
    // the Jones rows they read come from L1
    for (int64_t bl = blockIdx.x * (int64_t)kSolveThreads + tid; bl < a.n_bl; bl += gstride) {
      const int2 ij = a.bl_ant[bl];
      float2 Mp[4];
      if (model) {
        block_model_f(a.jones + (size_t)(k - 1) * a.n_ant * 4, ij, Sprev, Mp);
        #pragma unroll
        for (int e = 0; e < 4; ++e) a.M[((size_t)(q - 1) * a.n_bl + bl) * 4 + e] = Mp[e];
      }
      if (corr) {
        float2 v[4];
        #pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = __ldg(a.Ablk + ((size_t)q * a.n_bl + bl) * 4 + e);
        const float2* D = a.Dtab + (size_t)bl * a.n_pairs + q * (q - 1) / 2;
        // M_j recomputed from the solved Jones matrices (L1/L2) with the arithmetic
        // that stored it, instead of read back from the [BK][n_bl][4] array in HBM
        #pragma unroll 2
        for (int j = 0; j < q; ++j) {
          const float2 d = __ldg(D + j);
          float2 mj[4];
          if (j == q - 1) {
            #pragma unroll
            for (int e = 0; e < 4; ++e) mj[e] = Mp[e];
          } else {
            block_model_f(a.jones + (size_t)(a.s0 + j) * a.n_ant * 4, ij, (float)a.src[3 * (a.s0 + j) + 2], mj);
          }
          #pragma unroll
          for (int e = 0; e < 4; ++e) v[e] = csub(v[e], cmul(mj[e], d));
        }
        #pragma unroll
        for (int e = 0; e < 4; ++e) a.avg[(size_t)bl * 4 + e] = v[e];
      }
    }
    if (!corr) break;
    if (!solve_barrier(a.sync, ++nbar, &s_flag)) {
      if (tid == 0) a.status[k] = kSolveStatusTimeout;
      return;
    }

    // ---- stage the rows of this CTA's antennas; start from J = I
    for (int idx = tid; idx < a.apc * a.n_ant; idx += kSolveThreads) {
      const int s = idx / a.n_ant, qq = idx - s * a.n_ant, p = blockIdx.x + s * G;
      if (p >= a.n_ant) continue;
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
      if (qq > p) {
        const float4* v = reinterpret_cast<const float4*>(a.avg + bl_index(a.n_ant, p, qq) * 4);
        r0 = __ldcg(v);
        r1 = __ldcg(v + 1);
      } else if (qq < p) {                   // V_pq = V_qp^H
        const float4* v = reinterpret_cast<const float4*>(a.avg + bl_index(a.n_ant, qq, p) * 4);
        const float4 w0 = __ldcg(v), w1 = __ldcg(v + 1);
        r0 = make_float4(w0.x, -w0.y, w1.x, -w1.y);
        r1 = make_float4(w0.z, -w0.w, w1.z, -w1.w);
      }
      // [slot][half][q] float4: entries (0, 1) and (2, 3) of V_pq in separate planes,
      // so consecutive q are consecutive 16-byte words (conflict-free row reads)
      float4* d = reinterpret_cast<float4*>(rows);
      d[((size_t)s * 2) * a.n_ant + qq] = r0;
      d[((size_t)s * 2 + 1) * a.n_ant + qq] = r1;
    }
    for (int i = tid; i < a.apc * 4; i += kSolveThreads)
      Jold[i] = make_float2((i & 3) == 0 || (i & 3) == 3 ? 1.f : 0.f, 0.f);
    const float Sf = (float)a.src[3 * k + 2];

    // ---- n_iter Jacobi sweeps
    for (int it = 1; it <= a.n_iter; ++it) {
      const bool first = it == 1, last = it == a.n_iter, average = (it & 1) == 0;
      if (!first) {
        const float4* src4 = reinterpret_cast<const float4*>(a.Jf[(it - 1) & 1]);
        float4* dst4 = reinterpret_cast<float4*>(Js);
        for (int i = tid; i < a.n_ant * 2; i += kSolveThreads) dst4[i] = __ldcg(src4 + i);
      }
      __syncthreads();
      float2* Jf_new = a.Jf[it & 1];
      for (int g0 = 0; g0 < nquad; g0 += kSolveWarps / wpq) {     // CTA-uniform trip count
        const int g = g0 + warp / wpq, wq = warp % wpq, sa = lane >> 3;
        const int s = 4 * g + sa, p = blockIdx.x + s * G;
        const bool live = g < nquad && s < a.apc && p < a.n_ant;
        float A[8], Cm[4];
        #pragma unroll
        for (int i = 0; i < 8; ++i) A[i] = 0.f;
        #pragma unroll
        for (int i = 0; i < 4; ++i) Cm[i] = 0.f;
        if (live) {
          const float4* row0 = reinterpret_cast<const float4*>(rows) + (size_t)s * 2 * a.n_ant;
          const float4* row1 = row0 + a.n_ant;
          const float4* Jq4 = reinterpret_cast<const float4*>(Js);
          const int qstep = 8 * wpq;
          for (int q0 = (lane & 7) + 8 * wq; q0 < a.n_ant; q0 += qstep * kSolveBatch) {
            float2 V[kSolveBatch][4], J[kSolveBatch][4];
            #pragma unroll
            for (int u = 0; u < kSolveBatch; ++u) {
              const int qq = q0 + qstep * u;
              float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0, j0 = v0, j1 = v0;
              if (qq < a.n_ant && qq != p) {   // V_pp = 0, and C excludes q = p
                v0 = row0[qq];
                v1 = row1[qq];
                if (first) {
                  j0 = make_float4(1.f, 0.f, 0.f, 0.f);
                  j1 = make_float4(0.f, 0.f, 1.f, 0.f);
                } else {
                  j0 = Jq4[2 * qq];
                  j1 = Jq4[2 * qq + 1];
                }
              }
              V[u][0] = make_float2(v0.x, v0.y); V[u][1] = make_float2(v0.z, v0.w);
              V[u][2] = make_float2(v1.x, v1.y); V[u][3] = make_float2(v1.z, v1.w);
              J[u][0] = make_float2(j0.x, j0.y); J[u][1] = make_float2(j0.z, j0.w);
              J[u][2] = make_float2(j1.x, j1.y); J[u][3] = make_float2(j1.z, j1.w);
            }
            #pragma unroll
            for (int u = 0; u < kSolveBatch; ++u) {
              const float2* Vq = V[u];
              const float2* Jq = J[u];
              // A += V J
              const float2 a0 = cadd(cmul(Vq[0], Jq[0]), cmul(Vq[1], Jq[2]));
              const float2 a1 = cadd(cmul(Vq[0], Jq[1]), cmul(Vq[1], Jq[3]));
              const float2 a2 = cadd(cmul(Vq[2], Jq[0]), cmul(Vq[3], Jq[2]));
              const float2 a3 = cadd(cmul(Vq[2], Jq[1]), cmul(Vq[3], Jq[3]));
              A[0] += a0.x; A[1] += a0.y; A[2] += a1.x; A[3] += a1.y;
              A[4] += a2.x; A[5] += a2.y; A[6] += a3.x; A[7] += a3.y;
              // C += J^H J
              Cm[0] += Jq[0].x * Jq[0].x + Jq[0].y * Jq[0].y + Jq[2].x * Jq[2].x + Jq[2].y * Jq[2].y;
              Cm[1] += Jq[1].x * Jq[1].x + Jq[1].y * Jq[1].y + Jq[3].x * Jq[3].x + Jq[3].y * Jq[3].y;
              const float2 c01 = cadd(cconjmul(Jq[0], Jq[1]), cconjmul(Jq[2], Jq[3]));
              Cm[2] += c01.x; Cm[3] += c01.y;
            }
          }
        }
        #pragma unroll
        for (int i = 0; i < 8; ++i) s_p32[warp][i][lane] = A[i];
        #pragma unroll
        for (int i = 0; i < 4; ++i) s_p32[warp][8 + i][lane] = Cm[i];
        __syncthreads();
        // FP64 sums: warp r (r = 0..3, one per SM sub-partition) of the quad takes
        // values 3r .. 3r+2 of the 12 sums (A: 8 reals, C: 4) for the quad's four
        // antennas: the W warps' FP32 partials of its lane position (fixed order),
        // then FP64 over the antenna's 8 lane positions (a reduce-scatter of 4
        // slots: 3 conversions, 4 additions); the totals go to shared memory as FP32
        // for the solve
        if (wq < 4 && g < nquad) {
          double v[4];
          #pragma unroll
          for (int i = 0; i < 3; ++i) {
            float x = s_p32[warp - wq][3 * wq + i][lane];
            for (int w = 1; w < wpq; ++w) x += s_p32[warp - wq + w][3 * wq + i][lane];
            v[i] = (double)x;
          }
          v[3] = 0.0;
          #pragma unroll
          for (int o = 4, n = 4; o >= 2; o >>= 1, n >>= 1) {
            const bool upper = (lane & o) != 0;
            #pragma unroll
            for (int i = 0; i < n / 2; ++i) {
              const double send = upper ? v[i] : v[i + n / 2];
              const double keep = upper ? v[i + n / 2] : v[i];
              v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
          }
          const double tot = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);   // lane j: slot j >> 1
          const int j = lane & 7;
          if (live && (j & 1) == 0 && j < 6) {
            s_tot[s * 12 + 3 * wq + (j >> 1)] = (float)tot;
            if (last) s_tot64[s * 12 + 3 * wq + (j >> 1)] = tot;
          }
        }
        __syncthreads();
        if (wq == 0 && g < nquad) {
          const int j = lane & 7;
          const unsigned m4 = __ballot_sync(0xffffffffu, live && j < 4);   // solving lanes
          if (live && j < 4) {
            // lane j: entry e = j.  Sweeps before the last: solve, iterate and
            // averaging in FP32 (on GB300 each dependent FP64 step of this tail cost
            // ~100 cycles); the last sweep in FP64, with its relative change (the
            // status) against the FP32 previous iterate
            const int e = j;
            const float2 Jo = Jold[s * 4 + e];
            float2 Jn;
            if (!last) {
              Jn = solve_entry<float>(s_tot + s * 12, Sf, e);
              if (average) Jn = make_float2(0.5f * (Jn.x + Jo.x), 0.5f * (Jn.y + Jo.y));
            } else {
              double2 Jd = solve_entry<double>(s_tot64 + s * 12, a.src[3 * k + 2], e);
              if (average) Jd = make_double2(0.5 * (Jd.x + (double)Jo.x), 0.5 * (Jd.y + (double)Jo.y));
              const double dx = Jd.x - (double)Jo.x, dy = Jd.y - (double)Jo.y;
              double dn = dx * dx + dy * dy, nn = Jd.x * Jd.x + Jd.y * Jd.y;
              int bad = !(isfinite(Jd.x) && isfinite(Jd.y));
              #pragma unroll
              for (int o = 1; o <= 2; o <<= 1) {
                dn += __shfl_xor_sync(m4, dn, o);
                nn += __shfl_xor_sync(m4, nn, o);
                bad |= __shfl_xor_sync(m4, bad, o);
              }
              Jn = make_float2((float)Jd.x, (float)Jd.y);
              a.jones[((size_t)k * a.n_ant + p) * 4 + e] = Jn;
              if (e == 0) {
                s_norm[3 * s] = dn;
                s_norm[3 * s + 1] = nn;
                s_norm[3 * s + 2] = (double)bad;
              }
            }
            Jold[s * 4 + e] = Jn;
            Jf_new[(size_t)p * 4 + e] = Jn;
          }
        }
        __syncthreads();                     // partials read before the next quad round
      }
      if (last && tid == 0) {
        double dn = 0.0, nn = 0.0, bad = 0.0;
        for (int s = 0; s < a.apc && blockIdx.x + s * G < a.n_ant; ++s) {
          dn += s_norm[3 * s]; nn += s_norm[3 * s + 1]; bad += s_norm[3 * s + 2];
        }
        a.part[3 * blockIdx.x] = dn;
        a.part[3 * blockIdx.x + 1] = nn;
        a.part[3 * blockIdx.x + 2] = bad;
      }
      if (!solve_barrier(a.sync, ++nbar, &s_flag)) {
        if (tid == 0) a.status[k] = kSolveStatusTimeout;
        return;
      }
    }
    // ---- status of source k (fixed summation order: deterministic)
    if (blockIdx.x == 0 && tid == 0) {
      double dn = 0.0, nn = 0.0, bad = 0.0;
      for (int c = 0; c < G; ++c) {
        dn += __ldcg(a.part + 3 * c);
        nn += __ldcg(a.part + 3 * c + 1);
        bad += __ldcg(a.part + 3 * c + 2);
      }
      const double rel = sqrt(dn / nn);
      a.status[k] = (bad != 0.0 || !isfinite(rel)) ? -4 : (rel > 1e-6 ? 1 : 0);
      a.rel[k] = rel;
    }
  }
}

}  // namespace rts
