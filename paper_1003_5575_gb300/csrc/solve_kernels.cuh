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
//     q-1 and the corrected average of source q, with the arithmetic of
//     k_block_model and k_block_correct (same values);
//   per antenna, one warp: antenna p belongs to CTA p % G (slot p / G).  Its
//     row V_pq, q = 0..n_ant-1 (V_qp = V_pq^H applied while staging, V_pp = 0),
//     is staged in shared memory once per source, and every sweep stages the
//     FP32 iterate of all antennas.  Lane l takes q = l, l + 32, ...: the
//     products and each lane's partial sums are FP32, the sum over the 32
//     lanes is FP64 (one reduce-scatter per warp), and the 2x2 solve is FP64,
//     as in k_als_sweep (which splits an antenna over 128 threads; one warp
//     per antenna here quarters the FP64 additions, which are slow on GB300).
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
constexpr int kSolveBatch = 2;             // q terms whose loads a lane issues together
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
  double2* J64;            // [n_ant][4] FP64 solution of the current source
  float2* Jf[2];           // [n_ant][4] FP32 iterates (sweep it writes Jf[it & 1])
  double* part;            // [G][3] per-CTA sums of the last sweep: dn, nn, non-finite
  int* status;             // [n_src] per source: 0, 1 (not converged), -4, kSolveStatusTimeout
  double* rel;             // [n_src] last relative change
  float2* jones;           // [n_src][n_ant][4] solved Jones matrices
  unsigned* sync;          // [2] barrier counter, abort flag (zero at launch)
};

// dynamic shared memory: rows [apc][n_ant][4] float2, iterate [n_ant][4] float2,
// previous FP64 iterate of the CTA's antennas [apc][4] double2
inline size_t block_solve_smem(int n_ant, int apc) {
  return (size_t)apc * n_ant * 4 * sizeof(float2) + (size_t)n_ant * 4 * sizeof(float2) +
         (size_t)apc * 4 * sizeof(double2);
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

// Grid-wide barrier number n (1, 2, ...) of a cooperative launch.  Returns
// false when the wait gave up (its own time limit, or another CTA's abort).
__device__ bool solve_barrier(unsigned* sync, unsigned n, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(sync, 1u);
    const unsigned target = n * gridDim.x;
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
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// at most 64 registers a thread: half of an SM, so the geometry kernels of later
// blocks (low-priority stream) keep running beside it
__global__ void __launch_bounds__(kSolveThreads, 2) k_block_solve(BlockSolveArgs a) {
  extern __shared__ __align__(16) unsigned char solve_smem[];
  float2* rows = reinterpret_cast<float2*>(solve_smem);                 // [apc][n_ant][4]
  float2* Js = rows + (size_t)a.apc * a.n_ant * 4;                       // [n_ant][4]
  double2* Jold = reinterpret_cast<double2*>(Js + (size_t)a.n_ant * 4);  // [apc][4]
  __shared__ double s_wpart[kSolveWarps][3];
  __shared__ double s_tot[kSolveWarps][12];
  __shared__ int s_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  const int64_t gstride = (int64_t)G * kSolveThreads;
  unsigned nbar = 0;

  for (int q = 0; q <= a.n_blk; ++q) {
    const int k = a.s0 + q;
    // ---- per baseline: model matrix of source q-1, corrected average of source q
    const bool model = q > 0, corr = q < a.n_blk;
    const double Sprev = model ? a.src[3 * (k - 1) + 2] : 0.0;
    for (int64_t bl = blockIdx.x * (int64_t)kSolveThreads + tid; bl < a.n_bl; bl += gstride) {
      float2 Mp[4];
      if (model) {
        const int2 ij = a.bl_ant[bl];
        M22<double2> Ji, Jj;
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          Ji.e[e] = __ldcg(a.J64 + (size_t)ij.x * 4 + e);
          Jj.e[e] = __ldcg(a.J64 + (size_t)ij.y * 4 + e);
        }
        const M22<double2> P = mmul_h(Ji, Jj);
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          Mp[e] = make_float2((float)(Sprev * P.e[e].x), (float)(Sprev * P.e[e].y));
          a.M[((size_t)(q - 1) * a.n_bl + bl) * 4 + e] = Mp[e];
        }
      }
      if (corr) {
        float2 v[4];
        #pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = __ldg(a.Ablk + ((size_t)q * a.n_bl + bl) * 4 + e);
        const float2* D = a.Dtab + (size_t)bl * a.n_pairs + q * (q - 1) / 2;
        for (int j = 0; j < q; ++j) {
          const float2 d = __ldg(D + j);
          #pragma unroll
          for (int e = 0; e < 4; ++e) {
            // sources before q - 1 were modelled by this thread in earlier rounds
            const float2 mj = j == q - 1 ? Mp[e] : a.M[((size_t)j * a.n_bl + bl) * 4 + e];
            v[e] = csub(v[e], cmul(mj, d));
          }
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
      float4* d = reinterpret_cast<float4*>(rows + ((size_t)s * a.n_ant + qq) * 4);
      d[0] = r0;
      d[1] = r1;
    }
    for (int i = tid; i < a.apc * 4; i += kSolveThreads)
      Jold[i] = make_double2((i & 3) == 0 || (i & 3) == 3 ? 1.0 : 0.0, 0.0);
    const double S = a.src[3 * k + 2];

    // ---- n_iter Jacobi sweeps
    for (int it = 1; it <= a.n_iter; ++it) {
      const bool first = it == 1, last = it == a.n_iter, average = (it & 1) == 0;
      if (!first) {
        const float4* src4 = reinterpret_cast<const float4*>(a.Jf[(it - 1) & 1]);
        float4* dst4 = reinterpret_cast<float4*>(Js);
        for (int i = tid; i < a.n_ant * 2; i += kSolveThreads) dst4[i] = __ldcg(src4 + i);
      }
      if (last && lane == 0) s_wpart[warp][0] = s_wpart[warp][1] = s_wpart[warp][2] = 0.0;
      __syncthreads();
      float2* Jf_new = a.Jf[it & 1];
      for (int s = warp; s < a.apc; s += kSolveWarps) {
        const int p = blockIdx.x + s * G;
        if (p >= a.n_ant) break;             // warp-uniform; later slots are out of range too
        const float4* row = reinterpret_cast<const float4*>(rows + (size_t)s * a.n_ant * 4);
        const float4* Jq4 = reinterpret_cast<const float4*>(Js);
        float A[8], Cm[4];
        #pragma unroll
        for (int i = 0; i < 8; ++i) A[i] = 0.f;
        #pragma unroll
        for (int i = 0; i < 4; ++i) Cm[i] = 0.f;
        for (int q0 = lane; q0 < a.n_ant; q0 += 32 * kSolveBatch) {
          float2 V[kSolveBatch][4], J[kSolveBatch][4];
          #pragma unroll
          for (int u = 0; u < kSolveBatch; ++u) {
            const int qq = q0 + 32 * u;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0, j0 = v0, j1 = v0;
            if (qq < a.n_ant && qq != p) {     // V_pp = 0, and C excludes q = p
              v0 = row[2 * qq];
              v1 = row[2 * qq + 1];
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
        double v[16];
        #pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (double)A[i];
        #pragma unroll
        for (int i = 0; i < 4; ++i) v[8 + i] = (double)Cm[i];
        #pragma unroll
        for (int i = 12; i < 16; ++i) v[i] = 0.0;
        const double wsum = warp_reduce_scatter16(v, lane);     // lane L: total L >> 1
        double* tot = s_tot[warp];
        if ((lane & 1) == 0 && lane < 24) tot[lane >> 1] = wsum;
        __syncwarp();
        if (lane < 4) {
          // J_p = A C^-1 / S in FP64, C = [c00 c01; conj(c01) c11]
          const int e = lane, r = e >> 1, c = e & 1;
          const double c00 = tot[8], c11 = tot[9];
          const double2 c01 = make_double2(tot[10], tot[11]);
          const double det = c00 * c11 - (c01.x * c01.x + c01.y * c01.y);
          const double sc = 1.0 / (det * S);
          const double2 i0c = c == 0 ? make_double2(c11 * sc, 0.0) : make_double2(-c01.x * sc, -c01.y * sc);
          const double2 i1c = c == 0 ? make_double2(-c01.x * sc, c01.y * sc) : make_double2(c00 * sc, 0.0);
          const double2 Ar0 = make_double2(r ? tot[4] : tot[0], r ? tot[5] : tot[1]);
          const double2 Ar1 = make_double2(r ? tot[6] : tot[2], r ? tot[7] : tot[3]);
          double2 Jn = cadd(cmul(Ar0, i0c), cmul(Ar1, i1c));
          const double2 Jo = Jold[s * 4 + e];
          if (average) Jn = make_double2(0.5 * (Jn.x + Jo.x), 0.5 * (Jn.y + Jo.y));
          const double dx = Jn.x - Jo.x, dy = Jn.y - Jo.y;
          double dn = dx * dx + dy * dy, nn = Jn.x * Jn.x + Jn.y * Jn.y;
          int bad = !(isfinite(Jn.x) && isfinite(Jn.y));
          #pragma unroll
          for (int o = 1; o <= 2; o <<= 1) {
            dn += __shfl_xor_sync(0xfu, dn, o);
            nn += __shfl_xor_sync(0xfu, nn, o);
            bad |= __shfl_xor_sync(0xfu, bad, o);
          }
          Jold[s * 4 + e] = Jn;
          const float2 Jf = make_float2((float)Jn.x, (float)Jn.y);
          Jf_new[(size_t)p * 4 + e] = Jf;
          if (last) {
            a.J64[(size_t)p * 4 + e] = Jn;
            a.jones[((size_t)k * a.n_ant + p) * 4 + e] = Jf;
            if (e == 0) {
              s_wpart[warp][0] += dn;
              s_wpart[warp][1] += nn;
              s_wpart[warp][2] += (double)bad;
            }
          }
        }
      }
      if (last) {
        __syncthreads();
        if (tid == 0) {
          double dn = 0.0, nn = 0.0, bad = 0.0;
          for (int w = 0; w < kSolveWarps; ++w) { dn += s_wpart[w][0]; nn += s_wpart[w][1]; bad += s_wpart[w][2]; }
          a.part[3 * blockIdx.x] = dn;
          a.part[3 * blockIdx.x + 1] = nn;
          a.part[3 * blockIdx.x + 2] = bad;
        }
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
