// Persistent solve of one block of sources in the blocked peel.
//
// Inside a block the sources are still solved one after another: source q
// needs the model matrices of sources 0..q-1 of its block for its corrected
// average (the closed-form D_jk correction of block_kernels.cuh), and each of
// its n_iter Jacobi ALS sweeps needs every antenna's previous iterate.  Issued
// as separate launches, that chain is n_iter + 2 small kernels per source,
// each a few microseconds of work behind a launch.  Here one cooperative
// launch runs the chain of a whole block: the CTAs stay resident and meet at
// grid-wide barriers, one after each source's corrected average and one
// after every sweep.
//
// Per source q of the block (G CTAs of kSolveThreads threads, G <= SMs):
//   corrected average (solve_correct): P_q = A_q - sum_{j<q} M_j D_jq for
//     every baseline, by 32 x 32-antenna tiles.  Every CTA takes an equal
//     share of the tiles' rows; a tile's column Jones matrices of sources
//     0 .. q-1 are staged in shared memory, and its rows stream through a
//     two-stage ring of asynchronous copies (a row's baselines are consecutive,
//     so its D terms are one contiguous run in the target-major dir_index
//     layout); M_j D = S_j D J_i J_k^H is recomputed from the solved FP32 Jones
//     matrices instead of read back from HBM.  The term that needs source q-1
//     also writes M_{q-1} for the block's pass.  Grid barrier.
//   rows: antenna p belongs to CTA p % G (slot p / G).  Its row V_pq,
//     q = 0..n_ant-1 (V_qp = V_pq^H applied while staging, V_pp = 0), is staged
//     in shared memory from P_q.
//   n_iter sweeps: every sweep stages the FP32 iterate of all antennas.  The
//     CTA's warps are split evenly over its slots; lane l of the w-th warp of a
//     slot takes the partners q = l + 32 w (+ 32 W u).  Products and per-lane
//     partial sums are FP32, a warp's lanes are added in FP32 by a shuffle tree,
//     and the W warps of a slot in FP64 (the normal-equation accumulation).  The
//     2x2 solve, the iterate and its averaging are FP32 in sweeps
//     1 .. n_iter-1; the last sweep converts the lane partials to FP64, solves
//     in FP64 and takes the relative change of its FP64 iterate against the
//     FP32 previous one in FP64 (the status compares that change with 1e-6,
//     and the FP32 rounding of a solve would move it by several per cent near
//     the threshold).  Grid barrier after each sweep.
// After the block's last source: its model matrices, and every source's
// status from the per-antenna norms of its last sweep (off the chain).
//
// FP64 arithmetic runs at 1/64 of the FP32 rate on GB300 and a warp
// instruction costs the same with 4 or 32 lanes active: the FP64 part of a
// sweep is a few conversions and additions per total, spread over four warps
// on the four sub-partitions.
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
constexpr int kTileAnt = 32;               // antennas per side of a correction tile
constexpr int kCorrMaxJ = 64;             // sources of a block at the most (RTS_BLOCK)
// shared memory of the correction: column Jones matrices [2][kTileAnt][kCorrMaxJ]
// float4, then two stages of kCorrStageBytes (a chunk of rows: D values, row
// Jones matrices, plain averages)
constexpr size_t kCorrColBytes = (size_t)2 * kTileAnt * kCorrMaxJ * sizeof(float4);
constexpr size_t kCorrStageBytes = 40960;
constexpr size_t kCorrBytes = kCorrColBytes + 2 * kCorrStageBytes;
constexpr int kSolveMaxApc = 16;           // antenna slots per CTA (one warp each at the most)
constexpr unsigned long long kSolveWaitNs = 2000000000ull;   // 2 s for one barrier wait
constexpr unsigned kSolveMaxSpins = 1u << 24;                // and at most this many polls
constexpr int kSolveStatusTimeout = -3;                      // status value (RTS_ECUDA)

struct BlockSolveArgs {
  const float2* Ablk;      // [BK][n_bl][4] plain averages of the block's directions
  const float2* Dtab;      // closed-form D_jk of the block (dir_index layout)
  const double* src;       // [n_src][3] (l, m, S), device copy of the source list
  int s0, n_blk;           // first source of the block, sources in it
  const int2* bl_ant;
  int n_ant;
  int64_t n_bl;
  int n_iter;
  int apc;                 // antenna slots per CTA: ceil(n_ant / G), at most kSolveMaxApc
  float2* P;               // [n_bl][4] corrected average of the current source
  float2* M;               // [BK][n_bl][4] model matrices of the block (written)
  float2* Jf[2];           // [n_ant][4] FP32 iterates (sweep it writes Jf[it & 1])
  double* part;            // [BK][n_ant][4] per antenna, last sweep: dn, nn, non-finite
  int* status;             // [n_src] per source: 0, 1 (not converged), -4, kSolveStatusTimeout
  double* rel;             // [n_src] last relative change
  float2* jones;           // [n_src][n_ant][4] solved Jones matrices
  unsigned* sync;          // [2] barrier counter, abort flag (zero at launch)
};

// dynamic shared memory: rows [apc][2][n_ant] float4 and iterate [2][n_ant]
// float4 (entries 0, 1 | 2, 3), in a space shared with the correction's chunks
// (kCorrBytes, and the status sums at the end); then
// the previous iterate of the CTA's antennas [apc][4] float2, FP64
// normal-equation totals of the last sweep [apc][12] double, normal-equation
// totals [apc][12] float
__host__ __device__ inline size_t solve_union_bytes(int n_ant, int apc) {
  const size_t rows = ((size_t)apc + 1) * n_ant * 2 * sizeof(float4);
  return rows > kCorrBytes ? rows : kCorrBytes;
}
inline size_t block_solve_smem(int n_ant, int apc) {
  return solve_union_bytes(n_ant, apc) + (size_t)apc * 4 * sizeof(float2) + (size_t)apc * 12 * sizeof(double) +
         (size_t)apc * 12 * sizeof(float);
}

// 1 / x: the correctly rounded FP32 reciprocal (no IEEE division sequence) for
// the FP32 sweeps, a plain division in FP64
__device__ __forceinline__ float solve_recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double solve_recip(double x) { return 1.0 / x; }

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
  const T sc = solve_recip(det * S);
  const C i0c = c == 0 ? cmk<C>(c11 * sc, 0) : cmk<C>(-c01.x * sc, -c01.y * sc);
  const C i1c = c == 0 ? cmk<C>(-c01.x * sc, c01.y * sc) : cmk<C>(c00 * sc, 0);
  const C Ar0 = cmk<C>(tot[4 * r], tot[4 * r + 1]);
  const C Ar1 = cmk<C>(tot[4 * r + 2], tot[4 * r + 3]);
  return cadd(cmul(Ar0, i0c), cmul(Ar1, i1c));
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
// n_cta CTAs take part, in two halves so that a CTA can work between them:
// solve_arrive counts the CTA in (its writes before the call, ordered by the
// CTA barrier, are released to every CTA whose acquire load sees the count);
// solve_wait returns once all n_cta have arrived, or false when the wait gave
// up (its own time limit, or another CTA's abort).
__device__ __forceinline__ void solve_arrive(unsigned* sync) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(sync) : "memory");
}

__device__ bool solve_wait(unsigned* sync, unsigned n, unsigned n_cta, int* s_flag) {
  if (threadIdx.x == 0) {
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

__device__ bool solve_barrier_n(unsigned* sync, unsigned n, unsigned n_cta, int* s_flag) {
  solve_arrive(sync);
  return solve_wait(sync, n, n_cta, s_flag);
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

// M = S J_i J_j^H in FP32 from the two antennas' solved FP32 Jones matrices,
// each as two float4 (entries 0, 1 | 2, 3): M[r][c] = S sum_k J_i[r][k] conj(J_j[c][k])
__device__ __forceinline__ void block_model4(float4 i0, float4 i1, float4 j0, float4 j1, float S, float2 (&M)[4]) {
  const float2 I00 = make_float2(i0.x, i0.y), I01 = make_float2(i0.z, i0.w);
  const float2 I10 = make_float2(i1.x, i1.y), I11 = make_float2(i1.z, i1.w);
  const float2 J00 = make_float2(j0.x, j0.y), J01 = make_float2(j0.z, j0.w);
  const float2 J10 = make_float2(j1.x, j1.y), J11 = make_float2(j1.z, j1.w);
  const float2 P[4] = {cadd(cmulc(I00, J00), cmulc(I01, J01)), cadd(cmulc(I00, J10), cmulc(I01, J11)),
                       cadd(cmulc(I10, J00), cmulc(I11, J01)), cadd(cmulc(I10, J10), cmulc(I11, J11))};
  #pragma unroll
  for (int e = 0; e < 4; ++e) M[e] = make_float2(S * P[e].x, S * P[e].y);
}

// the same from a source's Jones matrices J [n_ant][4] in global memory; they
// are written during the launch by other CTAs, so they are read from L2
__device__ __forceinline__ void block_model_cg(const float2* J, int2 ij, float S, float2 (&M)[4]) {
  const float4* J4 = reinterpret_cast<const float4*>(J);
  block_model4(__ldcg(J4 + 2 * ij.x), __ldcg(J4 + 2 * ij.x + 1), __ldcg(J4 + 2 * ij.y), __ldcg(J4 + 2 * ij.y + 1),
               S, M);
}

// Reduce 8 doubles over the 32 lanes of a warp (a fixed shuffle tree: three
// levels exchange half of the remaining values, two add the last one); lane L
// ends with the warp total of value (L >> 2) & 7.
__device__ __forceinline__ double warp_reduce_scatter8d(double (&v)[8], int lane) {
  #pragma unroll
  for (int o = 16, n = 8; o >= 4; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
    #pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double send = upper ? v[i] : v[i + n / 2];
      const double keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double r = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
  return r + __shfl_xor_sync(0xffffffffu, r, 1);
}

__device__ __forceinline__ void solve_cp16(void* smem, const void* gmem) {     // L2 only
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void solve_cp8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void solve_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void solve_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }


// One chunk's rows of a correction tile (see solve_correct): JL term lanes per
// baseline (JL >= q where q < 8, else 8), kSolveThreads / (kTileAnt JL) rows at a time;
// thread (row s, column c, term lane l) sums the terms j = l (mod JL) of its
// baseline, and the JL lanes are added by a fixed shuffle tree that leaves
// each lane max(1, 8 / JL) of the 8 floats.  Stage layout: D [R][kTileAnt][q]
// float2 at 0, row Jones [R][2][q] float4 at offJ, plain averages
// [R][kTileAnt][2] float4 at offA.  CTA-uniform.
template <int JL>
__device__ void solve_correct_rows(const BlockSolveArgs& a, int q, const unsigned char* st, size_t offJ,
                                   size_t offA, const float4* JC, const float* Sj, int I0, int K0, int nK, int r0,
                                   int nrows) {
  constexpr int RP = kSolveThreads / (kTileAnt * JL);      // rows per pass
  constexpr int F = JL >= 8 ? 1 : 8 / JL;                 // floats a lane ends with
  const int tid = threadIdx.x, jl = tid & (JL - 1), c = (tid / JL) & (kTileAnt - 1), rs = tid / (JL * kTileAnt);
  for (int rr0 = 0; rr0 < nrows; rr0 += RP) {
    const int rr = rr0 + rs, r = r0 + rr, i = I0 + r;
    const int k0 = max(K0, i + 1), nk = K0 + nK - k0;
    const bool valid = rr < nrows && c < nk;
    const int col = k0 - K0 + c;
    float2 acc[4];
    #pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
    const int64_t bl = valid ? bl_index(a.n_ant, i, K0 + col) : 0;
    if (valid) {
      const float2* Dd = reinterpret_cast<const float2*>(st) + ((size_t)rr * kTileAnt + c) * q;
      const float4* JR = reinterpret_cast<const float4*>(st + offJ) + (size_t)rr * 2 * q;
      const float4* Jk0 = JC + (size_t)col * kCorrMaxJ;
      const float4* Jk1 = JC + ((size_t)kTileAnt + col) * kCorrMaxJ;
      #pragma unroll 4
      for (int j = jl; j < q; j += JL) {
        // M_j D = S_j D J_i J_k^H: w_rm = S_j D J_i[r][m], then acc[2r + c] +=
        // sum_m w_rm conj(J_k[c][m])
        const float4 i0 = JR[j], i1 = JR[q + j], k0 = Jk0[j], k1 = Jk1[j];
        const float2 d = Dd[j];
        const float S = Sj[j];
        if (j == q - 1) {                      // the model matrix of source q-1, for the pass
          float2 M[4];
          block_model4(i0, i1, k0, k1, S, M);
          float4* dm = reinterpret_cast<float4*>(a.M + ((size_t)(q - 1) * a.n_bl + bl) * 4);
          dm[0] = make_float4(M[0].x, M[0].y, M[1].x, M[1].y);
          dm[1] = make_float4(M[2].x, M[2].y, M[3].x, M[3].y);
        }
        const float2 sd = make_float2(S * d.x, S * d.y);
        const float2 w00 = cmul(sd, make_float2(i0.x, i0.y)), w01 = cmul(sd, make_float2(i0.z, i0.w));
        const float2 w10 = cmul(sd, make_float2(i1.x, i1.y)), w11 = cmul(sd, make_float2(i1.z, i1.w));
        auto cfma = [](float2 acc2, float2 w, float kx, float ky) {     // acc + w conj(k)
          acc2.x = fmaf(w.x, kx, fmaf(w.y, ky, acc2.x));
          acc2.y = fmaf(w.y, kx, fmaf(-w.x, ky, acc2.y));
          return acc2;
        };
        acc[0] = cfma(cfma(acc[0], w00, k0.x, k0.y), w01, k0.z, k0.w);
        acc[1] = cfma(cfma(acc[1], w00, k1.x, k1.y), w01, k1.z, k1.w);
        acc[2] = cfma(cfma(acc[2], w10, k0.x, k0.y), w11, k0.z, k0.w);
        acc[3] = cfma(cfma(acc[3], w10, k1.x, k1.y), w11, k1.z, k1.w);
      }
    }
    float v[8] = {acc[0].x, acc[0].y, acc[1].x, acc[1].y, acc[2].x, acc[2].y, acc[3].x, acc[3].y};
    #pragma unroll
    for (int o = JL / 2, n = 8; o >= 1; o >>= 1, n >>= 1) {
      if (n >= 2) {                           // exchange halves: the upper lane keeps the upper half
        const bool upper = (jl & o) != 0;
        #pragma unroll
        for (int u = 0; u < n / 2; ++u) {
          const float send = upper ? v[u] : v[u + n / 2];
          const float keep = upper ? v[u + n / 2] : v[u];
          v[u] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      } else {                                // JL = 16: the pair adds its one value
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
      }
    }
    const int base = JL == 16 ? (jl >> 1) : jl * F;
    if (valid && (JL < 16 || (jl & 1) == 0)) {
      const float* AR = reinterpret_cast<const float*>(st + offA) + ((size_t)rr * kTileAnt + c) * 8 + base;
      float* P = reinterpret_cast<float*>(a.P + bl * 4) + base;
      if (F >= 4) {                            // 16-byte accesses (the floats of a baseline are 32-byte aligned)
        #pragma unroll
        for (int f = 0; f < F; f += 4) {
          const float4 A4 = *reinterpret_cast<const float4*>(AR + f);
          *reinterpret_cast<float4*>(P + f) = make_float4(A4.x - v[f], A4.y - v[f + 1], A4.z - v[f + 2], A4.w - v[f + 3]);
        }
      } else if (F == 2) {
        const float2 A2 = *reinterpret_cast<const float2*>(AR);
        *reinterpret_cast<float2*>(P) = make_float2(A2.x - v[0], A2.y - v[1]);
      } else {
        P[0] = AR[0] - v[0];
      }
    }
  }
}

// Corrected average of source q >= 1 of the block, P_q = A_q - sum_{j<q} M_j D_jq,
// with M_j = S_j J_i^j J_k^jH recomputed from the solved FP32 Jones matrices.
// The baselines (i < k) are cut into tiles of kTileAnt x kTileAnt antennas
// (row group g1 <= column group g2); CTA c takes an equal share of all tiles'
// rows (in tile, row order: parts of at most two tiles).  The Jones matrices
// of the tile's column antennas for sources 0 .. q-1 are staged
// in shared memory once per tile; the tile's rows go in chunks of as many rows
// as a stage holds (all of them for small q), two stages filled by
// asynchronous copies one chunk ahead (spread over all threads): the row's D values (its
// baselines are consecutive, so its terms are one contiguous run of memory in
// the dir_index layout), its antenna's Jones matrices and its plain averages.
// CTA-uniform.
__device__ void solve_correct(const BlockSolveArgs& a, int q, unsigned char* smem, float* Sj) {
  const int tid = threadIdx.x;
  const int n_ant = a.n_ant, G = gridDim.x;
  const int ngr = (n_ant + kTileAnt - 1) / kTileAnt, n_tiles = ngr * (ngr + 1) / 2;
  float4* JC = reinterpret_cast<float4*>(smem);                              // [2][kTileAnt][kCorrMaxJ]
  unsigned char* ring = smem + kCorrColBytes;                                // [2][kCorrStageBytes]
  const float4* J4 = reinterpret_cast<const float4*>(a.jones);
  const int64_t dbase = dir_index(a.n_bl, 0, 0, q);
  for (int j = tid; j < q; j += kSolveThreads) Sj[j] = (float)a.src[3 * (a.s0 + j) + 2];   // read after a barrier below
  // rows per chunk, and the stage layout
  const int R = max(1, min(kTileAnt, (int)(kCorrStageBytes / ((size_t)q * kTileAnt * 8 + (size_t)q * 32 + 1024))));
  const size_t offJ = (size_t)R * kTileAnt * q * sizeof(float2), offA = offJ + (size_t)R * 2 * q * sizeof(float4);
  // this CTA's share of the tiles' rows, in (tile, row) order: at most two tiles
  const int64_t n_rows_all = (int64_t)n_tiles * kTileAnt;
  const int64_t gr_end = n_rows_all * (blockIdx.x + 1) / G;
  for (int64_t gr = n_rows_all * blockIdx.x / G; gr < gr_end;) {
    const int t = (int)(gr / kTileAnt), rlo = (int)(gr - (int64_t)t * kTileAnt);
    const int rhi = (int)min((int64_t)kTileAnt, rlo + (gr_end - gr));
    gr += rhi - rlo;
    int g1 = 0, rest = t;
    while (rest >= ngr - g1) { rest -= ngr - g1; ++g1; }
    const int g2 = g1 + rest;
    const int I0 = g1 * kTileAnt, K0 = g2 * kTileAnt;
    const int nI = min(kTileAnt, n_ant - I0), nK = min(kTileAnt, n_ant - K0);
    const int r_hi = min(rhi, nI);             // rows rlo .. r_hi - 1 of the tile
    if (r_hi <= rlo) continue;                 // CTA-uniform
    const int n_ch = (r_hi - rlo + R - 1) / R;
    auto issue = [&](int ch) {
      unsigned char* st = ring + (size_t)(ch & 1) * kCorrStageBytes;
      const int nr = min(R, r_hi - rlo - ch * R);
      // D runs of the chunk's rows, spread over all threads: element x of row rr
      for (int idx = tid; idx < nr * kTileAnt * q; idx += kSolveThreads) {
        const int rr = idx / (kTileAnt * q), x = idx - rr * kTileAnt * q;
        const int i = I0 + rlo + ch * R + rr, k0 = max(K0, i + 1), nk = K0 + nK - k0;
        if (x < nk * q)
          solve_cp8(reinterpret_cast<float2*>(st) + (size_t)rr * kTileAnt * q + x,
                    a.Dtab + dbase + bl_index(n_ant, i, k0) * q + x);
      }
      // row Jones matrices (x = plane + 2 j) and plain averages (x = half + 2 column)
      for (int idx = tid; idx < nr * 2 * q; idx += kSolveThreads) {
        const int rr = idx / (2 * q), x = idx - rr * 2 * q, i = I0 + rlo + ch * R + rr;
        solve_cp16(reinterpret_cast<float4*>(st + offJ) + (size_t)rr * 2 * q + (x & 1) * q + (x >> 1),
                   J4 + ((size_t)(a.s0 + (x >> 1)) * n_ant + i) * 2 + (x & 1));
      }
      for (int idx = tid; idx < nr * 2 * kTileAnt; idx += kSolveThreads) {
        const int rr = idx / (2 * kTileAnt), x = idx - rr * 2 * kTileAnt;
        const int i = I0 + rlo + ch * R + rr, k0 = max(K0, i + 1), nk = K0 + nK - k0;
        if (x < 2 * nk)
          solve_cp16(reinterpret_cast<float4*>(st + offA) + (size_t)rr * kTileAnt * 2 + x,
                     reinterpret_cast<const float4*>(a.Ablk + ((size_t)q * a.n_bl + bl_index(n_ant, i, k0)) * 4) + x);
      }
      solve_cp_commit();
    };
    // the column antennas' Jones matrices, sources 0 .. q-1: JC[plane][col][j]
    for (int x = tid; x < 2 * nK * q; x += kSolveThreads) {
      const int plane = x & 1, col = (x >> 1) % nK, j = (x >> 1) / nK;
      solve_cp16(JC + ((size_t)plane * kTileAnt + col) * kCorrMaxJ + j,
                 J4 + ((size_t)(a.s0 + j) * n_ant + K0 + col) * 2 + plane);
    }
    solve_cp_commit();
    issue(0);
    for (int ch = 0; ch < n_ch; ++ch) {
      if (ch + 1 < n_ch) {
        issue(ch + 1);
        solve_cp_wait<1>();
      } else {
        solve_cp_wait<0>();
      }
      __syncthreads();
      const unsigned char* st = ring + (size_t)(ch & 1) * kCorrStageBytes;
      const int r0 = rlo + ch * R, nrows = min(R, r_hi - r0);
      if (q >= 8) solve_correct_rows<8>(a, q, st, offJ, offA, JC, Sj, I0, K0, nK, r0, nrows);
      else if (q >= 4) solve_correct_rows<4>(a, q, st, offJ, offA, JC, Sj, I0, K0, nK, r0, nrows);
      else if (q >= 2) solve_correct_rows<2>(a, q, st, offJ, offA, JC, Sj, I0, K0, nK, r0, nrows);
      else solve_correct_rows<1>(a, q, st, offJ, offA, JC, Sj, I0, K0, nK, r0, nrows);
      __syncthreads();                       // stage ch & 1 read before chunk ch + 2 refills it
    }
  }
}

static_assert(kSolveWarps == 16 && kSolveThreads == 16 * kTileAnt,
              "a correction pass: at least one row of kTileAnt columns x 16 term lanes");

// at most 96 registers a thread (three quarters of an SM's register file), so a CTA
// of the geometry kernels of later blocks (low-priority stream) keeps running beside it
__global__ void __maxnreg__(96) k_block_solve(BlockSolveArgs a) {
  extern __shared__ __align__(16) unsigned char solve_smem[];
  const int n_ant = a.n_ant;
  // the rows and the staged iterate share their space with the correction's tiles
  float4* rows = reinterpret_cast<float4*>(solve_smem);                      // [apc][2][n_ant]
  float4* Js = rows + (size_t)a.apc * 2 * n_ant;                              // [2][n_ant]
  float2* Jold = reinterpret_cast<float2*>(solve_smem + solve_union_bytes(n_ant, a.apc));   // [apc][4]
  double* s_tot64 = reinterpret_cast<double*>(Jold + (size_t)a.apc * 4);      // [apc][12]
  float* s_tot = reinterpret_cast<float*>(s_tot64 + (size_t)a.apc * 12);      // [apc][12]
  __shared__ float s_wp[kSolveWarps][12];                     // each warp's 12 sums
  __shared__ double s_wp64[kSolveWarps][12];                  // the same in FP64 (last sweep)
  __shared__ float s_S[kCorrMaxJ];                            // fluxes of the block's sources (correction)
  __shared__ int s_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  // W warps per slot (the slot count rounded up to a power of two)
  const int sp = a.apc <= 1 ? 1 : (a.apc <= 2 ? 2 : (a.apc <= 4 ? 4 : (a.apc <= 8 ? 8 : 16)));
  const int W = kSolveWarps / sp;
  const int slot = warp / W, wi = warp - slot * W;
  const int my_p = blockIdx.x + slot * G;
  const bool my_live = slot < a.apc && my_p < n_ant;
  const int n_row = a.apc * n_ant;
  unsigned nbar = 0;

  for (int q = 0; q < a.n_blk; ++q) {
    const int k = a.s0 + q;
    // ---- corrected average of source q (source 0 of the block: its plain average)
    if (q > 0) {
      solve_correct(a, q, solve_smem, s_S);
      solve_arrive(a.sync);
      if (!solve_wait(a.sync, ++nbar, (unsigned)G, &s_flag)) {
        if (tid == 0) a.status[k] = kSolveStatusTimeout;
        return;
      }
    }
    // ---- rows of this CTA's antennas: [slot][half][q], entries (0, 1) and (2, 3)
    // of V_pq in separate planes, consecutive q in consecutive 16-byte words
    // (conflict-free row reads); V_pq = V_qp^H for q < p, V_pp = 0
    {
      const float2* Pq = q > 0 ? a.P : a.Ablk;
      for (int idx0 = tid; idx0 < n_row; idx0 += 2 * kSolveThreads) {
        float4 w[2][2];
        #pragma unroll
        for (int u = 0; u < 2; ++u) {        // both elements' loads before either store
          const int idx = idx0 + u * kSolveThreads;
          w[u][0] = w[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          const int s = idx / n_ant, qq = idx - s * n_ant, p = blockIdx.x + s * G;
          if (idx < n_row && p < n_ant && qq != p) {
            const float4* P4 = reinterpret_cast<const float4*>(Pq + bl_index(n_ant, min(p, qq), max(p, qq)) * 4);
            w[u][0] = __ldcg(P4);
            w[u][1] = __ldcg(P4 + 1);
          }
        }
        #pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int idx = idx0 + u * kSolveThreads;
          const int s = idx / n_ant, qq = idx - s * n_ant, p = blockIdx.x + s * G;
          if (idx < n_row && p < n_ant) {
            float4 r0 = w[u][0], r1 = w[u][1];
            if (qq < p) {
              r0 = make_float4(w[u][0].x, -w[u][0].y, w[u][1].x, -w[u][1].y);
              r1 = make_float4(w[u][0].z, -w[u][0].w, w[u][1].z, -w[u][1].w);
            }
            rows[((size_t)s * 2) * n_ant + qq] = r0;
            rows[((size_t)s * 2 + 1) * n_ant + qq] = r1;
          }
        }
      }
    }
    for (int i = tid; i < a.apc * 4; i += kSolveThreads)
      Jold[i] = make_float2((i & 3) == 0 || (i & 3) == 3 ? 1.f : 0.f, 0.f);
    const float Sf = (float)a.src[3 * k + 2];

    // ---- n_iter Jacobi sweeps, one grid barrier each
    for (int it = 1; it <= a.n_iter; ++it) {
      const bool first = it == 1, last = it == a.n_iter, average = (it & 1) == 0;
      if (!first) {
        const float4* J4 = reinterpret_cast<const float4*>(a.Jf[(it - 1) & 1]);
        for (int i = tid; i < 2 * n_ant; i += kSolveThreads) Js[(i & 1) * n_ant + (i >> 1)] = __ldcg(J4 + i);
      }
      __syncthreads();
      // normal-equation terms of this warp's slot: A = sum_q V_pq J_q (8 reals),
      // C = sum_q J_q^H J_q (c00, c11, re c01, im c01); per-lane FP32 partials
      float v[16];
      #pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
      if (my_live) {
        const float4* row0 = rows + (size_t)slot * 2 * n_ant;
        const float4* row1 = row0 + n_ant;
        #pragma unroll 2
        for (int qq = lane + 32 * wi; qq < n_ant; qq += 32 * W) {
          const float4 v0 = row0[qq], v1 = row1[qq];    // V_pp = 0 in the row
          float4 j0 = first ? make_float4(1.f, 0.f, 0.f, 0.f) : Js[qq];
          float4 j1 = first ? make_float4(0.f, 0.f, 1.f, 0.f) : Js[n_ant + qq];
          if (qq == my_p) j0 = j1 = make_float4(0.f, 0.f, 0.f, 0.f);   // C excludes q = p
          // A += V J (entries row-major, complex interleaved)
          v[0] = fmaf(v0.x, j0.x, v[0]); v[0] = fmaf(-v0.y, j0.y, v[0]);
          v[0] = fmaf(v0.z, j1.x, v[0]); v[0] = fmaf(-v0.w, j1.y, v[0]);
          v[1] = fmaf(v0.x, j0.y, v[1]); v[1] = fmaf(v0.y, j0.x, v[1]);
          v[1] = fmaf(v0.z, j1.y, v[1]); v[1] = fmaf(v0.w, j1.x, v[1]);
          v[2] = fmaf(v0.x, j0.z, v[2]); v[2] = fmaf(-v0.y, j0.w, v[2]);
          v[2] = fmaf(v0.z, j1.z, v[2]); v[2] = fmaf(-v0.w, j1.w, v[2]);
          v[3] = fmaf(v0.x, j0.w, v[3]); v[3] = fmaf(v0.y, j0.z, v[3]);
          v[3] = fmaf(v0.z, j1.w, v[3]); v[3] = fmaf(v0.w, j1.z, v[3]);
          v[4] = fmaf(v1.x, j0.x, v[4]); v[4] = fmaf(-v1.y, j0.y, v[4]);
          v[4] = fmaf(v1.z, j1.x, v[4]); v[4] = fmaf(-v1.w, j1.y, v[4]);
          v[5] = fmaf(v1.x, j0.y, v[5]); v[5] = fmaf(v1.y, j0.x, v[5]);
          v[5] = fmaf(v1.z, j1.y, v[5]); v[5] = fmaf(v1.w, j1.x, v[5]);
          v[6] = fmaf(v1.x, j0.z, v[6]); v[6] = fmaf(-v1.y, j0.w, v[6]);
          v[6] = fmaf(v1.z, j1.z, v[6]); v[6] = fmaf(-v1.w, j1.w, v[6]);
          v[7] = fmaf(v1.x, j0.w, v[7]); v[7] = fmaf(v1.y, j0.z, v[7]);
          v[7] = fmaf(v1.z, j1.w, v[7]); v[7] = fmaf(v1.w, j1.z, v[7]);
          // C += J^H J: c00, c11, c01 = sum_r conj(J_r0) J_r1
          v[8] = fmaf(j0.x, j0.x, v[8]); v[8] = fmaf(j0.y, j0.y, v[8]);
          v[8] = fmaf(j1.x, j1.x, v[8]); v[8] = fmaf(j1.y, j1.y, v[8]);
          v[9] = fmaf(j0.z, j0.z, v[9]); v[9] = fmaf(j0.w, j0.w, v[9]);
          v[9] = fmaf(j1.z, j1.z, v[9]); v[9] = fmaf(j1.w, j1.w, v[9]);
          v[10] = fmaf(j0.x, j0.z, v[10]); v[10] = fmaf(j0.y, j0.w, v[10]);
          v[10] = fmaf(j1.x, j1.z, v[10]); v[10] = fmaf(j1.y, j1.w, v[10]);
          v[11] = fmaf(j0.x, j0.w, v[11]); v[11] = fmaf(-j0.y, j0.z, v[11]);
          v[11] = fmaf(j1.x, j1.w, v[11]); v[11] = fmaf(-j1.y, j1.z, v[11]);
        }
      }
      if (!last) {
        const float wsum = warp_reduce_scatter16f(v, lane);
        if ((lane & 1) == 0 && (lane >> 1) < 12) s_wp[warp][lane >> 1] = wsum;
      } else {
        // the last sweep's sums, which the FP64 solve and the status read: the
        // lane partials converted to FP64 and every later addition in FP64
        #pragma unroll
        for (int h = 0; h < 2; ++h) {
          double d[8];
          #pragma unroll
          for (int u = 0; u < 8; ++u) d[u] = (h == 0 || u < 4) ? (double)v[8 * h + u] : 0.0;
          const double dsum = warp_reduce_scatter8d(d, lane);
          const int u = 8 * h + ((lane >> 2) & 7);
          if ((lane & 3) == 0 && u < 12) s_wp64[warp][u] = dsum;
        }
      }
      __syncthreads();
      // totals: total i = 12 s + u (slot s, value u) on warp i & 3 (the four
      // sub-partitions), the slot's W warp sums added in FP64 in a fixed order
      // (the last sweep's warp sums are FP64 from the lane partials on)
      if (tid < 128) {
        for (int i = (tid & 31) * 4 + (tid >> 5); i < 12 * a.apc; i += 128) {
          const int s = i / 12, u = i - 12 * s, w0 = s * W;
          double tot;
          if (!last) {
            tot = (double)s_wp[w0][u];
            for (int w = 1; w < W; ++w) tot += (double)s_wp[w0 + w][u];
          } else {
            tot = s_wp64[w0][u];
            for (int w = 1; w < W; ++w) tot += s_wp64[w0 + w][u];
            s_tot64[i] = tot;
          }
          s_tot[i] = (float)tot;
        }
      }
      __syncthreads();
      // ---- 2x2 solves: lane (slot tid / 4, entry tid % 4) of the first warps.
      // Sweeps before the last: solve, iterate and averaging in FP32; the last
      // sweep in FP64, with its relative change against the FP32 previous iterate
      float2* Jf_new = a.Jf[it & 1];
      if (warp < (4 * a.apc + 31) / 32) {
        const int s = tid >> 2, e = tid & 3, p = blockIdx.x + s * G;
        const bool live = s < a.apc && p < n_ant;
        float2 Jn = make_float2(0.f, 0.f);
        if (!last) {
          if (live) {
            const float2 Jo = Jold[s * 4 + e];
            Jn = solve_entry<float>(s_tot + s * 12, Sf, e);
            if (average) Jn = make_float2(0.5f * (Jn.x + Jo.x), 0.5f * (Jn.y + Jo.y));
          }
        } else {
          double dn = 0.0, nn = 0.0;
          int bad = 0;
          if (live) {
            const float2 Jo = Jold[s * 4 + e];
            double2 Jd = solve_entry<double>(s_tot64 + s * 12, a.src[3 * k + 2], e);
            if (average) Jd = make_double2(0.5 * (Jd.x + (double)Jo.x), 0.5 * (Jd.y + (double)Jo.y));
            const double dx = Jd.x - (double)Jo.x, dy = Jd.y - (double)Jo.y;
            dn = dx * dx + dy * dy;
            nn = Jd.x * Jd.x + Jd.y * Jd.y;
            bad = !(isfinite(Jd.x) && isfinite(Jd.y));
            Jn = make_float2((float)Jd.x, (float)Jd.y);
            a.jones[((size_t)k * n_ant + p) * 4 + e] = Jn;
          }
          #pragma unroll
          for (int o = 1; o <= 2; o <<= 1) {
            dn += __shfl_xor_sync(0xffffffffu, dn, o);
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
          }
          if (live && e == 0) {
            double* pt = a.part + ((size_t)q * n_ant + p) * 4;
            pt[0] = dn;
            pt[1] = nn;
            pt[2] = (double)bad;
          }
        }
        if (live) {
          Jold[s * 4 + e] = Jn;
          Jf_new[(size_t)p * 4 + e] = Jn;
        }
      }
      solve_arrive(a.sync);
      if (!solve_wait(a.sync, ++nbar, (unsigned)G, &s_flag)) {
        if (tid == 0) a.status[k] = kSolveStatusTimeout;
        return;
      }
    }
  }

  // ---- after the block's last source (no barrier needed: the launch ends here):
  // its model matrices, then every source's status from the per-antenna norms
  {
    const int q = a.n_blk - 1, k = a.s0 + q;
    const float S = (float)a.src[3 * k + 2];
    const float2* J = a.jones + (size_t)k * n_ant * 4;
    for (int64_t bl = (int64_t)blockIdx.x * kSolveThreads + tid; bl < a.n_bl; bl += (int64_t)G * kSolveThreads) {
      float2 M[4];
      block_model_cg(J, a.bl_ant[bl], S, M);
      float4* d = reinterpret_cast<float4*>(a.M + ((size_t)q * a.n_bl + bl) * 4);
      d[0] = make_float4(M[0].x, M[0].y, M[1].x, M[1].y);
      d[1] = make_float4(M[2].x, M[2].y, M[3].x, M[3].y);
    }
  }
  double* s_red = reinterpret_cast<double*>(solve_smem);          // [3][kSolveThreads]
  for (int q = blockIdx.x; q < a.n_blk; q += G) {                  // CTA-uniform
    double dn = 0.0, nn = 0.0, bad = 0.0;
    for (int p = tid; p < n_ant; p += kSolveThreads) {
      const double* pt = a.part + ((size_t)q * n_ant + p) * 4;
      dn += __ldcg(pt);
      nn += __ldcg(pt + 1);
      bad += __ldcg(pt + 2);
    }
    s_red[tid] = dn;
    s_red[kSolveThreads + tid] = nn;
    s_red[2 * kSolveThreads + tid] = bad;
    __syncthreads();
    for (int o = kSolveThreads / 2; o > 0; o >>= 1) {     // fixed order: deterministic
      if (tid < o) {
        s_red[tid] += s_red[tid + o];
        s_red[kSolveThreads + tid] += s_red[kSolveThreads + tid + o];
        s_red[2 * kSolveThreads + tid] += s_red[2 * kSolveThreads + tid + o];
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double rel = sqrt(s_red[0] / s_red[kSolveThreads]);
      a.status[a.s0 + q] = (s_red[2 * kSolveThreads] != 0.0 || !isfinite(rel)) ? -4 : (rel > 1e-6 ? 1 : 0);
      a.rel[a.s0 + q] = rel;
    }
    __syncthreads();
  }
}

}  // namespace rts
