// The phase step alone: the per-channel phase of one direction on chosen
// (time, baseline) pairs, formed exactly as the streaming, blocked and adjoint
// kernels form it (common.cuh): FP64 delay tau = u l + v m + w (n - 1), two
// Q0.64 fixed-point phases A = frac(tau nu_0 / c), B = frac(tau dnu / c), and
// channel c at A + c B (mod 2^64, the integer wrap being the reduction modulo
// one turn).  Used to check that phase against a direct FP64 evaluation.
#pragma once
#include "common.cuh"

namespace rts {

// out[pair][c] in turns, [-1/2, 1/2): the Q0.64 phase (rounded == 0), or the
// FP32 value the kernels pass to the hardware sin/cos (rounded == 1: rounded to
// Q0.32, then converted).  Pairs whose time or baseline index is out of range
// get NaN in every channel.
__global__ void __launch_bounds__(256) k_phase_table(const double* __restrict__ uvw, const int2* __restrict__ bl_ant,
                                                     int n_ant, int n_chan, int n_time, int64_t n_bl, SrcDir d,
                                                     double nu0_c, double dnu_c, int n_pair,
                                                     const int* __restrict__ tb, int rounded,
                                                     double* __restrict__ out) {
  const int64_t n = (int64_t)n_pair * n_chan;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int pair = (int)(i / n_chan), c = (int)(i - (int64_t)pair * n_chan);
    const int t = tb[2 * pair];
    const int64_t bl = tb[2 * pair + 1];
    if (t < 0 || t >= n_time || bl < 0 || bl >= n_bl) {
      out[i] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const int2 ij = bl_ant[bl];
    const double tau = delay_m(uvw, n_ant, t, ij.x, ij.y, d);
    const unsigned long long ph = frac_q64(tau * nu0_c) + (unsigned long long)c * frac_q64(tau * dnu_c);
    out[i] = rounded ? (double)q64_to_turns(ph) : (double)(long long)ph * (1.0 / kTwo64);
  }
}

}  // namespace rts
