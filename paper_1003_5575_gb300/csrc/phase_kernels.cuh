// The phase step alone: the per-channel phase of one direction on chosen
// (time, baseline) pairs, formed exactly as the streaming, blocked and adjoint
// kernels form it (common.cuh): FP64 delay tau = u l + v m + w (n - 1), two
// Q0.64 fixed-point phases A = frac(tau nu_0 / c), B = frac(tau dnu / c), and
// channel c at A + c B (mod 2^64, the integer wrap being the reduction modulo
// one turn).  Used to check that phase against a direct FP64 evaluation.
#pragma once
#include "common.cuh"

namespace rts {

// out[pair][c] in turns, [-1/2, 1/2): form 0, the Q0.64 phase of the baseline's
// FP64 delay (the streaming, predict and adjoint kernels); form 1, that phase
// as the FP32 value the kernels pass to the hardware sin/cos (rounded to Q0.32,
// then converted); form 2, the Q0.64 phase as the blocked schedule forms it,
// the difference of the two antennas' Q0.64 phases (their FP64 delays
// tau_i = u_i l + v_i m + w_i (n - 1)).  Pairs whose time or baseline index is
// out of range get NaN in every channel.
__global__ void __launch_bounds__(256) k_phase_table(const double* __restrict__ uvw, const int2* __restrict__ bl_ant,
                                                     int n_ant, int n_chan, int n_time, int64_t n_bl, SrcDir d,
                                                     double nu0_c, double dnu_c, int n_pair,
                                                     const int* __restrict__ tb, int form,
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
    unsigned long long A, B;
    if (form == 2) {
      const double* ui = uvw + ((size_t)t * n_ant + ij.x) * 3;
      const double* uj = uvw + ((size_t)t * n_ant + ij.y) * 3;
      const double ti = ui[0] * d.l + ui[1] * d.m + ui[2] * d.nm1, tj = uj[0] * d.l + uj[1] * d.m + uj[2] * d.nm1;
      A = frac_q64(ti * nu0_c) - frac_q64(tj * nu0_c);
      B = frac_q64(ti * dnu_c) - frac_q64(tj * dnu_c);
    } else {
      const double tau = delay_m(uvw, n_ant, t, ij.x, ij.y, d);
      A = frac_q64(tau * nu0_c);
      B = frac_q64(tau * dnu_c);
    }
    const unsigned long long ph = A + (unsigned long long)c * B;
    out[i] = form == 1 ? (double)q64_to_turns(ph) : (double)(long long)ph * (1.0 / kTwo64);
  }
}

}  // namespace rts
