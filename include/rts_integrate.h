/* rts_integrate.h - C ABI of the GB300 visibility integrator (librtspeel.so).
 *
 * Section 3 of Edgar et al. (arXiv:1003.5575), the first stage of the RTS
 * pipeline: the visibility integrator takes the correlator's 0.5 s samples and
 * integrates them into 2, 4 and 8 s groups, integrating baselines between
 * widely separated tiles for shorter times, because the Earth's rotation
 * changes their delays faster (coherence loss).  A visibility integrated for
 * 2 s appears four times in an 8 s cadence.
 *
 * Reading (R19 of the design notes): baseline b averages len[b] consecutive
 * fine samples (len[b] divides n_fine); output slot s of baseline b is the
 * mean of fine samples s len[b] .. (s + 1) len[b] - 1 for s < n_fine / len[b],
 * and the remaining slots up to n_slot are zero.  The group lengths come from
 * the caller, or from rts_integrate_lengths, which picks for each baseline the
 * longest allowed group whose baseline-length cut it passes.  Layouts:
 *   fine  [n_fine][n_bl][n_chan][4] complex64 (the cube layout of rts_peel.h)
 *   out   [n_slot][n_bl][n_chan][4] complex64
 * Sums are FP32 over at most n_fine samples, scaled by 1 / len.
 *
 * Ownership: the caller owns every pointer it passes; the handle owns a device
 * copy of the group lengths.  Calls are asynchronous on `stream`.  Errors:
 * RTS_OK (0) or a negative code of rts_peel.h; text from rts_integrate_last_error.
 */
#ifndef RTS_INTEGRATE_H
#define RTS_INTEGRATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rts_integ_t rts_integ_t;

/* Group length per baseline from its length |uvw_i - uvw_j| (metres, from the
 * antenna positions h_uvw [n_ant][3] at one time): baselines shorter than
 * cut_m[0] get len_for[0] fine samples, those in [cut_m[k-1], cut_m[k]) get
 * len_for[k], the rest len_for[n_cut].  cut_m ascending, n_cut 0 .. 8.
 * h_len receives [n_bl] in the baseline order of rts_peel.h.  Host only.
 * RTS_EINVAL for bad arguments. */
int rts_integrate_lengths(int32_t n_ant, const double* h_uvw, int32_t n_cut, const double* cut_m,
                          const int32_t* len_for, int32_t* h_len);

/* A handle for cubes of n_fine samples x n_bl baselines x n_chan channels with
 * the group lengths h_len [n_bl] (each >= 1 and dividing n_fine) and n_slot
 * output slots (>= n_fine / min len, <= n_fine).  RTS_EINVAL, RTS_ENOMEM, RTS_ECUDA. */
int rts_integrate_init(int32_t n_fine, int64_t n_bl, int32_t n_chan, const int32_t* h_len,
                       int32_t n_slot, rts_integ_t** out);

/* Integrate one cadence: d_fine -> d_out (device, 16-byte aligned, not
 * overlapping).  RTS_EINVAL for bad arguments, RTS_ECUDA for a failed launch. */
int rts_integrate_run(rts_integ_t* h, const void* d_fine, void* d_out, void* stream);

const char* rts_integrate_last_error(const rts_integ_t* h);
void rts_integrate_destroy(rts_integ_t* h);

#ifdef __cplusplus
}
#endif
#endif
