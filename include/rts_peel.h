/* rts_peel.h - C ABI of the GB300 calibrate-and-peel library (librtspeel.so).
 *
 * The library implements the per-source loop of the Calibration-Measurement
 * Loop (CML) of the MWA Real Time System (Edgar et al., arXiv:1003.5575,
 * Section 3, the CML item of the stage list: the CML steps sequentially
 * through a list of calibrator sources, reducing calibration to a set of
 * linear equations per source whose unknowns include a 2x2 Jones matrix per
 * tile in the direction of the calibrator).  For each source in list order it
 * phase-rotates every 2x2 visibility to the source direction, averages over
 * the cadence, solves per-antenna Jones matrices by alternating least squares
 * and subtracts the predicted source from the residual.
 *
 * Conventions (the paper prints no formula for the loop; these are the
 * standard measurement-equation readings the library follows):
 *   V_ij(t,c)  = sum_k S_k J_i^k J_j^kH exp(-2 pi i phi_k(t,ij,c))
 *   phi_k      = (u l_k + v m_k + w (n_k - 1)) nu_c / c_light  [turns],
 *                n_k = sqrt(1 - l_k^2 - m_k^2), (u,v,w)_ij = uvw_i - uvw_j
 *   baselines  i < j (no autocorrelations), index
 *              bl(i,j) = i*n_ant - i*(i+1)/2 + (j - i - 1)
 *   2x2 layout [XX, XY, YX, YY] row major, complex = interleaved (re, im)
 *   cube       vis[n_time][n_bl][n_chan][4] complex
 *              (complex64 in RTS_PREC_MIXED, complex128 in RTS_PREC_FP64)
 *              device cubes and averages (d_vis, d_resid, d_avg) start on a
 *              16-byte boundary (the kernels move a polarisation pair per
 *              16-byte access; a misaligned pointer is RTS_EINVAL)
 *   Jones      jones[n_src][n_ant][4] complex, same precision as the cube;
 *              device Jones arrays (d_jones, d_gain, d_slope) also start
 *              on a 16-byte boundary (RTS_EINVAL otherwise)
 *   sources    host double [n_src][3] = (l, m, S in Jy), in peel order
 *
 * Ownership: the caller owns every pointer it passes; "d_" pointers are
 * device memory, "h_" pointers host memory.  The handle owns the device
 * workspace and frees it in rts_peel_destroy.  rts_peel_init allocates the
 * workspace of the peel (the paper's advice in Section 5 to pre-allocate all
 * workspace at initialisation): the per-source buffers, the blocked
 * schedule's geometry tables, streams and solve set-up, and the Taylor
 * cadence's moments, so rts_peel_cadence, _cadence_taylor, _cadence_host,
 * _predict, _rotate_average and _solve allocate nothing.  Two workspaces whose
 * size depends on how the handle is used are allocated on first use and kept:
 * the adjoint's (first rts_peel_grad or rts_peel_offsets: 88 bytes per
 * baseline for each of max_sources sources) and the pipeline's two
 * device cubes and page-locked staging (first rts_peel_pipeline_submit); a
 * warm-up call before real-time use moves that allocation out of the loop.  Calls are asynchronous on `stream` (a cudaStream_t, NULL
 * = legacy default stream) unless an h_status pointer is given, which makes
 * the call wait for its stream.  A handle must not be used from two host
 * threads at once.
 *
 * Errors: every int-returning call returns RTS_OK (0) or a negative code; the
 * text of the last error is available from rts_peel_last_error.  Invalid
 * arguments are rejected on the host before any device work.  No call aborts
 * the process or traps on the device.
 */
#ifndef RTS_PEEL_H
#define RTS_PEEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTS_OK               0
#define RTS_NOT_CONVERGED    1   /* per-source status only */
#define RTS_EINVAL         (-1)  /* bad argument */
#define RTS_ENOMEM         (-2)  /* device allocation failed */
#define RTS_ECUDA          (-3)  /* CUDA runtime error (launch, copy, device) */
#define RTS_ENONFINITE     (-4)  /* NaN/Inf in averaged data or in a Jones solve */

#define RTS_PREC_MIXED 0  /* complex64 cube; FP64 phase and normal-equation sums */
#define RTS_PREC_FP64  1  /* complex128 cube; FP64 everywhere (plain comparator) */

typedef struct rts_peel_t rts_peel_t;   /* opaque handle */

typedef struct rts_peel_config {
  int32_t n_ant;        /* tiles, 2 .. 8192 */
  int32_t n_chan;       /* channels, 1 .. 65536 */
  int32_t n_time;       /* time samples per cadence, 1 .. 1024 */
  int32_t n_iter;       /* ALS sweeps per source, 1 .. 10000 (20 is the default reading) */
  int32_t precision;    /* RTS_PREC_MIXED or RTS_PREC_FP64 */
  int32_t max_sources;  /* largest n_src any call will pass, >= 1 */
  const double* uvw;    /* host [n_time][n_ant][3] antenna (u, v, w) in metres; copied */
  const double* freq_hz;/* host [n_chan] channel centres in Hz; must be uniformly spaced
                           (nu_c = nu_0 + c dnu to 1e-9 relative); copied */
  int32_t sources_per_pass; /* RTS_PREC_MIXED only: 1 = one streaming pass per source
                           (subtract k fused with the average of k+1); 8, 16, 32 or 64 =
                           one pass per block of that many sources, the averages inside a
                           block corrected in closed form (same results); 0 = library
                           default (RTS_BLOCK) */
  int32_t block_kernel;  /* blocked peel only: RTS_BLOCK_AUTO (0: the tcgen05 pass when
                           n_chan <= 768, else the mma.sync pass when n_chan <= 960, else
                           the FP32 pass), RTS_BLOCK_FMA (the FP32 FMA pass),
                           RTS_BLOCK_TENSOR (TF32 mma.sync with split operands;
                           n_chan <= 960, else RTS_EINVAL), RTS_BLOCK_TCGEN05 (tcgen05.mma
                           with TMEM accumulators, TF32 with split operands; n_chan <= 768,
                           else RTS_EINVAL).  All give FP32-level accuracy. */
  int32_t solve_kernel;  /* blocked peel only: RTS_SOLVE_AUTO (0: the corrected averages,
                           ALS sweeps and model matrices of a whole block in one
                           cooperative launch whose CTAs meet at grid-wide barriers, when
                           the device supports cooperative launches and the rows of
                           ceil(n_ant / n_SM) antennas fit in shared memory, about
                           n_ant <= 900 on GB300; otherwise as RTS_SOLVE_LAUNCHES),
                           RTS_SOLVE_LAUNCHES (1: one launch per ALS sweep, per
                           correction and per model step).  The cooperative launch
                           solves the 2x2 systems of the sweeps before the last in
                           FP32 and the last in FP64, the per-step launches every
                           sweep in FP64; both accumulate the normal equations'
                           cross-thread sums in FP64, and their results agree to
                           FP32 rounding (statuses outside a band around 1e-6). */
  int32_t grad_kernel;   /* RTS_PREC_MIXED adjoint (rts_peel_grad, rts_peel_offsets):
                           RTS_GRAD_AUTO (0: phasors factorised per 16-channel group into
                           two shared-memory tables, T1[q] T2[r], when the tables of all
                           n_src sources fit in shared memory, about n_src <= 580 on
                           GB300; otherwise as RTS_GRAD_DIRECT), RTS_GRAD_DIRECT (1: one
                           hardware sin/cos per source and sample).  FP32-level accuracy
                           either way; RTS_PREC_FP64 always evaluates every phasor in FP64. */
  int32_t band_n_chan;   /* channel sharding (Section 3.1: channel groups on separate
                           workers, combined centrally): 0 = the handle's channels are the
                           whole band; else the band has band_n_chan uniform channels and
                           freq_hz are its channels band_chan0 .. band_chan0 + n_chan - 1.
                           A shard's averages are normalised by the whole band's sample
                           count and its in-block corrections are taken over the whole
                           band, so the shards' partial averages add up to the band's.
                           Shard handles peel only through the rts_peel_shard_* calls
                           (blocked peel, RTS_PREC_MIXED, sources_per_pass > 1). */
  int32_t band_chan0;    /* this handle's first channel in the band (0 when band_n_chan = 0) */
} rts_peel_config;

#define RTS_GRAD_AUTO   0
#define RTS_GRAD_DIRECT 1

#define RTS_SOLVE_AUTO     0
#define RTS_SOLVE_LAUNCHES 1

#define RTS_BLOCK_AUTO   0
#define RTS_BLOCK_FMA    1
#define RTS_BLOCK_TENSOR 2
#define RTS_BLOCK_TCGEN05 3

#define RTS_BLOCK 64   /* default sources per streaming pass of the blocked peel */

/* Validate `cfg`, allocate the device workspace on the current device, copy
 * uvw and frequencies.  On success *out is a new handle.  Errors: RTS_EINVAL
 * (cfg, sizes, non-uniform channels, non-finite uvw), RTS_ENOMEM, RTS_ECUDA;
 * *out is then NULL and the message is available from rts_peel_last_error(NULL). */
int rts_peel_init(const rts_peel_config* cfg, rts_peel_t** out);

/* Replace the antenna uvw for the next cadence (host [n_time][n_ant][3] metres).
 * Ordered on `stream` before later calls on that stream. */
int rts_peel_set_uvw(rts_peel_t* h, const double* h_uvw, void* stream);

/* One cadence of the calibrate-and-peel loop (Section 3, CML).
 *   d_vis    [n_time][n_bl][n_chan][4] input visibilities (read only)
 *   d_resid  same shape; receives the residual after all n_src sources are
 *            subtracted.  d_resid == d_vis peels in place.  Other overlap is
 *            undefined.
 *   n_src    0 .. max_sources;  h_src  host [n_src][3] (l, m, S), peel order;
 *            l^2 + m^2 < 1, S > 0 and finite.
 *   d_jones  [n_src][n_ant][4] receives each source's solved Jones matrices.
 *   h_status optional host [n_src]: 0 converged, 1 not converged (last relative
 *            change of the ALS sweep > 1e-6), RTS_ENONFINITE.  When given,
 *            the call waits for the stream and returns RTS_ENONFINITE if any
 *            source hit a non-finite value.
 * Each source: average in its direction (fused with the previous source's
 * subtraction), n_iter Jacobi ALS sweeps from J = I with every second sweep
 * averaged with the previous iterate, then subtraction. */
int rts_peel_cadence(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src,
                     const double* h_src, void* d_jones, int32_t* h_status, void* stream);

/* One cadence with the gains Taylor-expanded in frequency (Section 3.1: when
 * consecutive channels are combined, the unknown tile gain may be
 * Taylor-expanded in frequency).  First order about the band centre:
 *   J_p^k(c) = G_p^k + x_c H_p^k,  x_c = (c - (n_chan - 1)/2) / n_chan,
 * so each source's model is S (G_i + x_c H_i)(G_j + x_c H_j)^H e^{-2 pi i phi}.
 * Each source in list order: one streaming pass subtracts the previous
 * source's model and takes three channel moments mean_{t,c} x_c^n R e^{+2 pi i phi}
 * (n = 0, 1, 2) of the residual in its direction; n_iter Jacobi ALS sweeps on
 * X_p = [G_p H_p] (2x4) from G = I, H = 0, every second averaged with the
 * previous iterate, each solving the 4x4 normal equations (FP64 sums and
 * Cholesky solve); then its model is subtracted.  One pass per source
 * whatever sources_per_pass says.
 *   d_vis, d_resid, n_src, h_src, h_status, stream: as rts_peel_cadence
 *            (status from the relative change of X in the last sweep).
 *   d_gain   [n_src][n_ant][4] complex64 receives G (the gain at the band centre).
 *   d_slope  [n_src][n_ant][4] complex64 receives H (the change of the gain
 *            across one band width).
 * RTS_PREC_MIXED handles only, n_chan >= 2 (else RTS_EINVAL). */
int rts_peel_cadence_taylor(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src,
                            const double* h_src, void* d_gain, void* d_slope, int32_t* h_status,
                            void* stream);

/* One cadence of a channel shard, step by step (Section 3.1: channel groups are
 * processed by separate workers and their numbers combined centrally).  Every
 * shard of the band runs the same calls with the same source list; between
 * the calls the caller sums the shards' partial averages, in place, across the
 * shards (an all-reduce of n_float floats per block of sources, e.g. NCCL on
 * `stream`), so every shard solves the same Jones matrices from the whole
 * band's averages and subtracts them from its own channels:
 *   rts_peel_shard_begin(h, ...)         first pass: partial averages of block 0
 *   loop: rts_peel_shard_partials(h, &p, &n); sum p[0..n) over the shards;
 *         rc = rts_peel_shard_step(h, h_status, stream)
 *         (solve the block, subtract it, partial averages of the next block;
 *          rc = 1: sum again and step again; rc = 0: the cadence is done)
 * d_vis, d_resid, n_src (>= 1), h_src, d_jones: as rts_peel_cadence, the cube
 * holding this handle's n_chan channels.  The source list is copied at begin.
 * d_partial: float [n_blk][n_bl][4][re, im] of the library's workspace, valid
 * until the next step.  All calls of a cadence use the same stream; the
 * partials are ready on it when begin / step return, and step orders its work
 * after what the caller enqueued on it.  h_status (may be NULL) is filled by the
 * final step, as in rts_peel_cadence.  Errors: RTS_EINVAL (a one-source-per-pass
 * handle, a call out of order, another stream), or as rts_peel_cadence; an
 * error ends the cadence. */
int rts_peel_shard_begin(rts_peel_t* h, const void* d_vis, void* d_resid, int32_t n_src, const double* h_src,
                         void* d_jones, void* stream);
int rts_peel_shard_partials(rts_peel_t* h, float** d_partial, int64_t* n_float);
int rts_peel_shard_step(rts_peel_t* h, int32_t* h_status, void* stream);

/* rts_peel_cadence on host buffers: copies h_vis to the caller's device buffer
 * d_work (cube-sized), peels it in place, copies the residual to h_resid and
 * the Jones matrices to h_jones ([n_src][n_ant][4]), and waits for the stream.
 * h_vis and h_resid may be the same buffer.  Page-locked host memory gives the
 * fastest copies. */
int rts_peel_cadence_host(rts_peel_t* h, const void* h_vis, void* h_resid, int32_t n_src,
                          const double* h_src, void* h_jones, int32_t* h_status,
                          void* d_work, void* stream);

/* Pipelined cadences on host buffers (the paper's Section 5 proposes streaming
 * the next data onto the GPU while the previous cadence is processed).
 * rts_peel_pipeline_submit enqueues, and returns without waiting:
 *   copy-in stream   h_vis -> one of two library-owned device cubes
 *   compute stream   the peel of that cube in place (after its copy-in)
 *   copy-out stream  residual -> h_resid, Jones and statuses -> library-owned
 *                    page-locked staging (after the peel)
 * so the copies of one cadence overlap the peel of the other.  The Jones
 * matrices (h_jones [n_src][n_ant][4]) and statuses (h_status [n_src], may be
 * NULL) are written to the caller's buffers when the cadence retires: in
 * rts_peel_pipeline_wait, or in the submit that reuses its slot.  At most two
 * cadences are in flight: a third submit first waits for the oldest one.  The
 * host buffers of a cadence must stay valid and untouched until it retires;
 * h_vis and h_resid must be page-locked (rts_host_alloc) for the copies to
 * overlap (h_jones and h_status may be ordinary memory).  The two device cubes
 * and the staging buffers are allocated on the first submit and kept.
 * rts_peel_pipeline_wait waits for every submitted cadence and returns
 * RTS_ENONFINITE if any source of any of them had a non-finite solve. */
int rts_peel_pipeline_submit(rts_peel_t* h, const void* h_vis, void* h_resid, int32_t n_src,
                             const double* h_src, void* h_jones, int32_t* h_status);
int rts_peel_pipeline_wait(rts_peel_t* h);

/* Model visibilities: d_vis = (accumulate ? d_vis : 0) +
 * sum_k S_k J_i^k J_j^kH exp(-2 pi i phi_k) for the n_src sources in h_src with
 * Jones d_jones [n_src][n_ant][4] (the predict step of the loop, for all sources). */
int rts_peel_predict(rts_peel_t* h, void* d_vis, int32_t n_src, const double* h_src,
                     const void* d_jones, int32_t accumulate, void* stream);

/* The average step alone: d_avg[n_bl][4] = mean_{t,c} vis exp(+2 pi i phi(l, m)). */
int rts_peel_rotate_average(rts_peel_t* h, const void* d_vis, double l, double m,
                            void* d_avg, void* stream);

/* The solve step alone: Jones d_jones[n_ant][4] for a source of flux S from its
 * averaged visibilities d_avg[n_bl][4]; optional *h_status as in rts_peel_cadence.
 * d_avg and d_jones start on a 16-byte boundary (else RTS_EINVAL). */
int rts_peel_solve(rts_peel_t* h, const void* d_avg, double S, void* d_jones,
                   int32_t* h_status, void* stream);

/* The relative change ||J_n - J_(n-1)||_F / ||J_n||_F of each source's last ALS
 * sweep in the last cadence run on this handle (rts_peel_cadence, _host,
 * _taylor; slot 0 after rts_peel_solve): the number each status compares with
 * 1e-6 (Section 3, CML: the per-source solve; the threshold is this library's
 * reading).  h_rel host [n_src] doubles, n_src <= the cadence's source count.
 * Copied on `stream` (pass the cadence's stream) and waited for.  RTS_EINVAL
 * for a NULL handle or pointer or n_src outside [0, max_sources]. */
int rts_peel_rel(rts_peel_t* h, int32_t n_src, double* h_rel, void* stream);

/* The phase step alone (Section 2: visibilities are Fourier samples of the
 * sky; the loop's phase rotation to a source direction): for n_pair
 * (time, baseline) pairs, d_tb DEVICE int32 [n_pair][2] = (t, bl), the phase of
 * direction (l, m) at every channel, d_phase DEVICE double [n_pair][n_chan], in
 * turns in [-1/2, 1/2), as the peel's kernels form it: the FP64 delay
 * tau = u l + v m + w (n - 1), the Q0.64 fixed-point phases A = frac(tau nu_0 / c)
 * and B = frac(tau dnu / c), and channel c at A + c B modulo one turn (exact
 * integer arithmetic).  form = 0 returns that Q0.64 phase (the streaming,
 * predict and adjoint kernels); form = 1 the FP32 value the kernels hand to the
 * hardware sin/cos (rounded to Q0.32 first); form = 2 the Q0.64 phase as the
 * blocked schedule forms it, from the two antennas' delays
 * tau_i = u_i l + v_i m + w_i (n - 1) (the same geometry: uvw_ij = uvw_i - uvw_j)
 * as the difference of their Q0.64 phases modulo one turn.  A pair with t or
 * bl out of range gets NaN.  Asynchronous on `stream`.  RTS_EINVAL for a NULL
 * handle or pointer, n_pair < 0, form not 0, 1 or 2, or a direction with
 * l^2 + m^2 >= 1. */
int rts_peel_phases(rts_peel_t* h, double l, double m, int32_t n_pair, const int32_t* d_tb,
                    int32_t form, double* d_phase, void* stream);

/* The solve step without any allocation, for callers that cannot call
 * cudaMalloc or create a handle: code that runs after a real-time pipeline has
 * frozen its memory at start-up, code inside another framework whose device
 * memory is owned by that framework's pool, or code in a stream-capture
 * region, where allocation calls are not allowed.  The paper has no
 * counterpart; this is an interface addition of this library.
 *   d_avg    device [n_bl][4] averaged visibilities (complex64 for
 *            RTS_PREC_MIXED, complex128 for RTS_PREC_FP64), as for rts_peel_solve
 *   n_ant    2 .. RTS_NOALLOC_MAX_ANT; larger arrays are rejected with RTS_EINVAL
 *   d_avg and d_jones start on a 16-byte boundary (else RTS_EINVAL)
 *   d_jones  device [n_ant][4] output, same precision as d_avg
 *   h_status optional host int: as in rts_peel_solve (the call then waits)
 * Scratch: one static device array of about 200 KB (sized for
 * RTS_NOALLOC_MAX_ANT antennas) that every device loading the library holds
 * until the process exits.  The first call on a device looks up that array's
 * device address; make that first call before any stream capture begins.
 * All calls share the array and it keeps the last call's contents, so calls
 * that overlap on the GPU (different streams, or different host threads on
 * one device) race with each other: serialise them.  Errors are reported by
 * the return code and rts_peel_last_error(NULL). */
#define RTS_NOALLOC_MAX_ANT 1024
int rts_peel_solve_noalloc(const void* d_avg, int32_t n_ant, double S, int32_t n_iter,
                           int32_t precision, void* d_jones, int32_t* h_status, void* stream);

/* Loss and gradient of the multi-source model (the adjoint of the predict step):
 *   L = sum_{t,bl,c} || V - sum_k S_k J_i^k J_j^kH exp(-2 pi i phi_k) ||_F^2
 *   d_vis   [n_time][n_bl][n_chan][4]; d_jones [n_src][n_ant][4];
 *   d_src   DEVICE double [n_src][3] (l, m, S)
 *   d_loss  device double[1] <- L
 *   d_gJ    device [n_src][n_ant][4] complex (cube precision) <- dL/dRe J + i dL/dIm J,
 *           or NULL
 *   d_gsrc  device double [n_src][3] <- (dL/dl, dL/dm, dL/dS), or NULL
 * Phasors are recomputed, never stored. */
int rts_peel_grad(rts_peel_t* h, const void* d_vis, int32_t n_src, const void* d_jones,
                  const double* d_src, double* d_loss, void* d_gJ, double* d_gsrc,
                  void* stream);

/* Ionospheric position offsets of the peeled sources (Section 3: each
 * calibrator's fit also returns a shift of its apparent position caused by
 * ionospheric refraction; Section 3.1: that fit needs six numbers per source
 * and is described by two, the ionosphere's response is a known function of
 * frequency, and workers send their numbers to a master that builds the
 * solution).  Reading: the shift of source k at channel c is
 * s_c (dl, dm) with s_c = (nu_ref/nu_c)^alpha (alpha = 2: refraction scales as
 * lambda^2; alpha = 0: a frequency-independent shift), and the six numbers are
 * the Gauss-Newton statistics of the loss L of rts_peel_grad at dl = dm = 0:
 *   H_pq = 2 (2 pi)^2 sum_{t,bl,c} a_p a_q w_c^2 ||S_k J_i J_j^H||_F^2,
 *   a_l = u - w l/n, a_m = v - w m/n, w_c = s_c nu_c / c,
 *   g = (dL/d dl, dL/d dm),  (dl, dm) = -H^-1 g, or (0, 0) where det H <= 0.
 * All six are sums over channels: GPUs holding different channel groups add
 * their d_out arrays (one all-reduce of 6 doubles per source, with a common
 * nu_ref) and call rts_offsets_solve on the sum.  The Jones matrices should be
 * ones calibrated without the shift (for instance from a previous cadence):
 * free per-antenna gains absorb most of a shift as antenna phase gradients.
 *   d_vis      [n_time][n_bl][n_chan][4] (cube precision); d_jones [n_src][n_ant][4]
 *   d_src      DEVICE double [n_src][3] (l, m, S)
 *   alpha      finite; nu_ref_hz > 0 (ignored when alpha == 0)
 *   d_out      device double [n_src][6] <- (H_ll, H_lm, H_mm, g_l, g_m, L)
 *   d_offsets  device double [n_src][2] <- (dl, dm) from this call's channels
 * n_src = 0 is a no-op; n_src > max_sources, a non-finite alpha or a bad
 * nu_ref_hz give RTS_EINVAL.  H and the solve are FP64; g and L come from the
 * adjoint sweep in the handle's precision.  The gradient workspace of
 * rts_peel_grad is reused (plus n_chan doubles on the first call with
 * alpha != 0). */
int rts_peel_offsets(rts_peel_t* h, const void* d_vis, int32_t n_src, const void* d_jones,
                     const double* d_src, double alpha, double nu_ref_hz, double* d_out,
                     double* d_offsets, void* stream);
/* (dl, dm) = -H^-1 g for each source from six numbers per source laid out as
 * rts_peel_offsets writes them (d_out [n_src][6], device), into d_offsets
 * [n_src][2] (device); (0, 0) where det H <= 0.  Needs no handle; errors
 * (RTS_EINVAL for n_src < 0 or NULL pointers, RTS_ECUDA for a failed launch)
 * are reported by the return code and rts_peel_last_error(NULL). */
int rts_offsets_solve(const double* d_out, int32_t n_src, double* d_offsets, void* stream);

/* Kernel timing and launch counts (the paper's Section 5 instruments every
 * kernel for bandwidth and FLOP counts; this is the same tracing hook).
 * Kernel classes, indices into the arrays below:                           */
#define RTS_K_AVERAGE      0  /* rotate + average (first source of a cadence) */
#define RTS_K_SUB_AVERAGE  1  /* subtract source k + average for source k+1 */
#define RTS_K_SUBTRACT     2  /* subtract the last source */
#define RTS_K_SOLVE        3  /* ALS sweeps + status of one source (timed as one group) */
#define RTS_K_PREDICT      4  /* model prediction */
#define RTS_K_GRAD         5  /* loss + adjoint sweep */
#define RTS_K_GRAD_REDUCE  6  /* adjoint reductions (per antenna / source / loss) */
#define RTS_K_BLOCK_PASS   7  /* blocked peel: subtract block b + average block b+1 */
#define RTS_K_BLOCK_FIX    8  /* blocked peel: in-block closed-form corrections, model matrices */
#define RTS_K_OFFSETS      9  /* position-offset normal equations and solve */
#define RTS_K_CLASSES     10
/* enable != 0: clear the counters and start bracketing every kernel (group)
 * with CUDA events on its stream; enable == 0: stop recording.  Launch
 * counts are always kept. */
int rts_peel_timing(rts_peel_t* h, int32_t enable);
/* Wait for the recorded events and return, per class, the summed device time
 * in ms (ms[RTS_K_CLASSES]), the number of timed groups (groups[RTS_K_CLASSES])
 * and the number of kernel launches since the last enable (launches[RTS_K_CLASSES]).
 * Any pointer may be NULL. */
int rts_peel_timing_read(rts_peel_t* h, double* ms, int64_t* groups, int64_t* launches);

/* The kernels the handle resolved at init (no paper counterpart: introspection
 * for benchmarks and tests).  *block_kernel: 0 when the handle peels one source
 * per pass, else RTS_BLOCK_FMA, RTS_BLOCK_TENSOR or RTS_BLOCK_TCGEN05 (the
 * choice RTS_BLOCK_AUTO made).  *solve_kernel: RTS_SOLVE_AUTO when the blocked
 * peel solves each block in one cooperative launch, else RTS_SOLVE_LAUNCHES.
 * Either pointer may be NULL.  RTS_EINVAL for a NULL handle. */
int rts_peel_kernels(const rts_peel_t* h, int32_t* block_kernel, int32_t* solve_kernel);

/* Measured FP64 fused multiply-add rate of the current device in TFLOP/s (no
 * paper counterpart: the roofline denominator of the RTS_PREC_FP64 path, which
 * is bound by FP64 arithmetic).  Runs a short kernel of independent FMA chains
 * on every SM (about a tenth of a second) and waits for it.  RTS_EINVAL for a
 * NULL pointer, RTS_ECUDA for a failed launch. */
int rts_fp64_rate(double* h_tflops);

/* Failure-detection self-test of the grid barrier the cooperative block solve
 * uses (no paper counterpart).  Launches n_cta CTAs (1 .. the device's
 * co-resident limit, at most 1024) on the current device, cooperatively, that
 * meet at `rounds` (1 .. 10000) barriers expecting n_cta + missing CTAs
 * (missing 0 or 1).  With missing = 0 every wait completes and
 * *h_completed = n_cta; with missing = 1 no wait can complete: each CTA's wait
 * runs out its 2 s limit or sees another CTA's abort flag, and the kernel
 * returns with *h_completed = 0 instead of hanging.  Synchronous; allocates
 * and frees a few bytes of device memory.  RTS_EINVAL for bad arguments,
 * RTS_ECUDA for a failed launch. */
int rts_barrier_selftest(int32_t n_cta, int32_t missing, int32_t rounds, int32_t* h_completed);

/* Page-locked host memory for the host-buffer calls (the paper, Section 4,
 * moved its host allocator to pinned memory for faster DMA).  rts_host_alloc
 * returns RTS_ENOMEM when the allocation fails; rts_host_free(NULL) is a no-op. */
int rts_host_alloc(uint64_t bytes, void** out);
int rts_host_free(void* p);

/* Message of the last failed call on `h` (or of the last failed rts_peel_init
 * when h is NULL).  The string stays valid until the next call on `h`. */
const char* rts_peel_last_error(const rts_peel_t* h);

/* Free the handle and its device workspace (NULL is accepted). */
void rts_peel_destroy(rts_peel_t* h);

#ifdef __cplusplus
}
#endif
#endif /* RTS_PEEL_H */
