/* FP64 CPU oracle of the calibrate-and-peel loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path includes, links or
 * calls this code; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code with the CUDA library.
 *
 * Layout conventions (all arrays row-major, complex = interleaved re, im):
 *   uvw   [n_time][n_ant][3]            antenna uvw, metres; baseline
 *                                        uvw_ij = uvw_i - uvw_j
 *   freq  [n_chan]                      Hz
 *   vis   [n_time][n_bl][n_chan][4]     2x2 visibility [XX, XY, YX, YY]
 *   avg   [n_bl][4]                     rotated + averaged visibility
 *   jones [n_src][n_ant][4]             2x2 Jones [XX, XY, YX, YY]
 *   lmS   [n_src][3]                    l, m (direction cosines), S (Jy)
 *   baseline bl(i, j), i < j: bl = i*n_ant - i*(i+1)/2 + (j - i - 1)
 */
#ifndef RTS_ORACLE_H
#define RTS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int64_t orc_n_baselines(int32_t n_ant);
int64_t orc_baseline_index(int32_t n_ant, int32_t i, int32_t j);
void    orc_baseline_antennas(int32_t n_ant, int32_t* ant_i, int32_t* ant_j);

double  orc_delay_m(const double* uvw, int32_t n_ant, int32_t t, int32_t i, int32_t j,
                    double l, double m);
double  orc_phase_turns(double tau_m, double freq_hz);

void orc_predict(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                 const double* freq, int32_t n_src, const double* lmS, const double* jones,
                 double* vis, int32_t accumulate);
void orc_rotate_average(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, const double* vis, double l, double m,
                        double* avg);
int32_t orc_als(int32_t n_ant, const double* avg, double S, int32_t n_iter,
                double* jones, double* rel_change);
void orc_subtract(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                  const double* freq, double* vis, double l, double m, double S,
                  const double* jones);
int32_t orc_peel(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                 const double* freq, double* vis, int32_t n_src, const double* lmS,
                 int32_t n_iter, double* jones, int32_t* status, double* avg_per_src,
                 double* rel_per_src);
void orc_loss_grad(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                   const double* freq, const double* vis, int32_t n_src, const double* lmS,
                   const double* jones, double* loss, double* g_jones, double* g_l,
                   double* g_m, double* g_S);
void orc_offsets(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                 const double* freq, const double* vis, int32_t n_src, const double* lmS,
                 const double* jones, double alpha, double nu_ref, double* out,
                 double* offsets);
/* gains Taylor-expanded in frequency, J_p(c) = G_p + x_c H_p (reading R16) */
void orc_predict_taylor(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, int32_t n_src, const double* lmS, const double* gain,
                        const double* slope, double* vis, int32_t accumulate);
int32_t orc_als_taylor(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                       const double* freq, const double* vis, double l, double m, double S,
                       int32_t n_iter, double* gain, double* slope, double* rel_change);
int32_t orc_peel_taylor(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, double* vis, int32_t n_src, const double* lmS,
                        int32_t n_iter, double* gain, double* slope, int32_t* status,
                        double* rel_per_src);
int32_t orc_taylor_rotation(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                            const double* freq, const double* vis, double l, double m, double S,
                            const double* gain, double* slope, double* g, double* h);
void orc_taylor_moments(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, const double* vis, double l, double m, double* mom);
void orc_taylor_dterm(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                      const double* freq, double lj, double mj, double lk, double mk, double* dterm);
/* gridder: radial gridding convolution function from a table (reading R18) */
void orc_grid(int32_t n_pix, double r_max, const double* gcf, int32_t n_tab, int32_t n_vis,
              int32_t n_pol, const double* xy, const double* vis, double* grid);
/* visibility integrator: per-baseline averaging of len[b] fine samples (reading R19) */
void orc_integrate(int32_t n_fine, int64_t n_bl, int32_t n_chan, const int32_t* len, int32_t n_slot,
                   const double* fine, double* out);
int32_t orc_num_threads(void);
void    orc_set_num_threads(int32_t n);   /* OpenMP threads of the later calls (timing only) */

#ifdef __cplusplus
}
#endif
#endif
