/* FP64 CPU oracle of the MWA calibrate-and-peel loop.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg, never by the product path.  Plain loops,
 * double precision throughout, libm sin/cos.  Shares no code with the CUDA
 * library.
 *
 * What it follows.  Section 3 of the paper (the Calibration-Measurement Loop
 * paragraph) states the method only in words: the CML steps sequentially
 * through a list of calibrator sources, reduces calibration to linear
 * equations per source, and fits a 2x2 Jones matrix per tile in the direction
 * of each calibrator.  Section 2 describes visibilities as Fourier samples of
 * the sky for each pair of receptors.  The paper prints no equation for the
 * loop, so the steps below are the standard measurement-equation reading,
 * each listed as a reading in the design notes:
 *
 *   model   V_ij(t,c) = sum_k  S_k J_i^k J_j^kH exp(-2 pi i phi_k)        (R1, R2)
 *   phase   phi_k = (u l + v m + w (n-1)) nu_c / c_light  [turns],
 *           n = sqrt(1 - l^2 - m^2), uvw_ij = uvw_i - uvw_j                 (R1)
 *   peel, for each source k in list order:                                  (R4)
 *     rotate + average   A_k(bl) = mean_{t,c} R(t,bl,c) exp(+2 pi i phi_k)  (R5)
 *     solve              per antenna p, Z_pq = S_k J_q^H,
 *                        J_p <- [sum_q A_pq Z_pq^H] [sum_q Z_pq Z_pq^H]^-1,
 *                        A_qp = A_pq^H; Jacobi sweep from J = I; on every
 *                        second sweep J <- (J_new + J_old)/2; fixed n_iter (R6)
 *     subtract           R(t,bl,c) -= S_k J_p J_q^H exp(-2 pi i phi_k)
 *   loss    L = sum ||V - sum_k S_k J_i J_j^H exp(-2 pi i phi_k)||_F^2 and its
 *           gradient w.r.t. (J, l, m, S) in the PyTorch convention
 *           dL/dRe + i dL/dIm (hand-derived adjoint, checked by differences).
 *   offsets Section 3 measures per calibrator a position offset (ionospheric
 *           refraction) as well as the Jones matrices; Section 3.1 says the
 *           fit needs six numbers per source and is described by two, that
 *           the ionosphere's response is a known function of frequency, and
 *           that workers send their numbers to a master that builds the
 *           solution.  Reading: the six numbers are the Gauss-Newton
 *           sufficient statistics of the two-parameter fit, additive over
 *           channel groups: J^T J (3), J^T r (2) and r^T r (1), with the shift
 *           at channel c equal to (nu_ref/nu_c)^alpha (dl, dm) (alpha = 2 for
 *           refraction), reported as (H_ll, H_lm, H_mm, g_l, g_m, L) with
 *           H = 2 J^T J, g = dL/d(dl, dm); the fit is -H^-1 g, or (0, 0)
 *           where det H <= 0 (no flux, zero gains, no baselines).
 *
 * Parallelism: baselines are independent in every streaming step; each
 * baseline's sums run serially in (t, c) order, and sums across baselines are
 * taken serially in baseline order afterwards, so results do not depend on
 * the thread count.
 */
#include "rts_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define C_LIGHT 299792458.0
#define TWO_PI 6.283185307179586476925286766559

typedef double complex cplx;
typedef struct { cplx e[4]; } mat2;      /* [0 1; 2 3] */

static mat2 m_load(const double* p) {
  mat2 r;
  for (int k = 0; k < 4; ++k) r.e[k] = p[2 * k] + I * p[2 * k + 1];
  return r;
}
static void m_store(double* p, mat2 a) {
  for (int k = 0; k < 4; ++k) { p[2 * k] = creal(a.e[k]); p[2 * k + 1] = cimag(a.e[k]); }
}
static mat2 m_zero(void) { mat2 r; for (int k = 0; k < 4; ++k) r.e[k] = 0; return r; }
static mat2 m_eye(void) { mat2 r = m_zero(); r.e[0] = 1; r.e[3] = 1; return r; }
static mat2 m_mul(mat2 a, mat2 b) {
  mat2 r;
  r.e[0] = a.e[0] * b.e[0] + a.e[1] * b.e[2];
  r.e[1] = a.e[0] * b.e[1] + a.e[1] * b.e[3];
  r.e[2] = a.e[2] * b.e[0] + a.e[3] * b.e[2];
  r.e[3] = a.e[2] * b.e[1] + a.e[3] * b.e[3];
  return r;
}
static mat2 m_herm(mat2 a) {
  mat2 r;
  r.e[0] = conj(a.e[0]); r.e[1] = conj(a.e[2]);
  r.e[2] = conj(a.e[1]); r.e[3] = conj(a.e[3]);
  return r;
}
static mat2 m_add(mat2 a, mat2 b) { for (int k = 0; k < 4; ++k) a.e[k] += b.e[k]; return a; }
static mat2 m_sub(mat2 a, mat2 b) { for (int k = 0; k < 4; ++k) a.e[k] -= b.e[k]; return a; }
static mat2 m_scale(mat2 a, cplx s) { for (int k = 0; k < 4; ++k) a.e[k] *= s; return a; }
static cplx m_trace(mat2 a) { return a.e[0] + a.e[3]; }
static double m_norm2(mat2 a) {
  double s = 0;
  for (int k = 0; k < 4; ++k) s += creal(a.e[k]) * creal(a.e[k]) + cimag(a.e[k]) * cimag(a.e[k]);
  return s;
}
/* closed-form 2x2 inverse: [d -b; -c a] / (ad - bc) */
static mat2 m_inv(mat2 a) {
  cplx det = a.e[0] * a.e[3] - a.e[1] * a.e[2];
  mat2 r;
  r.e[0] = a.e[3] / det; r.e[1] = -a.e[1] / det;
  r.e[2] = -a.e[2] / det; r.e[3] = a.e[0] / det;
  return r;
}
static int m_finite(mat2 a) {
  for (int k = 0; k < 4; ++k)
    if (!isfinite(creal(a.e[k])) || !isfinite(cimag(a.e[k]))) return 0;
  return 1;
}

void orc_set_num_threads(int32_t n) {
  if (n > 0) omp_set_num_threads(n);
}

int32_t orc_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- baselines ---------------------------------------------------------- */

int64_t orc_n_baselines(int32_t n_ant) { return (int64_t)n_ant * (n_ant - 1) / 2; }

int64_t orc_baseline_index(int32_t n_ant, int32_t i, int32_t j) {
  return (int64_t)i * n_ant - (int64_t)i * (i + 1) / 2 + (j - i - 1);
}

/* inverse map by enumeration: rows i = 0.., columns j = i+1.. */
void orc_baseline_antennas(int32_t n_ant, int32_t* ant_i, int32_t* ant_j) {
  int64_t b = 0;
  for (int32_t i = 0; i < n_ant; ++i)
    for (int32_t j = i + 1; j < n_ant; ++j) { ant_i[b] = i; ant_j[b] = j; ++b; }
}

/* ---- geometry and phase (reading R1) ------------------------------------ */

double orc_delay_m(const double* uvw, int32_t n_ant, int32_t t, int32_t i, int32_t j,
                   double l, double m) {
  const double* a = uvw + ((int64_t)t * n_ant + i) * 3;
  const double* b = uvw + ((int64_t)t * n_ant + j) * 3;
  double u = a[0] - b[0], v = a[1] - b[1], w = a[2] - b[2];
  double n = sqrt(1.0 - l * l - m * m);
  return u * l + v * m + w * (n - 1.0);
}

/* phase in turns, reduced to [-1/2, 1/2] by x - round(x) */
double orc_phase_turns(double tau_m, double freq_hz) {
  double x = tau_m * freq_hz / C_LIGHT;
  return x - nearbyint(x);
}

static cplx phasor(double turns, double sign) {       /* exp(sign * 2 pi i turns) */
  double a = TWO_PI * turns;
  return cos(a) + I * sign * sin(a);
}

static int32_t* g_ai;
static int32_t* g_aj;
static int32_t g_map_n = -1;
static void antenna_map(int32_t n_ant, int32_t** ai, int32_t** aj) {
  if (g_map_n != n_ant) {
    int64_t nb = orc_n_baselines(n_ant);
    free(g_ai); free(g_aj);
    g_ai = (int32_t*)malloc(sizeof(int32_t) * (nb > 0 ? nb : 1));
    g_aj = (int32_t*)malloc(sizeof(int32_t) * (nb > 0 ? nb : 1));
    orc_baseline_antennas(n_ant, g_ai, g_aj);
    g_map_n = n_ant;
  }
  *ai = g_ai; *aj = g_aj;
}

static double* vis_at(double* vis, int64_t n_bl, int32_t n_chan, int32_t t, int64_t bl, int32_t c) {
  return vis + (((int64_t)t * n_bl + bl) * n_chan + c) * 8;
}

/* ---- predict: V += sum_k S_k J_i J_j^H exp(-2 pi i phi_k) (R1, R2) ------- */

void orc_predict(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                 const double* freq, int32_t n_src, const double* lmS, const double* jones,
                 double* vis, int32_t accumulate) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t i = ai[bl], j = aj[bl];
    for (int32_t t = 0; t < n_time; ++t)
      for (int32_t c = 0; c < n_chan; ++c) {
        double* out = vis_at(vis, n_bl, n_chan, t, bl, c);
        mat2 v = accumulate ? m_load(out) : m_zero();
        for (int32_t k = 0; k < n_src; ++k) {
          double l = lmS[3 * k], m = lmS[3 * k + 1], S = lmS[3 * k + 2];
          mat2 Ji = m_load(jones + ((int64_t)k * n_ant + i) * 8);
          mat2 Jj = m_load(jones + ((int64_t)k * n_ant + j) * 8);
          mat2 M = m_scale(m_mul(Ji, m_herm(Jj)), S);
          double phi = orc_phase_turns(orc_delay_m(uvw, n_ant, t, i, j, l, m), freq[c]);
          v = m_add(v, m_scale(M, phasor(phi, -1.0)));
        }
        m_store(out, v);
      }
  }
}

/* ---- rotate + average (R5): A(bl) = mean_{t,c} V exp(+2 pi i phi) -------- */

void orc_rotate_average(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, const double* vis, double l, double m,
                        double* avg) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  double inv_n = 1.0 / ((double)n_time * n_chan);
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t i = ai[bl], j = aj[bl];
    mat2 acc = m_zero();
    for (int32_t t = 0; t < n_time; ++t) {
      double tau = orc_delay_m(uvw, n_ant, t, i, j, l, m);
      for (int32_t c = 0; c < n_chan; ++c) {
        mat2 v = m_load(vis_at((double*)vis, n_bl, n_chan, t, bl, c));
        acc = m_add(acc, m_scale(v, phasor(orc_phase_turns(tau, freq[c]), +1.0)));
      }
    }
    m_store(avg + bl * 8, m_scale(acc, inv_n));
  }
}

/* ---- ALS solve for one source (R6) --------------------------------------
 * Returns 0 when the last relative change ||J_new - J_old||_F / ||J_new||_F
 * is <= 1e-6, 1 when it is larger, -4 when a non-finite value appears.    */

int32_t orc_als(int32_t n_ant, const double* avg, double S, int32_t n_iter,
                double* jones, double* rel_change) {
  mat2* J = (mat2*)malloc(sizeof(mat2) * n_ant);
  mat2* Jn = (mat2*)malloc(sizeof(mat2) * n_ant);
  for (int32_t p = 0; p < n_ant; ++p) J[p] = m_eye();
  double rel = 0.0;
  int finite = 1;
  for (int32_t it = 1; it <= n_iter; ++it) {
    for (int32_t p = 0; p < n_ant; ++p) {
      mat2 A = m_zero(), C = m_zero();
      for (int32_t q = 0; q < n_ant; ++q) {
        if (q == p) continue;
        mat2 Vpq = p < q ? m_load(avg + orc_baseline_index(n_ant, p, q) * 8)
                         : m_herm(m_load(avg + orc_baseline_index(n_ant, q, p) * 8));
        mat2 Z = m_scale(m_herm(J[q]), S);          /* Z_pq = B J_q^H, B = S I */
        A = m_add(A, m_mul(Vpq, m_herm(Z)));
        C = m_add(C, m_mul(Z, m_herm(Z)));
      }
      Jn[p] = m_mul(A, m_inv(C));
    }
    if (it % 2 == 0)
      for (int32_t p = 0; p < n_ant; ++p) Jn[p] = m_scale(m_add(Jn[p], J[p]), 0.5);
    double dn = 0.0, nn = 0.0;
    for (int32_t p = 0; p < n_ant; ++p) {
      dn += m_norm2(m_sub(Jn[p], J[p]));
      nn += m_norm2(Jn[p]);
      if (!m_finite(Jn[p])) finite = 0;
    }
    rel = sqrt(dn / nn);
    mat2* tmp = J; J = Jn; Jn = tmp;
  }
  for (int32_t p = 0; p < n_ant; ++p) m_store(jones + (int64_t)p * 8, J[p]);
  free(J); free(Jn);
  if (rel_change) *rel_change = rel;
  if (!finite || !isfinite(rel)) return -4;
  return rel > 1e-6 ? 1 : 0;
}

/* ---- subtract one source: R -= S J_i J_j^H exp(-2 pi i phi) -------------- */

void orc_subtract(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                  const double* freq, double* vis, double l, double m, double S,
                  const double* jones) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t i = ai[bl], j = aj[bl];
    mat2 M = m_scale(m_mul(m_load(jones + (int64_t)i * 8), m_herm(m_load(jones + (int64_t)j * 8))), S);
    for (int32_t t = 0; t < n_time; ++t) {
      double tau = orc_delay_m(uvw, n_ant, t, i, j, l, m);
      for (int32_t c = 0; c < n_chan; ++c) {
        double* p = vis_at(vis, n_bl, n_chan, t, bl, c);
        m_store(p, m_sub(m_load(p), m_scale(M, phasor(orc_phase_turns(tau, freq[c]), -1.0))));
      }
    }
  }
}

/* ---- the peel: average, solve, subtract for each source in list order ---- */

int32_t orc_peel(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                 const double* freq, double* vis, int32_t n_src, const double* lmS,
                 int32_t n_iter, double* jones, int32_t* status, double* avg_per_src,
                 double* rel_per_src) {
  int64_t n_bl = orc_n_baselines(n_ant);
  double* avg = (double*)malloc(sizeof(double) * 8 * (n_bl > 0 ? n_bl : 1));
  int32_t worst = 0;
  for (int32_t k = 0; k < n_src; ++k) {
    double l = lmS[3 * k], m = lmS[3 * k + 1], S = lmS[3 * k + 2];
    double* Jk = jones + (int64_t)k * n_ant * 8;
    orc_rotate_average(n_ant, n_chan, n_time, uvw, freq, vis, l, m, avg);
    if (avg_per_src) memcpy(avg_per_src + (int64_t)k * n_bl * 8, avg, sizeof(double) * 8 * n_bl);
    double rel = 0.0;
    int32_t st = orc_als(n_ant, avg, S, n_iter, Jk, &rel);
    if (status) status[k] = st;
    if (rel_per_src) rel_per_src[k] = rel;
    if (st < 0) worst = st;
    orc_subtract(n_ant, n_chan, n_time, uvw, freq, vis, l, m, S, Jk);
  }
  free(avg);
  return worst;
}

/* ---- loss and its gradient ------------------------------------------------
 * R = V - sum_k M_k exp(-2 pi i phi_k), M_k = S_k J_i J_j^H,  L = sum ||R||^2.
 * With G_k = sum_{t,c} R exp(+2 pi i phi_k) and
 *      H_k^l = sum_{t,c} R exp(+2 pi i phi_k) d(phi_k)/dl,
 *      d(phi)/dl = (u - w l/n) nu / c_light  (turns per unit l), same for m:
 *   dL/dJ_i  += -2 S_k G_k J_j          dL/dJ_j += -2 S_k G_k^H J_i
 *   dL/dS_k  += -2 Re tr(G_k^H J_i J_j^H)
 *   dL/dl_k  += -4 pi Im tr(H_k^lH M_k)  (and m likewise).                  */

void orc_loss_grad(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                   const double* freq, const double* vis, int32_t n_src, const double* lmS,
                   const double* jones, double* loss, double* g_jones, double* g_l,
                   double* g_m, double* g_S) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  int64_t nkb = (int64_t)n_src * n_bl;
  mat2* G = (mat2*)calloc((size_t)(nkb > 0 ? nkb : 1), sizeof(mat2));
  mat2* Hl = (mat2*)calloc((size_t)(nkb > 0 ? nkb : 1), sizeof(mat2));
  mat2* Hm = (mat2*)calloc((size_t)(nkb > 0 ? nkb : 1), sizeof(mat2));
  double* bl_loss = (double*)calloc((size_t)(n_bl > 0 ? n_bl : 1), sizeof(double));
  mat2* Mk = (mat2*)malloc(sizeof(mat2) * (nkb > 0 ? nkb : 1));
  for (int32_t k = 0; k < n_src; ++k)
    for (int64_t bl = 0; bl < n_bl; ++bl) {
      mat2 Ji = m_load(jones + ((int64_t)k * n_ant + ai[bl]) * 8);
      mat2 Jj = m_load(jones + ((int64_t)k * n_ant + aj[bl]) * 8);
      Mk[k * n_bl + bl] = m_scale(m_mul(Ji, m_herm(Jj)), lmS[3 * k + 2]);
    }
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t i = ai[bl], j = aj[bl];
    double* phi = (double*)malloc(sizeof(double) * (n_src > 0 ? n_src : 1));
    for (int32_t t = 0; t < n_time; ++t) {
      const double* a = uvw + ((int64_t)t * n_ant + i) * 3;
      const double* b = uvw + ((int64_t)t * n_ant + j) * 3;
      double u = a[0] - b[0], w = a[2] - b[2], v = a[1] - b[1];
      for (int32_t c = 0; c < n_chan; ++c) {
        mat2 R = m_load(vis_at((double*)vis, n_bl, n_chan, t, bl, c));
        for (int32_t k = 0; k < n_src; ++k) {
          phi[k] = orc_phase_turns(orc_delay_m(uvw, n_ant, t, i, j, lmS[3 * k], lmS[3 * k + 1]), freq[c]);
          R = m_sub(R, m_scale(Mk[k * n_bl + bl], phasor(phi[k], -1.0)));
        }
        bl_loss[bl] += m_norm2(R);
        for (int32_t k = 0; k < n_src; ++k) {
          double l = lmS[3 * k], m = lmS[3 * k + 1];
          double n = sqrt(1.0 - l * l - m * m);
          double dphi_dl = (u - w * l / n) * freq[c] / C_LIGHT;
          double dphi_dm = (v - w * m / n) * freq[c] / C_LIGHT;
          mat2 Rr = m_scale(R, phasor(phi[k], +1.0));
          G[k * n_bl + bl] = m_add(G[k * n_bl + bl], Rr);
          Hl[k * n_bl + bl] = m_add(Hl[k * n_bl + bl], m_scale(Rr, dphi_dl));
          Hm[k * n_bl + bl] = m_add(Hm[k * n_bl + bl], m_scale(Rr, dphi_dm));
        }
      }
    }
    free(phi);
  }
  double L = 0.0;
  for (int64_t bl = 0; bl < n_bl; ++bl) L += bl_loss[bl];
  *loss = L;
  if (g_jones) memset(g_jones, 0, sizeof(double) * 8 * n_src * (size_t)n_ant);
  for (int32_t k = 0; k < n_src; ++k) {
    double S = lmS[3 * k + 2];
    double gl = 0.0, gm = 0.0, gS = 0.0;
    for (int64_t bl = 0; bl < n_bl; ++bl) {
      int32_t i = ai[bl], j = aj[bl];
      mat2 Ji = m_load(jones + ((int64_t)k * n_ant + i) * 8);
      mat2 Jj = m_load(jones + ((int64_t)k * n_ant + j) * 8);
      mat2 Gk = G[k * n_bl + bl];
      mat2 M = Mk[k * n_bl + bl];
      if (g_jones) {
        double* gi = g_jones + ((int64_t)k * n_ant + i) * 8;
        double* gj = g_jones + ((int64_t)k * n_ant + j) * 8;
        m_store(gi, m_add(m_load(gi), m_scale(m_mul(Gk, Jj), -2.0 * S)));
        m_store(gj, m_add(m_load(gj), m_scale(m_mul(m_herm(Gk), Ji), -2.0 * S)));
      }
      gS += -2.0 * creal(m_trace(m_mul(m_herm(Gk), m_mul(Ji, m_herm(Jj)))));
      gl += -4.0 * M_PI * cimag(m_trace(m_mul(m_herm(Hl[k * n_bl + bl]), M)));
      gm += -4.0 * M_PI * cimag(m_trace(m_mul(m_herm(Hm[k * n_bl + bl]), M)));
    }
    if (g_l) g_l[k] = gl;
    if (g_m) g_m[k] = gm;
    if (g_S) g_S[k] = gS;
  }
  free(G); free(Hl); free(Hm); free(bl_loss); free(Mk);
}

/* ---- ionospheric position offsets (Gauss-Newton normal equations) ----------
 * Offset model: at channel c source k sits at (l + s_c dl, m + s_c dm),
 * s_c = (nu_ref/nu_c)^alpha (alpha = 2: refraction, which scales as lambda^2;
 * alpha = 0: a frequency-independent shift).  At dl = dm = 0 the derivative of
 * source k's model is  D_p = M_k e^{-2 pi i phi_k} (-2 pi i) s_c a_p nu_c/c,
 * a_l = u - w l/n, a_m = v - w m/n, and with R the residual of all sources
 *   H_pq = 2 Re sum tr(D_p^H D_q),  g_p = -2 Re sum tr(R^H D_p),  L = sum ||R||^2.
 * out[k][6] = (H_ll, H_lm, H_mm, g_l, g_m, L), offsets[k][2] = -H^-1 g.      */

void orc_offsets(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                 const double* freq, const double* vis, int32_t n_src, const double* lmS,
                 const double* jones, double alpha, double nu_ref, double* out,
                 double* offsets) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  int64_t nkb = (int64_t)n_src * n_bl;
  double* part = (double*)calloc((size_t)(nkb > 0 ? nkb : 1) * 5, sizeof(double));
  double* bl_loss = (double*)calloc((size_t)(n_bl > 0 ? n_bl : 1), sizeof(double));
  mat2* Mk = (mat2*)malloc(sizeof(mat2) * (nkb > 0 ? nkb : 1));
  for (int32_t k = 0; k < n_src; ++k)
    for (int64_t bl = 0; bl < n_bl; ++bl) {
      mat2 Ji = m_load(jones + ((int64_t)k * n_ant + ai[bl]) * 8);
      mat2 Jj = m_load(jones + ((int64_t)k * n_ant + aj[bl]) * 8);
      Mk[k * n_bl + bl] = m_scale(m_mul(Ji, m_herm(Jj)), lmS[3 * k + 2]);
    }
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t i = ai[bl], j = aj[bl];
    mat2* Mph = (mat2*)malloc(sizeof(mat2) * (n_src > 0 ? n_src : 1));
    for (int32_t t = 0; t < n_time; ++t) {
      const double* a = uvw + ((int64_t)t * n_ant + i) * 3;
      const double* b = uvw + ((int64_t)t * n_ant + j) * 3;
      double u = a[0] - b[0], v = a[1] - b[1], w = a[2] - b[2];
      for (int32_t c = 0; c < n_chan; ++c) {
        mat2 R = m_load(vis_at((double*)vis, n_bl, n_chan, t, bl, c));
        for (int32_t k = 0; k < n_src; ++k) {
          double phi = orc_phase_turns(orc_delay_m(uvw, n_ant, t, i, j, lmS[3 * k], lmS[3 * k + 1]), freq[c]);
          Mph[k] = m_scale(Mk[k * n_bl + bl], phasor(phi, -1.0));
          R = m_sub(R, Mph[k]);
        }
        bl_loss[bl] += m_norm2(R);
        double s_c = pow(nu_ref / freq[c], alpha);
        for (int32_t k = 0; k < n_src; ++k) {
          double l = lmS[3 * k], m = lmS[3 * k + 1];
          double n = sqrt(1.0 - l * l - m * m);
          cplx f = -2.0 * M_PI * I * s_c * freq[c] / C_LIGHT;
          mat2 Dl = m_scale(Mph[k], f * (u - w * l / n));
          mat2 Dm = m_scale(Mph[k], f * (v - w * m / n));
          double* o = part + ((int64_t)k * n_bl + bl) * 5;
          o[0] += 2.0 * creal(m_trace(m_mul(m_herm(Dl), Dl)));
          o[1] += 2.0 * creal(m_trace(m_mul(m_herm(Dl), Dm)));
          o[2] += 2.0 * creal(m_trace(m_mul(m_herm(Dm), Dm)));
          o[3] += -2.0 * creal(m_trace(m_mul(m_herm(R), Dl)));
          o[4] += -2.0 * creal(m_trace(m_mul(m_herm(R), Dm)));
        }
      }
    }
    free(Mph);
  }
  double L = 0.0;
  for (int64_t bl = 0; bl < n_bl; ++bl) L += bl_loss[bl];
  for (int32_t k = 0; k < n_src; ++k) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t bl = 0; bl < n_bl; ++bl)
      for (int q = 0; q < 5; ++q) acc[q] += part[((int64_t)k * n_bl + bl) * 5 + q];
    double* o = out + 6 * (int64_t)k;
    for (int q = 0; q < 5; ++q) o[q] = acc[q];
    o[5] = L;
    double hll = acc[0], hlm = acc[1], hmm = acc[2], gl = acc[3], gm = acc[4];
    double det = hll * hmm - hlm * hlm;       /* no step where H is singular */
    offsets[2 * k] = det > 0.0 ? -(hmm * gl - hlm * gm) / det : 0.0;
    offsets[2 * k + 1] = det > 0.0 ? -(hll * gm - hlm * gl) / det : 0.0;
  }
  free(part); free(bl_loss); free(Mk);
}

/* ---- gains Taylor-expanded in frequency ------------------------------------
 * Section 3.1: combining consecutive channels helps the calibration because the
 * unknown tile gain can then be Taylor-expanded in frequency.  Reading (R16):
 * first order about the band centre,
 *   J_p(c) = G_p + x_c H_p,   x_c = (nu_c - nu_mid) / (n_chan dnu),
 *   nu_mid = (nu_0 + nu_last) / 2, dnu the channel spacing,
 * so the model of source k on baseline (i, j) at channel c is
 *   S_k (G_i + x_c H_i)(G_j + x_c H_j)^H exp(-2 pi i phi_k).
 * The solve is the same Jacobi alternating least squares with the 2 x 4
 * unknown X_p = [G_p H_p]: with the rotated residual R~ = R exp(+2 pi i phi_k)
 * and Z_pq(c) = S [W_q(c); x_c W_q(c)] (4 x 2), W_q(c) = (G_q + x_c H_q)^H,
 *   X_p <- [sum_q sum_{t,c} R~_pq Z_pq^H] [sum_q sum_{t,c} Z_pq Z_pq^H]^-1
 * (R~_qp = R~_pq^H), from G = I, H = 0, every second sweep averaged with the
 * previous iterate, fixed n_iter; status from ||X_new - X_old|| / ||X_new||.
 * Sums run over every sample (t, c), as the least-squares problem states.   */

static double taylor_x(const double* freq, int32_t n_chan, int32_t c) {
  if (n_chan < 2) return 0.0;
  double dnu = (freq[n_chan - 1] - freq[0]) / (n_chan - 1);
  double mid = 0.5 * (freq[0] + freq[n_chan - 1]);
  return (freq[c] - mid) / (n_chan * dnu);
}

/* Gauss-Jordan inverse of an n x n complex matrix (partial pivoting); 0 if singular */
static int c_inverse(int n, const cplx* a, cplx* inv) {
  cplx m[4][8];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) m[r][c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (cabs(m[r][col]) > cabs(m[piv][col])) piv = r;
    if (cabs(m[piv][col]) == 0.0) return 0;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) { cplx tmp = m[col][c]; m[col][c] = m[piv][c]; m[piv][c] = tmp; }
    cplx d = m[col][col];
    for (int c = 0; c < 2 * n; ++c) m[col][c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      cplx f = m[r][col];
      for (int c = 0; c < 2 * n; ++c) m[r][c] -= f * m[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) inv[r * n + c] = m[r][n + c];
  return 1;
}

/* The common slope rotation (reading R27).  Rotating every slope by the same
 * Hermitian K, H_p -> H_p + i G_p K, changes the model
 * S (G_i + x H_i)(G_j + x H_j)^H only at second order in x (the first-order
 * terms cancel), so the Jacobi sweeps, which move one antenna at a time, barely
 * move the iterate along it.  After every sweep from the second on, one Newton
 * step from K = 0 on the least-squares cost restricted to that direction,
 *   f(K) = sum_{i<j} sum_{t,c} || R~_ij - S (G_i + x (H_i + i G_i K))(G_j + x (H_j + i G_j K))^H ||^2,
 * with K = sum_a k_a B_a over the Hermitian basis
 *   B_0 = [1 0; 0 0], B_1 = [0 0; 0 1], B_2 = [0 1; 1 0], B_3 = [0 -i; i 0].
 * With r the residual at K = 0 and <X, Y> = tr(X^H Y):
 *   dm/dk_a         = S x^2 i (G_i B_a H_j^H - H_i B_a G_j^H)
 *   d2m/dk_a dk_b   = S x^2 G_i (B_a B_b + B_b B_a) G_j^H
 *   g_a  = -2 Re sum <r, dm/dk_a>
 *   h_ab =  2 Re sum <dm/dk_a, dm/dk_b> - 2 Re sum <r, d2m/dk_a dk_b>
 * and k = -h^-1 g when every Cholesky pivot of h exceeds 1e-6 of its largest
 * diagonal entry (else no step: along a flat direction the step is not
 * defined).  Returns 1 when the step was taken.  The solve takes the step only
 * with three channels or more: with two, x_c^2 is the same at both, the change
 * along K is one that G can absorb, and the direction is part of a flat set.  g_out [4], h_out [16]
 * (optional) receive g and h. */
static const cplx kRotB[4][4] = {{1, 0, 0, 0}, {0, 0, 0, 1}, {0, 1, 1, 0}, {0, -I, I, 0}};

static int rotation_step(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* freq,
                         const mat2* Rr, double S, const mat2* G, mat2* H, double* g_out, double* h_out) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int64_t n_s = (int64_t)n_time * n_chan;
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  mat2 B[4], W[4][4];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k) B[a].e[k] = kRotB[a][k];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) W[a][b] = m_add(m_mul(B[a], B[b]), m_mul(B[b], B[a]));
  double g[4] = {0, 0, 0, 0}, h[16] = {0};
#pragma omp parallel for schedule(static) reduction(+ : g[:4], h[:16])
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t p = ai[bl], q = aj[bl];
    mat2 D[4], E[4][4];
    for (int a = 0; a < 4; ++a)
      D[a] = m_scale(m_sub(m_mul(m_mul(G[p], B[a]), m_herm(H[q])), m_mul(m_mul(H[p], B[a]), m_herm(G[q]))),
                     I * S);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) E[a][b] = m_scale(m_mul(m_mul(G[p], W[a][b]), m_herm(G[q])), S);
    for (int32_t t = 0; t < n_time; ++t)
      for (int32_t c = 0; c < n_chan; ++c) {
        double x = taylor_x(freq, n_chan, c), x2 = x * x, x4 = x2 * x2;
        mat2 Ap = m_add(G[p], m_scale(H[p], x)), Aq = m_add(G[q], m_scale(H[q], x));
        mat2 r = m_sub(Rr[bl * n_s + (int64_t)t * n_chan + c], m_scale(m_mul(Ap, m_herm(Aq)), S));
        for (int a = 0; a < 4; ++a) {
          cplx rd = 0;
          for (int k = 0; k < 4; ++k) rd += conj(r.e[k]) * D[a].e[k];
          g[a] += -2.0 * x2 * creal(rd);
          for (int b = 0; b < 4; ++b) {
            cplx dd = 0, re = 0;
            for (int k = 0; k < 4; ++k) {
              dd += conj(D[a].e[k]) * D[b].e[k];
              re += conj(r.e[k]) * E[a][b].e[k];
            }
            h[4 * a + b] += 2.0 * x4 * creal(dd) - 2.0 * x2 * creal(re);
          }
        }
      }
  }
  if (g_out) memcpy(g_out, g, sizeof(g));
  if (h_out) memcpy(h_out, h, sizeof(h));
  /* Cholesky h = L L^T with the pivot test, then k = -h^-1 g */
  double L[4][4] = {{0}}, dmax = 0.0;
  for (int a = 0; a < 4; ++a) dmax = fmax(dmax, h[5 * a]);
  if (!(dmax > 0.0)) return 0;
  for (int j = 0; j < 4; ++j) {
    double d = h[5 * j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 1e-6 * dmax)) return 0;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < 4; ++i) {
      double v = h[4 * i + j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  double y[4], k[4];
  for (int i = 0; i < 4; ++i) {
    double v = -g[i];
    for (int j = 0; j < i; ++j) v -= L[i][j] * y[j];
    y[i] = v / L[i][i];
  }
  for (int i = 3; i >= 0; --i) {
    double v = y[i];
    for (int j = i + 1; j < 4; ++j) v -= L[j][i] * k[j];
    k[i] = v / L[i][i];
  }
  mat2 K = m_zero();
  for (int a = 0; a < 4; ++a) K = m_add(K, m_scale(B[a], k[a]));
  for (int32_t p = 0; p < n_ant; ++p) H[p] = m_add(H[p], m_scale(m_mul(G[p], K), I));
  return 1;
}

void orc_predict_taylor(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, int32_t n_src, const double* lmS, const double* gain,
                        const double* slope, double* vis, int32_t accumulate) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    int32_t i = ai[bl], j = aj[bl];
    for (int32_t t = 0; t < n_time; ++t)
      for (int32_t c = 0; c < n_chan; ++c) {
        double x = taylor_x(freq, n_chan, c);
        double* out = vis_at(vis, n_bl, n_chan, t, bl, c);
        mat2 v = accumulate ? m_load(out) : m_zero();
        for (int32_t k = 0; k < n_src; ++k) {
          double l = lmS[3 * k], m = lmS[3 * k + 1], S = lmS[3 * k + 2];
          int64_t oi = ((int64_t)k * n_ant + i) * 8, oj = ((int64_t)k * n_ant + j) * 8;
          mat2 Ji = m_add(m_load(gain + oi), m_scale(m_load(slope + oi), x));
          mat2 Jj = m_add(m_load(gain + oj), m_scale(m_load(slope + oj), x));
          mat2 M = m_scale(m_mul(Ji, m_herm(Jj)), S);
          double phi = orc_phase_turns(orc_delay_m(uvw, n_ant, t, i, j, l, m), freq[c]);
          v = m_add(v, m_scale(M, phasor(phi, -1.0)));
        }
        m_store(out, v);
      }
  }
}

int32_t orc_als_taylor(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                       const double* freq, const double* vis, double l, double m, double S,
                       int32_t n_iter, double* gain, double* slope, double* rel_change) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int64_t n_s = (int64_t)n_time * n_chan;
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  /* the residual rotated to the source, per baseline and sample */
  mat2* Rr = (mat2*)malloc(sizeof(mat2) * (size_t)(n_bl * n_s > 0 ? n_bl * n_s : 1));
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl)
    for (int32_t t = 0; t < n_time; ++t) {
      double tau = orc_delay_m(uvw, n_ant, t, ai[bl], aj[bl], l, m);
      for (int32_t c = 0; c < n_chan; ++c)
        Rr[bl * n_s + (int64_t)t * n_chan + c] =
            m_scale(m_load(vis_at((double*)vis, n_bl, n_chan, t, bl, c)), phasor(orc_phase_turns(tau, freq[c]), +1.0));
    }
  mat2* G = (mat2*)malloc(sizeof(mat2) * n_ant);
  mat2* H = (mat2*)malloc(sizeof(mat2) * n_ant);
  mat2* Gn = (mat2*)malloc(sizeof(mat2) * n_ant);
  mat2* Hn = (mat2*)malloc(sizeof(mat2) * n_ant);
  for (int32_t p = 0; p < n_ant; ++p) { G[p] = m_eye(); H[p] = m_zero(); }
  double rel = 0.0;
  int finite = 1;
  for (int32_t it = 1; it <= n_iter; ++it) {
#pragma omp parallel for schedule(static)
    for (int32_t p = 0; p < n_ant; ++p) {
      cplx A[2][4] = {{0}}, C[16] = {0}, Ci[16];
      for (int32_t q = 0; q < n_ant; ++q) {
        if (q == p) continue;
        int64_t bl = p < q ? orc_baseline_index(n_ant, p, q) : orc_baseline_index(n_ant, q, p);
        for (int32_t t = 0; t < n_time; ++t)
          for (int32_t c = 0; c < n_chan; ++c) {
            double x = taylor_x(freq, n_chan, c);
            mat2 R = Rr[bl * n_s + (int64_t)t * n_chan + c];
            if (p > q) R = m_herm(R);
            mat2 W = m_herm(m_add(G[q], m_scale(H[q], x)));     /* W_q(c) */
            cplx Z[4][2];                                        /* S [W; x W] */
            for (int r = 0; r < 2; ++r)
              for (int s = 0; s < 2; ++s) { Z[r][s] = S * W.e[2 * r + s]; Z[2 + r][s] = S * x * W.e[2 * r + s]; }
            for (int r = 0; r < 2; ++r)                          /* A += R Z^H */
              for (int s = 0; s < 4; ++s)
                for (int u = 0; u < 2; ++u) A[r][s] += R.e[2 * r + u] * conj(Z[s][u]);
            for (int r = 0; r < 4; ++r)                          /* C += Z Z^H */
              for (int s = 0; s < 4; ++s)
                for (int u = 0; u < 2; ++u) C[4 * r + s] += Z[r][u] * conj(Z[s][u]);
          }
      }
      if (!c_inverse(4, C, Ci))
        for (int k = 0; k < 16; ++k) Ci[k] = NAN;
      cplx X[2][4];
      for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 4; ++s) {
          X[r][s] = 0.0;
          for (int u = 0; u < 4; ++u) X[r][s] += A[r][u] * Ci[4 * u + s];
        }
      for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) { Gn[p].e[2 * r + s] = X[r][s]; Hn[p].e[2 * r + s] = X[r][2 + s]; }
    }
    if (it % 2 == 0)
      for (int32_t p = 0; p < n_ant; ++p) {
        Gn[p] = m_scale(m_add(Gn[p], G[p]), 0.5);
        Hn[p] = m_scale(m_add(Hn[p], H[p]), 0.5);
      }
    if (it >= 2 && n_chan >= 3) rotation_step(n_ant, n_chan, n_time, freq, Rr, S, Gn, Hn, NULL, NULL);
    double dn = 0.0, nn = 0.0;
    for (int32_t p = 0; p < n_ant; ++p) {
      dn += m_norm2(m_sub(Gn[p], G[p])) + m_norm2(m_sub(Hn[p], H[p]));
      nn += m_norm2(Gn[p]) + m_norm2(Hn[p]);
      if (!m_finite(Gn[p]) || !m_finite(Hn[p])) finite = 0;
    }
    rel = sqrt(dn / nn);
    mat2* tmp = G; G = Gn; Gn = tmp;
    tmp = H; H = Hn; Hn = tmp;
  }
  for (int32_t p = 0; p < n_ant; ++p) {
    m_store(gain + (int64_t)p * 8, G[p]);
    m_store(slope + (int64_t)p * 8, H[p]);
  }
  free(Rr); free(G); free(H); free(Gn); free(Hn);
  if (rel_change) *rel_change = rel;
  if (!finite || !isfinite(rel)) return -4;
  return rel > 1e-6 ? 1 : 0;
}

/* One slope-rotation step (rotation_step above) of source (l, m, S) on the
 * cube vis at the iterate (gain, slope), exposed for the tests: slope is
 * updated in place when the step is taken (returns 1), g [4] and h [16]
 * receive the gradient and Hessian of f at K = 0. */
int32_t orc_taylor_rotation(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                            const double* freq, const double* vis, double l, double m, double S,
                            const double* gain, double* slope, double* g, double* h) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int64_t n_s = (int64_t)n_time * n_chan;
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  mat2* Rr = (mat2*)malloc(sizeof(mat2) * (size_t)(n_bl * n_s > 0 ? n_bl * n_s : 1));
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl)
    for (int32_t t = 0; t < n_time; ++t) {
      double tau = orc_delay_m(uvw, n_ant, t, ai[bl], aj[bl], l, m);
      for (int32_t c = 0; c < n_chan; ++c)
        Rr[bl * n_s + (int64_t)t * n_chan + c] =
            m_scale(m_load(vis_at((double*)vis, n_bl, n_chan, t, bl, c)), phasor(orc_phase_turns(tau, freq[c]), +1.0));
    }
  mat2* G = (mat2*)malloc(sizeof(mat2) * n_ant);
  mat2* H = (mat2*)malloc(sizeof(mat2) * n_ant);
  for (int32_t p = 0; p < n_ant; ++p) {
    G[p] = m_load(gain + (int64_t)p * 8);
    H[p] = m_load(slope + (int64_t)p * 8);
  }
  int taken = rotation_step(n_ant, n_chan, n_time, freq, Rr, S, G, H, g, h);
  for (int32_t p = 0; p < n_ant; ++p) m_store(slope + (int64_t)p * 8, H[p]);
  free(Rr); free(G); free(H);
  return taken;
}

int32_t orc_peel_taylor(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, double* vis, int32_t n_src, const double* lmS,
                        int32_t n_iter, double* gain, double* slope, int32_t* status,
                        double* rel_per_src) {
  int32_t worst = 0;
  for (int32_t k = 0; k < n_src; ++k) {
    double l = lmS[3 * k], m = lmS[3 * k + 1], S = lmS[3 * k + 2];
    double* Gk = gain + (int64_t)k * n_ant * 8;
    double* Hk = slope + (int64_t)k * n_ant * 8;
    int32_t st = orc_als_taylor(n_ant, n_chan, n_time, uvw, freq, vis, l, m, S, n_iter, Gk, Hk,
                                rel_per_src ? rel_per_src + k : NULL);
    if (status) status[k] = st;
    if (st < 0) worst = st;
    /* subtract S (G_i + x H_i)(G_j + x H_j)^H exp(-2 pi i phi) */
    double one[3] = {l, m, -S};
    orc_predict_taylor(n_ant, n_chan, n_time, uvw, freq, 1, one, Gk, Hk, vis, 1);
  }
  return worst;
}

/* ---- gridder (Section 6, the gridding equation) ---------------------------
 * V_grid(x, y) = sum_i f(r_i) V_i over visibilities with r_i < r_max, where
 * r_i = |(x, y) - (x_i, y_i)| is the distance from the pixel centre (integer
 * coordinates) to the visibility, in pixels, and the gridding convolution
 * function f is radial (reading R18): the linear interpolation of the table
 * gcf[0 .. n_tab-1] sampled at r_k = k r_max / (n_tab - 1).  Visibilities
 * outside [0, n_pix) in either coordinate are not gridded.  Each of n_pol
 * complex values per visibility goes to its own plane.  Plain scatter in
 * input order, FP64.                                                        */

static double gcf_at(const double* gcf, int32_t n_tab, double r_max, double r) {
  double s = r / r_max * (n_tab - 1);
  int32_t k = (int32_t)floor(s);
  if (k >= n_tab - 1) return gcf[n_tab - 1];
  double w = s - k;
  return gcf[k] + w * (gcf[k + 1] - gcf[k]);
}

void orc_grid(int32_t n_pix, double r_max, const double* gcf, int32_t n_tab, int32_t n_vis,
              int32_t n_pol, const double* xy, const double* vis, double* grid) {
  int64_t plane = (int64_t)n_pix * n_pix;
  memset(grid, 0, sizeof(double) * 2 * plane * n_pol);
  for (int32_t i = 0; i < n_vis; ++i) {
    double x = xy[2 * i], y = xy[2 * i + 1];
    if (!(x >= 0.0 && x < n_pix && y >= 0.0 && y < n_pix)) continue;
    int32_t x0 = (int32_t)ceil(x - r_max), x1 = (int32_t)floor(x + r_max);
    int32_t y0 = (int32_t)ceil(y - r_max), y1 = (int32_t)floor(y + r_max);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > n_pix - 1) x1 = n_pix - 1;
    if (y1 > n_pix - 1) y1 = n_pix - 1;
    for (int32_t py = y0; py <= y1; ++py)
      for (int32_t px = x0; px <= x1; ++px) {
        double r = sqrt((px - x) * (px - x) + (py - y) * (py - y));
        if (!(r < r_max)) continue;
        double f = gcf_at(gcf, n_tab, r_max, r);
        for (int32_t p = 0; p < n_pol; ++p) {
          double* g = grid + 2 * ((int64_t)p * plane + (int64_t)py * n_pix + px);
          g[0] += f * vis[2 * ((int64_t)i * n_pol + p)];
          g[1] += f * vis[2 * ((int64_t)i * n_pol + p) + 1];
        }
      }
  }
}

/* ---- visibility integrator (Section 3, the first stage of the RTS) ---------
 * The correlator delivers a sample every dt (0.5 s); the integrator averages
 * them into longer groups, shorter for baselines between widely separated
 * tiles (their delays change faster with the Earth's rotation).  Reading R19:
 * baseline b averages len[b] consecutive fine samples (len[b] divides n_fine),
 * output slot s of baseline b is the mean of fine samples s len[b] ..
 * (s + 1) len[b] - 1, for s < n_fine / len[b]; the remaining slots (up to
 * n_slot) are zero.  fine [n_fine][n_bl][n_chan][4], out [n_slot][n_bl][n_chan][4]. */

void orc_integrate(int32_t n_fine, int64_t n_bl, int32_t n_chan, const int32_t* len, int32_t n_slot,
                   const double* fine, double* out) {
  int64_t per_t = n_bl * n_chan * 4;                 /* complex values per time sample */
  memset(out, 0, sizeof(double) * 2 * per_t * n_slot);
  for (int64_t b = 0; b < n_bl; ++b) {
    int32_t L = len[b];
    for (int32_t s = 0; s < n_fine / L && s < n_slot; ++s)
      for (int32_t c = 0; c < n_chan; ++c)
        for (int32_t e = 0; e < 4; ++e) {
          double re = 0.0, im = 0.0;
          for (int32_t t = s * L; t < (s + 1) * L; ++t) {
            const double* x = fine + 2 * ((int64_t)t * per_t + (b * n_chan + c) * 4 + e);
            re += x[0];
            im += x[1];
          }
          double* o = out + 2 * ((int64_t)s * per_t + (b * n_chan + c) * 4 + e);
          o[0] = re / L;
          o[1] = im / L;
        }
  }
}

/* ---- Taylor-gain moments and pair terms (for the blocked Taylor schedule) ---
 * mom[n][bl][4] = mean_{t,c} x_c^n R(t,bl,c) exp(+2 pi i phi) (n = 0, 1, 2), the
 * residual's channel moments in direction (l, m); and, for two directions j
 * and k, dterm[p][bl] = mean_{t,c} x_c^p exp(2 pi i (phi_k - phi_j)) (p = 0..4),
 * the plain definitions (direct sums) of the terms that correct source k's
 * moments for the model of an earlier source j of the same block:
 *   M_n(k) = M_n^plain(k) - sum_j sum_m P_m,j D^(n+m)_jk,
 *   P_0 = S G_i G_j^H, P_1 = S (G_i H_j^H + H_i G_j^H), P_2 = S H_i H_j^H.      */

void orc_taylor_moments(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                        const double* freq, const double* vis, double l, double m, double* mom) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  double inv_n = 1.0 / ((double)n_time * n_chan);
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    mat2 acc[3] = {m_zero(), m_zero(), m_zero()};
    for (int32_t t = 0; t < n_time; ++t) {
      double tau = orc_delay_m(uvw, n_ant, t, ai[bl], aj[bl], l, m);
      for (int32_t c = 0; c < n_chan; ++c) {
        double x = taylor_x(freq, n_chan, c);
        mat2 y = m_scale(m_load(vis_at((double*)vis, n_bl, n_chan, t, bl, c)), phasor(orc_phase_turns(tau, freq[c]), +1.0));
        acc[0] = m_add(acc[0], y);
        acc[1] = m_add(acc[1], m_scale(y, x));
        acc[2] = m_add(acc[2], m_scale(y, x * x));
      }
    }
    for (int n = 0; n < 3; ++n) m_store(mom + ((int64_t)n * n_bl + bl) * 8, m_scale(acc[n], inv_n));
  }
}

void orc_taylor_dterm(int32_t n_ant, int32_t n_chan, int32_t n_time, const double* uvw,
                      const double* freq, double lj, double mj, double lk, double mk, double* dterm) {
  int64_t n_bl = orc_n_baselines(n_ant);
  int32_t *ai, *aj;
  antenna_map(n_ant, &ai, &aj);
  double inv_n = 1.0 / ((double)n_time * n_chan);
#pragma omp parallel for schedule(static)
  for (int64_t bl = 0; bl < n_bl; ++bl) {
    cplx acc[5] = {0, 0, 0, 0, 0};
    for (int32_t t = 0; t < n_time; ++t) {
      double tj = orc_delay_m(uvw, n_ant, t, ai[bl], aj[bl], lj, mj);
      double tk = orc_delay_m(uvw, n_ant, t, ai[bl], aj[bl], lk, mk);
      for (int32_t c = 0; c < n_chan; ++c) {
        double x = taylor_x(freq, n_chan, c), xp = 1.0;
        cplx z = phasor(orc_phase_turns(tk, freq[c]), +1.0) * phasor(orc_phase_turns(tj, freq[c]), -1.0);
        for (int p = 0; p < 5; ++p, xp *= x) acc[p] += xp * z;
      }
    }
    for (int p = 0; p < 5; ++p) {
      dterm[2 * ((int64_t)p * n_bl + bl)] = creal(acc[p]) * inv_n;
      dterm[2 * ((int64_t)p * n_bl + bl) + 1] = cimag(acc[p]) * inv_n;
    }
  }
}
