/*
 * FP64 oracle of the learned face flux (TEST INFRASTRUCTURE ONLY, see
 * oracle.h).
 *
 * The paper has no learned flux: it solves every face with the Riemann
 * solvers of Sec. 2.4 and names neural surrogates only as future work in its
 * summary (Sec. 8).  The learned flux of this build replaces the HLLD solve
 * of a face by a network's correction of the HLLE flux, kept only where the
 * correction passes two checks, with HLLD as the fallback.  This file writes
 * that definition out step by step, in FP64, in the order the build defines
 * it (every quantity in the face frame of Sec. 2.4: w = (rho, vn, vt1, vt2,
 * p, Bt1, Bt2), normal field bn on both sides):
 *
 *  1. scales: rho_L and c = max(c_f,L, c_f,R), the fast magnetosonic speeds
 *     along the face normal (the outer-speed estimate of the HLLD solver);
 *  2. the 14 dimensionless features: the left state without its density
 *     and bn, each divided by its natural scale (c for speeds, rho_L c^2 for
 *     pressures, sqrt(rho_L) c for fields), then the jump dW = W_R - W_L on
 *     the same scales (density on rho_L) as d (1 + |dW|), d = dW / |dW|
 *     (zero where the states coincide): an invertible encoding of the two
 *     states that keeps the jump's direction whatever its size;
 *  3. the network output y (7 numbers), the MLP of mlp.c;
 *  4. the flux scales k = (rho_L c, rho_L c^2 (x3), rho_L c^3 gamma /
 *     (gamma - 1), sqrt(rho_L) c^2 (x2));
 *  5. the HLLE flux F_E between the outer speeds S_L = min(vn_L, vn_R) - c,
 *     S_R = max(vn_L, vn_R) + c (upwind side when the fan lies on one side
 *     of the face), and the dimensionless jump
 *     J = (S_R - S_L) sqrt(sum_q ((U_R,q - U_L,q) / k_q)^2);
 *  6. the candidate F = F_E + k J y (a hydro face carries no induction
 *     flux);
 *  7. acceptance: for every component |F_q - F_E,q| <= tau (S_R - S_L)
 *     |U_R,q - U_L,q| + 0.02 k_q (within a fraction tau of the HLL
 *     dissipation bracket around F_E), and the HLL-fan states the candidate
 *     implies keep rho > 0 and p > 0: by the jump condition across the outer
 *     wave at S, F - F_side = S (U* - U_side), those are U_L + (F - F_L) /
 *     S_L where S_L < 0 and U_R + (F - F_R) / S_R where S_R > 0 (for
 *     F = F_E both are the HLL state);
 *  8. a rejected face takes the HLLD flux of mhd.c.
 *
 * The network's training target (orc_learned_target) is the HLLD flux in the
 * same form: y = (F_HLLD - F_E) / (k J), zero where J <= 1e-9.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle_internal.h"

#define LF_NIN 14
#define LF_NOUT 7

/* steps 1, 2 and 4: scales, features x[14] and flux scales k[7] */
static void lf_scales(double gamma, const double* wl, const double* wr, double bn, double* x,
                      double* k) {
  const double cl = orc_fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  const double cr = orc_fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  const double rho = wl[0], c = cl > cr ? cl : cr, sq = sqrt(rho);
  const double sv = c, sp = rho * c * c, sb = sq * c;
  if (x) {
    x[0] = wl[1] / sv; x[1] = wl[2] / sv; x[2] = wl[3] / sv;
    x[3] = wl[4] / sp; x[4] = wl[5] / sb; x[5] = wl[6] / sb;
    x[6] = bn / sb;
    const double scale[7] = {rho, sv, sv, sv, sp, sb, sb};
    double dw[7], m = 0.0;
    for (int q = 0; q < 7; ++q) {
      dw[q] = (wr[q] - wl[q]) / scale[q];
      m += dw[q] * dw[q];
    }
    m = sqrt(m);
    for (int q = 0; q < 7; ++q) x[7 + q] = m > 0.0 ? dw[q] / m * (1.0 + m) : 0.0;
  }
  k[0] = rho * c;
  k[1] = k[2] = k[3] = rho * c * c;
  k[4] = rho * c * c * c * gamma / (gamma - 1.0);
  k[5] = k[6] = sq * c * c;
}

/* step 5: HLLE flux, outer speeds, conserved states and fluxes of the two
 * sides, and the jump J */
typedef struct {
  double ul[7], ur[7], fl[7], fr[7], fe[7];
  double sl, sr, J;
} LfHll;

static void lf_hlle(double gamma, const double* wl, const double* wr, double bn, const double* k,
                    LfHll* h) {
  double ptl, ptr;
  orc_side_flux(gamma, wl, bn, h->ul, h->fl, &ptl);
  orc_side_flux(gamma, wr, bn, h->ur, h->fr, &ptr);
  const double cl = orc_fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  const double cr = orc_fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  const double c = cl > cr ? cl : cr;
  h->sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - c;
  h->sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + c;
  double s2 = 0.0;
  for (int q = 0; q < 7; ++q) {
    const double du = h->ur[q] - h->ul[q];
    s2 += (du / k[q]) * (du / k[q]);
    if (h->sl >= 0.0) {
      h->fe[q] = h->fl[q];                 /* the whole fan moves right */
    } else if (h->sr <= 0.0) {
      h->fe[q] = h->fr[q];                 /* the whole fan moves left */
    } else {
      /* flux of the single HLL state between S_L and S_R */
      h->fe[q] = (h->sr * h->fl[q] - h->sl * h->fr[q] + h->sl * h->sr * du) / (h->sr - h->sl);
    }
  }
  h->J = (h->sr - h->sl) * sqrt(s2);
}

/* rho and p of a conserved face-frame state (normal field bn) */
static void lf_rho_p(double gamma, const double* u, double bn, double* rho, double* p) {
  *rho = u[0];
  if (!(u[0] > 0.0)) { *p = -1.0; return; }
  const double ke = 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
  const double me = 0.5 * (bn * bn + u[5] * u[5] + u[6] * u[6]);
  *p = (gamma - 1.0) * (u[4] - ke - me);
}

int orc_learned_flux(double gamma, const double* wl, const double* wr, double bn,
                     const double* params, double tau, int mhd, double* flux, double* info) {
  static const int dims[5] = {14, 128, 128, 128, 7};
  double x[LF_NIN], y[LF_NOUT], k[7], F[7];
  lf_scales(gamma, wl, wr, bn, x, k);                    /* steps 1, 2, 4 */
  orc_mlp_forward(4, dims, params, 1, x, y);             /* step 3 */
  LfHll h;
  lf_hlle(gamma, wl, wr, bn, k, &h);                     /* step 5 */
  for (int q = 0; q < 7; ++q) F[q] = h.fe[q] + k[q] * h.J * y[q];   /* step 6 */
  if (!mhd) F[5] = F[6] = 0.0;
  /* step 7: the bracket around F_E, then positivity in the HLL fan */
  int ok = 1;
  double m_br = INFINITY, m_pos = INFINITY;
  for (int q = 0; q < 7; ++q) {
    const double tol = tau * (h.sr - h.sl) * fabs(h.ur[q] - h.ul[q]) + 0.02 * k[q];
    const double d = fabs(F[q] - h.fe[q]);
    if (!(d <= tol)) ok = 0;
    if (h.J > 0.0) {
      const double m = (tol - d) / (k[q] * h.J);
      if (m < m_br) m_br = m;
    }
  }
  for (int side = 0; side < 2; ++side) {
    const double s = side == 0 ? h.sl : h.sr;
    if (side == 0 ? !(s < 0.0) : !(s > 0.0)) continue;
    const double* u = side == 0 ? h.ul : h.ur;
    const double* f = side == 0 ? h.fl : h.fr;
    double us[7], rho, p;
    for (int q = 0; q < 7; ++q) us[q] = u[q] + (F[q] - f[q]) / s;
    lf_rho_p(gamma, us, bn, &rho, &p);
    if (!(rho > 0.0 && p > 0.0)) ok = 0;
    if (info && h.J > 0.0) {
      /* margins of the positivity test in units of the network output: a
       * change dy moves the implied state by k J dy / |S| per component,
       * and p by at most (gamma - 1) (k_E + |v| (k_Mn + k_Mt1 + k_Mt2) +
       * |v|^2 / 2 k_rho + |B_t| (k_Bt1 + k_Bt2)) J dy / |S| */
      const double a = h.J / fabs(s);
      const double r = rho > 0.0 ? rho : 1e-300;
      const double v = sqrt(us[1] * us[1] + us[2] * us[2] + us[3] * us[3]) / r;
      const double b = sqrt(us[5] * us[5] + us[6] * us[6]);
      const double dp = (gamma - 1.0) * (k[4] + v * (k[1] + k[2] + k[3]) + 0.5 * v * v * k[0] +
                                         b * (k[5] + k[6])) * a;
      const double mr = rho / (k[0] * a);
      if (mr < m_pos) m_pos = mr;
      if (rho > 0.0 && p / dp < m_pos) m_pos = p / dp;   /* p exists only where rho > 0 */
    }
  }
  if (info) {
    for (int q = 0; q < 7; ++q) { info[q] = F[q]; info[8 + q] = k[q]; }
    info[7] = h.J;
    info[15] = m_br;
    info[16] = m_pos;
    for (int q = 0; q < 7; ++q) info[17 + q] = y[q];
  }
  if (ok) {
    memcpy(flux, F, sizeof F);
    return 1;
  }
  orc_hlld(gamma, wl, wr, bn, flux);                     /* step 8 */
  if (!mhd) flux[5] = flux[6] = 0.0;
  return 0;
}

void orc_learned_target(double gamma, const double* wl, const double* wr, double bn, double* y) {
  double k[7], fd[7];
  LfHll h;
  lf_scales(gamma, wl, wr, bn, NULL, k);
  lf_hlle(gamma, wl, wr, bn, k, &h);
  orc_hlld(gamma, wl, wr, bn, fd);
  for (int q = 0; q < 7; ++q) y[q] = h.J > 1e-9 ? (fd[q] - h.fe[q]) / (k[q] * h.J) : 0.0;
}

void orc_learned_features(double gamma, const double* wl, const double* wr, double bn,
                          double* x, double* k) {
  lf_scales(gamma, wl, wr, bn, x, k);
}

void orc_learned_flux_batch(double gamma, int n, const double* wl, const double* wr,
                            const double* bn, const double* params, double tau, int mhd,
                            double* flux, int* accepted, double* info) {
#pragma omp parallel for schedule(static)
  for (int f = 0; f < n; ++f)
    accepted[f] = orc_learned_flux(gamma, wl + 7 * (long)f, wr + 7 * (long)f, bn[f], params, tau,
                                   mhd, flux + 7 * (long)f, info ? info + 24 * (long)f : NULL);
}
