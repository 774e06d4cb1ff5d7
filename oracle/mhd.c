/*
 * FP64 oracle: one finite-volume MHD step as the Aether.jl paper
 * (arXiv 2608.14048, Sec. 2) states it.  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).  Plain loops, explicit ghost zones, one pass per operation.
 */
#include "oracle.h"
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Mesh and geometry (Sec. 2.3)                                         */
/* ------------------------------------------------------------------ */

int orc_mesh_init(Mesh* m, const orc_grid* g, int ng) {
  m->n[0] = g->nx; m->n[1] = g->ny; m->n[2] = g->nz;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || ng < 1) return -1;
  m->ng = ng;
  for (int d = 0; d < 3; ++d) {
    m->N[d] = m->n[d] + 2 * ng + 1;
    m->lo[d] = g->lo[d];
    m->hi[d] = g->hi[d];
    m->dx[d] = (g->hi[d] - g->lo[d]) / m->n[d];
    m->bc[d] = g->bc[d];
    if (!(m->dx[d] > 0)) return -1;
  }
  m->coord = g->coord;
  m->size = (long)m->N[0] * m->N[1] * m->N[2];
  return 0;
}

/* Face coordinate of face index i along axis d (face i is the lower face
 * of cell i). */
double orc_xf(const Mesh* m, int d, int i) { return m->lo[d] + i * m->dx[d]; }

/* Exact face area of the lower face of cell (i,j,k) normal to axis d. */
double orc_area(const Mesh* m, int d, int i, int j, int k) {
  if (m->coord == ORC_CART) {
    if (d == 0) return m->dx[1] * m->dx[2];
    if (d == 1) return m->dx[0] * m->dx[2];
    return m->dx[0] * m->dx[1];
  }
  /* spherical-polar (r, theta, phi) */
  double rm = orc_xf(m, 0, i), rp = orc_xf(m, 0, i + 1);
  double tm = orc_xf(m, 1, j), tp = orc_xf(m, 1, j + 1);
  double dphi = m->dx[2];
  (void)k;
  if (d == 0) return rm * rm * (cos(tm) - cos(tp)) * dphi;
  if (d == 1) return 0.5 * (rp * rp - rm * rm) * sin(tm) * dphi;
  return 0.5 * (rp * rp - rm * rm) * (tp - tm);
}

/* Exact cell volume. */
double orc_volume(const Mesh* m, int i, int j, int k) {
  if (m->coord == ORC_CART) return m->dx[0] * m->dx[1] * m->dx[2];
  double rm = orc_xf(m, 0, i), rp = orc_xf(m, 0, i + 1);
  double tm = orc_xf(m, 1, j), tp = orc_xf(m, 1, j + 1);
  (void)k;
  return (rp * rp * rp - rm * rm * rm) / 3.0 * (cos(tm) - cos(tp)) * m->dx[2];
}

/* Exact length of the edge along axis d that starts at the lower corner of
 * cell (i,j,k) (edge along x1 at (x2f(j), x3f(k)), and so on). */
double orc_edge(const Mesh* m, int d, int i, int j, int k) {
  if (m->coord == ORC_CART) return m->dx[d];
  double r = orc_xf(m, 0, i);
  (void)k;
  if (d == 0) return m->dx[0];
  if (d == 1) return r * m->dx[1];
  return r * sin(orc_xf(m, 1, j)) * m->dx[2];
}

/* Physical cell widths at the volume-weighted centroid, used by Eq. 11. */
void orc_widths(const Mesh* m, int i, int j, int k, double* w) {
  if (m->coord == ORC_CART) {
    w[0] = m->dx[0]; w[1] = m->dx[1]; w[2] = m->dx[2];
    return;
  }
  double rm = orc_xf(m, 0, i), rp = orc_xf(m, 0, i + 1);
  double tm = orc_xf(m, 1, j), tp = orc_xf(m, 1, j + 1);
  (void)k;
  double rc = 0.75 * (pow(rp, 4) - pow(rm, 4)) / (pow(rp, 3) - pow(rm, 3));
  double tc = (sin(tp) - sin(tm) - tp * cos(tp) + tm * cos(tm)) /
              (cos(tm) - cos(tp));
  w[0] = m->dx[0];
  w[1] = rc * m->dx[1];
  w[2] = rc * sin(tc) * m->dx[2];
}

/* ------------------------------------------------------------------ */
/* Ghost zones: periodic or outflow, one axis at a time so that edge and  */
/* corner ghosts (all 26 neighbours, Sec. 2.3) are filled.              */
/* ------------------------------------------------------------------ */

static void fill_axis(const Mesh* m, double* a, int d, int is_face_d) {
  int n = m->n[d], ng = m->ng;
  int lo[3], hi[3];
  for (int e = 0; e < 3; ++e) {
    if (e <= d) { lo[e] = -ng; hi[e] = m->n[e] + ng; }  /* own axis, or
                                                           already filled */
    else { lo[e] = 0; hi[e] = m->n[e]; }                 /* incl. last face */
  }
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int c[3] = {i, j, k};
        if (d == 0 && !(i < 0 || i >= n)) continue;
        if (d == 1 && !(j < 0 || j >= n)) continue;
        if (d == 2 && !(k < 0 || k >= n)) continue;
        int p = c[d];
        int s;
        if (m->bc[d] == ORC_PERIODIC) {
          s = ((p % n) + n) % n;
        } else if (is_face_d) {      /* outflow, normal face field */
          if (p >= 0 && p <= n) continue;   /* faces 0..n are real */
          s = p < 0 ? 0 : n;
        } else {                     /* outflow, zero gradient */
          s = p < 0 ? 0 : n - 1;
        }
        int src[3] = {i, j, k};
        src[d] = s;
        a[IDX(m, i, j, k)] = a[IDX(m, src[0], src[1], src[2])];
      }
}

void orc_fill_ghosts(const Mesh* m, double** u, int nu, double** b) {
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < nu; ++v) fill_axis(m, u[v], d, 0);
    if (b)
      for (int f = 0; f < 3; ++f) fill_axis(m, b[f], d, f == d);
  }
}

/* ------------------------------------------------------------------ */
/* Conserved -> primitive (Sec. 2.1, Eq. 5) with floors                 */
/* ------------------------------------------------------------------ */

/* Dual-energy selection (Sec. 2.8): the internal energy from the total,
 * eint = E - kinetic - magnetic, is untrusted when it is below alpha_switch
 * times the kinetic plus magnetic energy (written as a product so that a
 * fluid at rest without field compares eint with 0). */
static int dual_use_entropy(const orc_params* p, double eint, double kin_mag) {
  return eint < p->alpha_switch * kin_mag;
}

/* Dual-energy synchronisation of the interior cells of a stage state
 * (Sec. 2.8), before its ghost fill: where eint is untrusted, E is
 * rewritten from S (eint = S rho^(gamma-1) / (gamma-1)); where eint exceeds
 * alpha_sync times the kinetic plus magnetic energy, S is resynchronised
 * from E; in between neither changes. */
static void dual_sync(const Mesh* m, const orc_params* p, double** u, double** b) {
#pragma omp parallel for collapse(2)
  for (int k = 0; k < m->n[2]; ++k)
    for (int j = 0; j < m->n[1]; ++j)
      for (int i = 0; i < m->n[0]; ++i) {
        long c = IDX(m, i, j, k);
        double rho = u[0][c];
        if (rho < p->rho_floor) rho = p->rho_floor;
        double v1 = u[1][c] / rho, v2 = u[2][c] / rho, v3 = u[3][c] / rho;
        double bc1 = 0, bc2 = 0, bc3 = 0;
        if (p->mhd) {
          bc1 = 0.5 * (b[0][c] + b[0][IDX(m, i + 1, j, k)]);
          bc2 = 0.5 * (b[1][c] + b[1][IDX(m, i, j + 1, k)]);
          bc3 = 0.5 * (b[2][c] + b[2][IDX(m, i, j, k + 1)]);
        }
        double km = 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3) +
                    0.5 * (bc1 * bc1 + bc2 * bc2 + bc3 * bc3);
        double eint = u[4][c] - km;
        double rg = pow(rho, p->gamma - 1.0);
        if (dual_use_entropy(p, eint, km)) {
          u[4][c] = u[5][c] * rg / (p->gamma - 1.0) + km;
        } else if (eint > p->alpha_sync * km) {
          u[5][c] = (p->gamma - 1.0) * eint / rg;
        }
      }
}

/* W = (rho, v1, v2, v3, p, B1, B2, B3) with cell-centred B the mean of the
 * two bounding face values (Sec. 2.5); with dual energy also w[8] = S/rho. */
static long cons_to_prim(const Mesh* m, const orc_params* p, double** u,
                         double** b, double** w) {
  long hits = 0;
  int ng = m->ng;
#pragma omp parallel for reduction(+ : hits) collapse(2)
  for (int k = -ng; k < m->n[2] + ng; ++k)
    for (int j = -ng; j < m->n[1] + ng; ++j)
      for (int i = -ng; i < m->n[0] + ng; ++i) {
        long c = IDX(m, i, j, k);
        double rho = u[0][c];
        if (rho < p->rho_floor) { rho = p->rho_floor; ++hits; }
        double v1 = u[1][c] / rho, v2 = u[2][c] / rho, v3 = u[3][c] / rho;
        double bc1 = 0, bc2 = 0, bc3 = 0;
        if (p->mhd) {
          bc1 = 0.5 * (b[0][c] + b[0][IDX(m, i + 1, j, k)]);
          bc2 = 0.5 * (b[1][c] + b[1][IDX(m, i, j + 1, k)]);
          bc3 = 0.5 * (b[2][c] + b[2][IDX(m, i, j, k + 1)]);
        }
        double ke = 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3);
        double me = 0.5 * (bc1 * bc1 + bc2 * bc2 + bc3 * bc3);
        double pr;
        if (p->iso) {
          pr = p->cs_iso * p->cs_iso * rho;
        } else if (p->dual && dual_use_entropy(p, u[4][c] - ke - me, ke + me)) {
          /* dual energy (Sec. 2.8): the subtraction is untrusted, the
           * pressure comes from the advected entropy */
          pr = u[5][c] * pow(rho, p->gamma - 1.0);
          if (pr < p->p_floor) { pr = p->p_floor; ++hits; }
        } else {
          pr = (p->gamma - 1.0) * (u[4][c] - ke - me);
          if (pr < p->p_floor) { pr = p->p_floor; ++hits; }
        }
        w[0][c] = rho; w[1][c] = v1; w[2][c] = v2; w[3][c] = v3;
        w[4][c] = pr;  w[5][c] = bc1; w[6][c] = bc2; w[7][c] = bc3;
        if (p->dual) w[8][c] = u[5][c] / rho;   /* specific entropy */
      }
  return hits;
}

/* ------------------------------------------------------------------ */
/* Reconstruction (Sec. 2.4): donor cell, PLM with the van Leer (1974)   */
/* harmonic-mean limiter, PPM (Colella & Woodward 1984).                 */
/* ------------------------------------------------------------------ */

static double vl_slope(double wm, double w0, double wp) {
  double dm = w0 - wm, dp = wp - w0;
  if (dm * dp > 0.0) return 2.0 * dm * dp / (dm + dp);
  return 0.0;
}

/* Fourth-order interface value between s1 and s2 (stencil s0..s3), kept
 * inside the range of its two neighbours. */
static double ppm_iface(double s0, double s1, double s2, double s3) {
  double a = (7.0 / 12.0) * (s1 + s2) - (1.0 / 12.0) * (s0 + s3);
  double lo = s1 < s2 ? s1 : s2, hi = s1 < s2 ? s2 : s1;
  if (a < lo) a = lo;
  if (a > hi) a = hi;
  return a;
}

/* Parabola limiter of CW84: flatten at an extremum, otherwise pull the
 * overshooting side back so the parabola stays monotone in the cell. */
static void ppm_limit(double w, double* al, double* ar) {
  double l = *al, r = *ar;
  if ((r - w) * (w - l) <= 0.0) {
    l = w; r = w;
  } else {
    double d = r - l, q = d * (w - 0.5 * (l + r)), d2 = d * d / 6.0;
    if (q > d2) l = 3.0 * w - 2.0 * r;
    else if (-d2 > q) r = 3.0 * w - 2.0 * l;
  }
  *al = l; *ar = r;
}

/* PPM5 (Sec. 2.4): the interface value of a cell from the quartic through
 * the five cell averages centred on it (upwind-biased toward that cell),
 * exact for cell averages of polynomials up to degree 4.  q[0..4] = cells
 * c-2..c+2; right: the value at c+1/2, left: at c-1/2. */
static double ppm5_right(const double* q) {
  return (2.0 * q[0] - 13.0 * q[1] + 47.0 * q[2] + 27.0 * q[3] - 3.0 * q[4]) / 60.0;
}
static double ppm5_left(const double* q) {
  return (-3.0 * q[0] + 27.0 * q[1] + 47.0 * q[2] - 13.0 * q[3] + 2.0 * q[4]) / 60.0;
}

/* clip an interface value into the range of the two cells it separates */
static double clip_pair(double a, double u0, double u1) {
  double lo = u0 < u1 ? u0 : u1, hi = u0 < u1 ? u1 : u0;
  if (a < lo) a = lo;
  if (a > hi) a = hi;
  return a;
}

/* s[0..5] = cells f-3..f+2 around face f (between s[2] and s[3]). */
static void recon_face(int recon, const double* s, double* wl, double* wr) {
  if (recon == ORC_DONOR) {
    *wl = s[2]; *wr = s[3];
  } else if (recon == ORC_PLM) {
    *wl = s[2] + 0.5 * vl_slope(s[1], s[2], s[3]);
    *wr = s[3] - 0.5 * vl_slope(s[2], s[3], s[4]);
  } else if (recon == ORC_PPM5) {
    /* cell s[2]: its two interface values from s[0..4]; cell s[3]: from
     * s[1..5]; each clipped into its face's neighbour range, then the
     * CW84 parabola limiter as in PPM */
    double l1 = clip_pair(ppm5_left(s), s[1], s[2]), r1 = clip_pair(ppm5_right(s), s[2], s[3]);
    double l2 = clip_pair(ppm5_left(s + 1), s[2], s[3]);
    double r2 = clip_pair(ppm5_right(s + 1), s[3], s[4]);
    ppm_limit(s[2], &l1, &r1);
    ppm_limit(s[3], &l2, &r2);
    *wl = r1; *wr = l2;
  } else {
    double im = ppm_iface(s[0], s[1], s[2], s[3]);   /* face f-1 */
    double i0 = ppm_iface(s[1], s[2], s[3], s[4]);   /* face f   */
    double ip = ppm_iface(s[2], s[3], s[4], s[5]);   /* face f+1 */
    double l1 = im, r1 = i0, l2 = i0, r2 = ip;
    ppm_limit(s[2], &l1, &r1);
    ppm_limit(s[3], &l2, &r2);
    *wl = r1; *wr = l2;
  }
}

void orc_recon_line(int recon, int n, const double* w, double* wl,
                    double* wr) {
  int reach = recon == ORC_DONOR ? 0 : (recon == ORC_PLM ? 1 : 2);   /* PPM, PPM5: 2 */
  for (int f = 0; f + 1 < n; ++f) {
    /* face between cells f and f+1: stencil cells f-2..f+3 */
    if (f - reach < 0 || f + 1 + reach > n - 1) {
      wl[f] = NAN; wr[f] = NAN;
      continue;
    }
    double s[6];
    for (int q = 0; q < 6; ++q) {
      int c = f - 2 + q;
      s[q] = (c >= 0 && c < n) ? w[c] : 0.0;
    }
    recon_face(recon, s, &wl[f], &wr[f]);
  }
}

/* ------------------------------------------------------------------ */
/* HLLD Riemann solver (Miyoshi & Kusano 2005), face frame (Sec. 2.4)    */
/* ------------------------------------------------------------------ */

static double fast_speed(double gamma, double rho, double p, double bn,
                         double bt1, double bt2) {
  double a2 = gamma * p / rho;
  double b2 = (bn * bn + bt1 * bt1 + bt2 * bt2) / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bn * bn / rho;
  if (disc < 0.0) disc = 0.0;
  return sqrt(0.5 * (s + sqrt(disc)));
}

/* Physical flux and conserved vector of one side, face frame. */
static void side_flux(double gamma, const double* w, double bn, double* u,
                      double* f, double* pt_out) {
  double rho = w[0], vn = w[1], v1 = w[2], v2 = w[3], p = w[4];
  double b1 = w[5], b2 = w[6];
  double bb = bn * bn + b1 * b1 + b2 * b2;
  double pt = p + 0.5 * bb;
  double e = p / (gamma - 1.0) + 0.5 * rho * (vn * vn + v1 * v1 + v2 * v2) +
             0.5 * bb;
  double vb = vn * bn + v1 * b1 + v2 * b2;
  u[0] = rho; u[1] = rho * vn; u[2] = rho * v1; u[3] = rho * v2; u[4] = e;
  u[5] = b1; u[6] = b2;
  f[0] = rho * vn;
  f[1] = rho * vn * vn + pt - bn * bn;
  f[2] = rho * vn * v1 - bn * b1;
  f[3] = rho * vn * v2 - bn * b2;
  f[4] = (e + pt) * vn - bn * vb;
  f[5] = b1 * vn - bn * v1;
  f[6] = b2 * vn - bn * v2;
  *pt_out = pt;
}

/* The two helpers above for the other files of the oracle (learned.c). */
double orc_fast_speed(double gamma, double rho, double p, double bn, double bt1, double bt2) {
  return fast_speed(gamma, rho, p, bn, bt1, bt2);
}
void orc_side_flux(double gamma, const double* w, double bn, double* u, double* f, double* pt) {
  side_flux(gamma, w, bn, u, f, pt);
}

/* Physical flux and conserved vector of one isothermal side (p = a2 rho),
 * face frame; the energy entries are zero. */
static void side_flux_iso(double a2, const double* w, double bn, double* u, double* f) {
  double rho = w[0], vn = w[1], v1 = w[2], v2 = w[3], b1 = w[5], b2 = w[6];
  double pt = a2 * rho + 0.5 * (bn * bn + b1 * b1 + b2 * b2);
  u[0] = rho; u[1] = rho * vn; u[2] = rho * v1; u[3] = rho * v2; u[4] = 0.0;
  u[5] = b1; u[6] = b2;
  f[0] = rho * vn;
  f[1] = rho * vn * vn + pt - bn * bn;
  f[2] = rho * vn * v1 - bn * b1;
  f[3] = rho * vn * v2 - bn * b2;
  f[4] = 0.0;
  f[5] = b1 * vn - bn * v1;
  f[6] = b2 * vn - bn * v2;
}

/* outer wave-speed estimates of both solvers: the fast speed with gamma = 1
 * and p = a2 rho is the isothermal fast speed */
static void iso_speeds(double a2, const double* wl, const double* wr, double bn, double* sl,
                       double* sr) {
  double cfl = fast_speed(1.0, wl[0], a2 * wl[0], bn, wl[5], wl[6]);
  double cfr = fast_speed(1.0, wr[0], a2 * wr[0], bn, wr[5], wr[6]);
  double cmax = cfl > cfr ? cfl : cfr;
  *sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - cmax;
  *sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + cmax;
}

void orc_hlle_iso(double cs, const double* wl, const double* wr, double bn, double* flux) {
  double a2 = cs * cs, ul[7], ur[7], fl[7], fr[7], sl, sr;
  side_flux_iso(a2, wl, bn, ul, fl);
  side_flux_iso(a2, wr, bn, ur, fr);
  iso_speeds(a2, wl, wr, bn, &sl, &sr);
  double bm = sl < 0.0 ? sl : 0.0, bp = sr > 0.0 ? sr : 0.0;
  for (int q = 0; q < 7; ++q)
    flux[q] = (bp * fl[q] - bm * fr[q] + bp * bm * (ur[q] - ul[q])) / (bp - bm);
}

#define HLLD_ISO_EPS 1e-12

void orc_hlld_iso(double cs, const double* wl, const double* wr, double bn, double* flux) {
  double a2 = cs * cs, ul[7], ur[7], fl[7], fr[7], sl, sr;
  side_flux_iso(a2, wl, bn, ul, fl);
  side_flux_iso(a2, wr, bn, ur, fr);
  iso_speeds(a2, wl, wr, bn, &sl, &sr);
  if (sl >= 0.0) { for (int q = 0; q < 7; ++q) flux[q] = fl[q]; return; }
  if (sr <= 0.0) { for (int q = 0; q < 7; ++q) flux[q] = fr[q]; return; }
  /* density and normal momentum are uniform inside the fan (no contact
   * wave): their fluxes there are the HLL fluxes, rho* is the HLL average
   * and the normal velocity of the transverse jump conditions is
   * u* = F_rho^HLL / rho* */
  double rs = (sr * ur[0] - sl * ul[0] - (fr[0] - fl[0])) / (sr - sl);
  double fm = (sr * fl[0] - sl * fr[0] + sl * sr * (ur[0] - ul[0])) / (sr - sl);
  double fmn = (sr * fl[1] - sl * fr[1] + sl * sr * (ur[1] - ul[1])) / (sr - sl);
  double us = fm / rs;
  double sq = sqrt(rs);
  double sgn = bn > 0.0 ? 1.0 : (bn < 0.0 ? -1.0 : 0.0);
  double ssl = us - fabs(bn) / sq, ssr = us + fabs(bn) / sq;
  /* outer star states: Rankine-Hugoniot conditions across S_L and S_R for
   * the transverse momentum and field, with rho* and u* fixed */
  double st[2][7], fs[2][7];
  const double* w[2] = {wl, wr};
  const double* uu[2] = {ul, ur};
  const double* ff[2] = {fl, fr};
  double s[2] = {sl, sr};
  for (int k = 0; k < 2; ++k) {
    double rho = w[k][0], vn = w[k][1];
    double den = rho * (s[k] - vn) * (s[k] - us) - bn * bn;
    double vt1 = w[k][2], vt2 = w[k][3], bt1 = w[k][5], bt2 = w[k][6];
    if (fabs(den) >= HLLD_ISO_EPS * (rho * (s[k] - vn) * (s[k] - vn) + bn * bn)) {
      double fv = bn * (us - vn) / den;
      double fb = (rho * (s[k] - vn) * (s[k] - vn) - bn * bn) / den;
      vt1 = w[k][2] - w[k][5] * fv;
      vt2 = w[k][3] - w[k][6] * fv;
      bt1 = w[k][5] * fb;
      bt2 = w[k][6] * fb;
    }
    st[k][0] = rs; st[k][1] = rs * us; st[k][2] = rs * vt1; st[k][3] = rs * vt2; st[k][4] = 0.0;
    st[k][5] = bt1; st[k][6] = bt2;
    for (int q = 2; q < 7; ++q) fs[k][q] = ff[k][q] + s[k] * (st[k][q] - uu[k][q]);
    fs[k][0] = fm;
    fs[k][1] = fmn;
    fs[k][4] = 0.0;
  }
  if (ssl >= 0.0) { for (int q = 0; q < 7; ++q) flux[q] = fs[0][q]; return; }
  if (ssr <= 0.0) { for (int q = 0; q < 7; ++q) flux[q] = fs[1][q]; return; }
  /* central state between the Alfven waves (equal densities on both sides) */
  double vl1 = st[0][2] / rs, vl2 = st[0][3] / rs, vr1 = st[1][2] / rs, vr2 = st[1][3] / rs;
  double vc1 = 0.5 * (vl1 + vr1) + 0.5 * (st[1][5] - st[0][5]) * sgn / sq;
  double vc2 = 0.5 * (vl2 + vr2) + 0.5 * (st[1][6] - st[0][6]) * sgn / sq;
  double bc1 = 0.5 * (st[0][5] + st[1][5]) + 0.5 * sq * (vr1 - vl1) * sgn;
  double bc2 = 0.5 * (st[0][6] + st[1][6]) + 0.5 * sq * (vr2 - vl2) * sgn;
  double uc[7] = {rs, rs * us, rs * vc1, rs * vc2, 0.0, bc1, bc2};
  for (int q = 0; q < 7; ++q) flux[q] = fs[0][q];
  for (int q = 2; q < 7; ++q) flux[q] += ssl * (uc[q] - st[0][q]);
  flux[4] = 0.0;
}

void orc_hlle(double gamma, const double* wl, const double* wr, double bn, double* flux) {
  double ul[7], ur[7], fl[7], fr[7], ptl, ptr;
  side_flux(gamma, wl, bn, ul, fl, &ptl);
  side_flux(gamma, wr, bn, ur, fr, &ptr);
  double cfl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  double cfr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  double cmax = cfl > cfr ? cfl : cfr;
  double sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - cmax;
  double sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + cmax;
  double bm = sl < 0.0 ? sl : 0.0;
  double bp = sr > 0.0 ? sr : 0.0;
  /* the HLL state integrates the conservation law over the fan [b-, b+] */
  for (int q = 0; q < 7; ++q)
    flux[q] = (bp * fl[q] - bm * fr[q] + bp * bm * (ur[q] - ul[q])) / (bp - bm);
}

#define HLLD_EPS 1e-12

int orc_hlld(double gamma, const double* wl, const double* wr, double bn,
             double* flux) {
  double ul[7], ur[7], fl[7], fr[7], ptl, ptr;
  side_flux(gamma, wl, bn, ul, fl, &ptl);
  side_flux(gamma, wr, bn, ur, fr, &ptr);

  double cfl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  double cfr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  double cmax = cfl > cfr ? cfl : cfr;
  double sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - cmax;
  double sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + cmax;

  if (sl > 0.0) { memcpy(flux, fl, sizeof fl); return 0; }
  if (sr < 0.0) { memcpy(flux, fr, sizeof fr); return 5; }

  double sul = sl - wl[1], sur = sr - wr[1];
  double den = sur * wr[0] - sul * wl[0];
  double sm = (sur * wr[0] * wr[1] - sul * wl[0] * wl[1] - ptr + ptl) / den;
  double pts = (sur * wr[0] * ptl - sul * wl[0] * ptr +
                wl[0] * wr[0] * sur * sul * (wr[1] - wl[1])) / den;

  /* single-star states */
  double us[2][7], rs[2];
  const double* ws[2] = {wl, wr};
  const double* uu[2] = {ul, ur};
  double ss[2] = {sl, sr};
  double pt[2] = {ptl, ptr};
  for (int a = 0; a < 2; ++a) {
    const double* w = ws[a];
    double su = ss[a] - w[1];
    double rho_s = w[0] * su / (ss[a] - sm);
    double dd = w[0] * su * (ss[a] - sm) - bn * bn;
    double v1s, v2s, b1s, b2s;
    if (fabs(dd) < HLLD_EPS * pts) {
      v1s = w[2]; v2s = w[3]; b1s = w[5]; b2s = w[6];
    } else {
      double fv = bn * (sm - w[1]) / dd;
      double fb = (w[0] * su * su - bn * bn) / dd;
      v1s = w[2] - w[5] * fv;
      v2s = w[3] - w[6] * fv;
      b1s = w[5] * fb;
      b2s = w[6] * fb;
    }
    double vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    double vbs = sm * bn + v1s * b1s + v2s * b2s;
    double es = (su * uu[a][4] - pt[a] * w[1] + pts * sm + bn * (vb - vbs)) /
                (ss[a] - sm);
    us[a][0] = rho_s; us[a][1] = rho_s * sm; us[a][2] = rho_s * v1s;
    us[a][3] = rho_s * v2s; us[a][4] = es; us[a][5] = b1s; us[a][6] = b2s;
    rs[a] = rho_s;
  }

  /* Alfven waves; degenerate when B_n^2 is negligible */
  double sql = sqrt(rs[0]), sqr = sqrt(rs[1]);
  double abn = fabs(bn);
  int degen = 0.5 * bn * bn < HLLD_EPS * pts;
  double ssl = degen ? sm : sm - abn / sql;
  double ssr = degen ? sm : sm + abn / sqr;

  int region;
  if (ssl >= 0.0) region = 1;
  else if (sm >= 0.0) region = 2;
  else if (ssr >= 0.0) region = 3;
  else region = 4;

  if (region == 1 || region == 4) {
    int a = region == 1 ? 0 : 1;
    const double* f = a ? fr : fl;
    const double* u = a ? ur : ul;
    for (int q = 0; q < 7; ++q) flux[q] = f[q] + ss[a] * (us[a][q] - u[q]);
    return region;
  }

  /* double-star states (shared velocity and field) */
  double sgn = bn > 0 ? 1.0 : (bn < 0 ? -1.0 : 0.0);
  double inv = 1.0 / (sql + sqr);
  double v1l = us[0][2] / rs[0], v2l = us[0][3] / rs[0];
  double v1r = us[1][2] / rs[1], v2r = us[1][3] / rs[1];
  double b1l = us[0][5], b2l = us[0][6], b1r = us[1][5], b2r = us[1][6];
  double v1ss = (sql * v1l + sqr * v1r + (b1r - b1l) * sgn) * inv;
  double v2ss = (sql * v2l + sqr * v2r + (b2r - b2l) * sgn) * inv;
  double b1ss = (sql * b1r + sqr * b1l + sql * sqr * (v1r - v1l) * sgn) * inv;
  double b2ss = (sql * b2r + sqr * b2l + sql * sqr * (v2r - v2l) * sgn) * inv;
  double vbss = sm * bn + v1ss * b1ss + v2ss * b2ss;
  int a = region == 2 ? 0 : 1;
  double sq = a ? sqr : sql;
  double vbs = sm * bn + us[a][2] / rs[a] * us[a][5] +
               us[a][3] / rs[a] * us[a][6];
  double sign_side = a ? 1.0 : -1.0;
  double ess = us[a][4] + sign_side * sq * (vbs - vbss) * sgn;
  double uss[7] = {rs[a], rs[a] * sm, rs[a] * v1ss, rs[a] * v2ss, ess,
                   b1ss, b2ss};
  const double* f = a ? fr : fl;
  const double* u = a ? ur : ul;
  double sst = a ? ssr : ssl;
  for (int q = 0; q < 7; ++q)
    flux[q] = f[q] + ss[a] * (us[a][q] - u[q]) + sst * (uss[q] - us[a][q]);
  return region;
}

int orc_lhlld(double gamma, const double* wl, const double* wr, double bn, double* flux) {
  int region = orc_hlld(gamma, wl, wr, bn, flux);
  if (region == 0 || region == 5) return region;   /* supersonic: no contact */
  /* the HLLD quantities the correction needs, recomputed as in orc_hlld */
  double ul[7], ur[7], fl[7], fr[7], ptl, ptr;
  side_flux(gamma, wl, bn, ul, fl, &ptl);
  side_flux(gamma, wr, bn, ur, fr, &ptr);
  double cfl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  double cfr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  double cmax = cfl > cfr ? cfl : cfr;
  double sl = (wl[1] < wr[1] ? wl[1] : wr[1]) - cmax;
  double sr = (wl[1] > wr[1] ? wl[1] : wr[1]) + cmax;
  double sul = sl - wl[1], sur = sr - wr[1];
  double den = sur * wr[0] - sul * wl[0];
  double sm = (sur * wr[0] * wr[1] - sul * wl[0] * wl[1] - ptr + ptl) / den;
  double d = wl[0] * wr[0] * sur * sul * (wr[1] - wl[1]) / den;
  /* local Mach number: the larger flow speed over the larger fast speed */
  double vl = sqrt(wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]);
  double vr = sqrt(wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]);
  double mach = (vl > vr ? vl : vr) / cmax;
  double phi = mach < 1.0 ? mach : 1.0;
  flux[1] += (phi - 1.0) * d;
  flux[4] += (phi - 1.0) * d * sm;
  return region;
}

/* ------------------------------------------------------------------ */
/* Upwind corner EMF (Gardiner & Stone 2005), Sec. 2.5                   */
/* ------------------------------------------------------------------ */

static double upwind(double mflux, double from_lower, double from_upper) {
  if (mflux > 0.0) return from_lower;
  if (mflux < 0.0) return from_upper;
  return 0.5 * (from_lower + from_upper);
}

double orc_corner_emf(double ea_m, double ea_p, double eb_m, double eb_p,
                      const double* eref, double fa_m, double fa_p,
                      double fb_m, double fb_p) {
  /* eref[2*rb + ca]: rb = 0 row b-1, 1 row b; ca = 0 column a-1, 1 col a */
  double r00 = eref[0], r01 = eref[1], r10 = eref[2], r11 = eref[3];
  /* half-cell differences along b next to the edge (upper and lower
   * quarter points), upwinded by the a-face mass flux of their row */
  double db_hi = upwind(fa_p, r10 - eb_m, r11 - eb_p);
  double db_lo = upwind(fa_m, eb_m - r00, eb_p - r01);
  /* half-cell differences along a, upwinded by the b-face mass flux */
  double da_hi = upwind(fb_p, r01 - ea_m, r11 - ea_p);
  double da_lo = upwind(fb_m, ea_m - r00, ea_p - r10);
  return 0.25 * (ea_m + ea_p + eb_m + eb_p) + 0.25 * (db_lo - db_hi) +
         0.25 * (da_lo - da_hi);
}

/* ------------------------------------------------------------------ */
/* One stage: L(src) and the register combination                        */
/* ------------------------------------------------------------------ */

typedef struct {
  double* w[9];      /* primitives (+ specific entropy with dual energy) */
  double* f[3][6];   /* hydro fluxes per direction (+ entropy flux) */
  double* e[3][2];   /* face EMFs per direction: component t1, t2 */
  double* edge[3];   /* corner EMFs, by component */
} Work;

static double* zalloc(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

static int work_alloc(Work* wk, const Mesh* m) {
  memset(wk, 0, sizeof *wk);
  for (int v = 0; v < 9; ++v) if (!(wk->w[v] = zalloc(m->size))) return -1;
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 6; ++v) if (!(wk->f[d][v] = zalloc(m->size))) return -1;
    for (int v = 0; v < 2; ++v) if (!(wk->e[d][v] = zalloc(m->size))) return -1;
    if (!(wk->edge[d] = zalloc(m->size))) return -1;
  }
  return 0;
}

static void work_free(Work* wk) {
  for (int v = 0; v < 9; ++v) free(wk->w[v]);
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 6; ++v) free(wk->f[d][v]);
    for (int v = 0; v < 2; ++v) free(wk->e[d][v]);
    free(wk->edge[d]);
  }
}

/* Spherical-polar geometric momentum sources from the total stress
 * T_ij = rho v_i v_j + P* delta_ij - B_i B_j (Eq. 12), with discrete
 * factors built from the same face areas and volumes as Eq. 8:
 * <1/r> = (A_r+ - A_r-)/(2V), <cot(theta)/r> = (A_t+ - A_t-)/V. */
static void sph_source(const Mesh* m, int i, int j, int k, const double* w,
                       int mhd, double* s) {
  double rho = w[0], v[3] = {w[1], w[2], w[3]};
  double b[3] = {0, 0, 0};
  if (mhd) { b[0] = w[5]; b[1] = w[6]; b[2] = w[7]; }
  double pstar = w[4] + 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  double T[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      T[a][c] = rho * v[a] * v[c] + (a == c ? pstar : 0.0) - b[a] * b[c];
  double V = orc_volume(m, i, j, k);
  double inv_r = (orc_area(m, 0, i + 1, j, k) - orc_area(m, 0, i, j, k)) /
                 (2.0 * V);
  double cot_r = (orc_area(m, 1, i, j + 1, k) - orc_area(m, 1, i, j, k)) / V;
  s[0] = (T[1][1] + T[2][2]) * inv_r;
  s[1] = T[2][2] * cot_r - T[0][1] * inv_r;
  s[2] = -T[2][0] * inv_r - T[2][1] * cot_r;
}

/* Computes fluxes, face EMFs and corner EMFs from the state (src_u, src_b)
 * and writes out = w0*A + w1*B + beta*dt*L(src).  out may alias A. */
static long stage(const Mesh* m, const orc_params* p, int recon, Work* wk,
                  double** src_u, double** src_b, double w0, double** a_u,
                  double** a_b, double w1, double** b_u, double** b_b,
                  double beta, double dt, double** out_u, double** out_b) {
  int mhd = p->mhd;
  int nu = p->dual ? 6 : 5;
  if (p->dual) {
    /* the sync reads each interior cell's bounding faces: on periodic axes
     * the face at index n is the image of face 0, set by the ghost fill, so
     * fill first, sync, then fill again to carry the synced E and S into
     * the ghost cells */
    orc_fill_ghosts(m, src_u, nu, mhd ? src_b : NULL);
    dual_sync(m, p, src_u, src_b);
  }
  orc_fill_ghosts(m, src_u, nu, mhd ? src_b : NULL);
  long hits = cons_to_prim(m, p, src_u, src_b, wk->w);

  /* --- fluxes along each direction (Sec. 2.4), cyclic face frame --- */
  for (int d = 0; d < 3; ++d) {
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      if (e == d) { lo[e] = 0; hi[e] = m->n[e]; }
      else { lo[e] = -1; hi[e] = m->n[e]; }   /* one ring for the EMFs */
    }
    /* primitive slots of the face frame: rho, vn, vt1, vt2, p, Bt1, Bt2 */
    int slot[7] = {0, 1 + d, 1 + t1, 1 + t2, 4, 5 + t1, 5 + t2};
#pragma omp parallel for collapse(2)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          int c[3] = {i, j, k};
          long fc = IDX(m, i, j, k);
          double wl[7], wr[7];
          for (int q = 0; q < 7; ++q) {
            if (!mhd && q >= 5) { wl[q] = wr[q] = 0.0; continue; }
            double s[6];
            for (int t = 0; t < 6; ++t) {
              int cc[3] = {c[0], c[1], c[2]};
              cc[d] = c[d] - 3 + t;
              if (cc[d] < -m->ng || cc[d] >= m->n[d] + m->ng) { s[t] = NAN; continue; }
              s[t] = wk->w[slot[q]][IDX(m, cc[0], cc[1], cc[2])];
            }
            recon_face(recon, s, &wl[q], &wr[q]);
          }
          /* the normal field is the stored face value on both sides */
          double bn = mhd ? src_b[d][fc] : 0.0;
          double fx[7];
          if (p->iso) {
            if (p->riemann == ORC_HLLE) orc_hlle_iso(p->cs_iso, wl, wr, bn, fx);
            else orc_hlld_iso(p->cs_iso, wl, wr, bn, fx);
          } else if (p->riemann == ORC_HLLE) {
            orc_hlle(p->gamma, wl, wr, bn, fx);
          } else if (p->riemann == ORC_LHLLD) {
            orc_lhlld(p->gamma, wl, wr, bn, fx);
          } else {
            orc_hlld(p->gamma, wl, wr, bn, fx);
          }
          wk->f[d][0][fc] = fx[0];
          wk->f[d][1 + d][fc] = fx[1];
          wk->f[d][1 + t1][fc] = fx[2];
          wk->f[d][1 + t2][fc] = fx[3];
          wk->f[d][4][fc] = fx[4];
          /* induction flux components are face EMFs: F(Bt1) = -E_t2,
           * F(Bt2) = +E_t1 */
          wk->e[d][0][fc] = fx[6];
          wk->e[d][1][fc] = -fx[5];
          if (p->dual) {
            /* entropy flux (Sec. 2.8): mass flux times the specific entropy
             * of the upwind side, reconstructed like the primitives */
            double s6[6], sl, sr;
            for (int t = 0; t < 6; ++t) {
              int cc[3] = {c[0], c[1], c[2]};
              cc[d] = c[d] - 3 + t;
              if (cc[d] < -m->ng || cc[d] >= m->n[d] + m->ng) { s6[t] = NAN; continue; }
              s6[t] = wk->w[8][IDX(m, cc[0], cc[1], cc[2])];
            }
            recon_face(recon, s6, &sl, &sr);
            wk->f[d][5][fc] = fx[0] >= 0.0 ? fx[0] * sl : fx[0] * sr;
          }
        }
  }

  /* --- corner EMFs (Sec. 2.5) --- */
  if (mhd) {
    for (int c = 0; c < 3; ++c) {
      int a = (c + 1) % 3, b = (c + 2) % 3;
      int lo[3], hi[3];
      for (int e = 0; e < 3; ++e) {
        lo[e] = 0;
        hi[e] = (e == c) ? m->n[e] - 1 : m->n[e];
      }
#pragma omp parallel for collapse(2)
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            int P[3] = {i, j, k};
            int Pa[3] = {i, j, k}, Pb[3] = {i, j, k}, Pab[3] = {i, j, k};
            Pa[a] -= 1; Pb[b] -= 1; Pab[a] -= 1; Pab[b] -= 1;
            long iP = IDX(m, P[0], P[1], P[2]);
            long iA = IDX(m, Pa[0], Pa[1], Pa[2]);
            long iB = IDX(m, Pb[0], Pb[1], Pb[2]);
            long iAB = IDX(m, Pab[0], Pab[1], Pab[2]);
            /* cell-centred reference E_c = -(v_a B_b - v_b B_a) */
            long cells[4] = {iAB, iB, iA, iP};  /* (b-1,a-1),(b-1,a),(b,a-1),(b,a) */
            double eref[4];
            for (int q = 0; q < 4; ++q) {
              long cc = cells[q];
              eref[q] = -(wk->w[1 + a][cc] * wk->w[5 + b][cc] -
                          wk->w[1 + b][cc] * wk->w[5 + a][cc]);
            }
            double ea_m = wk->e[a][1][iB], ea_p = wk->e[a][1][iP];
            double eb_m = wk->e[b][0][iA], eb_p = wk->e[b][0][iP];
            double fa_m = wk->f[a][0][iB], fa_p = wk->f[a][0][iP];
            double fb_m = wk->f[b][0][iA], fb_p = wk->f[b][0][iP];
            wk->edge[c][iP] = orc_corner_emf(ea_m, ea_p, eb_m, eb_p, eref,
                                             fa_m, fa_p, fb_m, fb_p);
          }
    }
  }

  /* --- conserved update, Eq. 8 (+ curvilinear sources, Eq. 12) --- */
#pragma omp parallel for collapse(2)
  for (int k = 0; k < m->n[2]; ++k)
    for (int j = 0; j < m->n[1]; ++j)
      for (int i = 0; i < m->n[0]; ++i) {
        long c = IDX(m, i, j, k);
        long cp[3] = {IDX(m, i + 1, j, k), IDX(m, i, j + 1, k),
                      IDX(m, i, j, k + 1)};
        double V = orc_volume(m, i, j, k);
        double Am[3], Ap[3];
        Am[0] = orc_area(m, 0, i, j, k); Ap[0] = orc_area(m, 0, i + 1, j, k);
        Am[1] = orc_area(m, 1, i, j, k); Ap[1] = orc_area(m, 1, i, j + 1, k);
        Am[2] = orc_area(m, 2, i, j, k); Ap[2] = orc_area(m, 2, i, j, k + 1);
        double src[5] = {0, 0, 0, 0, 0};
        if (m->coord == ORC_SPH) {
          double wc[8];
          for (int v = 0; v < 8; ++v) wc[v] = wk->w[v][c];
          double s[3];
          sph_source(m, i, j, k, wc, mhd, s);
          src[1] = s[0]; src[2] = s[1]; src[3] = s[2];
        }
        for (int v = 0; v < nu; ++v) {
          double div = 0.0;
          for (int d = 0; d < 3; ++d)
            div += Ap[d] * wk->f[d][v][cp[d]] - Am[d] * wk->f[d][v][c];
          double rhs = -div / V + (v < 5 ? src[v] : 0.0);
          double base = w0 * a_u[v][c];
          if (w1 != 0.0) base += w1 * b_u[v][c];
          out_u[v][c] = base + beta * dt * rhs;
        }
      }

  /* --- constrained transport, Eq. 9 --- */
  if (mhd) {
    for (int d = 0; d < 3; ++d) {
      int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
      int hi[3];
      for (int q = 0; q < 3; ++q) hi[q] = m->n[q] - 1;
      if (m->bc[d] == ORC_OUTFLOW) hi[d] = m->n[d];  /* both end faces */
#pragma omp parallel for collapse(2)
      for (int k = 0; k <= hi[2]; ++k)
        for (int j = 0; j <= hi[1]; ++j)
          for (int i = 0; i <= hi[0]; ++i) {
            int P[3] = {i, j, k};
            int Q1[3] = {i, j, k}, Q2[3] = {i, j, k};
            Q1[e1] += 1; Q2[e2] += 1;
            long c = IDX(m, i, j, k);
            long q1 = IDX(m, Q1[0], Q1[1], Q1[2]);
            long q2 = IDX(m, Q2[0], Q2[1], Q2[2]);
            /* circulation: [E_e2 l_e2] across e1  -  [E_e1 l_e1] across e2 */
            double circ =
                wk->edge[e2][q1] * orc_edge(m, e2, Q1[0], Q1[1], Q1[2]) -
                wk->edge[e2][c] * orc_edge(m, e2, P[0], P[1], P[2]) -
                (wk->edge[e1][q2] * orc_edge(m, e1, Q2[0], Q2[1], Q2[2]) -
                 wk->edge[e1][c] * orc_edge(m, e1, P[0], P[1], P[2]));
            double A = orc_area(m, d, i, j, k);
            double base = w0 * a_b[d][c];
            if (w1 != 0.0) base += w1 * b_b[d][c];
            out_b[d][c] = base - beta * dt * circ / A;
          }
    }
  }
  return hits;
}

/* ------------------------------------------------------------------ */
/* State marshalling                                                     */
/* ------------------------------------------------------------------ */

int orc_ghost_width(int recon) {
  return (recon == ORC_PPM || recon == ORC_PPM5) ? 3 : (recon == ORC_PLM ? 2 : 1);
}

void orc_load(const Mesh* m, const double* cons, const double* b1,
              const double* b2, const double* b3, double** u, int nu,
              double** b) {
  int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  long ncell = (long)nx * ny * nz;
  for (int v = 0; v < nu; ++v)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          u[v][IDX(m, i, j, k)] = cons[v * ncell + ((long)k * ny + j) * nx + i];
  if (!b) return;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i)
        b[0][IDX(m, i, j, k)] = b1[((long)k * ny + j) * (nx + 1) + i];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i)
        b[1][IDX(m, i, j, k)] = b2[((long)k * (ny + 1) + j) * nx + i];
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        b[2][IDX(m, i, j, k)] = b3[((long)k * ny + j) * nx + i];
}

void orc_store(const Mesh* m, double** u, int nu, double** b, double* cons,
               double* b1, double* b2, double* b3) {
  int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  long ncell = (long)nx * ny * nz;
  for (int v = 0; v < nu; ++v)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          cons[v * ncell + ((long)k * ny + j) * nx + i] = u[v][IDX(m, i, j, k)];
  if (!b) return;
  /* periodic directions: the last face is the image of the first */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        int s = (i == nx && m->bc[0] == ORC_PERIODIC) ? 0 : i;
        b1[((long)k * ny + j) * (nx + 1) + i] = b[0][IDX(m, s, j, k)];
      }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int s = (j == ny && m->bc[1] == ORC_PERIODIC) ? 0 : j;
        b2[((long)k * (ny + 1) + j) * nx + i] = b[1][IDX(m, i, s, k)];
      }
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int s = (k == nz && m->bc[2] == ORC_PERIODIC) ? 0 : k;
        b3[((long)k * ny + j) * nx + i] = b[2][IDX(m, i, j, s)];
      }
}

void orc_dual_init(const orc_grid* g, const orc_params* p, double* cons, const double* b1,
                   const double* b2, const double* b3) {
  Mesh m;
  if (orc_mesh_init(&m, g, 1) != 0) return;
  int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  long ncell = (long)nx * ny * nz;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        double rho = cons[c];
        if (rho < p->rho_floor) rho = p->rho_floor;
        double m1 = cons[ncell + c], m2 = cons[2 * ncell + c], m3 = cons[3 * ncell + c];
        double bc[3] = {0, 0, 0};
        if (p->mhd) {
          bc[0] = 0.5 * (b1[((long)k * ny + j) * (nx + 1) + i] +
                         b1[((long)k * ny + j) * (nx + 1) + i + 1]);
          bc[1] = 0.5 * (b2[((long)k * (ny + 1) + j) * nx + i] +
                         b2[((long)k * (ny + 1) + j + 1) * nx + i]);
          bc[2] = 0.5 * (b3[((long)k * ny + j) * nx + i] +
                         b3[((long)(k + 1) * ny + j) * nx + i]);
        }
        double km = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / rho +
                    0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
        double pr = (p->gamma - 1.0) * (cons[4 * ncell + c] - km);
        if (pr < p->p_floor) pr = p->p_floor;
        cons[5 * ncell + c] = pr / pow(rho, p->gamma - 1.0);
      }
}

/* ------------------------------------------------------------------ */
/* Public: one step (Sec. 2.6)                                           */
/* ------------------------------------------------------------------ */

int orc_mhd_step(const orc_grid* g, const orc_params* p, double dt,
                 double* cons, double* b1, double* b2, double* b3,
                 long* floor_hits) {
  Mesh m;
  if (orc_mesh_init(&m, g, orc_ghost_width(p->recon)) != 0) return -1;
  int nu = p->dual ? 6 : 5;   /* dual energy: S is the sixth cell variable */
  double *A[6] = {0}, *Ab[3], *B[6] = {0}, *Bb[3];
  for (int v = 0; v < nu; ++v) { A[v] = zalloc(m.size); B[v] = zalloc(m.size); }
  for (int d = 0; d < 3; ++d) { Ab[d] = zalloc(m.size); Bb[d] = zalloc(m.size); }
  Work wk;
  if (work_alloc(&wk, &m) != 0) return -2;
  orc_load(&m, cons, b1, b2, b3, A, nu, p->mhd ? Ab : NULL);

  long hits = 0;
  if (p->integrator == ORC_VL2) {
    /* van Leer predictor-corrector: half step with donor-cell states from
     * U^n, then a full step from U^n with fluxes of U^{n+1/2} */
    hits += stage(&m, p, ORC_DONOR, &wk, A, Ab, 1.0, A, Ab, 0.0, NULL, NULL,
                  0.5, dt, B, Bb);
    hits += stage(&m, p, p->recon, &wk, B, Bb, 1.0, A, Ab, 0.0, NULL, NULL,
                  1.0, dt, A, Ab);
  } else if (p->integrator == ORC_RK3) {
    /* SSP-RK3 (Shu & Osher 1988; Sec. 2.6): u1 = u + dt L(u);
     * u2 = 3/4 u + 1/4 u1 + 1/4 dt L(u1); u' = 1/3 u + 2/3 u2 + 2/3 dt L(u2),
     * with a third register for u2 */
    double *C[6] = {0}, *Cb[3];
    for (int v = 0; v < nu; ++v) C[v] = zalloc(m.size);
    for (int d = 0; d < 3; ++d) Cb[d] = zalloc(m.size);
    hits += stage(&m, p, p->recon, &wk, A, Ab, 1.0, A, Ab, 0.0, NULL, NULL,
                  1.0, dt, B, Bb);
    hits += stage(&m, p, p->recon, &wk, B, Bb, 0.75, A, Ab, 0.25, B, Bb, 0.25,
                  dt, C, Cb);
    hits += stage(&m, p, p->recon, &wk, C, Cb, 1.0 / 3.0, A, Ab, 2.0 / 3.0, C, Cb,
                  2.0 / 3.0, dt, A, Ab);
    for (int v = 0; v < nu; ++v) free(C[v]);
    for (int d = 0; d < 3; ++d) free(Cb[d]);
  } else {
    /* two-register SSP-RK2 (Eq. 10): u2 <- u1; u1 <- u1 + dt L(u1);
     * u1 <- 1/2 u2 + 1/2 u1 + 1/2 dt L(u1) */
    hits += stage(&m, p, p->recon, &wk, A, Ab, 1.0, A, Ab, 0.0, NULL, NULL,
                  1.0, dt, B, Bb);
    hits += stage(&m, p, p->recon, &wk, B, Bb, 0.5, A, Ab, 0.5, B, Bb, 0.5,
                  dt, A, Ab);
  }
  if (p->mhd) orc_fill_ghosts(&m, A, nu, Ab);
  orc_store(&m, A, nu, p->mhd ? Ab : NULL, cons, b1, b2, b3);
  if (floor_hits) *floor_hits = hits;
  work_free(&wk);
  for (int v = 0; v < nu; ++v) { free(A[v]); free(B[v]); }
  for (int d = 0; d < 3; ++d) { free(Ab[d]); free(Bb[d]); }
  return 0;
}

double orc_mhd_dt(const orc_grid* g, const orc_params* p, const double* cons,
                  const double* b1, const double* b2, const double* b3) {
  Mesh m;
  if (orc_mesh_init(&m, g, 1) != 0) return NAN;
  int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  long ncell = (long)nx * ny * nz;
  double dtmin = INFINITY;
#pragma omp parallel for reduction(min : dtmin) collapse(2)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        double rho = cons[c];
        if (rho < p->rho_floor) rho = p->rho_floor;
        double v[3] = {cons[ncell + c] / rho, cons[2 * ncell + c] / rho,
                       cons[3 * ncell + c] / rho};
        double bc[3] = {0, 0, 0};
        if (p->mhd) {
          bc[0] = 0.5 * (b1[((long)k * ny + j) * (nx + 1) + i] +
                         b1[((long)k * ny + j) * (nx + 1) + i + 1]);
          bc[1] = 0.5 * (b2[((long)k * (ny + 1) + j) * nx + i] +
                         b2[((long)k * (ny + 1) + j + 1) * nx + i]);
          bc[2] = 0.5 * (b3[((long)k * ny + j) * nx + i] +
                         b3[((long)(k + 1) * ny + j) * nx + i]);
        }
        double pr, gam = p->gamma;
        if (p->iso) {
          /* isothermal: the fast speed with gamma = 1 and p = cs^2 rho */
          pr = p->cs_iso * p->cs_iso * rho;
          gam = 1.0;
        } else {
          double km = 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) +
                      0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
          double eint = cons[4 * ncell + c] - km;
          if (p->dual && dual_use_entropy(p, eint, km))
            pr = cons[5 * ncell + c] * pow(rho, p->gamma - 1.0);
          else
            pr = (p->gamma - 1.0) * eint;
          if (pr < p->p_floor) pr = p->p_floor;
        }
        double w[3];
        orc_widths(&m, i, j, k, w);
        for (int d = 0; d < 3; ++d) {
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          double cf = fast_speed(gam, rho, pr, bc[d], bc[t1], bc[t2]);
          double dtd = w[d] / (fabs(v[d]) + cf);
          if (dtd < dtmin) dtmin = dtd;
        }
      }
  return p->cfl * 1.0 * dtmin;
}

void orc_mhd_diag(const orc_grid* g, const orc_params* p, const double* cons,
                  const double* b1, const double* b2, const double* b3,
                  orc_diag* out) {
  Mesh m;
  memset(out, 0, sizeof *out);
  if (orc_mesh_init(&m, g, 1) != 0) return;
  int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  long ncell = (long)nx * ny * nz;
  double rel = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        double V = orc_volume(&m, i, j, k);
        out->mass += cons[c] * V;
        for (int d = 0; d < 3; ++d) out->mom[d] += cons[(1 + d) * ncell + c] * V;
        out->energy += cons[4 * ncell + c] * V;
        if (!p->mhd) continue;
        double f[6] = {b1[((long)k * ny + j) * (nx + 1) + i],
                       b1[((long)k * ny + j) * (nx + 1) + i + 1],
                       b2[((long)k * (ny + 1) + j) * nx + i],
                       b2[((long)k * (ny + 1) + j + 1) * nx + i],
                       b3[((long)k * ny + j) * nx + i],
                       b3[((long)(k + 1) * ny + j) * nx + i]};
        double a[6] = {orc_area(&m, 0, i, j, k), orc_area(&m, 0, i + 1, j, k),
                       orc_area(&m, 1, i, j, k), orc_area(&m, 1, i, j + 1, k),
                       orc_area(&m, 2, i, j, k), orc_area(&m, 2, i, j, k + 1)};
        double div = a[1] * f[1] - a[0] * f[0] + a[3] * f[3] - a[2] * f[2] +
                     a[5] * f[5] - a[4] * f[4];
        double den = 0.0;
        for (int q = 0; q < 6; ++q) den += a[q] * fabs(f[q]);
        if (den > 0.0 && fabs(div) / den > rel) rel = fabs(div) / den;
      }
  out->max_divb_rel = rel;
}

/* ------------------------------------------------------------------ */
/* L(U) for other integrators (dust.c): the stage above with zero base   */
/* weights and beta*dt = 1 returns exactly the right-hand side of Eq. 8  */
/* (flux divergence plus curvilinear sources) in `out`.                  */
/* ------------------------------------------------------------------ */
long orc_rhs(const Mesh* m, const orc_params* p, int recon, double** u, double** b,
             double** out_u, double** out_b) {
  Work wk;
  if (work_alloc(&wk, m) != 0) return -1;
  long hits = stage(m, p, recon, &wk, u, b, 0.0, u, b, 0.0, NULL, NULL, 1.0, 1.0, out_u,
                    out_b);
  work_free(&wk);
  return hits;
}
