/*
 * FP64 oracle: multifluid dust (paper Sec. 2.2, Eqs. 6-7) with the IMEX2P
 * integrator of Sec. 2.6.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Gas: hydro (B = 0), adiabatic or isothermal, reconstruction + HLLD (= HLLC
 * at B = 0) as in mhd.c.  Dust: N pressureless species, same reconstruction,
 * Rusanov flux with speed max(|v_n,L|, |v_n,R|).  Drag rho_k (v - v_k) / t_k
 * on species k and the opposite reaction on the gas, integrated implicitly;
 * t_k is a constant per species, or rho_k / K_k for the constant-coefficient
 * law.  With the adiabatic closure the drift energy the drag removes becomes
 * gas heat (total energy conserved); the isothermal closure has no energy
 * equation.
 *
 * IMEX2P (reading): the two-stage IMEX pair of Ascher, Ruuth & Spiteri with
 * implicit weight gamma = lambda = 1 + 1/sqrt 2 (stiffly accurate, L-stable)
 * and explicit weights delta = 1 - 1/(2 gamma) >= 0:
 *   U2   = U^n + g dt L(U^n) + g dt R(U2)
 *   U^n+1 = U^n + dt [d L(U^n) + (1-d) L(U2)] + dt [(1-g) R(U2) + g R(U^n+1)]
 * Each implicit stage is one closed-form drag solve with h = g dt.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "oracle_internal.h"

#define IMEX_G (1.0 + 1.0 / 1.4142135623730951)
#define IMEX_D (1.0 - 1.0 / (2.0 * IMEX_G))

/* Implicit drag for one cell and one velocity component: v' = v* + h drag(v').
 * Dust: v_k' = (v_k* + a_k v_g') / (1 + a_k), a_k = h / t_k.
 * Gas:  v_g' = (rho_g v_g* + sum_k rho_k w_k v_k*) / (rho_g + sum_k rho_k w_k),
 *       w_k = a_k / (1 + a_k).  Closed form of the arrowhead system (Sec. 2.2). */
void orc_drag_solve(int nd, double h, double rho_g, const double* rho_d,
                    const double* t_stop, double* v_g, double* v_d) {
  double num = rho_g * (*v_g), den = rho_g;
  for (int k = 0; k < nd; ++k) {
    double a = h / t_stop[k];
    double w = a / (1.0 + a);
    num += rho_d[k] * w * v_d[k];
    den += rho_d[k] * w;
  }
  double vg = num / den;
  for (int k = 0; k < nd; ++k) {
    double a = h / t_stop[k];
    v_d[k] = (v_d[k] + a * vg) / (1.0 + a);
  }
  *v_g = vg;
}

/* Drag solve on every interior cell of (gas u[5], dust d[4 nd]) in place. */
static long drag_cells(const Mesh* m, const orc_dust_params* dp, int iso, double h,
                       double** u, double** d) {
  int nd = dp->nd;
  long hits = 0;
#pragma omp parallel for collapse(2) reduction(+ : hits)
  for (int k = 0; k < m->n[2]; ++k)
    for (int j = 0; j < m->n[1]; ++j)
      for (int i = 0; i < m->n[0]; ++i) {
        long c = IDX(m, i, j, k);
        double rd[32], vd[32], vd0[32], ts[32];
        double rg = u[0][c];
        for (int s = 0; s < nd; ++s) rd[s] = d[4 * s][c];
        /* the drag leaves the densities alone, so t_k = rho_k / K_k of the
         * stage's density holds through the implicit solve */
        for (int s = 0; s < nd; ++s)
          ts[s] = dp->law == ORC_DRAG_COEFF ? rd[s] / dp->t_stop[s] : dp->t_stop[s];
        double ke_before = 0.0, ke_after = 0.0;
        for (int q = 0; q < 3; ++q) {
          double vg = u[1 + q][c] / rg;
          for (int s = 0; s < nd; ++s) {
            vd[s] = rd[s] > 0 ? d[4 * s + 1 + q][c] / rd[s] : 0.0;
            vd0[s] = vd[s];
          }
          orc_drag_solve(nd, h, rg, rd, ts, &vg, vd);
          u[1 + q][c] = rg * vg;
          for (int s = 0; s < nd; ++s) {
            d[4 * s + 1 + q][c] = rd[s] * vd[s];
            ke_before += 0.5 * rd[s] * vd0[s] * vd0[s];
            ke_after += 0.5 * rd[s] * vd[s] * vd[s];
          }
        }
        /* total energy conserved: the dust kinetic energy lost to drag
         * (and the gas kinetic change) is accounted in the gas total E;
         * the isothermal closure carries its energy slot unchanged */
        if (!iso) u[4][c] -= ke_after - ke_before;
        /* dust floor: reset to the floor with zero velocity */
        for (int s = 0; s < nd; ++s)
          if (d[4 * s][c] < dp->rho_floor_dust) {
            d[4 * s][c] = dp->rho_floor_dust;
            d[4 * s + 1][c] = d[4 * s + 2][c] = d[4 * s + 3][c] = 0.0;
            ++hits;
          }
      }
  return hits;
}

/* Explicit right-hand side of the dust species: pressureless Rusanov fluxes
 * (Sec. 2.2) of reconstructed primitives (rho_k, v_k) plus, in spherical
 * coordinates, the pressureless form of the curvilinear sources (Eq. 12). */
static void dust_rhs(const Mesh* m, int recon, const orc_dust_params* dp, double** d,
                     double** rhs) {
  int nd = dp->nd;
  orc_fill_ghosts(m, d, 4 * nd, NULL);
  double *w[4], *f[3][4];
  for (int q = 0; q < 4; ++q) w[q] = (double*)calloc((size_t)m->size, sizeof(double));
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 4; ++q) f[a][q] = (double*)calloc((size_t)m->size, sizeof(double));
  int ng = m->ng;
  for (int s = 0; s < nd; ++s) {
    double** ds = d + 4 * s;
    /* primitives (rho, v) with the dust floor */
    for (int k = -ng; k < m->n[2] + ng; ++k)
      for (int j = -ng; j < m->n[1] + ng; ++j)
        for (int i = -ng; i < m->n[0] + ng; ++i) {
          long c = IDX(m, i, j, k);
          double r = ds[0][c];
          if (r < dp->rho_floor_dust) r = dp->rho_floor_dust;
          w[0][c] = r;
          for (int q = 0; q < 3; ++q) w[1 + q][c] = ds[1 + q][c] / r;
        }
    for (int a = 0; a < 3; ++a) {
#pragma omp parallel for collapse(2)
      for (int k = 0; k <= m->n[2]; ++k)
        for (int j = 0; j <= m->n[1]; ++j)
          for (int i = 0; i <= m->n[0]; ++i) {
            int c3[3] = {i, j, k};
            /* only faces of interior cells along a; others stay unused */
            int ok = 1;
            for (int e = 0; e < 3; ++e)
              if (e != a && c3[e] >= m->n[e]) ok = 0;
            if (!ok) continue;
            long fc = IDX(m, i, j, k);
            double wl[4], wr[4];
            for (int q = 0; q < 4; ++q) {
              double st[6];
              for (int t = 0; t < 6; ++t) {
                int cc[3] = {i, j, k};
                cc[a] = c3[a] - 3 + t;
                st[t] = (cc[a] < -ng || cc[a] >= m->n[a] + ng)
                            ? NAN
                            : w[q][IDX(m, cc[0], cc[1], cc[2])];
              }
              /* same reconstruction as the gas (s[2] | s[3] around the face) */
              double tmpl, tmpr;
              double line[6];
              memcpy(line, st, sizeof line);
              {
                /* reuse the line reconstruction on the 6-point stencil */
                double wl6[5], wr6[5];
                orc_recon_line(recon, 6, line, wl6, wr6);
                tmpl = wl6[2];
                tmpr = wr6[2];
              }
              wl[q] = tmpl;
              wr[q] = tmpr;
            }
            double vnl = wl[1 + a], vnr = wr[1 + a];
            double sp = fabs(vnl) > fabs(vnr) ? fabs(vnl) : fabs(vnr);
            double ul[4] = {wl[0], wl[0] * wl[1], wl[0] * wl[2], wl[0] * wl[3]};
            double ur[4] = {wr[0], wr[0] * wr[1], wr[0] * wr[2], wr[0] * wr[3]};
            for (int q = 0; q < 4; ++q) {
              double fl = ul[q] * vnl, fr = ur[q] * vnr;
              f[a][q][fc] = 0.5 * (fl + fr) - 0.5 * sp * (ur[q] - ul[q]);
            }
          }
    }
    /* divergence and curvilinear sources */
#pragma omp parallel for collapse(2)
    for (int k = 0; k < m->n[2]; ++k)
      for (int j = 0; j < m->n[1]; ++j)
        for (int i = 0; i < m->n[0]; ++i) {
          long c = IDX(m, i, j, k);
          long cp[3] = {IDX(m, i + 1, j, k), IDX(m, i, j + 1, k), IDX(m, i, j, k + 1)};
          double V = orc_volume(m, i, j, k);
          double Am[3] = {orc_area(m, 0, i, j, k), orc_area(m, 1, i, j, k),
                          orc_area(m, 2, i, j, k)};
          double Ap[3] = {orc_area(m, 0, i + 1, j, k), orc_area(m, 1, i, j + 1, k),
                          orc_area(m, 2, i, j, k + 1)};
          double src[4] = {0, 0, 0, 0};
          if (m->coord == ORC_SPH) {
            double r = w[0][c], v[3] = {w[1][c], w[2][c], w[3][c]};
            double inv_r = (Ap[0] - Am[0]) / (2.0 * V);
            double cot_r = (Ap[1] - Am[1]) / V;
            double T11 = r * v[1] * v[1], T22 = r * v[2] * v[2];
            double T01 = r * v[0] * v[1], T20 = r * v[2] * v[0], T21 = r * v[2] * v[1];
            src[1] = (T11 + T22) * inv_r;
            src[2] = T22 * cot_r - T01 * inv_r;
            src[3] = -T20 * inv_r - T21 * cot_r;
          }
          for (int q = 0; q < 4; ++q) {
            double div = 0.0;
            for (int a = 0; a < 3; ++a) div += Ap[a] * f[a][q][cp[a]] - Am[a] * f[a][q][c];
            rhs[4 * s + q][c] = -div / V + src[q];
          }
        }
  }
  for (int q = 0; q < 4; ++q) free(w[q]);
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 4; ++q) free(f[a][q]);
}

/* L(U) for gas and dust, with the optional uniform gas acceleration g
 * (momentum source rho g, energy source M . g). */
static long full_rhs(const Mesh* m, const orc_params* p, const orc_dust_params* dp, double** u,
                     double** d, double** lu, double** ld) {
  long hits = orc_rhs(m, p, p->recon, u, NULL, lu, NULL);
  dust_rhs(m, p->recon, dp, d, ld);
  const double* g = dp->gas_accel;
  if (g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0) {
    for (int k = 0; k < m->n[2]; ++k)
      for (int j = 0; j < m->n[1]; ++j)
        for (int i = 0; i < m->n[0]; ++i) {
          long c = IDX(m, i, j, k);
          for (int q = 0; q < 3; ++q) lu[1 + q][c] += u[0][c] * g[q];
          lu[4][c] += u[1][c] * g[0] + u[2][c] * g[1] + u[3][c] * g[2];
        }
  }
  return hits;
}

static void load_dust(const Mesh* m, int nd, const double* dust, double** d) {
  int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  long nc = (long)nx * ny * nz;
  for (int a = 0; a < 4 * nd; ++a)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          d[a][IDX(m, i, j, k)] = dust[a * nc + ((long)k * ny + j) * nx + i];
}

static void store_dust(const Mesh* m, int nd, double** d, double* dust) {
  int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  long nc = (long)nx * ny * nz;
  for (int a = 0; a < 4 * nd; ++a)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          dust[a * nc + ((long)k * ny + j) * nx + i] = d[a][IDX(m, i, j, k)];
}

int orc_dust_step(const orc_grid* g, const orc_params* p, const orc_dust_params* dp,
                  double dt, double* cons, double* dust, long* floor_hits) {
  if (p->mhd || dp->nd < 0 || dp->nd > 32) return -1;
  if (dp->law != ORC_DRAG_TSTOP && dp->law != ORC_DRAG_COEFF) return -1;
  Mesh m;
  if (orc_mesh_init(&m, g, orc_ghost_width(p->recon)) != 0) return -1;
  int nd = dp->nd, nv = 4 * nd;
  double *U[5], *X[5], *A[5], *Lu[5];
  double *D[128], *XD[128], *AD[128], *LD[128];
  for (int v = 0; v < 5; ++v) {
    U[v] = calloc((size_t)m.size, sizeof(double));
    X[v] = calloc((size_t)m.size, sizeof(double));
    A[v] = calloc((size_t)m.size, sizeof(double));
    Lu[v] = calloc((size_t)m.size, sizeof(double));
  }
  for (int v = 0; v < nv; ++v) {
    D[v] = calloc((size_t)m.size, sizeof(double));
    XD[v] = calloc((size_t)m.size, sizeof(double));
    AD[v] = calloc((size_t)m.size, sizeof(double));
    LD[v] = calloc((size_t)m.size, sizeof(double));
  }
  orc_load(&m, cons, NULL, NULL, NULL, U, 5, NULL);
  load_dust(&m, nd, dust, D);
  const double gI = IMEX_G, dE = IMEX_D, h = IMEX_G * dt;
  long hits = 0;

  /* stage 2: X = U^n + g dt L(U^n); A = U^n + d dt L(U^n); U2 = drag(X) */
  hits += full_rhs(&m, p, dp, U, D, Lu, LD);
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        long c = IDX(&m, i, j, k);
        for (int v = 0; v < 5; ++v) {
          X[v][c] = U[v][c] + gI * dt * Lu[v][c];
          A[v][c] = U[v][c] + dE * dt * Lu[v][c];
        }
        for (int v = 0; v < nv; ++v) {
          XD[v][c] = D[v][c] + gI * dt * LD[v][c];
          AD[v][c] = D[v][c] + dE * dt * LD[v][c];
        }
      }
  /* U2 = drag(X) stored in U/D; dt R(U2) = (U2 - X) / g */
  for (int v = 0; v < 5; ++v) memcpy(U[v], X[v], (size_t)m.size * sizeof(double));
  for (int v = 0; v < nv; ++v) memcpy(D[v], XD[v], (size_t)m.size * sizeof(double));
  hits += drag_cells(&m, dp, p->iso, h, U, D);
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        long c = IDX(&m, i, j, k);
        for (int v = 0; v < 5; ++v) A[v][c] += (1.0 - gI) * (U[v][c] - X[v][c]) / gI;
        for (int v = 0; v < nv; ++v) AD[v][c] += (1.0 - gI) * (D[v][c] - XD[v][c]) / gI;
      }

  /* stage 3: Y = A + (1 - d) dt L(U2); U^n+1 = drag(Y) */
  hits += full_rhs(&m, p, dp, U, D, Lu, LD);
  for (int k = 0; k < m.n[2]; ++k)
    for (int j = 0; j < m.n[1]; ++j)
      for (int i = 0; i < m.n[0]; ++i) {
        long c = IDX(&m, i, j, k);
        for (int v = 0; v < 5; ++v) U[v][c] = A[v][c] + (1.0 - dE) * dt * Lu[v][c];
        for (int v = 0; v < nv; ++v) D[v][c] = AD[v][c] + (1.0 - dE) * dt * LD[v][c];
      }
  hits += drag_cells(&m, dp, p->iso, h, U, D);

  orc_store(&m, U, 5, NULL, cons, NULL, NULL, NULL);
  store_dust(&m, nd, D, dust);
  if (floor_hits) *floor_hits = hits;
  for (int v = 0; v < 5; ++v) { free(U[v]); free(X[v]); free(A[v]); free(Lu[v]); }
  for (int v = 0; v < nv; ++v) { free(D[v]); free(XD[v]); free(AD[v]); free(LD[v]); }
  return 0;
}

/* Eq. 11 with Cmax = 1/lambda (IMEX2P); gas sound speed, dust c = 0. */
double orc_dust_dt(const orc_grid* g, const orc_params* p, const orc_dust_params* dp,
                   const double* cons, const double* dust) {
  Mesh m;
  if (orc_mesh_init(&m, g, 1) != 0) return NAN;
  int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  long nc = (long)nx * ny * nz;
  double dtmin = INFINITY;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long c = ((long)k * ny + j) * nx + i;
        double rho = cons[c];
        if (rho < p->rho_floor) rho = p->rho_floor;
        double v[3] = {cons[nc + c] / rho, cons[2 * nc + c] / rho, cons[3 * nc + c] / rho};
        double cs;
        if (p->iso) {
          cs = p->cs_iso;
        } else {
          double pr = (p->gamma - 1.0) *
                      (cons[4 * nc + c] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
          if (pr < p->p_floor) pr = p->p_floor;
          cs = sqrt(p->gamma * pr / rho);
        }
        double w[3];
        orc_widths(&m, i, j, k, w);
        for (int d = 0; d < 3; ++d) {
          double t = w[d] / (fabs(v[d]) + cs);
          if (t < dtmin) dtmin = t;
        }
        for (int s = 0; s < dp->nd; ++s) {
          double r = dust[(4 * s) * nc + c];
          if (!(r > 0)) continue;
          for (int d = 0; d < 3; ++d) {
            double vk = fabs(dust[(4 * s + 1 + d) * nc + c] / r);
            if (vk > 0 && w[d] / vk < dtmin) dtmin = w[d] / vk;
          }
        }
      }
  return p->cfl * (1.0 / IMEX_G) * dtmin;
}
