/*
 * FP64 CPU oracle for the finite-volume MHD step of the Aether.jl paper
 * (arXiv 2608.14048).  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark call this code; the CUDA
 * library never links, includes or calls it, and it shares no header, helper
 * or constant with the CUDA path.
 *
 * Everything here is plain double-precision loops over explicitly ghosted
 * arrays, one operation per pass, in the order the paper states them:
 *   ghost fill (Sec. 2.3) -> conserved->primitive (Sec. 2.1, Eq. 5, floors)
 *   -> per-direction reconstruction + face-frame Riemann solve (Sec. 2.4)
 *   -> upwinded corner EMFs and constrained transport (Sec. 2.5, Eq. 9)
 *   -> finite-volume update (Eq. 8) + curvilinear sources (Eq. 12)
 *   -> two-stage integrator (Sec. 2.6, Eq. 10) ; CFL step (Eq. 11).
 * Dust (Sec. 2.2, Eqs. 6-7) and the IMEX2P integrator (Sec. 2.6) live in
 * dust.c; the learned-flux MLP reference lives in mlp.c.
 *
 * Array conventions (caller-owned, row-major, i fastest):
 *   cons[5][nz][ny][nx]  : rho, M1, M2, M3, E
 *   b1[nz][ny][nx+1], b2[nz][ny+1][nx], b3[nz+1][ny][nx] : face-averaged
 *   normal field.  In a periodic direction the last face equals the first.
 */
#ifndef AETHER_ORACLE_H
#define AETHER_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CART = 0, ORC_SPH = 1 };
enum { ORC_PERIODIC = 0, ORC_OUTFLOW = 1 };
enum { ORC_DONOR = 0, ORC_PLM = 1, ORC_PPM = 2, ORC_PPM5 = 3 };
enum { ORC_VL2 = 0, ORC_RK2 = 1, ORC_RK3 = 2 };
enum { ORC_HLLD = 0, ORC_HLLE = 1, ORC_LHLLD = 2 };

typedef struct {
  int nx, ny, nz;     /* interior cells along x1, x2, x3 */
  int coord;          /* ORC_CART or ORC_SPH (r, theta, phi) */
  double lo[3], hi[3];
  int bc[3];          /* per axis: ORC_PERIODIC or ORC_OUTFLOW (both sides) */
} orc_grid;

typedef struct {
  double gamma;
  double rho_floor, p_floor;
  int recon;          /* reconstruction of the final (or only) stage */
  int integrator;     /* ORC_VL2, ORC_RK2 or ORC_RK3 */
  double cfl;         /* Courant factor C of Eq. 11 */
  int mhd;            /* 1: MHD; 0: hydro (face arrays ignored, B = 0) */
  int riemann;        /* ORC_HLLD (Sec. 2.4 default), ORC_HLLE or ORC_LHLLD */
  int iso;            /* 1: isothermal closure p = cs_iso^2 rho (Sec. 2.1): no
                         energy equation (the energy slot is carried, unused) */
  double cs_iso;      /* isothermal sound speed */
  int dual;           /* 1: dual-energy formalism (Sec. 2.8): the state carries a
                         sixth cell variable S = p / rho^(gamma-1) */
  double alpha_switch, alpha_sync;  /* its thresholds (1e-3, 1e-1 by default) */
} orc_params;

typedef struct {
  double mass, mom[3], energy;  /* volume integrals over the interior */
  double max_divb_rel;          /* max |sum_f +-A_f B_f| / sum_f A_f |B_f| */
  long floor_hits;              /* cells where a floor was applied */
} orc_diag;

/* Dual-energy formalism (Sec. 2.8): the entropy S = p / rho^(gamma-1) of
 * every interior cell from its conserved state (cons[5] of a 6-variable
 * state; p from E with the floors of the cons->prim conversion). */
void orc_dual_init(const orc_grid* g, const orc_params* p, double* cons, const double* b1,
                   const double* b2, const double* b3);

/* One full step of length dt (both stages), in place.  Returns 0 on
 * success, a negative value on bad arguments. */
int orc_mhd_step(const orc_grid* g, const orc_params* p, double dt,
                 double* cons, double* b1, double* b2, double* b3,
                 long* floor_hits);

/* Eq. 11: C * Cmax * min over cells and directions of dx_d/(|v_d|+c_d);
 * Cmax = 1 for VL2 and RK2. */
double orc_mhd_dt(const orc_grid* g, const orc_params* p, const double* cons,
                  const double* b1, const double* b2, const double* b3);

void orc_mhd_diag(const orc_grid* g, const orc_params* p, const double* cons,
                  const double* b1, const double* b2, const double* b3,
                  orc_diag* out);

/* Single-face HLLD flux (Miyoshi & Kusano 2005) in the face frame.
 * wl, wr: (rho, vn, vt1, vt2, p, Bt1, Bt2); bn: normal field (both sides).
 * flux: (rho, Mn, Mt1, Mt2, E, Bt1, Bt2).  Returns the region index
 * 0..5 (L, *L, **L, **R, *R, R) that supplied the flux. */
int orc_hlld(double gamma, const double* wl, const double* wr, double bn,
             double* flux);

/* Single-face low-dissipation HLLD (LHLLD; Sec. 2.4 after Minoshima &
 * Miyoshi 2021, as read here): the HLLD flux with the pressure dissipation
 * at the contact scaled by the local Mach number.  HLLD's star total
 * pressure is p_T* = pbar + D, pbar the average of p_TL and p_TR weighted
 * by rho_a (S_a - u_a), and D = rho_L rho_R (S_R - u_R)(S_L - u_L)(u_R - u_L)
 * / den the term that grows with the sound speed.  Inside the fan the
 * normal-momentum flux carries D and the energy flux S_M D; LHLLD replaces
 * them with phi D and phi S_M D, phi = min(1, max(|v_L|, |v_R|) /
 * max(c_f,L, c_f,R)).  phi = 1 (local Mach >= 1) gives HLLD exactly; with
 * B = 0 it is the low-dissipation HLLC (LHLLC).  Returns the region. */
int orc_lhlld(double gamma, const double* wl, const double* wr, double bn, double* flux);

/* Single-face HLLE flux (Harten, Lax & van Leer 1983; Einfeldt 1988;
 * Sec. 2.4), same frames as orc_hlld: the flux of the single averaged state
 * of the HLL fan between the outer wave-speed estimates
 *   S_L = min(vn_L, vn_R) - max(c_f,L, c_f,R),
 *   S_R = max(vn_L, vn_R) + max(c_f,L, c_f,R)
 * (the estimates the HLLD solver uses), with b- = min(S_L, 0) and
 * b+ = max(S_R, 0) so that a supersonic face takes the upwind flux. */
void orc_hlle(double gamma, const double* wl, const double* wr, double bn, double* flux);

/* Isothermal solvers (p = cs^2 rho; Sec. 2.1, 2.4), same frames with the
 * pressure slot of w unused and a zero energy flux.
 * orc_hlld_iso: the isothermal HLLD of Mignone (2007): density and normal
 * momentum are uniform inside the fan (no contact wave), with the HLL
 * fluxes there; rho* = the HLL average and u* = F_rho^HLL / rho*; outer
 * transverse states across the fast waves, a central state between the
 * Alfven waves S*_L,R = u* -+ |Bn|/sqrt(rho*).
 * orc_hlle_iso: HLLE with the same outer speeds. */
void orc_hlld_iso(double cs, const double* wl, const double* wr, double bn, double* flux);
void orc_hlle_iso(double cs, const double* wl, const double* wr, double bn, double* flux);

/* Reconstruction of one 1-D line: w[0..n-1] -> left/right states at the
 * n-1 interior faces (face f lies between cells f and f+1; faces whose
 * stencil leaves the line are set to NaN). */
void orc_recon_line(int recon, int n, const double* w, double* wl, double* wr);

/* Corner EMF of the upwind scheme of Gardiner & Stone (2005) at one edge,
 * exposed for unit tests.  ea_m, ea_p: a-face EMFs at rows b-1, b;
 * eb_m, eb_p: b-face EMFs at columns a-1, a; eref[2][2] indexed
 * [row b-1 / b][column a-1 / a]; fa_m, fa_p: a-face mass fluxes at rows
 * b-1, b; fb_m, fb_p: b-face mass fluxes at columns a-1, a. */
double orc_corner_emf(double ea_m, double ea_p, double eb_m, double eb_p,
                      const double* eref, double fa_m, double fa_p,
                      double fb_m, double fb_p);

/* ---- multifluid dust (dust.c) ---------------------------------------- */
enum { ORC_DRAG_TSTOP = 0, ORC_DRAG_COEFF = 1 };

typedef struct {
  int nd;                 /* number of dust species N */
  const double* t_stop;   /* [nd] ORC_DRAG_TSTOP: constant stopping times t_k;
                             ORC_DRAG_COEFF: drag coefficients K_k */
  double rho_floor_dust;
  double gas_accel[3];    /* uniform external acceleration on the gas only
                             (explicit term; used by the forced-relaxation
                             test, zero otherwise) */
  int law;                /* drag law (Sec. 2.2): constant stopping time, or
                             constant coefficient, t_k = rho_k / K_k */
} orc_dust_params;

/* Closed-form implicit drag solve of one cell and one velocity component
 * (Sec. 2.2): given weight h, gas (rho_g, v_g*) and dust (rho_k, v_k*),
 * returns the v' solving v' = v* + h * drag(v'). */
void orc_drag_solve(int nd, double h, double rho_g, const double* rho_d,
                    const double* t_stop, double* v_g, double* v_d);

/* One IMEX2P step of hydro gas (adiabatic, or isothermal with p->iso) + nd
 * pressureless dust species.  dust[nd][4][nz][ny][nx] holds (rho_k, M1_k,
 * M2_k, M3_k). */
int orc_dust_step(const orc_grid* g, const orc_params* p,
                  const orc_dust_params* dp, double dt, double* cons,
                  double* dust, long* floor_hits);

double orc_dust_dt(const orc_grid* g, const orc_params* p,
                   const orc_dust_params* dp, const double* cons,
                   const double* dust);

/* ---- learned-flux MLP reference (mlp.c) ----------------------------- */
/* Dense MLP with SiLU hidden activations and a linear output layer.
 * dims[0..nl] are layer widths; params packs, per layer l, W_l[out][in]
 * followed by b_l[out]. */
void orc_mlp_forward(int nl, const int* dims, const double* params, int n,
                     const double* x, double* y);
/* Gradient of 0.5/n * sum |y - target|^2 w.r.t. params; returns the loss. */
double orc_mlp_grad(int nl, const int* dims, const double* params, int n,
                    const double* x, const double* target, double* grad);

/* ---- learned face flux (learned.c; no counterpart in the paper) ------ */
/* The learned flux of one face in the face frame of orc_hlld, with the
 * 14-128-128-128-7 network params (FP64, packed as for orc_mlp_forward):
 * features, network, F = F_E + k J y, acceptance (tau: the fraction of the
 * HLL dissipation bracket; positivity of the implied HLL-fan states), HLLD
 * fallback; mhd = 0: hydro face (no induction fluxes).  Returns 1 where the
 * network's flux is accepted, 0 where HLLD replaced it.  info (24 doubles,
 * may be NULL): [0..6] the candidate F, [7] J, [8..14] k, [15] the
 * bracket margin and [16] the positivity margin, both in units of the
 * network output and positive where the check passes (the decision can
 * only flip under a change of y larger than min(info[15], info[16]) in
 * magnitude), [17..23] the network output y.  The batch form takes n
 * faces (wl, wr [n][7], bn [n]) and 24 info doubles per face. */
int orc_learned_flux(double gamma, const double* wl, const double* wr, double bn,
                     const double* params, double tau, int mhd, double* flux, double* info);
void orc_learned_flux_batch(double gamma, int n, const double* wl, const double* wr,
                            const double* bn, const double* params, double tau, int mhd,
                            double* flux, int* accepted, double* info);
/* The network's training target of one face: y = (F_HLLD - F_E) / (k J),
 * zero where J <= 1e-9. */
void orc_learned_target(double gamma, const double* wl, const double* wr, double bn, double* y);
/* The features x[14] and flux scales k[7] of one face. */
void orc_learned_features(double gamma, const double* wl, const double* wr, double bn,
                          double* x, double* k);

#ifdef __cplusplus
}
#endif
#endif
