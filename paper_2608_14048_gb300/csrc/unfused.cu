// Unfused stage: one kernel per operation of Sec. 2.4-2.6 with intermediate
// arrays in HBM (primitives, face fluxes, face and corner EMFs).  This path
// keeps every intermediate inspectable; the fused path (fused.cu) computes
// the same quantities per tile in shared memory.
#include "runtime.hpp"

namespace aeth {

template <typename R>
void launch_fill(const BlockPtrs<R>& P, R* const* arrs, int nv, cudaStream_t st);

// ------------------------------------------------------------------------
// conserved -> primitive over cells -g..n+g-1 (Eq. 5, floors of Sec. 2.1)
// ------------------------------------------------------------------------
template <typename R, bool P64>
__global__ void k_prim(Layout L, ConstArr8<R> u, Arr8<R> w, int mhd, double gamma,
                       R rho_floor, R p_floor, double cs2, unsigned long long* floor_hits) {
  const int g = L.g;
  const int i = blockIdx.x * blockDim.x + threadIdx.x - g;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - g;
  const int k = blockIdx.z * blockDim.z + threadIdx.z - g;
  if (i >= L.n[0] + g || j >= L.n[1] + g || k >= L.n[2] + g) return;
  const long long c = L.idx(i, j, k);
  int hits = 0;
  R rho = u.p[0][c];
  if (rho < rho_floor) { rho = rho_floor; ++hits; }
  const R v1 = u.p[1][c] / rho, v2 = u.p[2][c] / rho, v3 = u.p[3][c] / rho;
  R b1 = 0, b2 = 0, b3 = 0;
  if (mhd) {
    b1 = R(0.5) * (u.p[5][c] + u.p[5][c + 1]);
    b2 = R(0.5) * (u.p[6][c] + u.p[6][c + L.sx]);
    b3 = R(0.5) * (u.p[7][c] + u.p[7][c + L.sx * L.sy]);
  }
  R pr;
  if (cs2 > 0.0) {
    pr = (R)cs2 * rho;   // isothermal closure: no energy, no pressure floor
  } else if (P64) {
    // FP64 subtraction in every cell, or only where the FP32 one cancels
    bool wide = true;
    if (L.p64_ratio > 0.0f) {
      const R ke = R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3);
      const R me = R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3);
      const R ei = u.p[4][c] - ke - me;
      wide = ke + me > (R)L.p64_ratio * ei;
      pr = (R)(gamma - 1.0) * ei;
    }
    if (wide) {
      const double r = rho;
      const double ke = 0.5 * r * ((double)v1 * v1 + (double)v2 * v2 + (double)v3 * v3);
      const double me = 0.5 * ((double)b1 * b1 + (double)b2 * b2 + (double)b3 * b3);
      pr = (R)((gamma - 1.0) * ((double)u.p[4][c] - ke - me));
    }
  } else {
    const R ke = R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3);
    const R me = R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3);
    pr = (R)(gamma - 1.0) * (u.p[4][c] - ke - me);
  }
  if (cs2 <= 0.0 && pr < p_floor) { pr = p_floor; ++hits; }
  w.p[0][c] = rho; w.p[1][c] = v1; w.p[2][c] = v2; w.p[3][c] = v3;
  w.p[4][c] = pr; w.p[5][c] = b1; w.p[6][c] = b2; w.p[7][c] = b3;
  if (hits) atomicAdd(floor_hits, (unsigned long long)hits);
}

// ------------------------------------------------------------------------
// per-direction face fluxes: faces 0..n along d, one ring across
// ------------------------------------------------------------------------
template <typename R, int RECON>
__global__ void k_flux(Layout L, ConstArr8<R> w, const R* __restrict__ bface, int d, int mhd,
                       int solver, R gamma, R* f0, R* f1, R* f2, R* f3, R* f4, R* e0, R* e1) {
  int c[3];
  c[0] = blockIdx.x * blockDim.x + threadIdx.x;
  c[1] = blockIdx.y * blockDim.y + threadIdx.y;
  c[2] = blockIdx.z * blockDim.z + threadIdx.z;
  for (int e = 0; e < 3; ++e) {
    if (e != d) c[e] -= 1;
    const int hi = L.n[e];
    if (c[e] > hi) return;
  }
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const long long fc = L.idx(c[0], c[1], c[2]);
  const long long sd = L.stride(d);
  const int slot[7] = {0, 1 + d, 1 + t1, 1 + t2, 4, 5 + t1, 5 + t2};
  const int nq = mhd ? 7 : 5;
  R wl[7], wr[7];
  for (int q = 0; q < 7; ++q) {
    if (q >= nq) { wl[q] = wr[q] = R(0); continue; }
    const R* a = w.p[slot[q]];
    R s[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int off = t - 3;
      const bool need = RECON >= 2 || (RECON == 1 && t >= 1 && t <= 4) || (RECON == 0 && (t == 2 || t == 3));
      s[t] = need ? a[fc + off * sd] : R(0);
    }
    recon_face<RECON>(s, wl[q], wr[q]);
  }
  const R bn = mhd ? bface[fc] : R(0);
  R fx[7];
  // solver: AETH_RIEMANN_HLLD / _HLLE / _LHLLD, or SOLVER_ISO_HLLD / _HLLE with
  // `gamma` holding the isothermal sound speed
  if (solver == AETH_RIEMANN_HLLE) hlle(gamma, wl, wr, bn, fx);
  else if (solver == SOLVER_ISO_HLLD) hlld_iso(gamma, wl, wr, bn, fx);
  else if (solver == SOLVER_ISO_HLLE) hlle_iso(gamma, wl, wr, bn, fx);
  else if (solver == AETH_RIEMANN_LHLLD) hlld<true>(gamma, wl, wr, bn, fx);
  else hlld(gamma, wl, wr, bn, fx);
  R* fo[5] = {f0, f1, f2, f3, f4};
  fo[0][fc] = fx[0];
  fo[1 + d][fc] = fx[1];
  fo[1 + t1][fc] = fx[2];
  fo[1 + t2][fc] = fx[3];
  fo[4][fc] = fx[4];
  if (mhd) {
    e0[fc] = fx[6];    // E_t1 =  F(B_t2)
    e1[fc] = -fx[5];   // E_t2 = -F(B_t1)
  }
}

// ------------------------------------------------------------------------
// corner EMFs (Sec. 2.5): edges along c at the lower corner of (i,j,k)
// ------------------------------------------------------------------------
template <typename R>
struct EmfArgs {
  const R* w[NPRIM];
  const R* f0[3];      // mass flux per direction
  const R* e[3][2];    // face EMFs per direction
  R* edge[3];
};

template <typename R>
__global__ void k_emf(Layout L, EmfArgs<R> A) {
  int P[3];
  P[0] = blockIdx.x * blockDim.x + threadIdx.x;
  P[1] = blockIdx.y * blockDim.y + threadIdx.y;
  P[2] = blockIdx.z * blockDim.z + threadIdx.z;
  if (P[0] > L.n[0] || P[1] > L.n[1] || P[2] > L.n[2]) return;
  const long long iP = L.idx(P[0], P[1], P[2]);
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    if (P[cc] >= L.n[cc]) continue;
    const int a = (cc + 1) % 3, b = (cc + 2) % 3;
    const long long sa = L.stride(a), sb = L.stride(b);
    const long long iA = iP - sa, iB = iP - sb, iAB = iP - sa - sb;
    auto eref = [&](long long x) {
      return -(A.w[1 + a][x] * A.w[5 + b][x] - A.w[1 + b][x] * A.w[5 + a][x]);
    };
    const R r00 = eref(iAB), r01 = eref(iB), r10 = eref(iA), r11 = eref(iP);
    A.edge[cc][iP] = corner_emf(A.e[a][1][iB], A.e[a][1][iP], A.e[b][0][iA], A.e[b][0][iP],
                                r00, r01, r10, r11, A.f0[a][iB], A.f0[a][iP],
                                A.f0[b][iA], A.f0[b][iP]);
  }
}

// ------------------------------------------------------------------------
// update: out = w0*A + w1*B + beta*dt*L  (Eq. 8 + Eq. 12; CT of Eq. 9)
// ------------------------------------------------------------------------
template <typename R>
struct UpdArgs {
  const R* a[NVAR];
  const R* b[NVAR];
  R* out[NVAR];
  const R* f[3][5];
  const R* edge[3];
  const R* w[NPRIM];
  R w0, w1, beta;
  const double* dt;
};

template <typename R>
__global__ void k_update(Layout L, Geometry<R> geo, UpdArgs<R> A, int mhd) {
  int P[3];
  P[0] = blockIdx.x * blockDim.x + threadIdx.x;
  P[1] = blockIdx.y * blockDim.y + threadIdx.y;
  P[2] = blockIdx.z * blockDim.z + threadIdx.z;
  if (P[0] > L.n[0] || P[1] > L.n[1] || P[2] > L.n[2]) return;
  const int i = P[0], j = P[1], k = P[2];
  const long long c = L.idx(i, j, k);
  const R dt = (R)(*A.dt);
  const R bdt = A.beta * dt;
  if (i < L.n[0] && j < L.n[1] && k < L.n[2]) {
    const long long cp[3] = {c + 1, c + L.sx, c + L.sx * L.sy};
    const R V = geo.vol(i, j, k);
    const R Am[3] = {geo.area[0](i, j, k), geo.area[1](i, j, k), geo.area[2](i, j, k)};
    const R Ap[3] = {geo.area[0](i + 1, j, k), geo.area[1](i, j + 1, k), geo.area[2](i, j, k + 1)};
    R src[5] = {0, 0, 0, 0, 0};
    if (L.coord == AETH_COORD_SPH) {
      // curvilinear momentum sources from the stress tensor (Eq. 12)
      const R rho = A.w[0][c], v[3] = {A.w[1][c], A.w[2][c], A.w[3][c]};
      R bb[3] = {0, 0, 0};
      if (mhd) { bb[0] = A.w[5][c]; bb[1] = A.w[6][c]; bb[2] = A.w[7][c]; }
      const R ps = A.w[4][c] + R(0.5) * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
      auto T = [&](int x, int y) { return rho * v[x] * v[y] + (x == y ? ps : R(0)) - bb[x] * bb[y]; };
      const R ir = geo.invr(i, j, k), ct = geo.cotr(i, j, k);
      src[1] = (T(1, 1) + T(2, 2)) * ir;
      src[2] = T(2, 2) * ct - T(0, 1) * ir;
      src[3] = -T(2, 0) * ir - T(2, 1) * ct;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R div = R(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) div += Ap[d] * A.f[d][v][cp[d]] - Am[d] * A.f[d][v][c];
      const R rhs = -div / V + src[v];
      R base = A.w0 * A.a[v][c];
      if (A.w1 != R(0)) base += A.w1 * A.b[v][c];
      A.out[v][c] = base + bdt * rhs;
    }
  }
  if (!mhd) return;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    const int hid = L.bc[d] == AETH_BC_OUTFLOW ? L.n[d] : L.n[d] - 1;
    if (P[d] > hid || P[e1] >= L.n[e1] || P[e2] >= L.n[e2]) continue;
    int Q1[3] = {i, j, k}, Q2[3] = {i, j, k};
    Q1[e1] += 1; Q2[e2] += 1;
    const long long q1 = c + L.stride(e1), q2 = c + L.stride(e2);
    const R circ = A.edge[e2][q1] * geo.edge[e2](Q1[0], Q1[1], Q1[2]) -
                   A.edge[e2][c] * geo.edge[e2](i, j, k) -
                   (A.edge[e1][q2] * geo.edge[e1](Q2[0], Q2[1], Q2[2]) -
                    A.edge[e1][c] * geo.edge[e1](i, j, k));
    const R Af = geo.area[d](i, j, k);
    R base = A.w0 * A.a[5 + d][c];
    if (A.w1 != R(0)) base += A.w1 * A.b[5 + d][c];
    const R nb = base - bdt * circ / Af;
    A.out[5 + d][c] = nb;
    // periodic axis: face n is the image of face 0; keep it current so
    // every reader (CFL, diagnostics) sees a consistent field
    if (L.bc[d] == AETH_BC_PERIODIC && P[d] == 0) A.out[5 + d][c + (long long)L.n[d] * L.stride(d)] = nb;
  }
}

// ------------------------------------------------------------------------
// one stage on one block
// ------------------------------------------------------------------------
template <typename R, bool P64>
static void stage_unfused(aeth_ctx* c, const BlockPtrs<R>& P, int recon, int src, R w0,
                          int has_b, R w1, R beta, int out) {
  const Layout& L = P.L;
  const int mhd = is_mhd(c);
  const int nv = mhd ? NVAR : 5;
  cudaStream_t st = c->stream;
  launch_fill<R>(P, P.reg[src], nv, st);

  ConstArr8<R> u{}, w{};
  Arr8<R> wo{};
  for (int v = 0; v < NVAR; ++v) { u.p[v] = P.reg[src][v]; w.p[v] = P.w[v]; wo.p[v] = P.w[v]; }
  const int g = L.g;
  dim3 blk(32, 4, 2);
  const bool iso = is_iso(c);
  const double cs2 = iso ? c->cfg.cs_iso * c->cfg.cs_iso : 0.0;
  const int solver = !iso ? c->cfg.riemann
                          : (c->cfg.riemann == AETH_RIEMANN_HLLE ? SOLVER_ISO_HLLE : SOLVER_ISO_HLLD);
  {
    const int ex = L.n[0] + 2 * g, ey = L.n[1] + 2 * g, ez = L.n[2] + 2 * g;
    dim3 grd((ex + 31) / 32, (ey + 3) / 4, (ez + 1) / 2);
    k_prim<R, P64><<<grd, blk, 0, st>>>(L, u, wo, mhd, c->cfg.gamma, (R)c->cfg.rho_floor,
                                        (R)c->cfg.p_floor, cs2, c->d_floor);
  }
  for (int d = 0; d < 3; ++d) {
    int ext[3];
    for (int e = 0; e < 3; ++e) ext[e] = e == d ? L.n[e] + 1 : L.n[e] + 2;
    dim3 grd((ext[0] + 31) / 32, (ext[1] + 3) / 4, (ext[2] + 1) / 2);
    const R* bf = P.reg[src][5 + d];
    R gm = (R)(iso ? c->cfg.cs_iso : c->cfg.gamma);
    // algorithmic traffic: 7 primitives read and 7 outputs written per face
    const double faces = (double)ext[0] * ext[1] * ext[2];
    prof_begin(c);
    if (recon == AETH_RECON_DONOR)
      k_flux<R, 0><<<grd, blk, 0, st>>>(L, w, bf, d, mhd, solver, gm, P.f[d][0], P.f[d][1], P.f[d][2],
                                        P.f[d][3], P.f[d][4], P.e[d][0], P.e[d][1]);
    else if (recon == AETH_RECON_PLM)
      k_flux<R, 1><<<grd, blk, 0, st>>>(L, w, bf, d, mhd, solver, gm, P.f[d][0], P.f[d][1], P.f[d][2],
                                        P.f[d][3], P.f[d][4], P.e[d][0], P.e[d][1]);
    else if (recon == AETH_RECON_PPM5)
      k_flux<R, 3><<<grd, blk, 0, st>>>(L, w, bf, d, mhd, solver, gm, P.f[d][0], P.f[d][1], P.f[d][2],
                                        P.f[d][3], P.f[d][4], P.e[d][0], P.e[d][1]);
    else
      k_flux<R, 2><<<grd, blk, 0, st>>>(L, w, bf, d, mhd, solver, gm, P.f[d][0], P.f[d][1], P.f[d][2],
                                        P.f[d][3], P.f[d][4], P.e[d][0], P.e[d][1]);
    prof_end(c, faces * (mhd ? 15 : 10) * sizeof(R));
  }
  dim3 grd((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 3) / 4, (L.n[2] + 1 + 1) / 2);
  if (mhd) {
    EmfArgs<R> ea{};
    for (int v = 0; v < NPRIM; ++v) ea.w[v] = P.w[v];
    for (int d = 0; d < 3; ++d) {
      ea.f0[d] = P.f[d][0];
      ea.e[d][0] = P.e[d][0];
      ea.e[d][1] = P.e[d][1];
      ea.edge[d] = P.edge[d];
    }
    k_emf<R><<<grd, blk, 0, st>>>(L, ea);
  }
  UpdArgs<R> ua{};
  for (int v = 0; v < NVAR; ++v) {
    ua.a[v] = P.reg[0][v];
    ua.b[v] = P.reg[1][v];
    ua.out[v] = P.reg[out][v];
  }
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 5; ++v) ua.f[d][v] = P.f[d][v];
    ua.edge[d] = P.edge[d];
  }
  for (int v = 0; v < NPRIM; ++v) ua.w[v] = P.w[v];
  ua.w0 = w0;
  ua.w1 = has_b ? w1 : R(0);
  ua.beta = beta;
  ua.dt = c->d_dt;
  k_update<R><<<grd, blk, 0, st>>>(L, P.geo, ua, mhd);
  c->n_launch += 3 + 1 + 3 + (mhd ? 1 : 0) + 1;
}

template <typename R, bool P64>
aeth_status step_unfused(aeth_ctx* c) {
  const int recon = c->cfg.recon;
  const int nb = (int)c->blocks.size();
  if (c->cfg.integrator == AETH_INT_VL2) {
    // predictor: U^{n+1/2} = U^n - dt/2 L_donor(U^n)   (register A -> B)
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), AETH_RECON_DONOR, 0, R(1), 0, R(0), R(0.5), 1);
    // corrector: U^{n+1} = U^n - dt L(U^{n+1/2})         (B -> A, in place)
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), recon, 1, R(1), 0, R(0), R(1), 0);
  } else if (c->cfg.integrator == AETH_INT_RK2) {
    // two-register SSP-RK2 (Eq. 10)
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), recon, 0, R(1), 0, R(0), R(1), 1);
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), recon, 1, R(0.5), 1, R(0.5), R(0.5), 0);
  } else if (c->cfg.integrator == AETH_INT_RK3) {
    // SSP-RK3 in two registers (the middle stage updates B in place)
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), recon, 0, R(1), 0, R(0), R(1), 1);
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), recon, 1, R(0.75), 1, R(0.25), R(0.25), 1);
    for (int b = 0; b < nb; ++b)
      stage_unfused<R, P64>(c, block_ptrs<R>(c, b), recon, 1, R(1.0 / 3.0), 1, R(2.0 / 3.0),
                            R(2.0 / 3.0), 0);
  } else {
    return fail(c, AETH_ERR_UNSUPPORTED, "integrator %d not available on the unfused path",
                c->cfg.integrator);
  }
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

template aeth_status step_unfused<float, false>(aeth_ctx*);
template aeth_status step_unfused<float, true>(aeth_ctx*);
template aeth_status step_unfused<double, false>(aeth_ctx*);

}  // namespace aeth
