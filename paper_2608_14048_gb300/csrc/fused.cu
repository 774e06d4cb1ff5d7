// Fused stage of the MHD step (Sec. 2.4-2.6) in three passes:
//
//  1. k_flux3: conserved->primitive, reconstruction and HLLD for all three
//     face directions of every cell in one sweep.  A CTA owns a TX x TY
//     column tile and marches along z: each x-y plane of primitives (with
//     the reconstruction halo) is staged in shared memory for the x- and
//     y-faces, while every thread keeps the z-stencil of its own column in a
//     register queue for the z-faces.  Each face is solved exactly once.
//     Outputs: hydro fluxes, face EMFs (the transverse induction fluxes) and
//     the cell-centred reference EMF of the upwind CT scheme.
//  2. k_emf_ref: corner EMFs of Gardiner & Stone (2005) from those arrays.
//  3. k_update_f: finite-volume update (Eq. 8, curvilinear sources of
//     Eq. 12) and constrained transport (Eq. 9) with the stage combination.
#include "runtime.hpp"

namespace aeth {

template <typename R>
void launch_fill(const BlockPtrs<R>& P, R* const* arrs, int nv, cudaStream_t st);

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;

bool fused_supported(const aeth_ctx*) { return true; }

template <typename R>
struct FluxOut {
  R* f[3][5];
  R* e[3][2];
  R* eref[3];
};

// Primitive variables of cell (i,j,k) (Eq. 5 with the floors of Sec. 2.1):
// w = (rho, v1, v2, v3, p, Bc1, Bc2, Bc3).  Returns the number of floors hit.
template <typename R, bool P64, bool MHD>
__device__ __forceinline__ int prim_cell(const Layout& L, const ConstArr8<R>& u, long long c,
                                         R gm1, R rho_floor, R p_floor, R* w) {
  int hits = 0;
  R rho = u.p[0][c];
  if (rho < rho_floor) { rho = rho_floor; ++hits; }
  const R ir = R(1) / rho;
  const R v1 = u.p[1][c] * ir, v2 = u.p[2][c] * ir, v3 = u.p[3][c] * ir;
  R b1 = 0, b2 = 0, b3 = 0;
  if (MHD) {
    b1 = R(0.5) * (u.p[5][c] + u.p[5][c + 1]);
    b2 = R(0.5) * (u.p[6][c] + u.p[6][c + L.sx]);
    b3 = R(0.5) * (u.p[7][c] + u.p[7][c + L.sx * L.sy]);
  }
  R pr;
  if (P64) {
    const double m1 = u.p[1][c], m2 = u.p[2][c], m3 = u.p[3][c];
    const double ke = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / (double)rho;
    const double me = 0.5 * ((double)b1 * b1 + (double)b2 * b2 + (double)b3 * b3);
    pr = (R)((double)gm1 * ((double)u.p[4][c] - ke - me));
  } else {
    pr = gm1 * (u.p[4][c] - R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3) -
                R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3));
  }
  if (pr < p_floor) { pr = p_floor; ++hits; }
  w[0] = rho; w[1] = v1; w[2] = v2; w[3] = v3; w[4] = pr; w[5] = b1; w[6] = b2; w[7] = b3;
  return hits;
}

__device__ __forceinline__ bool in_prim_range(const Layout& L, int i, int j, int k) {
  return i >= -L.g && i < L.n[0] + L.g && j >= -L.g && j < L.n[1] + L.g && k >= -L.g &&
         k < L.n[2] + L.g;
}

// Reconstruct face states of one variable from a stencil with stride.
template <int RECON, typename R, typename Get>
__device__ __forceinline__ void recon_var(Get get, R& wl, R& wr) {
  constexpr int RL = RECON + 1;
  R s[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int off = t - 3;   // cell offset from the face's right cell
    s[t] = (off >= -RL && off <= RECON) ? get(off) : R(0);
  }
  recon_face<RECON>(s, wl, wr);
}

// Solve one face of direction D and store its outputs.
template <int D, typename R>
__device__ __forceinline__ void store_face(const FluxOut<R>& o, long long fc, const R* fx) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  o.f[D][0][fc] = fx[0];
  o.f[D][1 + D][fc] = fx[1];
  o.f[D][1 + T1][fc] = fx[2];
  o.f[D][1 + T2][fc] = fx[3];
  o.f[D][4][fc] = fx[4];
  o.e[D][0][fc] = fx[6];    // E_t1 =  F(B_t2)
  o.e[D][1][fc] = -fx[5];   // E_t2 = -F(B_t1)
}

// two CTAs per SM in FP32 (<= 128 registers); FP64 takes the full file
template <typename R, bool P64, int RECON, bool MHD>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1)
    k_flux3(Layout L, ConstArr8<R> u, FluxOut<R> o, R gamma, R rho_floor, R p_floor, int kchunk,
            unsigned long long* floor_hits) {
  constexpr int RL = RECON + 1, RH = RECON;
  constexpr int WX = TX + RL + RH, WY = TY + RL + RH;
  constexpr int QN = RL + RH + 1;
  __shared__ R sw[NPRIM][WY][WX];

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i0 = -1 + (int)blockIdx.x * TX, j0 = -1 + (int)blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int k0 = -1 + (int)blockIdx.z * kchunk;
  const int k1 = min(nz, k0 + kchunk - 1);
  const bool active = i <= nx && j <= ny;
  const R gm1 = gamma - R(1);
  int hits = 0;

  // z register queue of the own column: planes k-RL .. k+RH, 7 variables
  // (the z-face normal field comes from the face array)
  R q[7][QN];
  auto load_q = [&](int slot, int kk) {
    R w[8];
    if (active && in_prim_range(L, i, j, kk)) {
      prim_cell<R, P64, MHD>(L, u, L.idx(i, j, kk), gm1, rho_floor, p_floor, w);
    } else {
      w[0] = R(1); w[1] = w[2] = w[3] = R(0); w[4] = R(1); w[5] = w[6] = w[7] = R(0);
    }
    // z-face frame order: rho, vz, vx, vy, p, Bx, By
    q[0][slot] = w[0]; q[1][slot] = w[3]; q[2][slot] = w[1]; q[3][slot] = w[2];
    q[4][slot] = w[4]; q[5][slot] = w[5]; q[6][slot] = w[6];
  };
#pragma unroll
  for (int t = 0; t < QN - 1; ++t) load_q(t + 1, k0 - RL + t);

  for (int k = k0; k <= k1; ++k) {
    __syncthreads();
    // stage plane k (tile + halo) in shared memory
    for (int t = threadIdx.x; t < WX * WY; t += NT) {
      const int rx = t % WX, ry = t / WX;
      const int ci = i0 - RL + rx, cj = j0 - RL + ry;
      R w[8];
      if (in_prim_range(L, ci, cj, k)) {
        hits += prim_cell<R, P64, MHD>(L, u, L.idx(ci, cj, k), gm1, rho_floor, p_floor, w);
      } else {
        w[0] = R(1); w[1] = w[2] = w[3] = R(0); w[4] = R(1); w[5] = w[6] = w[7] = R(0);
      }
#pragma unroll
      for (int v = 0; v < NPRIM; ++v) sw[v][ry][rx] = w[v];
    }
    // advance the z queue: drop plane k-RL-1, add plane k+RH
#pragma unroll
    for (int v = 0; v < 7; ++v)
#pragma unroll
      for (int t = 0; t < QN - 1; ++t) q[v][t] = q[v][t + 1];
    load_q(QN - 1, k + RH);
    __syncthreads();
    if (!active) continue;

    const long long fc = L.idx(i, j, k);
    const int sx = tx + RL, sy = ty + RL;
    R wl[7], wr[7], fx[7];
    // ---- x-face (i-1/2, j, k): frame (rho, vx, vy, vz, p, By, Bz)
    if (i >= 0 && k >= -1) {
      const int slot[7] = {0, 1, 2, 3, 4, 6, 7};
#pragma unroll
      for (int v = 0; v < 7; ++v) {
        if (!MHD && v >= 5) { wl[v] = wr[v] = R(0); continue; }
        recon_var<RECON>([&](int off) { return sw[slot[v]][sy][sx + off]; }, wl[v], wr[v]);
      }
      const R bn = MHD ? u.p[5][fc] : R(0);
      hlld(gamma, wl, wr, bn, fx);
      store_face<0>(o, fc, fx);
    }
    // ---- y-face (i, j-1/2, k): frame (rho, vy, vz, vx, p, Bz, Bx)
    if (j >= 0) {
      const int slot[7] = {0, 2, 3, 1, 4, 7, 5};
#pragma unroll
      for (int v = 0; v < 7; ++v) {
        if (!MHD && v >= 5) { wl[v] = wr[v] = R(0); continue; }
        recon_var<RECON>([&](int off) { return sw[slot[v]][sy + off][sx]; }, wl[v], wr[v]);
      }
      const R bn = MHD ? u.p[6][fc] : R(0);
      hlld(gamma, wl, wr, bn, fx);
      store_face<1>(o, fc, fx);
    }
    // ---- z-face (i, j, k-1/2): frame (rho, vz, vx, vy, p, Bx, By)
    if (k >= 0) {
#pragma unroll
      for (int v = 0; v < 7; ++v) {
        if (!MHD && v >= 5) { wl[v] = wr[v] = R(0); continue; }
        recon_var<RECON>([&](int off) { return q[v][off + RL]; }, wl[v], wr[v]);
      }
      const R bn = MHD ? u.p[7][fc] : R(0);
      hlld(gamma, wl, wr, bn, fx);
      store_face<2>(o, fc, fx);
    }
    // ---- cell-centred reference EMF, E = -v x B
    if (MHD) {
      const R vx = sw[1][sy][sx], vy = sw[2][sy][sx], vz = sw[3][sy][sx];
      const R bx = sw[5][sy][sx], by = sw[6][sy][sx], bz = sw[7][sy][sx];
      o.eref[0][fc] = -(vy * bz - vz * by);
      o.eref[1][fc] = -(vz * bx - vx * bz);
      o.eref[2][fc] = -(vx * by - vy * bx);
    }
  }
  if (hits) atomicAdd(floor_hits, (unsigned long long)hits);
}

// ------------------------------------------------------------------------
// corner EMFs from face EMFs, mass fluxes and the reference EMF arrays
// ------------------------------------------------------------------------
template <typename R>
struct EmfRefArgs {
  const R* eref[3];
  const R* f0[3];
  const R* e[3][2];
  R* edge[3];
};

template <typename R>
__global__ void __launch_bounds__(256) k_emf_ref(Layout L, EmfRefArgs<R> A) {
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
    const R* er = A.eref[cc];
    A.edge[cc][iP] = corner_emf(A.e[a][1][iB], A.e[a][1][iP], A.e[b][0][iA], A.e[b][0][iP],
                                er[iAB], er[iB], er[iA], er[iP], A.f0[a][iB], A.f0[a][iP],
                                A.f0[b][iA], A.f0[b][iP]);
  }
}

// ------------------------------------------------------------------------
// update: out = w0*A + w1*B + beta*dt*L (Eq. 8 + Eq. 12), CT (Eq. 9)
// ------------------------------------------------------------------------
template <typename R>
struct UpdFArgs {
  const R* a[NVAR];
  const R* b[NVAR];
  const R* src[NVAR];
  R* out[NVAR];
  const R* f[3][5];
  const R* edge[3];
  R w0, w1, beta;
  const double* dt;
};

template <typename R, bool P64, bool MHD, bool SPH>
__global__ void __launch_bounds__(256) k_update_f(Layout L, Geometry<R> geo, UpdFArgs<R> A,
                                                 R gamma, R rho_floor, R p_floor) {
  int P[3];
  P[0] = blockIdx.x * blockDim.x + threadIdx.x;
  P[1] = blockIdx.y * blockDim.y + threadIdx.y;
  P[2] = blockIdx.z * blockDim.z + threadIdx.z;
  if (P[0] > L.n[0] || P[1] > L.n[1] || P[2] > L.n[2]) return;
  const int i = P[0], j = P[1], k = P[2];
  const long long c = L.idx(i, j, k);
  const R bdt = A.beta * (R)(*A.dt);
  const bool has_b = A.w1 != R(0);
  if (i < L.n[0] && j < L.n[1] && k < L.n[2]) {
    const long long cp[3] = {c + 1, c + L.sx, c + L.sx * L.sy};
    R V, Am[3], Ap[3];
    if (SPH) {
      V = geo.vol(i, j, k);
      Am[0] = geo.area[0](i, j, k); Ap[0] = geo.area[0](i + 1, j, k);
      Am[1] = geo.area[1](i, j, k); Ap[1] = geo.area[1](i, j + 1, k);
      Am[2] = geo.area[2](i, j, k); Ap[2] = geo.area[2](i, j, k + 1);
    } else {
      V = geo.vol(0, 0, 0);
      Am[0] = Ap[0] = geo.area[0](0, 0, 0);
      Am[1] = Ap[1] = geo.area[1](0, 0, 0);
      Am[2] = Ap[2] = geo.area[2](0, 0, 0);
    }
    R src[5] = {0, 0, 0, 0, 0};
    if (SPH) {
      // curvilinear momentum sources from the stress tensor (Eq. 12) of
      // the stage state
      ConstArr8<R> s;
#pragma unroll
      for (int v = 0; v < NVAR; ++v) s.p[v] = A.src[v];
      R w[8];
      prim_cell<R, P64, MHD>(L, s, c, gamma - R(1), rho_floor, p_floor, w);
      const R rho = w[0], vv[3] = {w[1], w[2], w[3]};
      const R bb[3] = {w[5], w[6], w[7]};
      const R ps = w[4] + R(0.5) * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
      auto T = [&](int x, int y) {
        return rho * vv[x] * vv[y] + (x == y ? ps : R(0)) - bb[x] * bb[y];
      };
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
      if (has_b) base += A.w1 * A.b[v][c];
      A.out[v][c] = base + bdt * rhs;
    }
  }
  if (!MHD) return;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    const int hid = L.bc[d] == AETH_BC_OUTFLOW ? L.n[d] : L.n[d] - 1;
    if (P[d] > hid || P[e1] >= L.n[e1] || P[e2] >= L.n[e2]) continue;
    int Q1[3] = {i, j, k}, Q2[3] = {i, j, k};
    Q1[e1] += 1; Q2[e2] += 1;
    const long long q1 = c + L.stride(e1), q2 = c + L.stride(e2);
    R circ;
    if (SPH) {
      circ = A.edge[e2][q1] * geo.edge[e2](Q1[0], Q1[1], Q1[2]) -
             A.edge[e2][c] * geo.edge[e2](i, j, k) -
             (A.edge[e1][q2] * geo.edge[e1](Q2[0], Q2[1], Q2[2]) -
              A.edge[e1][c] * geo.edge[e1](i, j, k));
    } else {
      const R l2 = geo.edge[e2](0, 0, 0), l1 = geo.edge[e1](0, 0, 0);
      circ = A.edge[e2][q1] * l2 - A.edge[e2][c] * l2 - (A.edge[e1][q2] * l1 - A.edge[e1][c] * l1);
    }
    const R Af = SPH ? geo.area[d](i, j, k) : geo.area[d](0, 0, 0);
    R base = A.w0 * A.a[5 + d][c];
    if (has_b) base += A.w1 * A.b[5 + d][c];
    const R nb = base - bdt * circ / Af;
    A.out[5 + d][c] = nb;
    if (L.bc[d] == AETH_BC_PERIODIC && P[d] == 0)
      A.out[5 + d][c + (long long)L.n[d] * L.stride(d)] = nb;
  }
}

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------
constexpr int KCHUNK = 32;

template <typename R, bool P64, int RECON, bool MHD>
static void launch_flux3(aeth_ctx* c, const BlockPtrs<R>& P, int src, const FluxOut<R>& o) {
  const Layout& L = P.L;
  ConstArr8<R> u{};
  for (int v = 0; v < NVAR; ++v) u.p[v] = P.reg[src][v];
  const int kc = std::min(KCHUNK, L.n[2] + 2);
  dim3 grd((L.n[0] + 2 + TX - 1) / TX, (L.n[1] + 2 + TY - 1) / TY, (L.n[2] + 2 + kc - 1) / kc);
  k_flux3<R, P64, RECON, MHD><<<grd, NT, 0, c->stream>>>(L, u, o, (R)c->cfg.gamma,
                                                         (R)c->cfg.rho_floor, (R)c->cfg.p_floor,
                                                         kc, c->d_floor);
}

template <typename R, bool P64, bool MHD>
static void stage_fused(aeth_ctx* c, const BlockPtrs<R>& P, int recon, int src, R w0, int has_b,
                        R w1, R beta, int out) {
  const Layout& L = P.L;
  cudaStream_t st = c->stream;
  const int nv = MHD ? NVAR : 5;
  launch_fill<R>(P, P.reg[src], nv, st);
  FluxOut<R> o{};
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 5; ++v) o.f[d][v] = P.f[d][v];
    o.e[d][0] = P.e[d][0];
    o.e[d][1] = P.e[d][1];
    o.eref[d] = P.w[d];   // the primitive scratch slots hold E_ref here
  }
  // algorithmic traffic of the flux pass: the stage state read once
  // (8 words), outputs written once (15 fluxes + 6 face EMFs + 3 E_ref)
  const double cells = (double)(L.n[0] + 2) * (L.n[1] + 2) * (L.n[2] + 2);
  prof_begin(c);
  if (recon == AETH_RECON_DONOR) launch_flux3<R, P64, 0, MHD>(c, P, src, o);
  else if (recon == AETH_RECON_PLM) launch_flux3<R, P64, 1, MHD>(c, P, src, o);
  else launch_flux3<R, P64, 2, MHD>(c, P, src, o);
  prof_end(c, cells * ((MHD ? 8 : 5) + (MHD ? 24 : 15)) * sizeof(R));

  dim3 blk(32, 4, 2);
  dim3 grd((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 3) / 4, (L.n[2] + 1 + 1) / 2);
  if (MHD) {
    EmfRefArgs<R> ea{};
    for (int d = 0; d < 3; ++d) {
      ea.eref[d] = P.w[d];
      ea.f0[d] = P.f[d][0];
      ea.e[d][0] = P.e[d][0];
      ea.e[d][1] = P.e[d][1];
      ea.edge[d] = P.edge[d];
    }
    k_emf_ref<R><<<grd, blk, 0, st>>>(L, ea);
  }
  UpdFArgs<R> ua{};
  for (int v = 0; v < NVAR; ++v) {
    ua.a[v] = P.reg[0][v];
    ua.b[v] = P.reg[1][v];
    ua.src[v] = P.reg[src][v];
    ua.out[v] = P.reg[out][v];
  }
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 5; ++v) ua.f[d][v] = P.f[d][v];
    ua.edge[d] = P.edge[d];
  }
  ua.w0 = w0;
  ua.w1 = has_b ? w1 : R(0);
  ua.beta = beta;
  ua.dt = c->d_dt;
  const R gm = (R)c->cfg.gamma, rf = (R)c->cfg.rho_floor, pf = (R)c->cfg.p_floor;
  if (L.coord == AETH_COORD_SPH)
    k_update_f<R, P64, MHD, true><<<grd, blk, 0, st>>>(L, P.geo, ua, gm, rf, pf);
  else
    k_update_f<R, P64, MHD, false><<<grd, blk, 0, st>>>(L, P.geo, ua, gm, rf, pf);
  c->n_launch += 3 + 1 + (MHD ? 1 : 0) + 1;
}

template <typename R, bool P64, bool MHD>
static aeth_status step_fused_T(aeth_ctx* c) {
  const int recon = c->cfg.recon;
  const int nb = (int)c->blocks.size();
  if (c->cfg.integrator == AETH_INT_VL2) {
    for (int b = 0; b < nb; ++b)
      stage_fused<R, P64, MHD>(c, block_ptrs<R>(c, b), AETH_RECON_DONOR, 0, R(1), 0, R(0), R(0.5), 1);
    for (int b = 0; b < nb; ++b)
      stage_fused<R, P64, MHD>(c, block_ptrs<R>(c, b), recon, 1, R(1), 0, R(0), R(1), 0);
  } else if (c->cfg.integrator == AETH_INT_RK2) {
    for (int b = 0; b < nb; ++b)
      stage_fused<R, P64, MHD>(c, block_ptrs<R>(c, b), recon, 0, R(1), 0, R(0), R(1), 1);
    for (int b = 0; b < nb; ++b)
      stage_fused<R, P64, MHD>(c, block_ptrs<R>(c, b), recon, 1, R(0.5), 1, R(0.5), R(0.5), 0);
  } else {
    return fail(c, AETH_ERR_UNSUPPORTED, "integrator %d not available", c->cfg.integrator);
  }
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

template <typename R, bool P64>
aeth_status step_fused(aeth_ctx* c) {
  return is_mhd(c) ? step_fused_T<R, P64, true>(c) : step_fused_T<R, P64, false>(c);
}

template aeth_status step_fused<float, false>(aeth_ctx*);
template aeth_status step_fused<float, true>(aeth_ctx*);
template aeth_status step_fused<double, false>(aeth_ctx*);

}  // namespace aeth

namespace aeth {
// Hydro-gas flux pass for other integrators (dust runs): the same fused
// prim + reconstruction + HLLD sweep, writing the stage's face fluxes.
template <typename R, bool P64>
void hydro_flux_pass(aeth_ctx* c, const BlockPtrs<R>& P, int recon, int src) {
  FluxOut<R> o{};
  for (int d = 0; d < 3; ++d) {
    for (int v = 0; v < 5; ++v) o.f[d][v] = P.f[d][v];
    o.e[d][0] = P.e[d][0];
    o.e[d][1] = P.e[d][1];
    o.eref[d] = P.w[d];
  }
  if (recon == AETH_RECON_DONOR) launch_flux3<R, P64, 0, false>(c, P, src, o);
  else if (recon == AETH_RECON_PLM) launch_flux3<R, P64, 1, false>(c, P, src, o);
  else launch_flux3<R, P64, 2, false>(c, P, src, o);
  c->n_launch += 1;
}
template void hydro_flux_pass<float, false>(aeth_ctx*, const BlockPtrs<float>&, int, int);
template void hydro_flux_pass<float, true>(aeth_ctx*, const BlockPtrs<float>&, int, int);
template void hydro_flux_pass<double, false>(aeth_ctx*, const BlockPtrs<double>&, int, int);
}  // namespace aeth
