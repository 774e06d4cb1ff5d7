// Multifluid dust (Sec. 2.2, Eqs. 6-7) with the IMEX2P integrator (Sec. 2.6).
//
// Per stage: ghost fill; the fused hydro-gas flux pass (HLLD at B = 0);
// one pressureless Rusanov flux pass per direction for all species; then one
// fused kernel that forms the explicit stage combination and solves the
// implicit drag of every cell in closed form (arrowhead system, O(N) per
// velocity component) in FP64, whatever the transport precision.
//
// The stage combinations run in the working precision; the drag solve runs
// in FP64 by default (aeth_config.drag_precision) and its few divisions are
// hoisted: 1/rho_k and 1/(1 + a_k) per species, one 1/den per cell.
//
// IMEX2P with implicit weight g = 1 + 1/sqrt 2 and explicit weight
// d = 1 - 1/(2g) in two registers (A, B):
//   stage 2: X = U^n + g dt L(U^n), W = U^n + d dt L(U^n), U2 = drag_h(X),
//            B <- U2, A <- W + (1-g)/g (U2 - X)          [(U2-X)/g = dt R(U2)]
//   stage 3: Y = A + (1-d) dt L(U2), A <- drag_h(Y)      (h = g dt)
#include "runtime.hpp"

namespace aeth {

template <typename R>
void launch_fill(const BlockPtrs<R>& P, R* const* arrs, int nv, cudaStream_t st);
template <typename R, bool P64>
void hydro_flux_pass(aeth_ctx* c, int block, int recon, int src);

// z depth of the update's CTAs: 1 (128 threads; 2 or 3 CTAs per SM at its
// 160-180 registers) measured 6-9% faster than 2 (256 threads, one CTA)
#ifndef AETH_DUST_BZ
#define AETH_DUST_BZ 1
#endif

constexpr double kImexG = 1.0 + 0.70710678118654752440;
constexpr double kImexD = 1.0 - 1.0 / (2.0 * kImexG);

// ------------------------------------------------------------------------
// Rusanov flux of all species across the lower D-face of each cell
// ------------------------------------------------------------------------
template <typename R, int RECON, int D>
__global__ void __launch_bounds__(256)
    k_dust_flux(Layout L, const R* __restrict__ dsrc, R* __restrict__ dflux, int nd,
                R dfloor) {
  int c3[3];
  c3[0] = blockIdx.x * blockDim.x + threadIdx.x;
  c3[1] = blockIdx.y * blockDim.y + threadIdx.y;
  c3[2] = blockIdx.z * blockDim.z + threadIdx.z;
#pragma unroll
  for (int e = 0; e < 3; ++e)
    if (c3[e] > L.n[e] || (e != D && c3[e] == L.n[e])) return;
  constexpr int RH = recon_reach<RECON>(), RL = RH + 1;
  const long long sz = L.size();
  const long long fc = L.idx(c3[0], c3[1], c3[2]);
  const long long sd = L.stride(D);
  for (int s = 0; s < nd; ++s) {
    const R* rho = dsrc + (long long)(4 * s) * sz;
    R st[4][6];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int off = t - 3;
      if (off < -RL || off > RH) {
        st[0][t] = st[1][t] = st[2][t] = st[3][t] = R(0);
        continue;
      }
      const long long cc = fc + off * sd;
      R r = rho[cc];
      if (r < dfloor) r = dfloor;
      const R ir = R(1) / r;
      st[0][t] = r;
#pragma unroll
      for (int q = 0; q < 3; ++q) st[1 + q][t] = rho[(long long)(1 + q) * sz + cc] * ir;
    }
    R wl[4], wr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) recon_face<RECON>(st[q], wl[q], wr[q]);
    const R vnl = wl[1 + D], vnr = wr[1 + D];
    const R sp = fmax(fabs(vnl), fabs(vnr));
    const R ul[4] = {wl[0], wl[0] * wl[1], wl[0] * wl[2], wl[0] * wl[3]};
    const R ur[4] = {wr[0], wr[0] * wr[1], wr[0] * wr[2], wr[0] * wr[3]};
    R* out = dflux + (long long)((D * nd + s) * 4) * sz;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      out[(long long)q * sz + fc] =
          R(0.5) * (ul[q] * vnl + ur[q] * vnr) - R(0.5) * sp * (ur[q] - ul[q]);
  }
}

// ------------------------------------------------------------------------
// stage combination + implicit drag (FP64), Cartesian blocks
// ------------------------------------------------------------------------
template <typename R>
struct DustUpd {
  R* ga[5];            // gas register A
  R* gb[5];            // gas register B
  const R* gf[3][5];   // gas fluxes
  R* da;               // dust register A (base)
  R* db;               // dust register B (base)
  const R* df;         // dust fluxes (base)
  double drag_c[32];   // per species: 1 / t_k (constant stopping time) or
                       // K_k (constant coefficient, t_k = rho_k / K_k)
  const double* dt;
  R dfloor;
};

// Stage combination in the working precision R, implicit drag in DT.
// SEL (DT = double, R = float): per-species precision -- the species whose
// implicit weight a_k = h / t_k exceeds sel_ratio are solved in FP64, the
// others in FP32; the gas sums over species (the denominator, the momentum
// numerators and the drag heating) accumulate in FP64.
// COEFF: the constant-coefficient drag law (drag_c = K_k, a_k = h K_k /
// rho_k per cell).  iso: isothermal gas, whose energy slot takes no drag
// heating.
template <typename R, typename DT, int NDMAX, bool SEL = false, bool COEFF = false>
__global__ void __launch_bounds__(256)
    k_dust_update(Layout L, R idx1, R idx2, R idx3, DustUpd<R> A, int nd, int stage,
                  unsigned long long* floor_hits, float sel_ratio, int iso) {
  // per-species drag constants of this stage, the same for every cell:
  // a_k = h / t_k, 1 / (1 + a_k), w_k = a_k / (1 + a_k) with h = g dt
  __shared__ DT s_ak[NDMAX], s_ia[NDMAX], s_wk[NDMAX];
  __shared__ float f_ak[SEL ? NDMAX : 1], f_ia[SEL ? NDMAX : 1], f_wk[SEL ? NDMAX : 1];
  __shared__ unsigned s_wide;   // SEL: bit s set = species s in FP64
  {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (SEL && tid == 0) s_wide = 0u;
    __syncthreads();
    if (tid < nd && tid < NDMAX) {
      const DT h = (DT)kImexG * (DT)(*A.dt);
      const DT a = h * (DT)A.drag_c[tid];
      const DT ia = DT(1) / (DT(1) + a);
      s_ak[tid] = a;
      s_ia[tid] = ia;
      s_wk[tid] = a * ia;
      if constexpr (SEL) {
        const float af = (float)h * (float)A.drag_c[tid];
        const float iaf = 1.0f / (1.0f + af);
        f_ak[tid] = af;
        f_ia[tid] = iaf;
        f_wk[tid] = af * iaf;
        if (a > (DT)sel_ratio) atomicOr(&s_wide, 1u << tid);
      }
    }
    __syncthreads();
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= L.n[0] || j >= L.n[1] || k >= L.n[2]) return;
  const long long c = L.idx(i, j, k);
  const long long sz = L.size();
  const long long st[3] = {1, L.sx, L.sx * L.sy};
  const R inv[3] = {idx1, idx2, idx3};
  const R dt = (R)(*A.dt);
  const R g = (R)kImexG, d = (R)kImexD;
  // explicit right-hand sides and the stage's pre-drag state X; the
  // register-A values stay in registers for the stage-2 combination (a
  // reload after the first stores would wait on each store in turn)
  R gx[5], ug[5];
  R dx[NDMAX][4], ud[NDMAX][4];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    R div = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) div += (A.gf[a][v][c + st[a]] - A.gf[a][v][c]) * inv[a];
    ug[v] = A.ga[v][c];
    gx[v] = ug[v] - (stage == 2 ? g : R(1) - d) * dt * div;
  }
#pragma unroll
  for (int s = 0; s < NDMAX; ++s) {
    if (s >= nd) break;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      R div = R(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R* f = A.df + (long long)(((a * nd + s) * 4 + q)) * sz;
        div += (f[c + st[a]] - f[c]) * inv[a];
      }
      ud[s][q] = A.da[(long long)(4 * s + q) * sz + c];
      dx[s][q] = ud[s][q] - (stage == 2 ? g : R(1) - d) * dt * div;
    }
  }
  // closed-form implicit drag with h = g dt (Sec. 2.2).  With
  // a_k = h / t_k, w_k = a_k / (1 + a_k):
  //   rho_g v_g' = (M_g* + sum_k w_k M_k*) * rho_g / (rho_g + sum_k rho_k w_k)
  //   M_k' = rho_k v_k' = (M_k* + rho_k a_k v_g') / (1 + a_k)
  //   dKE_k = (M_k'^2 - M_k*^2) / (2 rho_k)
  // 1/rho_k and 1/den come from one division (simultaneous inversion,
  // Montgomery 1987: prefix products, one reciprocal, back-substitution).
  R gy[5], dy[NDMAX][4];
  const DT rg = gx[0];
  gy[0] = gx[0];
  if constexpr (COEFF) {
    // constant-coefficient law (Sec. 2.2): t_k = rho_k / K_k with the
    // stage's dust density, which the drag leaves unchanged, so the weight
    // a_k = h K_k / rho_k is fixed per cell through the solve; a species
    // with no density (rho_k <= 0) feels no drag
    const DT h = (DT)kImexG * (DT)(*A.dt);
    DT rk[NDMAX], ak[NDMAX], ia[NDMAX], irk[NDMAX];
    DT den = rg;
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
      rk[s] = dx[s][0];
      irk[s] = rk[s] > DT(0) ? DT(1) / rk[s] : DT(0);
      ak[s] = h * (DT)A.drag_c[s] * irk[s];
      ia[s] = DT(1) / (DT(1) + ak[s]);
      den += rk[s] * ak[s] * ia[s];
      dy[s][0] = dx[s][0];
    }
    const DT inv_den = DT(1) / den;
    DT dke2 = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      DT num = gx[1 + q];
#pragma unroll
      for (int s = 0; s < NDMAX; ++s) {
        if (s >= nd) break;
        num += ak[s] * ia[s] * (DT)dx[s][1 + q];
      }
      const DT vg = num * inv_den;
      gy[1 + q] = (R)(rg * vg);
#pragma unroll
      for (int s = 0; s < NDMAX; ++s) {
        if (s >= nd) break;
        const DT m0 = dx[s][1 + q];
        const DT m1 = (m0 + rk[s] * ak[s] * vg) * ia[s];
        dy[s][1 + q] = (R)m1;
        dke2 += (m1 - m0) * (m1 + m0) * irk[s];
      }
    }
    gy[4] = iso ? gx[4] : (R)((DT)gx[4] - DT(0.5) * dke2);
  } else if constexpr (SEL) {
    // per-species precision: FP64 for the stiff species (s_wide), FP32 for
    // the rest; one FP64 division for the denominator, reciprocals of the
    // densities in each species' own precision
    const unsigned wide = s_wide;
    DT den = rg;
    DT ir64[NDMAX];    // 1 / rho_k of the FP64 species (0 for rho_k <= 0)
    float ir32[NDMAX]; // the same for the FP32 species
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
      dy[s][0] = dx[s][0];
      ir64[s] = DT(0);
      ir32[s] = 0.0f;
      if ((wide >> s) & 1u) {
        den += (DT)dx[s][0] * s_wk[s];
        if ((DT)dx[s][0] > DT(0)) ir64[s] = DT(1) / (DT)dx[s][0];
      } else {
        den += (DT)((float)dx[s][0] * f_wk[s]);
        if ((float)dx[s][0] > 0.0f) ir32[s] = 1.0f / (float)dx[s][0];
      }
    }
    const DT inv_den = DT(1) / den;
    DT dke2 = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      DT num = gx[1 + q];
#pragma unroll
      for (int s = 0; s < NDMAX; ++s) {
        if (s >= nd) break;
        if ((wide >> s) & 1u) num += s_wk[s] * (DT)dx[s][1 + q];
        else num += (DT)(f_wk[s] * (float)dx[s][1 + q]);
      }
      const DT vg = num * inv_den;
      gy[1 + q] = (R)(rg * vg);
      const float vgf = (float)vg;
#pragma unroll
      for (int s = 0; s < NDMAX; ++s) {
        if (s >= nd) break;
        const R r = dx[s][0];
        if ((wide >> s) & 1u) {
          const DT rk = r, m0 = dx[s][1 + q];
          const DT m1 = (m0 + rk * s_ak[s] * vg) * s_ia[s];
          dy[s][1 + q] = (R)m1;
          dke2 += (m1 - m0) * (m1 + m0) * ir64[s];
        } else {
          const float rk = (float)r, m0 = (float)dx[s][1 + q];
          const float m1 = (m0 + rk * f_ak[s] * vgf) * f_ia[s];
          dy[s][1 + q] = (R)m1;
          dke2 += (DT)((m1 - m0) * (m1 + m0) * ir32[s]);
        }
      }
    }
    gy[4] = iso ? gx[4] : (R)((DT)gx[4] - DT(0.5) * dke2);
  } else {
  DT rk[NDMAX], rak[NDMAX], ir[NDMAX];
  DT den = rg;
#pragma unroll
  for (int s = 0; s < NDMAX; ++s) {
    if (s >= nd) break;
    rk[s] = dx[s][0];
    rak[s] = rk[s] * s_ak[s];
    den += rk[s] * s_wk[s];
    dy[s][0] = dx[s][0];
  }
  DT inv_den;
  if constexpr (sizeof(DT) == 8 && NDMAX <= 8) {
    // prefix products x_0 ... x_{s-1} of the densities (a non-positive
    // density enters as 1 and gets 1/rho = 0); at most 8 factors of the
    // density range stay far inside the FP64 exponent range
    DT pre[NDMAX];
    DT acc = DT(1);
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
      pre[s] = acc;
      acc *= rk[s] > DT(0) ? rk[s] : DT(1);
    }
    const DT q = DT(1) / (acc * den);   // the one division
    inv_den = q * acc;
    DT ip = q * den;                    // 1 / (x_0 ... x_{nd-1})
#pragma unroll
    for (int s = NDMAX - 1; s >= 0; --s) {
      if (s >= nd) continue;
      ir[s] = rk[s] > DT(0) ? ip * pre[s] : DT(0);
      ip *= rk[s] > DT(0) ? rk[s] : DT(1);   // 1 / (x_0 ... x_{s-1})
    }
  } else {
    inv_den = DT(1) / den;
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
      ir[s] = rk[s] > DT(0) ? DT(1) / rk[s] : DT(0);
    }
  }
  DT dke2 = 0;   // twice the change of the dust kinetic energy
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    DT m0[NDMAX];
    DT num = gx[1 + q];   // rho_g v_g* = M_g*
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
      m0[s] = (DT)dx[s][1 + q];
      num += s_wk[s] * m0[s];   // rho_k w_k v_k* = w_k M_k*
    }
    const DT vg = num * inv_den;
    gy[1 + q] = (R)(rg * vg);
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
      const DT m1 = (m0[s] + rak[s] * vg) * s_ia[s];
      dy[s][1 + q] = (R)m1;
      dke2 += (m1 - m0[s]) * (m1 + m0[s]) * ir[s];
    }
  }
  const DT dke = DT(0.5) * dke2;
  // total energy conserved: drift energy becomes gas heat (the isothermal
  // closure carries its energy slot unchanged)
  gy[4] = iso ? gx[4] : (R)((DT)gx[4] - dke);
  }
  int hits = 0;
#pragma unroll
  for (int s = 0; s < NDMAX; ++s) {
    if (s >= nd) break;
    if (dy[s][0] < A.dfloor) {
      dy[s][0] = A.dfloor;
      dy[s][1] = dy[s][2] = dy[s][3] = R(0);
      ++hits;
    }
  }
  if (stage == 2) {
    // A <- W + (1-g)/g (U2 - X), with W = U^n + d dt L = (1 - d/g) U^n + (d/g) X
    const R cw = (R(1) - g) / g, cu = R(1) - d / g, cx = d / g;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      A.gb[v][c] = gy[v];
      A.ga[v][c] = cu * ug[v] + cx * gx[v] + cw * (gy[v] - gx[v]);
    }
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long o = (long long)(4 * s + q) * sz + c;
        A.db[o] = dy[s][q];
        A.da[o] = cu * ud[s][q] + cx * dx[s][q] + cw * (dy[s][q] - dx[s][q]);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) A.ga[v][c] = gy[v];
#pragma unroll
    for (int s = 0; s < NDMAX; ++s) {
      if (s >= nd) break;
#pragma unroll
      for (int q = 0; q < 4; ++q) A.da[(long long)(4 * s + q) * sz + c] = dy[s][q];
    }
  }
  if (hits) atomicAdd(floor_hits, (unsigned long long)hits);
}

// Ghost fill of n cell-centred arrays at base + a * sz, one axis.
template <typename R>
__global__ void __launch_bounds__(256) k_fill_cells(Layout L, R* base, int narr, int d) {
  const int g = L.g;
  int lo[3], ext[3];
  for (int e = 0; e < 3; ++e) {
    if (e < d) { lo[e] = -g; ext[e] = L.n[e] + 2 * g + 1; }
    else if (e == d) { lo[e] = 0; ext[e] = 2 * g + 1; }
    else { lo[e] = 0; ext[e] = L.n[e] + 1; }
  }
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int t1 = blockIdx.y * blockDim.y + threadIdx.y;
  const int t2 = blockIdx.z * blockDim.z + threadIdx.z;
  if (t0 >= ext[0] || t1 >= ext[1] || t2 >= ext[2]) return;
  int c[3] = {t0 + lo[0], t1 + lo[1], t2 + lo[2]};
  const int n = L.n[d];
  const int t = c[d];
  c[d] = t < g ? t - g : n + (t - g);
  const int p = c[d];
  int s;
  if (L.bc[d] == AETH_BC_PERIODIC) s = ((p % n) + n) % n;
  else s = p < 0 ? 0 : n - 1;
  int sc[3] = {c[0], c[1], c[2]};
  sc[d] = s;
  const long long dst = L.idx(c[0], c[1], c[2]), srcx = L.idx(sc[0], sc[1], sc[2]);
  const long long sz = L.size();
  // eight arrays at a time, every source loaded before the stores (the
  // stores go through the same base, so interleaving them would serialise
  // the round trips)
  for (int a0 = 0; a0 < narr; a0 += 8) {
    R v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (a0 + q < narr) v[q] = base[(a0 + q) * sz + srcx];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (a0 + q < narr) base[(a0 + q) * sz + dst] = v[q];
  }
}

template <typename R, bool P64>
static void stage_dust(aeth_ctx* c, int b, int src, int stage) {
  const BlockPtrs<R> P = block_ptrs<R>(c, b);
  const BlockInfo& B = c->blocks[b];
  const Layout& L = P.L;
  const int nd = c->cfg.n_dust;
  cudaStream_t s = c->stream;
  launch_fill<R>(P, P.reg[src], 5, s);
  c->n_launch += 3;
  const long long sz = L.size();
  (void)sz;
  for (int d = 0; d < 3; ++d) {
    int ext[3];
    for (int e = 0; e < 3; ++e)
      ext[e] = e < d ? L.n[e] + 2 * L.g + 1 : (e == d ? 2 * L.g + 1 : L.n[e] + 1);
    dim3 fb(32, 4, 2), fg((ext[0] + 31) / 32, (ext[1] + 3) / 4, (ext[2] + 1) / 2);
    k_fill_cells<R><<<fg, fb, 0, s>>>(L, P.dust[src], 4 * nd, d);
  }
  c->n_launch += 3;
  hydro_flux_pass<R, P64>(c, b, c->cfg.recon, src);
  dim3 blk(32, 4, 2);
  dim3 grd((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 3) / 4, (L.n[2] + 1 + 1) / 2);
  const R dfl = (R)1e-20;
  const R* dsrc = P.dust[src];
  switch (c->cfg.recon) {
    case AETH_RECON_DONOR:
      k_dust_flux<R, 0, 0><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 0, 1><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 0, 2><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      break;
    case AETH_RECON_PLM:
      k_dust_flux<R, 1, 0><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 1, 1><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 1, 2><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      break;
    case AETH_RECON_PPM5:
      k_dust_flux<R, 3, 0><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 3, 1><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 3, 2><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      break;
    default:
      k_dust_flux<R, 2, 0><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 2, 1><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
      k_dust_flux<R, 2, 2><<<grd, blk, 0, s>>>(L, dsrc, P.dflux, nd, dfl);
  }
  DustUpd<R> u{};
  for (int v = 0; v < 5; ++v) {
    u.ga[v] = P.reg[0][v];
    u.gb[v] = P.reg[1][v];
    for (int a = 0; a < 3; ++a) u.gf[a][v] = P.f[a][v];
  }
  u.da = P.dust[0];
  u.db = P.dust[1];
  u.df = P.dflux;
  const bool coeff = c->cfg.drag_law == AETH_DRAG_LAW_COEFF;
  for (int q = 0; q < nd; ++q) u.drag_c[q] = coeff ? c->t_stop[q] : 1.0 / c->t_stop[q];
  u.dt = c->d_dt;
  u.dfloor = dfl;
  // inverse cell widths (Cartesian: area / volume = 1 / dx_d)
  const R i1 = (R)(B.desc.nx / (B.desc.x1max - B.desc.x1min));
  const R i2 = (R)(B.desc.ny / (B.desc.x2max - B.desc.x2min));
  const R i3 = (R)(B.desc.nz / (B.desc.x3max - B.desc.x3min));
  // the update: CTAs of 32 x 4 x AETH_DUST_BZ cells (its registers allow
  // few CTAs per SM)
  const dim3 blk2(32, 4, AETH_DUST_BZ);
  dim3 grd2((L.n[0] + 31) / 32, (L.n[1] + 3) / 4, (L.n[2] + AETH_DUST_BZ - 1) / AETH_DUST_BZ);
  const bool d64 = c->cfg.drag_precision == AETH_DRAG_FP64;
  const int iso = is_iso(c) ? 1 : 0;
  const float ratio = (float)c->cfg.drag_ratio;
  auto launch = [&](auto kernel) {
    kernel<<<grd2, blk2, 0, s>>>(L, i1, i2, i3, u, nd, stage, c->d_floor, ratio, iso);
  };
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    if (c->cfg.drag_precision == AETH_DRAG_SEL64) {
      // per-species precision: FP64 for the species with h / t_k > drag_ratio
      if (nd <= 8) launch(k_dust_update<R, double, 8, true>);
      else launch(k_dust_update<R, double, 32, true>);
      done = true;
    }
  }
  if (done) {
  } else if (coeff) {
    if (nd <= 8) d64 ? launch(k_dust_update<R, double, 8, false, true>)
                     : launch(k_dust_update<R, R, 8, false, true>);
    else d64 ? launch(k_dust_update<R, double, 32, false, true>)
             : launch(k_dust_update<R, R, 32, false, true>);
  } else if (nd <= 8) {
    d64 ? launch(k_dust_update<R, double, 8>) : launch(k_dust_update<R, R, 8>);
  } else {
    d64 ? launch(k_dust_update<R, double, 32>) : launch(k_dust_update<R, R, 32>);
  }
  c->n_launch += 3 + 1;
}

template <typename R, bool P64>
aeth_status step_dust(aeth_ctx* c) {
  const int nb = (int)c->blocks.size();
  for (int b = 0; b < nb; ++b) stage_dust<R, P64>(c, b, 0, 2);
  for (int b = 0; b < nb; ++b) stage_dust<R, P64>(c, b, 1, 3);
  AETH_CK(c, cudaGetLastError());
  return AETH_OK;
}

template aeth_status step_dust<float, false>(aeth_ctx*);
template aeth_status step_dust<float, true>(aeth_ctx*);
template aeth_status step_dust<double, false>(aeth_ctx*);

}  // namespace aeth
