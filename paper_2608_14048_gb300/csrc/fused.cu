// Fused stage of the MHD step (Sec. 2.4-2.6) in three passes:
//
// Every pass is ONE launch over all mesh blocks of the context: a device
// table holds each block's layout, geometry and array pointers, and each
// pass kind has a prefix sum of tiles per block, so a CTA finds its block
// by binary search.  The flux pass is persistent (grid-stride over tiles,
// grid sized to the SM count); uneven block sizes only change the number
// of tiles per block.
//
//  1. k_flux3 (flux3.cuh): conserved->primitive, reconstruction and the
//     Riemann solver for all three face directions of every cell in one
//     sweep; hydro fluxes, face EMFs and the cell-centred reference EMF.
//  2. k_emf_ref: corner EMFs of Gardiner & Stone (2005) from those arrays.
//  3. k_update_f: finite-volume update (Eq. 8, curvilinear sources of
//     Eq. 12) and constrained transport (Eq. 9) with the stage combination.
#include "flux3.cuh"

namespace aeth {

template <typename R>
void launch_fill(const BlockPtrs<R>& P, R* const* arrs, int nv, cudaStream_t st);

// resident CTAs per SM requested for the update pass (registers 65536 /
// (256 * UPD_MINB)): the loads of a cell are hoisted above its stores, so
// the register cap trades memory-level parallelism per thread for threads
#ifndef AETH_UPD_MINB
#define AETH_UPD_MINB 3
#endif

bool fused_supported(const aeth_ctx*) { return true; }

// Tile coordinates of the 32x4x2 elementwise passes.
struct CellTile {
  int b, P[3];
  bool ok;
};

template <typename R>
__device__ __forceinline__ CellTile cell_tile(const BlockPtrs<R>& B, int loc, const int* ext_add) {
  CellTile ct;
  ct.b = 0;
  const Layout& L = B.L;
  const int ntx = ceil_div_d(L.n[0] + ext_add[0], CELL_BX);
  const int nty = ceil_div_d(L.n[1] + ext_add[1], CELL_BY);
  const int bx = loc % ntx, by = (loc / ntx) % nty, bz = loc / (ntx * nty);
  ct.P[0] = bx * CELL_BX + (int)(threadIdx.x % CELL_BX);
  ct.P[1] = by * CELL_BY + (int)((threadIdx.x / CELL_BX) % CELL_BY);
  ct.P[2] = bz * CELL_BZ + (int)(threadIdx.x / (CELL_BX * CELL_BY));
  ct.ok = true;
  return ct;
}

// ------------------------------------------------------------------------
// 2. corner EMFs from face EMFs, mass fluxes and the reference EMF arrays
// ------------------------------------------------------------------------
template <typename R, typename Src>
__global__ void __launch_bounds__(256) k_emf_ref(Src S, int t0, int t1) {
  const int add[3] = {1, 1, 1};
  for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
    int loc;
    const BlockPtrs<R>& A = S.get(t, loc);
    const CellTile ct = cell_tile(A, loc, add);
    const Layout L = A.L;
    const int* P = ct.P;
    if (P[0] > L.n[0] || P[1] > L.n[1] || P[2] > L.n[2]) continue;
    const long long iP = L.idx(P[0], P[1], P[2]);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      if (P[cc] >= L.n[cc]) continue;
      const int a = (cc + 1) % 3, b = (cc + 2) % 3;
      const long long sa = L.stride(a), sb = L.stride(b);
      const long long iA = iP - sa, iB = iP - sb, iAB = iP - sa - sb;
      const R* er = A.w[cc];
      A.edge[cc][iP] = corner_emf(A.e[a][1][iB], A.e[a][1][iP], A.e[b][0][iA], A.e[b][0][iP],
                                  er[iAB], er[iB], er[iA], er[iP], A.f[a][0][iB], A.f[a][0][iP],
                                  A.f[b][0][iA], A.f[b][0][iP]);
    }
  }
}

// ------------------------------------------------------------------------
// 3. update: out = w0*A + w1*B + beta*dt*L (Eq. 8 + Eq. 12), CT (Eq. 9)
// ------------------------------------------------------------------------
// CT inputs of the three lower faces of one cell (Eq. 9): circulation of
// the corner EMFs around each face, face area, and the two register values.
template <typename R>
struct CtIn {
  R circ[3], area[3], b0[3], b1[3];
  bool on[3];
};

template <typename R, bool MHD, bool SPH>
__device__ __forceinline__ CtIn<R> ct_gather(const BlockPtrs<R>& B, const int* P, long long c,
                                             bool has_b) {
  CtIn<R> t;
  const Layout& L = B.L;
  const Geometry<R>& geo = B.geo;
  const int i = P[0], j = P[1], k = P[2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    t.on[d] = false;
    t.circ[d] = t.area[d] = t.b0[d] = t.b1[d] = R(0);
    if constexpr (MHD) {
      const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
      // faces 0..n-1, and face n on an outflow axis (across a block link
      // face n is also updated by the block above, from the same inputs,
      // and the mirror pass then copies that value)
      const int hid = L.bc[d] == AETH_BC_OUTFLOW ? L.n[d] : L.n[d] - 1;
      if (P[d] > hid || P[e1] >= L.n[e1] || P[e2] >= L.n[e2]) continue;
      t.on[d] = true;
      int Q1[3] = {i, j, k}, Q2[3] = {i, j, k};
      Q1[e1] += 1; Q2[e2] += 1;
      const long long q1 = c + L.stride(e1), q2 = c + L.stride(e2);
      if (SPH) {
        t.circ[d] = B.edge[e2][q1] * geo.edge[e2](Q1[0], Q1[1], Q1[2]) -
                    B.edge[e2][c] * geo.edge[e2](i, j, k) -
                    (B.edge[e1][q2] * geo.edge[e1](Q2[0], Q2[1], Q2[2]) -
                     B.edge[e1][c] * geo.edge[e1](i, j, k));
      } else {
        const R l2 = geo.edge[e2](0, 0, 0), l1 = geo.edge[e1](0, 0, 0);
        t.circ[d] = B.edge[e2][q1] * l2 - B.edge[e2][c] * l2 - (B.edge[e1][q2] * l1 - B.edge[e1][c] * l1);
      }
      t.area[d] = SPH ? geo.area[d](i, j, k) : geo.area[d](0, 0, 0);
      t.b0[d] = B.reg[0][5 + d][c];
      if (has_b) t.b1[d] = B.reg[1][5 + d][c];
    }
  }
  return t;
}

template <typename R, bool MHD>
__device__ __forceinline__ void ct_store(const BlockPtrs<R>& B, const int* P, long long c,
                                         R* const* outp, const CtIn<R>& t, R w0, R w1, R bdt,
                                         bool has_b) {
  if constexpr (MHD) {
    const Layout& L = B.L;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!t.on[d]) continue;
      R base = w0 * t.b0[d];
      if (has_b) base += w1 * t.b1[d];
      const R nb = base - bdt * t.circ[d] / t.area[d];
      outp[5 + d][c] = nb;
      // periodic axis: face n is the image of face 0 (across a block link
      // the mirror pass after the update writes face n from the block above)
      if (L.bc[d] == AETH_BC_PERIODIC && P[d] == 0)
        outp[5 + d][c + (long long)L.n[d] * L.stride(d)] = nb;
    }
  }
}

template <typename R, bool P64, bool MHD, bool SPH, bool DUAL = false>
__device__ __forceinline__ void update_cell(const BlockPtrs<R>& B, const int* P, int src, int out,
                                            R w0, R w1, R bdt, R gamma, R rho_floor, R p_floor,
                                            R cs2) {
  const Layout& L = B.L;
  const Geometry<R>& geo = B.geo;
  const int i = P[0], j = P[1], k = P[2];
  const long long c = L.idx(i, j, k);
  const bool has_b = w1 != R(0);
  R* const* outp = B.reg[out];
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
    R srcv[5] = {0, 0, 0, 0, 0};
    if (SPH) {
      // curvilinear momentum sources from the stress tensor (Eq. 12) of
      // the stage state
      ConstArr8<R> s;
#pragma unroll
      for (int v = 0; v < NVAR; ++v) s.p[v] = B.reg[src][v];
      R w[8];
      if (cs2 > R(0)) prim_cell<R, P64, MHD, true>(L, s, c, cs2, rho_floor, p_floor, w);
      else prim_cell<R, P64, MHD>(L, s, c, gamma - R(1), rho_floor, p_floor, w);
      const R rho = w[0], vv[3] = {w[1], w[2], w[3]};
      const R bb[3] = {w[5], w[6], w[7]};
      const R ps = w[4] + R(0.5) * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
      auto T = [&](int x, int y) {
        return rho * vv[x] * vv[y] + (x == y ? ps : R(0)) - bb[x] * bb[y];
      };
      const R ir = geo.invr(i, j, k), ct = geo.cotr(i, j, k);
      srcv[1] = (T(1, 1) + T(2, 2)) * ir;
      srcv[2] = T(2, 2) * ct - T(0, 1) * ir;
      srcv[3] = -T(2, 0) * ir - T(2, 1) * ct;
    }
    // every input of the cell is loaded before the first store: the stores
    // go through pointer arrays the compiler cannot prove disjoint from the
    // loads, so interleaving them would serialise the memory round trips
    R fm[3][5], fp[3][5], u0[5], u1[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        fp[d][v] = B.f[d][v][cp[d]];
        fm[d][v] = B.f[d][v][c];
      }
      u0[v] = B.reg[0][v][c];
      u1[v] = has_b ? B.reg[1][v][c] : R(0);
    }
    // dual energy: the entropy and its face fluxes (scratch slots 3..5)
    R sfm[3], sfp[3], s0 = R(0), s1 = R(0);
    if constexpr (DUAL) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        sfp[d] = B.w[3 + d][cp[d]];
        sfm[d] = B.w[3 + d][c];
      }
      s0 = B.ent[0][c];
      s1 = has_b ? B.ent[1][c] : R(0);
    }
    CtIn<R> ct = ct_gather<R, MHD, SPH>(B, P, c, has_b);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R div = R(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) div += Ap[d] * fp[d][v] - Am[d] * fm[d][v];
      const R rhs = -div / V + srcv[v];
      R base = w0 * u0[v];
      if (has_b) base += w1 * u1[v];
      outp[v][c] = base + bdt * rhs;
    }
    if constexpr (DUAL) {
      R div = R(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) div += Ap[d] * sfp[d] - Am[d] * sfm[d];
      R base = w0 * s0;
      if (has_b) base += w1 * s1;
      B.ent[out][c] = base + bdt * (-div / V);
    }
    ct_store<R, MHD>(B, P, c, outp, ct, w0, w1, bdt, has_b);
    return;
  }
  // cells on the upper face layer (index n along some axis) update only the
  // face field
  CtIn<R> ct = ct_gather<R, MHD, SPH>(B, P, c, has_b);
  ct_store<R, MHD>(B, P, c, outp, ct, w0, w1, bdt, has_b);
}

// COORD: 0 every block Cartesian, 1 every block spherical, 2 mixed (the
// coordinate system is then read per tile).
// cs2 > 0: the isothermal closure (the spherical sources take p = cs2 rho)
template <typename R, bool P64, bool MHD, int COORD, typename Src, bool DUAL = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? AETH_UPD_MINB : 2)
    k_update_f(Src S, int t0, int t1, int src, int out, R w0, R w1, R beta,
               const double* __restrict__ dt, R gamma, R rho_floor, R p_floor, R cs2) {
  const int add[3] = {1, 1, 1};
  const R bdt = beta * (R)(*dt);
  for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
    int loc;
    const BlockPtrs<R>& B = S.get(t, loc);
    const CellTile ct = cell_tile(B, loc, add);
    if (ct.P[0] > B.L.n[0] || ct.P[1] > B.L.n[1] || ct.P[2] > B.L.n[2]) continue;
    if (COORD == 1 || (COORD == 2 && B.L.coord == AETH_COORD_SPH))
      update_cell<R, P64, MHD, true, DUAL>(B, ct.P, src, out, w0, w1, bdt, gamma, rho_floor,
                                           p_floor, cs2);
    else
      update_cell<R, P64, MHD, false, DUAL>(B, ct.P, src, out, w0, w1, bdt, gamma, rho_floor,
                                            p_floor, cs2);
  }
}

// ------------------------------------------------------------------------
// 3'. the same update for FP32 Cartesian blocks, four consecutive x cells
// per thread: 16-byte loads and stores (the flux and corner-EMF arrays
// through the read-only path), the x-neighbour of the fourth cell as one
// scalar.  A thread's four cells sit at i = 4m .. 4m + 3, so the group is
// 16-byte aligned (interior cell 0 at x offset 4, row pitch a multiple of
// 4, every array 256-byte aligned).  Groups that reach the block's upper
// face layers (i + 3 >= n_x, j = n_y or k = n_z) take the per-cell path.
// One 32 x 4 x 2 cell tile per CTA of 64 threads.  COORD 1 (every block
// spherical) and 2 (mixed): a spherical block's groups take update4_sph,
// with the curvilinear geometry and sources.
// ------------------------------------------------------------------------
__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float at4(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

// Corner EMFs of four consecutive x cells per thread (FP32 blocks; the
// upwind corner EMF uses no geometry, so Cartesian and spherical blocks
// alike): every operand is a 16-byte load at the group's own column or a
// y / z neighbour, or, for the x-shifted operands (the b = x side of E_y,
// the a = x side of E_z), the same load shifted by one scalar from column
// i - 1.  Groups at the upper x end take the per-cell path.
__device__ __forceinline__ float4 shl(const float4& v, float s) {
  return make_float4(s, v.x, v.y, v.z);
}

template <typename Src>
__global__ void __launch_bounds__(64) k_emf_v4(Src S, int t0) {
  int loc;
  const BlockPtrs<float>& A = S.get(t0 + (int)blockIdx.x, loc);
  const Layout& L = A.L;
  const int ntx = ceil_div_d(L.n[0] + 1, CELL_BX), nty = ceil_div_d(L.n[1] + 1, CELL_BY);
  const int bx = loc % ntx, by = (loc / ntx) % nty, bz = loc / (ntx * nty);
  const int i4 = bx * CELL_BX + 4 * ((int)threadIdx.x % (CELL_BX / 4));
  const int j = by * CELL_BY + ((int)threadIdx.x / (CELL_BX / 4)) % CELL_BY;
  const int k = bz * CELL_BZ + (int)threadIdx.x / ((CELL_BX / 4) * CELL_BY);
  if (i4 > L.n[0] || j > L.n[1] || k > L.n[2]) return;
  if (i4 + 3 >= L.n[0]) {
    for (int q = 0; q < 4 && i4 + q <= L.n[0]; ++q) {
      const int P[3] = {i4 + q, j, k};
      const long long iP = L.idx(P[0], P[1], P[2]);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        if (P[cc] >= L.n[cc]) continue;
        const int a = (cc + 1) % 3, b = (cc + 2) % 3;
        const long long sa = L.stride(a), sb = L.stride(b);
        const long long iA = iP - sa, iB = iP - sb, iAB = iP - sa - sb;
        const float* er = A.w[cc];
        A.edge[cc][iP] = corner_emf(A.e[a][1][iB], A.e[a][1][iP], A.e[b][0][iA], A.e[b][0][iP],
                                    er[iAB], er[iB], er[iA], er[iP], A.f[a][0][iB],
                                    A.f[a][0][iP], A.f[b][0][iA], A.f[b][0][iP]);
      }
    }
    return;
  }
  const long long c = L.idx(i4, j, k);
  const long long sy = L.sx, sz = L.sx * L.sy;
  auto emf4 = [&](const float4& ea_m, const float4& ea_p, const float4& eb_m, const float4& eb_p,
                  const float4& r00, const float4& r01, const float4& r10, const float4& r11,
                  const float4& fa_m, const float4& fa_p, const float4& fb_m,
                  const float4& fb_p) {
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      o[q] = corner_emf(at4(ea_m, q), at4(ea_p, q), at4(eb_m, q), at4(eb_p, q), at4(r00, q),
                        at4(r01, q), at4(r10, q), at4(r11, q), at4(fa_m, q), at4(fa_p, q),
                        at4(fb_m, q), at4(fb_p, q));
    return make_float4(o[0], o[1], o[2], o[3]);
  };
  // E_x (a = y, b = z): every operand aligned
  {
    const float* er = A.w[0];
    st4(A.edge[0] + c,
        emf4(ldg4(A.e[1][1] + c - sz), ldg4(A.e[1][1] + c), ldg4(A.e[2][0] + c - sy),
             ldg4(A.e[2][0] + c), ldg4(er + c - sy - sz), ldg4(er + c - sz), ldg4(er + c - sy),
             ldg4(er + c), ldg4(A.f[1][0] + c - sz), ldg4(A.f[1][0] + c),
             ldg4(A.f[2][0] + c - sy), ldg4(A.f[2][0] + c)));
  }
  // E_y (a = z, b = x): the b side shifted by one column
  if (j < L.n[1]) {
    const float* er = A.w[1];
    const float4 ea_p = ldg4(A.e[2][1] + c), fa_p = ldg4(A.f[2][0] + c);
    const float4 ea_m = shl(ea_p, __ldg(A.e[2][1] + c - 1));
    const float4 fa_m = shl(fa_p, __ldg(A.f[2][0] + c - 1));
    const float4 rA = ldg4(er + c - sz), rP = ldg4(er + c);
    st4(A.edge[1] + c,
        emf4(ea_m, ea_p, ldg4(A.e[0][0] + c - sz), ldg4(A.e[0][0] + c),
             shl(rA, __ldg(er + c - sz - 1)), shl(rP, __ldg(er + c - 1)), rA, rP, fa_m, fa_p,
             ldg4(A.f[0][0] + c - sz), ldg4(A.f[0][0] + c)));
  }
  // E_z (a = x, b = y): the a side shifted by one column
  if (k < L.n[2]) {
    const float* er = A.w[2];
    const float4 eb_p = ldg4(A.e[1][0] + c), fb_p = ldg4(A.f[1][0] + c);
    const float4 eb_m = shl(eb_p, __ldg(A.e[1][0] + c - 1));
    const float4 fb_m = shl(fb_p, __ldg(A.f[1][0] + c - 1));
    const float4 rB = ldg4(er + c - sy), rP = ldg4(er + c);
    st4(A.edge[2] + c,
        emf4(ldg4(A.e[0][1] + c - sy), ldg4(A.e[0][1] + c), eb_m, eb_p,
             shl(rB, __ldg(er + c - sy - 1)), rB, shl(rP, __ldg(er + c - 1)), rP,
             ldg4(A.f[0][0] + c - sy), ldg4(A.f[0][0] + c), fb_m, fb_p));
  }
}

// resident CTAs per SM requested for it (its per-cell path for the face
// layers holds the most registers)
#ifndef AETH_UPD4_MINB
#define AETH_UPD4_MINB 16
#endif
// 0: the one-cell-per-thread corner-EMF pass everywhere
#ifndef AETH_EMF_V4
#define AETH_EMF_V4 1
#endif
// 0: the one-cell-per-thread update pass everywhere
#ifndef AETH_UPD_V4
#define AETH_UPD_V4 1
#endif

// The update of four consecutive x cells of a spherical block (a group
// with i + 3 < n_x, j < n_y, k < n_z): update_cell<float, P64, MHD, true>
// cell by cell, in the same expressions, with 16-byte loads and stores of
// the state, fluxes and corner EMFs, and the geometry factors of Sec. 2.3
// from their 1-D tables.  The curvilinear sources (Eq. 12) of the four
// cells are formed first, from the stage state, before any store.
template <bool P64, bool MHD>
__device__ __forceinline__ void update4_sph(const BlockPtrs<float>& B, int i4, int j, int k,
                                            int src, int out, float w0, float w1, float bdt,
                                            float gamma, float rho_floor, float p_floor,
                                            float cs2) {
  const Layout& L = B.L;
  const Geometry<float>& geo = B.geo;
  const long long c = L.idx(i4, j, k);
  const long long sy = L.sx, sz = L.sx * L.sy;
  const bool has_b = w1 != 0.0f;
  float* const* outp = B.reg[out];
  float srcv[4][3];
  {
    ConstArr8<float> s;
#pragma unroll
    for (int v = 0; v < NVAR; ++v) s.p[v] = B.reg[src][v];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float w[8];
      if (cs2 > 0.0f) prim_cell<float, P64, MHD, true>(L, s, c + q, cs2, rho_floor, p_floor, w);
      else prim_cell<float, P64, MHD>(L, s, c + q, gamma - 1.0f, rho_floor, p_floor, w);
      const float rho = w[0], vv[3] = {w[1], w[2], w[3]};
      const float bb[3] = {w[5], w[6], w[7]};
      const float ps = w[4] + 0.5f * (bb[0] * bb[0] + bb[1] * bb[1] + bb[2] * bb[2]);
      auto T = [&](int x, int y) {
        return rho * vv[x] * vv[y] + (x == y ? ps : 0.0f) - bb[x] * bb[y];
      };
      const float ir = geo.invr(i4 + q, j, k), ct = geo.cotr(i4 + q, j, k);
      srcv[q][0] = (T(1, 1) + T(2, 2)) * ir;
      srcv[q][1] = T(2, 2) * ct - T(0, 1) * ir;
      srcv[q][2] = -T(2, 0) * ir - T(2, 1) * ct;
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float4 fx = ldg4(B.f[0][v] + c);
    const float fx4 = __ldg(B.f[0][v] + c + 4);
    const float4 fy0 = ldg4(B.f[1][v] + c), fy1 = ldg4(B.f[1][v] + c + sy);
    const float4 fz0 = ldg4(B.f[2][v] + c), fz1 = ldg4(B.f[2][v] + c + sz);
    const float4 u0 = ld4(B.reg[0][v] + c);
    const float4 u1 = has_b ? ld4(B.reg[1][v] + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    float r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i4 + q;
      const float fxp = q < 3 ? at4(fx, q + 1) : fx4;
      float div = 0.0f;
      div += geo.area[0](i + 1, j, k) * fxp - geo.area[0](i, j, k) * at4(fx, q);
      div += geo.area[1](i, j + 1, k) * at4(fy1, q) - geo.area[1](i, j, k) * at4(fy0, q);
      div += geo.area[2](i, j, k + 1) * at4(fz1, q) - geo.area[2](i, j, k) * at4(fz0, q);
      const float rhs = -div / geo.vol(i, j, k) + (v >= 1 && v <= 3 ? srcv[q][v - 1] : 0.0f);
      float base = w0 * at4(u0, q);
      if (has_b) base += w1 * at4(u1, q);
      r[q] = base + bdt * rhs;
    }
    st4(outp[v] + c, make_float4(r[0], r[1], r[2], r[3]));
  }
  if constexpr (MHD) {
    // corner EMFs times edge lengths around the three lower faces (Eq. 9)
    const float4 e0c = ldg4(B.edge[0] + c), e0y = ldg4(B.edge[0] + c + sy),
                 e0z = ldg4(B.edge[0] + c + sz);
    const float4 e1c = ldg4(B.edge[1] + c), e1z = ldg4(B.edge[1] + c + sz);
    const float4 e2c = ldg4(B.edge[2] + c), e2y = ldg4(B.edge[2] + c + sy);
    const float e1x4 = __ldg(B.edge[1] + c + 4), e2x4 = __ldg(B.edge[2] + c + 4);
    float nb[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float4 b0 = ld4(B.reg[0][5 + d] + c);
      const float4 b1 = has_b ? ld4(B.reg[1][5 + d] + c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i4 + q;
        const float e1xp = q < 3 ? at4(e1c, q + 1) : e1x4;
        const float e2xp = q < 3 ? at4(e2c, q + 1) : e2x4;
        const Sep<float>& l0 = geo.edge[0];
        const Sep<float>& l1 = geo.edge[1];
        const Sep<float>& l2 = geo.edge[2];
        float circ;
        if (d == 0)
          circ = at4(e2y, q) * l2(i, j + 1, k) - at4(e2c, q) * l2(i, j, k) -
                 (at4(e1z, q) * l1(i, j, k + 1) - at4(e1c, q) * l1(i, j, k));
        else if (d == 1)
          circ = at4(e0z, q) * l0(i, j, k + 1) - at4(e0c, q) * l0(i, j, k) -
                 (e2xp * l2(i + 1, j, k) - at4(e2c, q) * l2(i, j, k));
        else
          circ = e1xp * l1(i + 1, j, k) - at4(e1c, q) * l1(i, j, k) -
                 (at4(e0y, q) * l0(i, j + 1, k) - at4(e0c, q) * l0(i, j, k));
        float base = w0 * at4(b0, q);
        if (has_b) base += w1 * at4(b1, q);
        nb[d][q] = base - bdt * circ / geo.area[d](i, j, k);
      }
      st4(outp[5 + d] + c, make_float4(nb[d][0], nb[d][1], nb[d][2], nb[d][3]));
    }
    // periodic axis: face n is the image of face 0
    if (L.bc[0] == AETH_BC_PERIODIC && i4 == 0) outp[5][c + L.n[0]] = nb[0][0];
    if (L.bc[1] == AETH_BC_PERIODIC && j == 0)
      st4(outp[6] + c + (long long)L.n[1] * sy, make_float4(nb[1][0], nb[1][1], nb[1][2], nb[1][3]));
    if (L.bc[2] == AETH_BC_PERIODIC && k == 0)
      st4(outp[7] + c + (long long)L.n[2] * sz, make_float4(nb[2][0], nb[2][1], nb[2][2], nb[2][3]));
  }
}

// resident CTAs per SM requested in contexts with spherical blocks
#ifndef AETH_UPD4_SPH_MINB
#define AETH_UPD4_SPH_MINB 12
#endif

template <bool P64, bool MHD, int COORD, typename Src>
__global__ void __launch_bounds__(64, COORD == 0 ? AETH_UPD4_MINB : AETH_UPD4_SPH_MINB)
    k_update_v4(Src S, int t0, int src, int out, float w0, float w1, float beta,
                const double* __restrict__ dt, float gamma, float rho_floor, float p_floor,
                float cs2) {
  const float bdt = beta * (float)(*dt);
  int loc;
  const BlockPtrs<float>& B = S.get(t0 + (int)blockIdx.x, loc);
  const Layout& L = B.L;
  const int ntx = ceil_div_d(L.n[0] + 1, CELL_BX), nty = ceil_div_d(L.n[1] + 1, CELL_BY);
  const int bx = loc % ntx, by = (loc / ntx) % nty, bz = loc / (ntx * nty);
  const int i4 = bx * CELL_BX + 4 * ((int)threadIdx.x % (CELL_BX / 4));
  const int j = by * CELL_BY + ((int)threadIdx.x / (CELL_BX / 4)) % CELL_BY;
  const int k = bz * CELL_BZ + (int)threadIdx.x / ((CELL_BX / 4) * CELL_BY);
  if (i4 > L.n[0] || j > L.n[1] || k > L.n[2]) return;
  const bool sph = COORD == 1 || (COORD == 2 && L.coord == AETH_COORD_SPH);
  if (i4 + 3 >= L.n[0] || j >= L.n[1] || k >= L.n[2]) {
    for (int q = 0; q < 4 && i4 + q <= L.n[0]; ++q) {
      const int P[3] = {i4 + q, j, k};
      if (sph)
        update_cell<float, P64, MHD, true>(B, P, src, out, w0, w1, bdt, gamma, rho_floor, p_floor,
                                           cs2);
      else
        update_cell<float, P64, MHD, false>(B, P, src, out, w0, w1, bdt, gamma, rho_floor,
                                            p_floor, cs2);
    }
    return;
  }
  if (sph) {
    update4_sph<P64, MHD>(B, i4, j, k, src, out, w0, w1, bdt, gamma, rho_floor, p_floor, cs2);
    return;
  }
  const long long c = L.idx(i4, j, k);
  const long long sy = L.sx, sz = L.sx * L.sy;
  const Geometry<float>& geo = B.geo;
  const float V = geo.vol(0, 0, 0);
  const float Ar[3] = {geo.area[0](0, 0, 0), geo.area[1](0, 0, 0), geo.area[2](0, 0, 0)};
  const bool has_b = w1 != 0.0f;
  float* const* outp = B.reg[out];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float4 fx = ldg4(B.f[0][v] + c);
    const float fx4 = __ldg(B.f[0][v] + c + 4);
    const float4 fy0 = ldg4(B.f[1][v] + c), fy1 = ldg4(B.f[1][v] + c + sy);
    const float4 fz0 = ldg4(B.f[2][v] + c), fz1 = ldg4(B.f[2][v] + c + sz);
    const float4 u0 = ld4(B.reg[0][v] + c);
    const float4 u1 = has_b ? ld4(B.reg[1][v] + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    float r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float fxp = q < 3 ? at4(fx, q + 1) : fx4;
      float div = 0.0f;
      div += Ar[0] * fxp - Ar[0] * at4(fx, q);
      div += Ar[1] * at4(fy1, q) - Ar[1] * at4(fy0, q);
      div += Ar[2] * at4(fz1, q) - Ar[2] * at4(fz0, q);
      float base = w0 * at4(u0, q);
      if (has_b) base += w1 * at4(u1, q);
      r[q] = base + bdt * (-div / V);
    }
    st4(outp[v] + c, make_float4(r[0], r[1], r[2], r[3]));
  }
  if constexpr (MHD) {
    // corner EMFs around the three lower faces of each cell (Eq. 9)
    const float l0 = geo.edge[0](0, 0, 0), l1 = geo.edge[1](0, 0, 0), l2 = geo.edge[2](0, 0, 0);
    const float4 e0c = ldg4(B.edge[0] + c), e0y = ldg4(B.edge[0] + c + sy),
                 e0z = ldg4(B.edge[0] + c + sz);
    const float4 e1c = ldg4(B.edge[1] + c), e1z = ldg4(B.edge[1] + c + sz);
    const float4 e2c = ldg4(B.edge[2] + c), e2y = ldg4(B.edge[2] + c + sy);
    const float e1x4 = __ldg(B.edge[1] + c + 4), e2x4 = __ldg(B.edge[2] + c + 4);
    float nb[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float4 b0 = ld4(B.reg[0][5 + d] + c);
      const float4 b1 = has_b ? ld4(B.reg[1][5 + d] + c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float e1xp = q < 3 ? at4(e1c, q + 1) : e1x4;
        const float e2xp = q < 3 ? at4(e2c, q + 1) : e2x4;
        float circ;
        if (d == 0)
          circ = at4(e2y, q) * l2 - at4(e2c, q) * l2 - (at4(e1z, q) * l1 - at4(e1c, q) * l1);
        else if (d == 1)
          circ = at4(e0z, q) * l0 - at4(e0c, q) * l0 - (e2xp * l2 - at4(e2c, q) * l2);
        else
          circ = e1xp * l1 - at4(e1c, q) * l1 - (at4(e0y, q) * l0 - at4(e0c, q) * l0);
        float base = w0 * at4(b0, q);
        if (has_b) base += w1 * at4(b1, q);
        nb[d][q] = base - bdt * circ / Ar[d];
      }
      st4(outp[5 + d] + c, make_float4(nb[d][0], nb[d][1], nb[d][2], nb[d][3]));
    }
    // periodic axis: face n is the image of face 0
    if (L.bc[0] == AETH_BC_PERIODIC && i4 == 0) outp[5][c + L.n[0]] = nb[0][0];
    if (L.bc[1] == AETH_BC_PERIODIC && j == 0)
      st4(outp[6] + c + (long long)L.n[1] * sy, make_float4(nb[1][0], nb[1][1], nb[1][2], nb[1][3]));
    if (L.bc[2] == AETH_BC_PERIODIC && k == 0)
      st4(outp[7] + c + (long long)L.n[2] * sz, make_float4(nb[2][0], nb[2][1], nb[2][2], nb[2][3]));
  }
}

// ------------------------------------------------------------------------
// Block links (Sec. 2.3): after an update, face n along the link axis of the
// block below takes the value of face 0 of the block above (both are the
// shared face; the block above's CT owns it).  blockIdx.y = link, threads
// over the face plane.
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_mirror_faces(const BlockPtrs<R>* __restrict__ tab,
                                                      const int3* __restrict__ links, int reg) {
  const int3 lk = links[blockIdx.y];   // (block below, axis, block above)
  const BlockPtrs<R>& A = tab[lk.x];
  const BlockPtrs<R>& B = tab[lk.z];
  const int d = lk.y, e1 = (d + 1) % 3, e2 = (d + 2) % 3;
  const int n1 = A.L.n[e1], n2 = A.L.n[e2];
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < (long long)n1 * n2;
       f += (long long)gridDim.x * blockDim.x) {
    int Q[3];
    Q[e1] = (int)(f % n1);
    Q[e2] = (int)(f / n1);
    Q[d] = 0;
    const R v = B.reg[reg][5 + d][B.L.idx(Q[0], Q[1], Q[2])];
    Q[d] = A.L.n[d];
    A.reg[reg][5 + d][A.L.idx(Q[0], Q[1], Q[2])] = v;
  }
}

// ------------------------------------------------------------------------
// dual-energy synchronisation of the interior cells of register `reg` at a
// stage start, before its ghost fill (Sec. 2.8): where the internal energy
// from E is below alpha_switch x (kinetic + magnetic), E is rewritten from
// the entropy, e = S rho^(gamma-1) / (gamma-1); above alpha_sync x
// (kinetic + magnetic), S is resynchronised from E; in between neither
// changes.  Each cell reads its own state and bounding faces only.
// ------------------------------------------------------------------------
template <typename R, bool MHD, typename Src>
__global__ void __launch_bounds__(256) k_dual_sync(Src S, int t0, int t1, int reg, R gm1,
                                                   R rho_floor, R a_switch, R a_sync) {
  const int add[3] = {1, 1, 1};
  for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
    int loc;
    const BlockPtrs<R>& B = S.get(t, loc);
    const CellTile ct = cell_tile(B, loc, add);
    const Layout& L = B.L;
    if (ct.P[0] >= L.n[0] || ct.P[1] >= L.n[1] || ct.P[2] >= L.n[2]) continue;
    const long long c = L.idx(ct.P[0], ct.P[1], ct.P[2]);
    R* const* u = B.reg[reg];
    R* ent = B.ent[reg];
    R rho = u[0][c];
    if (rho < rho_floor) rho = rho_floor;
    const R ir = R(1) / rho;
    const R v1 = u[1][c] * ir, v2 = u[2][c] * ir, v3 = u[3][c] * ir;
    R km = R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3);
    if (MHD) {
      const R b1 = R(0.5) * (u[5][c] + u[5][c + 1]);
      const R b2 = R(0.5) * (u[6][c] + u[6][c + L.sx]);
      const R b3 = R(0.5) * (u[7][c] + u[7][c + L.sx * L.sy]);
      km += R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3);
    }
    const R eint = u[4][c] - km;
    const R rg = pow(rho, gm1);
    if (eint < a_switch * km) u[4][c] = ent[c] * rg / gm1 + km;
    else if (eint > a_sync * km) ent[c] = gm1 * eint / rg;
  }
}

// ------------------------------------------------------------------------
// ghost fill of one register, one axis per launch (Sec. 2.3); LINKS and ENT
// compile the linked-block and entropy copies in only where the context has
// them (each costs registers in the plain fill)
// ------------------------------------------------------------------------
template <typename R, typename Src, bool LINKS, bool ENT>
__global__ void __launch_bounds__(256) k_fill_b(Src S, int t0, int t1, int reg, int nv, int d) {
  for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
    int loc;
    const BlockPtrs<R>& B = S.get(t, loc);
    const Layout L = B.L;
    const int g = L.g;
    int lo[3], ext[3];
    for (int e = 0; e < 3; ++e) {
      if (e < d) { lo[e] = -g; ext[e] = L.n[e] + 2 * g + 1; }
      else if (e == d) { lo[e] = 0; ext[e] = 2 * g + 1; }
      else { lo[e] = 0; ext[e] = L.n[e] + 1; }
    }
    // threads run linearly over the slab (x fastest): every lane busy even
    // where the slab is only 2g+1 cells thick along x
    const long long el = (long long)loc * FILL_TILE + threadIdx.x;
    if (el >= (long long)ext[0] * ext[1] * ext[2]) continue;
    const int t0c = (int)(el % ext[0]);
    const int t1c = (int)((el / ext[0]) % ext[1]);
    const int t2c = (int)(el / ((long long)ext[0] * ext[1]));
    int c[3] = {t0c + lo[0], t1c + lo[1], t2c + lo[2]};
    const int n = L.n[d];
    const int tt = c[d];
    c[d] = tt < g ? tt - g : n + (tt - g);
    const int p = c[d];
    const long long dst = L.idx(c[0], c[1], c[2]);
    // a linked side copies from the neighbouring block's cells (and faces)
    // beyond it: cells n_nb + p on the low side, p - n on the high side
    const int lk = LINKS ? L.lnk[d][p < 0 ? 0 : 1] : -1;
    const BlockPtrs<R>& SB = (lk < 0 || lk == L.self) ? B : B.tab[lk];
    // every source is loaded before the first store (the stores go through
    // pointer arrays the compiler cannot prove disjoint from the loads)
    R val[NVAR];
    bool on[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      on[v] = false;
      if (v >= nv) continue;
      const bool face_d = (v == 5 + d);
      int s;
      if (lk >= 0) {
        s = p < 0 ? SB.L.n[d] + p : p - n;
      } else if (L.bc[d] == AETH_BC_PERIODIC) {
        s = ((p % n) + n) % n;
      } else if (face_d) {
        if (p >= 0 && p <= n) continue;
        s = p < 0 ? 0 : n;
      } else {
        s = p < 0 ? 0 : n - 1;
      }
      int sc[3] = {c[0], c[1], c[2]};
      sc[d] = s;
      val[v] = SB.reg[reg][v][SB.L.idx(sc[0], sc[1], sc[2])];
      on[v] = true;
    }
#pragma unroll
    for (int v = 0; v < NVAR; ++v)
      if (on[v]) B.reg[reg][v][dst] = val[v];
    // dual energy: the entropy is a cell variable like the density
    if constexpr (ENT) {
      R* e = B.ent[reg];
      int sc[3] = {c[0], c[1], c[2]};
      if (lk >= 0) sc[d] = p < 0 ? SB.L.n[d] + p : p - n;
      else sc[d] = L.bc[d] == AETH_BC_PERIODIC ? ((p % n) + n) % n : (p < 0 ? 0 : n - 1);
      e[dst] = SB.ent[reg][SB.L.idx(sc[0], sc[1], sc[2])];
    }
  }
}

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------
template <typename R, bool LINKS, bool ENT>
static void launch_fill_axes(aeth_ctx* c, int reg, int nv, int block) {
  for (int d = 0; d < 3; ++d) {
    with_src<R>(c, PK_FILL0 + d, block, [&](auto S, TileRange r) {
      if (r.t1 <= r.t0) return;
      k_fill_b<R, decltype(S), LINKS, ENT><<<r.t1 - r.t0, 256, 0, c->stream>>>(S, r.t0, r.t1,
                                                                               reg, nv, d);
    });
  }
  c->n_launch += 3;
}

template <typename R>
static void launch_fill_all(aeth_ctx* c, int reg, int nv, int block) {
  const bool links = !c->links.empty(), ent = is_dual(c);
  if (links && ent) launch_fill_axes<R, true, true>(c, reg, nv, block);
  else if (links) launch_fill_axes<R, true, false>(c, reg, nv, block);
  else if (ent) launch_fill_axes<R, false, true>(c, reg, nv, block);
  else launch_fill_axes<R, false, false>(c, reg, nv, block);
}

template <typename R>
void mlp_flux_pass(aeth_ctx* c, int block);

template <typename R, bool P64, bool MHD>
static void flux_pass(aeth_ctx* c, int recon, int src, int block) {
  if (c->cfg.riemann == AETH_RIEMANN_MLP && c->d_mlp) {
    // learned flux: dump the face states, then the tensor-core network
    // (with HLLD fallback) solves them block by block
    flux_pass_solver<R, P64, MHD, 1>(c, recon, src, block);
    if (block >= 0) {
      mlp_flux_pass<R>(c, block);
    } else {
      for (int b = 0; b < (int)c->blocks.size(); ++b) mlp_flux_pass<R>(c, b);
    }
    return;
  }
  const bool hlle = c->cfg.riemann == AETH_RIEMANN_HLLE;
  if (is_dual(c)) {
    // dual energy: FP64 or FP32 states (the pressure of untrusted cells
    // comes from the entropy, not from an FP64 energy difference)
    if (hlle) flux_pass_solver<R, false, MHD, 2, true>(c, recon, src, block);
    else if (c->cfg.riemann == AETH_RIEMANN_LHLLD)
      flux_pass_solver<R, false, MHD, 5, true>(c, recon, src, block);
    else flux_pass_solver<R, false, MHD, 0, true>(c, recon, src, block);
    return;
  }
  if (is_iso(c)) {
    // the isothermal pressure cs^2 rho needs no FP64 energy difference
    if (hlle) flux_pass_solver<R, false, MHD, 4>(c, recon, src, block);
    else flux_pass_solver<R, false, MHD, 3>(c, recon, src, block);
  } else if (hlle) {
    flux_pass_solver<R, P64, MHD, 2>(c, recon, src, block);
  } else if (c->cfg.riemann == AETH_RIEMANN_LHLLD) {
    flux_pass_solver<R, P64, MHD, 5>(c, recon, src, block);
  } else {
    flux_pass_solver<R, P64, MHD, 0>(c, recon, src, block);
  }
}

// Algorithmic HBM bytes of one flux pass: every cell's stage state read
// once and its outputs (15 fluxes + 6 face EMFs + 3 E_ref) written once.
// The isothermal closure needs neither the energy entry nor the energy
// fluxes (the pass still writes those as zeros for the update pass); dual
// energy adds the entropy read and its three face fluxes.
static double flux_algo_bytes(const aeth_ctx* c, bool mhd) {
  double cells = 0;
  for (const auto& B : c->blocks)
    cells += (double)(B.L.n[0] + 2) * (B.L.n[1] + 2) * (B.L.n[2] + 2);
  const int e = is_iso(c) ? 1 : 0, s = is_dual(c) ? 1 : 0;
  return cells * ((mhd ? 8 : 5) - e + s + (mhd ? 24 : 15) - 3 * e + 3 * s) * (double)c->elem;
}

template <typename R, bool P64, bool MHD>
static void stage_fused(aeth_ctx* c, int recon, int src, R w0, R w1, R beta, int out) {
  const bool dual = !P64 && is_dual(c);   // dual energy runs FP64 or FP32 states
  if (dual) {
    with_src<R>(c, PK_CELL, -1, [&](auto S, TileRange r) {
      k_dual_sync<R, MHD><<<r.t1 - r.t0, 256, 0, c->stream>>>(
          S, r.t0, r.t1, src, (R)(c->cfg.gamma - 1.0), (R)c->cfg.rho_floor,
          (R)c->cfg.alpha_switch, (R)c->cfg.alpha_sync);
    });
    c->n_launch += 1;
  }
  launch_fill_all<R>(c, src, MHD ? NVAR : 5, -1);
  prof_begin(c);
  flux_pass<R, P64, MHD>(c, recon, src, -1);
  prof_end(c, flux_algo_bytes(c, MHD));
  int nsph = 0;
  for (const auto& B : c->blocks) nsph += B.L.coord == AETH_COORD_SPH;
  const int mode = nsph == 0 ? 0 : (nsph == (int)c->blocks.size() ? 1 : 2);
  with_src<R>(c, PK_CELL, -1, [&](auto S, TileRange r) {
    bool emf_done = false;
    if constexpr (sizeof(R) == 4) {
      if (MHD && AETH_EMF_V4) {   // geometry-free: every block
        k_emf_v4<<<r.t1 - r.t0, (CELL_BX / 4) * CELL_BY * CELL_BZ, 0, c->stream>>>(S, r.t0);
        emf_done = true;
      }
    }
    if (MHD && !emf_done) k_emf_ref<R><<<r.t1 - r.t0, 256, 0, c->stream>>>(S, r.t0, r.t1);
    const R g = (R)c->cfg.gamma, rf = (R)c->cfg.rho_floor, pf = (R)c->cfg.p_floor;
    const R cs2 = is_iso(c) ? (R)(c->cfg.cs_iso * c->cfg.cs_iso) : R(0);
    const int n = r.t1 - r.t0;
    using Src = decltype(S);
    auto upd = [&](auto kernel) {
      kernel<<<n, 256, 0, c->stream>>>(S, r.t0, r.t1, src, out, w0, w1, beta, c->d_dt, g, rf, pf,
                                       cs2);
    };
    if constexpr (!P64) {
      if (dual) {
        if (mode == 0) upd(k_update_f<R, P64, MHD, 0, Src, true>);
        else if (mode == 1) upd(k_update_f<R, P64, MHD, 1, Src, true>);
        else upd(k_update_f<R, P64, MHD, 2, Src, true>);
        return;
      }
    }
    if constexpr (sizeof(R) == 4) {
      if (AETH_UPD_V4) {
        // FP32: four x cells per thread, one tile per CTA (Cartesian and
        // spherical groups; the groups at the upper face layers per cell)
        auto v4 = [&](auto kernel) {
          kernel<<<n, (CELL_BX / 4) * CELL_BY * CELL_BZ, 0, c->stream>>>(
              S, r.t0, src, out, (float)w0, (float)w1, (float)beta, c->d_dt, (float)g,
              (float)rf, (float)pf, (float)cs2);
        };
        if (mode == 0) v4(k_update_v4<P64, MHD, 0, Src>);
        else if (mode == 1) v4(k_update_v4<P64, MHD, 1, Src>);
        else v4(k_update_v4<P64, MHD, 2, Src>);
        return;
      }
    }
    if (mode == 0) upd(k_update_f<R, P64, MHD, 0, Src>);
    else if (mode == 1) upd(k_update_f<R, P64, MHD, 1, Src>);
    else upd(k_update_f<R, P64, MHD, 2, Src>);
  });
  if (MHD && !c->links.empty()) {
    k_mirror_faces<R><<<dim3(64, (unsigned)c->links.size()), 256, 0, c->stream>>>(
        dtab<R>(c), c->d_links, out);
    c->n_launch += 1;
  }
  c->n_launch += MHD ? 2 : 1;
}

template <typename R, bool P64, bool MHD>
static aeth_status step_fused_T(aeth_ctx* c) {
  const int recon = c->cfg.recon;
  if (c->cfg.riemann == AETH_RIEMANN_MLP && !c->d_mlp)
    return fail(c, AETH_ERR_STATE, "learned flux selected: call aeth_load_mlp first");
  if (c->cfg.integrator == AETH_INT_VL2) {
    // predictor: U^{n+1/2} = U^n - dt/2 L_donor(U^n)   (register A -> B)
    stage_fused<R, P64, MHD>(c, AETH_RECON_DONOR, 0, R(1), R(0), R(0.5), 1);
    // corrector: U^{n+1} = U^n - dt L(U^{n+1/2})         (B -> A, in place)
    stage_fused<R, P64, MHD>(c, recon, 1, R(1), R(0), R(1), 0);
  } else if (c->cfg.integrator == AETH_INT_RK2) {
    stage_fused<R, P64, MHD>(c, recon, 0, R(1), R(0), R(1), 1);
    stage_fused<R, P64, MHD>(c, recon, 1, R(0.5), R(0.5), R(0.5), 0);
  } else if (c->cfg.integrator == AETH_INT_RK3) {
    // SSP-RK3 in two registers: B = A + dt L(A); B = 3/4 A + 1/4 B +
    // 1/4 dt L(B) (in place: every cell reads only its own A and B);
    // A = 1/3 A + 2/3 B + 2/3 dt L(B)
    stage_fused<R, P64, MHD>(c, recon, 0, R(1), R(0), R(1), 1);
    stage_fused<R, P64, MHD>(c, recon, 1, R(0.75), R(0.25), R(0.25), 1);
    stage_fused<R, P64, MHD>(c, recon, 1, R(1.0 / 3.0), R(2.0 / 3.0), R(2.0 / 3.0), 0);
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

// Hydro-gas flux pass of one block for other integrators (dust runs).
template <typename R, bool P64>
void hydro_flux_pass(aeth_ctx* c, int block, int recon, int src) {
  flux_pass<R, P64, false>(c, recon, src, block);
}
template void hydro_flux_pass<float, false>(aeth_ctx*, int, int, int);
template void hydro_flux_pass<float, true>(aeth_ctx*, int, int, int);
template void hydro_flux_pass<double, false>(aeth_ctx*, int, int, int);

}  // namespace aeth
