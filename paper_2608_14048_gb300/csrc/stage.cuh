// Per-cell helpers shared by the stage kernels (fused flux pass, learned
// flux): primitive recovery and stencil reconstruction.
#pragma once
#include "runtime.hpp"

namespace aeth {

// Primitive variables of cell (i,j,k) (Eq. 5 with the floors of Sec. 2.1):
// w = (rho, v1, v2, v3, p, Bc1, Bc2, Bc3).  Returns the number of floors hit.
// ISO: isothermal closure, p = gm1 * rho with gm1 holding cs^2 (the energy
// entry is not read and no pressure floor applies).
template <typename R, bool P64, bool MHD, bool ISO = false>
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
  if (ISO) {
    pr = gm1 * rho;
  } else if (P64) {
    // FP64 subtraction of Eq. 5 in every cell, or (p64_ratio > 0) only where
    // the FP32 one would cancel: kinetic + magnetic > ratio x internal
    bool wide = true;
    if (L.p64_ratio > 0.0f) {
      const R ke = R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3);
      const R me = R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3);
      const R ei = u.p[4][c] - ke - me;
      wide = ke + me > (R)L.p64_ratio * ei;
      pr = gm1 * ei;
    }
    if (wide) {
      const double m1 = u.p[1][c], m2 = u.p[2][c], m3 = u.p[3][c];
      const double ke = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / (double)rho;
      const double me = 0.5 * ((double)b1 * b1 + (double)b2 * b2 + (double)b3 * b3);
      pr = (R)((double)gm1 * ((double)u.p[4][c] - ke - me));
    }
  } else {
    pr = gm1 * (u.p[4][c] - R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3) -
                R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3));
  }
  if (!ISO && pr < p_floor) { pr = p_floor; ++hits; }
  w[0] = rho; w[1] = v1; w[2] = v2; w[3] = v3; w[4] = pr; w[5] = b1; w[6] = b2; w[7] = b3;
  return hits;
}

// Same, with the 8 state arrays at base + v * pitch.
template <typename R, bool P64, bool MHD, bool ISO = false>
__device__ __forceinline__ int prim_cell_s(const Layout& L, const R* __restrict__ base,
                                           long long pitch, long long c, R gm1, R rho_floor,
                                           R p_floor, R* w) {
  ConstArr8<R> u;
#pragma unroll
  for (int v = 0; v < NVAR; ++v) u.p[v] = base + v * pitch;
  return prim_cell<R, P64, MHD, ISO>(L, u, c, gm1, rho_floor, p_floor, w);
}

// Dual energy (Sec. 2.8): the primitives of cell c with the pressure from
// the entropy S = ent[c] where the internal energy from E is below
// alpha_switch times the kinetic plus magnetic energy, else from E; the
// floors of Eq. 5; sp = S / rho, the specific entropy the faces
// reconstruct.
template <typename R, bool MHD>
__device__ __forceinline__ int prim_cell_dual(const Layout& L, const R* __restrict__ base,
                                              long long pitch, const R* __restrict__ ent,
                                              long long c, R gm1, R rho_floor, R p_floor,
                                              R alpha_switch, R* w, R& sp) {
  int hits = 0;
  const R* u0 = base;
  R rho = u0[c];
  if (rho < rho_floor) { rho = rho_floor; ++hits; }
  const R ir = R(1) / rho;
  const R v1 = u0[pitch + c] * ir, v2 = u0[2 * pitch + c] * ir, v3 = u0[3 * pitch + c] * ir;
  R b1 = 0, b2 = 0, b3 = 0;
  if (MHD) {
    b1 = R(0.5) * (u0[5 * pitch + c] + u0[5 * pitch + c + 1]);
    b2 = R(0.5) * (u0[6 * pitch + c] + u0[6 * pitch + c + L.sx]);
    b3 = R(0.5) * (u0[7 * pitch + c] + u0[7 * pitch + c + L.sx * L.sy]);
  }
  // the internal energy in the same arithmetic as prim_cell, so that a run
  // whose cells all trust E reproduces the plain run bit for bit
  const R ke = R(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3);
  const R me = R(0.5) * (b1 * b1 + b2 * b2 + b3 * b3);
  const R eint = u0[4 * pitch + c] - ke - me;
  const R S = ent[c];
  R pr = eint < alpha_switch * (ke + me) ? S * pow(rho, gm1) : gm1 * eint;
  if (pr < p_floor) { pr = p_floor; ++hits; }
  w[0] = rho; w[1] = v1; w[2] = v2; w[3] = v3; w[4] = pr; w[5] = b1; w[6] = b2; w[7] = b3;
  sp = S * ir;
  return hits;
}

__device__ __forceinline__ bool in_prim_range(const Layout& L, int i, int j, int k) {
  return i >= -L.g && i < L.n[0] + L.g && j >= -L.g && j < L.n[1] + L.g && k >= -L.g &&
         k < L.n[2] + L.g;
}

// Reconstruct face states of one variable from a stencil with stride.
template <int RECON, typename R, typename Get>
__device__ __forceinline__ void recon_var(Get get, R& wl, R& wr) {
  constexpr int RH = recon_reach<RECON>(), RL = RH + 1;
  R s[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int off = t - 3;   // cell offset from the face's right cell
    s[t] = (off >= -RL && off <= RH) ? get(off) : R(0);
  }
  recon_face<RECON>(s, wl, wr);
}

}  // namespace aeth
