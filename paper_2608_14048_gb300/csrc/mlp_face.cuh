// Face features, output scaling, training targets, flux composition and
// the acceptance test of the learned Riemann flux, shared by the sample
// kernel and the mma.sync and tcgen05 network kernels.
#pragma once

#include "common.cuh"

// norm of the scaled jump in J: 0 = max over components, 2 = Euclidean
#ifndef AETH_MLP_JNORM
#define AETH_MLP_JNORM 2
#endif

namespace aeth {

// ------------------------------------------------------------------------
// features and output scaling (face frame, as the HLLD solver)
// ------------------------------------------------------------------------
struct FaceScale {
  float rho, c, sq;   // rho_L, c_ref, sqrt(rho_L)
};

template <typename R>
__device__ __forceinline__ R fast_speed_mlp(R gamma, R rho, R p, R bn, R b1, R b2) {
  return fast_speed(gamma, rho, p, bn, b1, b2);
}

template <typename R>
__device__ __forceinline__ FaceScale mlp_features(const R* wl, const R* wr, R bn, R gamma,
                                                  float* x) {
  const R cl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  const R cr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  FaceScale s;
  s.rho = (float)wl[0];
  s.c = (float)fmax(cl, cr);
  s.sq = sqrtf(s.rho);
  const float ic = 1.0f / s.c, ip = 1.0f / (s.rho * s.c * s.c), ib = 1.0f / (s.sq * s.c);
  // the left state (rho_L = 1 dropped) and the normal field
  x[0] = (float)wl[1] * ic;  x[1] = (float)wl[2] * ic;  x[2] = (float)wl[3] * ic;
  x[3] = (float)wl[4] * ip;  x[4] = (float)wl[5] * ib;  x[5] = (float)wl[6] * ib;
  x[6] = (float)bn * ib;
  // the jump W_R - W_L on the same scales: its direction d = dW / |dW| at
  // full resolution whatever the jump size (BF16 inputs would lose a jump
  // below 2^-9 of the state if the two states came separately), with the
  // size in the length, x = d (1 + |dW|)
  const float sc7[7] = {1.0f / s.rho, ic, ic, ic, ip, ib, ib};
  float dw[7], m2 = 0.0f;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    dw[q] = (float)(wr[q] - wl[q]) * sc7[q];
    m2 += dw[q] * dw[q];
  }
  const float m = sqrtf(m2);
  const float f = m > 0.0f ? (1.0f + m) / m : 0.0f;
#pragma unroll
  for (int q = 0; q < 7; ++q) x[7 + q] = dw[q] * f;
  x[14] = 0.0f; x[15] = 0.0f;
  return s;
}

// Scale of each flux: rho c | rho c^2 (x3) | rho c^3 gamma/(gamma-1) |
// sqrt(rho) c^2 (x2).  The energy flux carries the internal energy
// p/(gamma-1), so its natural size grows as gamma -> 1.
__device__ __forceinline__ void mlp_scale_out(const FaceScale& s, float gamma, float* k) {
  const float c2 = s.c * s.c;
  k[0] = s.rho * s.c;
  k[1] = k[2] = k[3] = s.rho * c2;
  k[4] = s.rho * c2 * s.c * gamma / (gamma - 1.0f);
  k[5] = k[6] = s.sq * c2;
}

// Conserved vector and physical flux of one face-frame state.
template <typename R>
__device__ __forceinline__ void side_uf(R gamma, const R* w, R bn, R* u, R* f) {
  const R rho = w[0], vn = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[5], b2 = w[6];
  const R bb = bn * bn + b1 * b1 + b2 * b2;
  const R pt = p + R(0.5) * bb;
  const R e = p / (gamma - R(1)) + R(0.5) * rho * (vn * vn + v1 * v1 + v2 * v2) + R(0.5) * bb;
  const R vb = vn * bn + v1 * b1 + v2 * b2;
  u[0] = rho; u[1] = rho * vn; u[2] = rho * v1; u[3] = rho * v2; u[4] = e; u[5] = b1; u[6] = b2;
  f[0] = rho * vn; f[1] = rho * vn * vn + pt - bn * bn; f[2] = rho * vn * v1 - bn * b1;
  f[3] = rho * vn * v2 - bn * b2; f[4] = (e + pt) * vn - bn * vb;
  f[5] = b1 * vn - bn * v1; f[6] = b2 * vn - bn * v2;
}

template <typename R>
__device__ __forceinline__ bool state_ok(R gamma, const R* u, R bn) {
  if (!(u[0] > R(0))) return false;
  const R ke = R(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
  const R me = R(0.5) * (bn * bn + u[5] * u[5] + u[6] * u[6]);
  return (gamma - R(1)) * (u[4] - ke - me) > R(0);
}

// HLLE flux and jump size of a face.  Davis speeds S_L = min(v_L, v_R) -
// c_max, S_R = max(v_L, v_R) + c_max; the HLLE flux F_E; the dimensionless
// jump J = (S_R - S_L) |dU / k| (k the flux scales; Euclidean norm over
// the 7 components by default, the smoother target for training, or the
// max norm).
// The HLL dissipation of component q is at most (S_R - S_L) |dU_q| / 4 <=
// k_q J / 4, so (F - F_E) / (k J) is O(1) for every consistent flux F.
template <typename R>
struct HllFace {
  R ul[7], fl[7], ur[7], fr[7], fe[7];
  R sl, sr, J;
};

template <typename R>
__device__ __forceinline__ void hll_face(R gamma, const R* wl, const R* wr, R bn, const float* k,
                                         HllFace<R>& h) {
  side_uf(gamma, wl, bn, h.ul, h.fl);
  side_uf(gamma, wr, bn, h.ur, h.fr);
  const R cl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  const R cr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  const R cm = fmax(cl, cr);
  h.sl = fmin(wl[1], wr[1]) - cm;
  h.sr = fmax(wl[1], wr[1]) + cm;
  R jm = R(0);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const R du = h.ur[q] - h.ul[q];
#if AETH_MLP_JNORM == 2
    jm += (du / (R)k[q]) * (du / (R)k[q]);
#else
    jm = fmax(jm, fabs(du) / (R)k[q]);
#endif
    if (h.sl >= R(0)) h.fe[q] = h.fl[q];
    else if (h.sr <= R(0)) h.fe[q] = h.fr[q];
    else h.fe[q] = (h.sr * h.fl[q] - h.sl * h.fr[q] + h.sl * h.sr * du) / (h.sr - h.sl);
  }
#if AETH_MLP_JNORM == 2
  jm = sqrt(jm);
#endif
  h.J = (h.sr - h.sl) * jm;
}

// Training target of the network: the HLLD flux fx as a correction of
// HLLE scaled by the jump, y_q = (fx_q - F_E,q) / (k_q J); zero where the
// states coincide to round-off (J < 1e-9: HLLD = HLLE there).
template <typename R>
__device__ __forceinline__ void mlp_target(R gamma, const R* wl, const R* wr, R bn, const R* fx,
                                           const float* k, float* y) {
  HllFace<R> h;
  hll_face(gamma, wl, wr, bn, k, h);
#pragma unroll
  for (int q = 0; q < 7; ++q)
    y[q] = h.J > R(1e-9) ? (float)((fx[q] - h.fe[q]) / ((R)k[q] * h.J)) : 0.0f;
}

// The learned flux F = F_E + k J y from the network output y, and its
// acceptance: F within tau of the HLL dissipation bracket around F_E (plus
// a 2e-2 k floor), and positive density and pressure in the intermediate
// states F implies in the HLL fan.  The flux is consistent by construction
// (F -> F_E -> the physical flux as the jump vanishes).  Returns false to
// reject the face (F is then undefined).
template <typename R>
__device__ __forceinline__ bool mlp_compose(R gamma, const R* wl, const R* wr, R bn, const float* y,
                                            const float* k, R tau, bool mhd, R* F) {
  HllFace<R> h;
  hll_face(gamma, wl, wr, bn, k, h);
#pragma unroll
  for (int q = 0; q < 7; ++q) F[q] = h.fe[q] + (R)k[q] * h.J * (R)y[q];
  if (!mhd) F[5] = F[6] = R(0);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const R tol = tau * (h.sr - h.sl) * fabs(h.ur[q] - h.ul[q]) + R(2e-2) * (R)k[q];
    if (!(fabs(F[q] - h.fe[q]) <= tol)) return false;
  }
  // the state between the outer wave at S and the face obeys the jump
  // condition across that wave, F - F_side = S (U* - U_side), so
  // U* = U_side + (F - F_side) / S (for F = F_E both give the HLL state)
  if (h.sl < R(0)) {
    R us[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) us[q] = h.ul[q] + (F[q] - h.fl[q]) / h.sl;
    if (!state_ok(gamma, us, bn)) return false;
  }
  if (h.sr > R(0)) {
    R us[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) us[q] = h.ur[q] + (F[q] - h.fr[q]) / h.sr;
    if (!state_ok(gamma, us, bn)) return false;
  }
  return true;
}

}  // namespace aeth
