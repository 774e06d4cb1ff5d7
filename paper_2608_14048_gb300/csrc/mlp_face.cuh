// Face features, output scaling and the acceptance test of the learned
// Riemann flux, shared by the mma.sync and the tcgen05 network kernels.
#pragma once

#include "common.cuh"

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
  x[0] = (float)wl[1] * ic;  x[1] = (float)wl[2] * ic;  x[2] = (float)wl[3] * ic;
  x[3] = (float)wl[4] * ip;  x[4] = (float)wl[5] * ib;  x[5] = (float)wl[6] * ib;
  x[6] = (float)wr[0] / s.rho;
  x[7] = (float)wr[1] * ic;  x[8] = (float)wr[2] * ic;  x[9] = (float)wr[3] * ic;
  x[10] = (float)wr[4] * ip; x[11] = (float)wr[5] * ib; x[12] = (float)wr[6] * ib;
  x[13] = (float)bn * ib;
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

// Accept the network's flux if it lies within tau of the HLL dissipation
// bracket around HLLE (plus a small absolute floor), and the intermediate
// states it implies in the HLL fan keep rho > 0 and p > 0.
template <typename R>
__device__ __forceinline__ bool mlp_accept(R gamma, const R* wl, const R* wr, R bn, const R* F,
                                           const float* scale, R tau) {
  R ul[7], fl[7], ur[7], fr[7];
  side_uf(gamma, wl, bn, ul, fl);
  side_uf(gamma, wr, bn, ur, fr);
  const R cl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  const R cr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  const R cm = fmax(cl, cr);
  const R sl = fmin(wl[1], wr[1]) - cm, sr = fmax(wl[1], wr[1]) + cm;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    R fh;
    if (sl >= R(0)) fh = fl[q];
    else if (sr <= R(0)) fh = fr[q];
    else fh = (sr * fl[q] - sl * fr[q] + sl * sr * (ur[q] - ul[q])) / (sr - sl);
    const R tol = tau * (sr - sl) * fabs(ur[q] - ul[q]) + R(2e-2) * (R)scale[q];
    if (!(fabs(F[q] - fh) <= tol)) return false;
  }
  if (sl < R(0)) {
    R us[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) us[q] = ul[q] - (F[q] - fl[q]) / sl;
    if (!state_ok(gamma, us, bn)) return false;
  }
  if (sr > R(0)) {
    R us[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) us[q] = ur[q] - (F[q] - fr[q]) / sr;
    if (!state_ok(gamma, us, bn)) return false;
  }
  return true;
}

}  // namespace aeth
