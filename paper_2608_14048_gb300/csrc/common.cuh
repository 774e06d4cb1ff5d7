// Device-side building blocks of the GB300 MHD step: memory layout, separable
// geometry factors, reconstruction and the HLLD Riemann solver.
//
// Layout (per mesh block, per variable): a padded 3-D array with `g` ghost
// layers on every side plus one extra point per axis so that face arrays
// (n+1 faces) share the cell arrays' shape.  i is fastest; rows start at a
// 16-byte boundary (x offset OX = 4 >= g).  The 8 state variables are
// rho, M1, M2, M3, E, B1f, B2f, B3f; B_df at index (i,j,k) is the face of
// cell (i,j,k) on its lower side along axis d.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace aeth {

constexpr int OX = 4;        // x offset of interior cell 0 (alignment)
constexpr int NVAR = 8;      // 5 conserved + 3 face fields
constexpr int NPRIM = 8;     // rho, v1, v2, v3, p, Bc1, Bc2, Bc3

struct Layout {
  int n[3];        // interior cells
  int g;           // ghost width
  int bc[3];       // 0 periodic, 1 outflow
  int coord;       // 0 Cartesian, 1 spherical-polar
  long long sx, sy, sz;   // padded extents (sx multiple of 4)
  __host__ __device__ long long idx(int i, int j, int k) const {
    return ((long long)(k + g) * sy + (j + g)) * sx + (i + OX);
  }
  __host__ __device__ long long stride(int d) const {
    return d == 0 ? 1 : (d == 1 ? sx : sx * sy);
  }
  __host__ __device__ long long size() const { return sx * sy * sz; }
};

// A separable geometric factor f(i,j,k) = x[i] * y[j] * z[k]; tables are
// indexed from -g (stored with an offset of g).
template <typename R>
struct Sep {
  const R* x;
  const R* y;
  const R* z;
  int g;
  __device__ __forceinline__ R operator()(int i, int j, int k) const {
    return x[i + g] * y[j + g] * z[k + g];
  }
};

// Exact face areas, volumes, edge lengths and curvilinear source factors of
// Sec. 2.3 (evaluated from 1-D tables built in FP64 on the host).
template <typename R>
struct Geometry {
  Sep<R> area[3];   // area of the lower face of cell (i,j,k) normal to d
  Sep<R> vol;       // cell volume
  Sep<R> edge[3];   // length of the edge along d at the lower corner
  Sep<R> invr;      // <1/r>        = (A_r+ - A_r-) / (2V)
  Sep<R> cotr;      // <cot(th)/r>  = (A_th+ - A_th-) / V
  Sep<R> width[3];  // physical widths at the centroid (Eq. 11)
};

template <typename R> struct Eps;
template <> struct Eps<double> { static constexpr double hlld = 1e-12; };
template <> struct Eps<float> { static constexpr float hlld = 1e-6f; };

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
template <> __device__ __forceinline__ float rsqrt_(float x) { return 1.0f / sqrtf(x); }

// ------------------------------------------------------------------------
// Reconstruction (Sec. 2.4)
// ------------------------------------------------------------------------

// van Leer (1974) harmonic-mean limited slope (undivided difference).
template <typename R>
__device__ __forceinline__ R vl_slope(R wm, R w0, R wp) {
  R dm = w0 - wm, dp = wp - w0;
  R q = dm * dp;
  return q > R(0) ? R(2) * q / (dm + dp) : R(0);
}

// Fourth-order interface value between s1 and s2, clipped to their range.
template <typename R>
__device__ __forceinline__ R ppm_iface(R s0, R s1, R s2, R s3) {
  R a = R(7.0 / 12.0) * (s1 + s2) - R(1.0 / 12.0) * (s0 + s3);
  R lo = fmin(s1, s2), hi = fmax(s1, s2);
  return fmin(fmax(a, lo), hi);
}

// Colella & Woodward (1984) parabola limiter.
template <typename R>
__device__ __forceinline__ void ppm_limit(R w, R& l, R& r) {
  if ((r - w) * (w - l) <= R(0)) {
    l = w; r = w;
  } else {
    R d = r - l, q = d * (w - R(0.5) * (l + r)), d2 = d * d * R(1.0 / 6.0);
    if (q > d2) l = R(3) * w - R(2) * r;
    else if (-d2 > q) r = R(3) * w - R(2) * l;
  }
}

// Face states from s[0..5] = cells f-3..f+2 around face f.
template <int RECON, typename R>
__device__ __forceinline__ void recon_face(const R* s, R& wl, R& wr) {
  if (RECON == 0) {
    wl = s[2]; wr = s[3];
  } else if (RECON == 1) {
    wl = s[2] + R(0.5) * vl_slope(s[1], s[2], s[3]);
    wr = s[3] - R(0.5) * vl_slope(s[2], s[3], s[4]);
  } else {
    R im = ppm_iface(s[0], s[1], s[2], s[3]);
    R i0 = ppm_iface(s[1], s[2], s[3], s[4]);
    R ip = ppm_iface(s[2], s[3], s[4], s[5]);
    R l1 = im, r1 = i0, l2 = i0, r2 = ip;
    ppm_limit(s[2], l1, r1);
    ppm_limit(s[3], l2, r2);
    wl = r1; wr = l2;
  }
}

// ------------------------------------------------------------------------
// HLLD (Miyoshi & Kusano 2005), face frame: W = (rho, vn, vt1, vt2, p, Bt1,
// Bt2), normal field bn shared by both sides.  Flux out: (rho, Mn, Mt1, Mt2,
// E, Bt1, Bt2).
// ------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ R fast_speed(R gamma, R rho, R p, R bn, R bt1, R bt2) {
  R a2 = gamma * p / rho;
  R b2 = (bn * bn + bt1 * bt1 + bt2 * bt2) / rho;
  R s = a2 + b2;
  R disc = fmax(s * s - R(4) * a2 * bn * bn / rho, R(0));
  return sqrt(R(0.5) * (s + sqrt(disc)));
}

template <typename R>
struct Side {
  R u[7];   // rho, Mn, Mt1, Mt2, E, Bt1, Bt2
  R f[7];
  R pt;
};

template <typename R>
__device__ __forceinline__ void side_state(R gamma, const R* w, R bn, Side<R>& s) {
  R rho = w[0], vn = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[5], b2 = w[6];
  R bb = bn * bn + b1 * b1 + b2 * b2;
  R pt = p + R(0.5) * bb;
  R e = p / (gamma - R(1)) + R(0.5) * rho * (vn * vn + v1 * v1 + v2 * v2) + R(0.5) * bb;
  R vb = vn * bn + v1 * b1 + v2 * b2;
  s.u[0] = rho; s.u[1] = rho * vn; s.u[2] = rho * v1; s.u[3] = rho * v2;
  s.u[4] = e; s.u[5] = b1; s.u[6] = b2;
  s.f[0] = rho * vn;
  s.f[1] = rho * vn * vn + pt - bn * bn;
  s.f[2] = rho * vn * v1 - bn * b1;
  s.f[3] = rho * vn * v2 - bn * b2;
  s.f[4] = (e + pt) * vn - bn * vb;
  s.f[5] = b1 * vn - bn * v1;
  s.f[6] = b2 * vn - bn * v2;
  s.pt = pt;
}

template <typename R>
__device__ void hlld(R gamma, const R* wl, const R* wr, R bn, R* flux) {
  Side<R> L, Rt;
  side_state(gamma, wl, bn, L);
  side_state(gamma, wr, bn, Rt);
  R cfl = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  R cfr = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  R cmax = fmax(cfl, cfr);
  R sl = fmin(wl[1], wr[1]) - cmax;
  R sr = fmax(wl[1], wr[1]) + cmax;
  if (sl > R(0)) {
#pragma unroll
    for (int q = 0; q < 7; ++q) flux[q] = L.f[q];
    return;
  }
  if (sr < R(0)) {
#pragma unroll
    for (int q = 0; q < 7; ++q) flux[q] = Rt.f[q];
    return;
  }
  R sul = sl - wl[1], sur = sr - wr[1];
  R den = sur * wr[0] - sul * wl[0];
  R sm = (sur * wr[0] * wr[1] - sul * wl[0] * wl[1] - Rt.pt + L.pt) / den;
  R pts = (sur * wr[0] * L.pt - sul * wl[0] * Rt.pt +
           wl[0] * wr[0] * sur * sul * (wr[1] - wl[1])) / den;

  // single-star states of both sides
  R us[2][7], vs1[2], vs2[2];
  R rs[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const R* w = a ? wr : wl;
    const Side<R>& S = a ? Rt : L;
    R sa = a ? sr : sl;
    R su = sa - w[1];
    R rho_s = w[0] * su / (sa - sm);
    R dd = w[0] * su * (sa - sm) - bn * bn;
    R v1s, v2s, b1s, b2s;
    if (fabs(dd) < Eps<R>::hlld * pts) {
      v1s = w[2]; v2s = w[3]; b1s = w[5]; b2s = w[6];
    } else {
      R fv = bn * (sm - w[1]) / dd;
      R fb = (w[0] * su * su - bn * bn) / dd;
      v1s = w[2] - w[5] * fv;
      v2s = w[3] - w[6] * fv;
      b1s = w[5] * fb;
      b2s = w[6] * fb;
    }
    R vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    R vbs = sm * bn + v1s * b1s + v2s * b2s;
    R es = (su * S.u[4] - S.pt * w[1] + pts * sm + bn * (vb - vbs)) / (sa - sm);
    us[a][0] = rho_s; us[a][1] = rho_s * sm; us[a][2] = rho_s * v1s;
    us[a][3] = rho_s * v2s; us[a][4] = es; us[a][5] = b1s; us[a][6] = b2s;
    rs[a] = rho_s; vs1[a] = v1s; vs2[a] = v2s;
  }
  R sql = sqrt(rs[0]), sqr = sqrt(rs[1]);
  R abn = fabs(bn);
  bool degen = R(0.5) * bn * bn < Eps<R>::hlld * pts;
  R ssl = degen ? sm : sm - abn / sql;
  R ssr = degen ? sm : sm + abn / sqr;

  int region;
  if (ssl >= R(0)) region = 1;
  else if (sm >= R(0)) region = 2;
  else if (ssr >= R(0)) region = 3;
  else region = 4;

  const int a = (region == 1 || region == 2) ? 0 : 1;
  const Side<R>& S = a ? Rt : L;
  const R sa = a ? sr : sl;
  if (region == 1 || region == 4) {
#pragma unroll
    for (int q = 0; q < 7; ++q) flux[q] = S.f[q] + sa * (us[a][q] - S.u[q]);
    return;
  }
  R sgn = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0));
  R inv = R(1) / (sql + sqr);
  R b1l = us[0][5], b2l = us[0][6], b1r = us[1][5], b2r = us[1][6];
  R v1ss = (sql * vs1[0] + sqr * vs1[1] + (b1r - b1l) * sgn) * inv;
  R v2ss = (sql * vs2[0] + sqr * vs2[1] + (b2r - b2l) * sgn) * inv;
  R b1ss = (sql * b1r + sqr * b1l + sql * sqr * (vs1[1] - vs1[0]) * sgn) * inv;
  R b2ss = (sql * b2r + sqr * b2l + sql * sqr * (vs2[1] - vs2[0]) * sgn) * inv;
  R vbss = sm * bn + v1ss * b1ss + v2ss * b2ss;
  R sq = a ? sqr : sql;
  R vbs = sm * bn + vs1[a] * us[a][5] + vs2[a] * us[a][6];
  R side_sign = a ? R(1) : R(-1);
  R ess = us[a][4] + side_sign * sq * (vbs - vbss) * sgn;
  R uss[7] = {rs[a], rs[a] * sm, rs[a] * v1ss, rs[a] * v2ss, ess, b1ss, b2ss};
  R sst = a ? ssr : ssl;
#pragma unroll
  for (int q = 0; q < 7; ++q)
    flux[q] = S.f[q] + sa * (us[a][q] - S.u[q]) + sst * (uss[q] - us[a][q]);
}

// Upwind selection of Gardiner & Stone (2005): lower-index value for a
// positive mass flux, upper for negative, mean for zero.
template <typename R>
__device__ __forceinline__ R upwind(R mflux, R lower, R upper) {
  return mflux > R(0) ? lower : (mflux < R(0) ? upper : R(0.5) * (lower + upper));
}

// Corner EMF at one edge (Sec. 2.5).  ea_m/ea_p: a-face EMFs at rows b-1/b;
// eb_m/eb_p: b-face EMFs at columns a-1/a; r[row][col] cell references;
// fa_*, fb_*: mass fluxes of those faces.
template <typename R>
__device__ __forceinline__ R corner_emf(R ea_m, R ea_p, R eb_m, R eb_p, R r00, R r01,
                                        R r10, R r11, R fa_m, R fa_p, R fb_m, R fb_p) {
  R db_hi = upwind(fa_p, r10 - eb_m, r11 - eb_p);
  R db_lo = upwind(fa_m, eb_m - r00, eb_p - r01);
  R da_hi = upwind(fb_p, r01 - ea_m, r11 - ea_p);
  R da_lo = upwind(fb_m, ea_m - r00, ea_p - r10);
  return R(0.25) * (ea_m + ea_p + eb_m + eb_p) + R(0.25) * (db_lo - db_hi) +
         R(0.25) * (da_lo - da_hi);
}

template <typename R>
struct Arr8 {
  R* p[NVAR];
};

template <typename R>
struct ConstArr8 {
  const R* p[NVAR];
};

}  // namespace aeth
