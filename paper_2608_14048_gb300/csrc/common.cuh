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
  int self;        // this block's index in its context
  int lnk[3][2];   // per axis, low / high side: the block whose cells lie
                   // beyond that side (its ghost cells are copied from
                   // there and the side's bc is not used), or -1
  float p64_ratio; // FP32 states with the FP64 pressure recovery: 0 = in
                   // every cell; > 0 = only where kinetic + magnetic energy
                   // exceeds p64_ratio x the internal energy (FP32 estimate)
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

// PPM5 (Sec. 2.4): interface values of a cell from the quartic through the
// five cell averages q[0..4] centred on it (upwind-biased toward the cell):
// at its upper face (right) and its lower face (left).
template <typename R>
__device__ __forceinline__ R ppm5_right(const R* q) {
  return (R(2) * q[0] - R(13) * q[1] + R(47) * q[2] + R(27) * q[3] - R(3) * q[4]) *
         R(1.0 / 60.0);
}
template <typename R>
__device__ __forceinline__ R ppm5_left(const R* q) {
  return (R(-3) * q[0] + R(27) * q[1] + R(47) * q[2] - R(13) * q[3] + R(2) * q[4]) *
         R(1.0 / 60.0);
}
template <typename R>
__device__ __forceinline__ R clip_pair(R a, R u0, R u1) {
  return fmin(fmax(a, fmin(u0, u1)), fmax(u0, u1));
}

// Cells a reconstruction reads on each side of a face beyond its two
// adjacent cells: donor 0, PLM 1, PPM and PPM5 2.
template <int RECON>
__host__ __device__ constexpr int recon_reach() { return RECON == 3 ? 2 : RECON; }

// Face states from s[0..5] = cells f-3..f+2 around face f.  RECON: 0 donor,
// 1 PLM, 2 PPM, 3 PPM5.
template <int RECON, typename R>
__device__ __forceinline__ void recon_face(const R* s, R& wl, R& wr) {
  if (RECON == 0) {
    wl = s[2]; wr = s[3];
  } else if (RECON == 1) {
    wl = s[2] + R(0.5) * vl_slope(s[1], s[2], s[3]);
    wr = s[3] - R(0.5) * vl_slope(s[2], s[3], s[4]);
  } else if (RECON == 3) {
    // each interface value clipped into its face's neighbour range, then
    // the CW84 parabola limiter as in PPM
    R l1 = clip_pair(ppm5_left(s), s[1], s[2]), r1 = clip_pair(ppm5_right(s), s[2], s[3]);
    R l2 = clip_pair(ppm5_left(s + 1), s[2], s[3]), r2 = clip_pair(ppm5_right(s + 1), s[3], s[4]);
    ppm_limit(s[2], l1, r1);
    ppm_limit(s[3], l2, r2);
    wl = r1; wr = l2;
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
  // one reciprocal of rho for the three quotients
  const R ir = R(1) / rho;
  const R a2 = gamma * p * ir;
  const R b2 = (bn * bn + bt1 * bt1 + bt2 * bt2) * ir;
  const R s = a2 + b2;
  const R disc = fmax(s * s - R(4) * a2 * bn * bn * ir, R(0));
  return sqrt(R(0.5) * (s + sqrt(disc)));
}

// Single-star state of one side (MK05): density, transverse velocity and
// field, total energy, from the side state and S_M, p_T*.
template <typename R>
__device__ __forceinline__ void hlld_star(R rho, R un, R v1, R v2, R b1, R b2, R e, R pt,
                                          R sa, R sm, R pts, R bn, R& rs, R& v1s, R& v2s,
                                          R& b1s, R& b2s, R& es) {
  const R su = sa - un;
  const R inv_ssm = R(1) / (sa - sm);
  rs = rho * su * inv_ssm;
  const R dd = rho * su * (sa - sm) - bn * bn;
  if (fabs(dd) < Eps<R>::hlld * pts) {
    v1s = v1; v2s = v2; b1s = b1; b2s = b2;
  } else {
    const R inv_dd = R(1) / dd;
    const R fv = bn * (sm - un) * inv_dd;
    const R fb = (rho * su * su - bn * bn) * inv_dd;
    v1s = v1 - b1 * fv;
    v2s = v2 - b2 * fv;
    b1s = b1 * fb;
    b2s = b2 * fb;
  }
  const R vb = un * bn + v1 * b1 + v2 * b2;
  const R vbs = sm * bn + v1s * b1s + v2s * b2s;
  es = (su * e - pt * un + pts * sm + bn * (vb - vbs)) * inv_ssm;
}

// HLLD flux.  Left/right states as scalars; all intermediate values stay in
// registers (no runtime-indexed arrays).  Returns the solver region
// 0..5 (L, *L, **L, **R, *R, R).
// LD: the low-dissipation variant LHLLD (Sec. 2.4, after Minoshima & Miyoshi
// 2021): HLLD's star total pressure is a weighted average of p_TL, p_TR plus
// D = rho_L rho_R (S_R - u_R)(S_L - u_L)(u_R - u_L) / den, the pressure
// dissipation that scales with the sound speed; inside the fan the flux
// carries D in the normal momentum and S_M D in the energy, and LHLLD
// scales both by phi = min(1, max(|v_L|, |v_R|) / max(c_f,L, c_f,R)).
template <bool LD = false, typename R>
__device__ __forceinline__ int hlld_s(R gamma, R rl, R ul, R vl, R wl, R pl, R byl, R bzl,
                                      R rr, R ur, R vr, R wr, R pr, R byr, R bzr, R bn,
                                      R* f) {
  // internal energies p / (gamma - 1): FP64 shares one division (a long
  // instruction sequence at the FP64 rate); FP32 keeps the single
  // approximate division, whose rounding the learned flux's engines rely on
  R eil, eir;
  if constexpr (sizeof(R) == 8) {
    const R igm1 = R(1) / (gamma - R(1));
    eil = pl * igm1;
    eir = pr * igm1;
  } else {
    const R gm1 = gamma - R(1);
    eil = pl / gm1;
    eir = pr / gm1;
  }
  const R bb_l = bn * bn + byl * byl + bzl * bzl;
  const R bb_r = bn * bn + byr * byr + bzr * bzr;
  const R ptl = pl + R(0.5) * bb_l, ptr = pr + R(0.5) * bb_r;
  const R el = eil + R(0.5) * rl * (ul * ul + vl * vl + wl * wl) + R(0.5) * bb_l;
  const R er = eir + R(0.5) * rr * (ur * ur + vr * vr + wr * wr) + R(0.5) * bb_r;
  // physical fluxes
  const R vbl = ul * bn + vl * byl + wl * bzl, vbr = ur * bn + vr * byr + wr * bzr;
  const R fl0 = rl * ul, fr0 = rr * ur;
  const R fl1 = rl * ul * ul + ptl - bn * bn, fr1 = rr * ur * ur + ptr - bn * bn;
  const R fl2 = rl * ul * vl - bn * byl, fr2 = rr * ur * vr - bn * byr;
  const R fl3 = rl * ul * wl - bn * bzl, fr3 = rr * ur * wr - bn * bzr;
  const R fl4 = (el + ptl) * ul - bn * vbl, fr4 = (er + ptr) * ur - bn * vbr;
  const R fl5 = byl * ul - bn * vl, fr5 = byr * ur - bn * vr;
  const R fl6 = bzl * ul - bn * wl, fr6 = bzr * ur - bn * wr;
  // fast speeds and outer waves
  const R cfl = fast_speed(gamma, rl, pl, bn, byl, bzl);
  const R cfr = fast_speed(gamma, rr, pr, bn, byr, bzr);
  const R cmax = fmax(cfl, cfr);
  const R sl = fmin(ul, ur) - cmax;
  const R sr = fmax(ul, ur) + cmax;
  if (sl > R(0)) {
    f[0] = fl0; f[1] = fl1; f[2] = fl2; f[3] = fl3; f[4] = fl4; f[5] = fl5; f[6] = fl6;
    return 0;
  }
  if (sr < R(0)) {
    f[0] = fr0; f[1] = fr1; f[2] = fr2; f[3] = fr3; f[4] = fr4; f[5] = fr5; f[6] = fr6;
    return 5;
  }
  const R sul = sl - ul, sur = sr - ur;
  const R inv_den = R(1) / (sur * rr - sul * rl);
  const R sm = (sur * rr * ur - sul * rl * ul - ptr + ptl) * inv_den;
  const R pts = (sur * rr * ptl - sul * rl * ptr + rl * rr * sur * sul * (ur - ul)) * inv_den;
  R rsl, v1sl, v2sl, b1sl, b2sl, esl;
  R rsr, v1sr, v2sr, b1sr, b2sr, esr;
  hlld_star(rl, ul, vl, wl, byl, bzl, el, ptl, sl, sm, pts, bn, rsl, v1sl, v2sl, b1sl, b2sl, esl);
  hlld_star(rr, ur, vr, wr, byr, bzr, er, ptr, sr, sm, pts, bn, rsr, v1sr, v2sr, b1sr, b2sr, esr);
  const R abn = fabs(bn);
  const bool degen = R(0.5) * bn * bn < Eps<R>::hlld * pts;
  // one reciprocal square root gives sqrt(rho*) and |Bn| / sqrt(rho*)
  const R ql = rsqrt(rsl), qr = rsqrt(rsr);
  const R sql = rsl * ql, sqr = rsr * qr;
  const R ssl = degen ? sm : sm - abn * ql;
  const R ssr = degen ? sm : sm + abn * qr;
  int region;
  if (ssl >= R(0)) region = 1;
  else if (sm >= R(0)) region = 2;
  else if (ssr >= R(0)) region = 3;
  else region = 4;
  const bool right = region >= 3;
  // selected side: physical flux, conserved vector, outer speed, star state
  const R s_a = right ? sr : sl;
  const R F0 = right ? fr0 : fl0, F1 = right ? fr1 : fl1, F2 = right ? fr2 : fl2;
  const R F3 = right ? fr3 : fl3, F4 = right ? fr4 : fl4, F5 = right ? fr5 : fl5;
  const R F6 = right ? fr6 : fl6;
  const R rho = right ? rr : rl, un = right ? ur : ul, v1 = right ? vr : vl, v2 = right ? wr : wl;
  const R u4 = right ? er : el, b1 = right ? byr : byl, b2 = right ? bzr : bzl;
  const R rs = right ? rsr : rsl, v1s = right ? v1sr : v1sl, v2s = right ? v2sr : v2sl;
  const R b1s = right ? b1sr : b1sl, b2s = right ? b2sr : b2sl, es = right ? esr : esl;
  // F* = F + S (U* - U)
  R g0 = F0 + s_a * (rs - rho);
  R g1 = F1 + s_a * (rs * sm - rho * un);
  R g2 = F2 + s_a * (rs * v1s - rho * v1);
  R g3 = F3 + s_a * (rs * v2s - rho * v2);
  R g4 = F4 + s_a * (es - u4);
  R g5 = F5 + s_a * (b1s - b1);
  R g6 = F6 + s_a * (b2s - b2);
  if constexpr (LD) {
    const R d = rl * rr * sur * sul * (ur - ul) * inv_den;
    const R vml = sqrt(ul * ul + vl * vl + wl * wl), vmr = sqrt(ur * ur + vr * vr + wr * wr);
    const R phi = fmin(R(1), fmax(vml, vmr) / cmax);
    g1 += (phi - R(1)) * d;
    g4 += (phi - R(1)) * d * sm;
  }
  if (region == 2 || region == 3) {
    // double-star states: shared velocity and field, sqrt(rho*) weighted
    const R sgn = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0));
    const R inv = R(1) / (sql + sqr);
    const R v1ss = (sql * v1sl + sqr * v1sr + (b1sr - b1sl) * sgn) * inv;
    const R v2ss = (sql * v2sl + sqr * v2sr + (b2sr - b2sl) * sgn) * inv;
    const R b1ss = (sql * b1sr + sqr * b1sl + sql * sqr * (v1sr - v1sl) * sgn) * inv;
    const R b2ss = (sql * b2sr + sqr * b2sl + sql * sqr * (v2sr - v2sl) * sgn) * inv;
    const R vbss = sm * bn + v1ss * b1ss + v2ss * b2ss;
    const R vbs = sm * bn + v1s * b1s + v2s * b2s;
    const R sq = right ? sqr : sql;
    const R ess = es + (right ? R(1) : R(-1)) * sq * (vbs - vbss) * sgn;
    const R sst = right ? ssr : ssl;
    // F** = F* + S* (U** - U*); rho** = rho* and u** = S_M, so the mass
    // and normal-momentum entries of U** - U* vanish
    g2 += sst * (rs * v1ss - rs * v1s);
    g3 += sst * (rs * v2ss - rs * v2s);
    g4 += sst * (ess - es);
    g5 += sst * (b1ss - b1s);
    g6 += sst * (b2ss - b2s);
  }
  f[0] = g0; f[1] = g1; f[2] = g2; f[3] = g3; f[4] = g4; f[5] = g5; f[6] = g6;
  return region;
}

// Array form: W = (rho, vn, vt1, vt2, p, Bt1, Bt2), flux (rho, Mn, Mt1, Mt2,
// E, Bt1, Bt2).
template <bool LD = false, typename R>
__device__ __forceinline__ int hlld(R gamma, const R* wl, const R* wr, R bn, R* flux) {
  return hlld_s<LD>(gamma, wl[0], wl[1], wl[2], wl[3], wl[4], wl[5], wl[6], wr[0], wr[1], wr[2],
                wr[3], wr[4], wr[5], wr[6], bn, flux);
}

// HLLE (Harten, Lax & van Leer 1983; Einfeldt 1988; Sec. 2.4): the flux of
// the single averaged state of the HLL fan between the outer speeds of the
// HLLD solver, S_L = min(vn) - max(c_f), S_R = max(vn) + max(c_f), with
// b- = min(S_L, 0), b+ = max(S_R, 0) (a supersonic face takes the upwind
// flux without a branch).  Same frames as hlld; returns 0.
template <typename R>
__device__ __forceinline__ int hlle(R gamma, const R* wl, const R* wr, R bn, R* f) {
  const R igm1 = R(1) / (gamma - R(1));
  auto side = [&](const R* w, R* u, R* fx) {
    const R rho = w[0], vn = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[5], b2 = w[6];
    const R bb = bn * bn + b1 * b1 + b2 * b2;
    const R pt = p + R(0.5) * bb;
    const R e = p * igm1 + R(0.5) * rho * (vn * vn + v1 * v1 + v2 * v2) + R(0.5) * bb;
    const R vb = vn * bn + v1 * b1 + v2 * b2;
    u[0] = rho; u[1] = rho * vn; u[2] = rho * v1; u[3] = rho * v2; u[4] = e; u[5] = b1; u[6] = b2;
    fx[0] = rho * vn; fx[1] = rho * vn * vn + pt - bn * bn; fx[2] = rho * vn * v1 - bn * b1;
    fx[3] = rho * vn * v2 - bn * b2; fx[4] = (e + pt) * vn - bn * vb;
    fx[5] = b1 * vn - bn * v1; fx[6] = b2 * vn - bn * v2;
  };
  R ul[7], ur[7], fl[7], fr[7];
  side(wl, ul, fl);
  side(wr, ur, fr);
  const R cm = fmax(fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]),
                    fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]));
  const R bm = fmin(fmin(wl[1], wr[1]) - cm, R(0));
  const R bp = fmax(fmax(wl[1], wr[1]) + cm, R(0));
  const R inv = R(1) / (bp - bm);
#pragma unroll
  for (int q = 0; q < 7; ++q) f[q] = (bp * fl[q] - bm * fr[q] + bp * bm * (ur[q] - ul[q])) * inv;
  return 0;
}

// ------------------------------------------------------------------------
// Isothermal closure p = cs^2 rho (Sec. 2.1): physical flux of one side
// (energy entries zero) and the outer speeds (the fast speed with gamma = 1
// and p = cs^2 rho).
// ------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void side_iso(R a2, const R* w, R bn, R* u, R* f) {
  const R rho = w[0], vn = w[1], v1 = w[2], v2 = w[3], b1 = w[5], b2 = w[6];
  const R pt = a2 * rho + R(0.5) * (bn * bn + b1 * b1 + b2 * b2);
  u[0] = rho; u[1] = rho * vn; u[2] = rho * v1; u[3] = rho * v2; u[4] = R(0); u[5] = b1; u[6] = b2;
  f[0] = rho * vn; f[1] = rho * vn * vn + pt - bn * bn; f[2] = rho * vn * v1 - bn * b1;
  f[3] = rho * vn * v2 - bn * b2; f[4] = R(0); f[5] = b1 * vn - bn * v1; f[6] = b2 * vn - bn * v2;
}

template <typename R>
__device__ __forceinline__ void iso_speeds(R a2, const R* wl, const R* wr, R bn, R& sl, R& sr) {
  const R cm = fmax(fast_speed(R(1), wl[0], a2 * wl[0], bn, wl[5], wl[6]),
                    fast_speed(R(1), wr[0], a2 * wr[0], bn, wr[5], wr[6]));
  sl = fmin(wl[1], wr[1]) - cm;
  sr = fmax(wl[1], wr[1]) + cm;
}

// Isothermal HLLE: HLL average between the outer speeds (branch-free form).
template <typename R>
__device__ __forceinline__ int hlle_iso(R cs, const R* wl, const R* wr, R bn, R* f) {
  const R a2 = cs * cs;
  R ul[7], ur[7], fl[7], fr[7], sl, sr;
  side_iso(a2, wl, bn, ul, fl);
  side_iso(a2, wr, bn, ur, fr);
  iso_speeds(a2, wl, wr, bn, sl, sr);
  const R bm = fmin(sl, R(0)), bp = fmax(sr, R(0));
  const R inv = R(1) / (bp - bm);
#pragma unroll
  for (int q = 0; q < 7; ++q) f[q] = (bp * fl[q] - bm * fr[q] + bp * bm * (ur[q] - ul[q])) * inv;
  return 0;
}

// Isothermal HLLD (Mignone 2007): no contact wave, so density and normal
// momentum are uniform inside the fan with the HLL fluxes there; rho* is
// the HLL average and u* = F_rho^HLL / rho* enters the jump conditions of
// the transverse components across the fast waves; a central state lies
// between the Alfven waves S*_L,R = u* -+ |Bn| / sqrt(rho*).
template <typename R>
__device__ __forceinline__ int hlld_iso(R cs, const R* wl, const R* wr, R bn, R* f) {
  const R a2 = cs * cs;
  R ul[7], ur[7], fl[7], fr[7], sl, sr;
  side_iso(a2, wl, bn, ul, fl);
  side_iso(a2, wr, bn, ur, fr);
  iso_speeds(a2, wl, wr, bn, sl, sr);
  if (sl >= R(0)) {
#pragma unroll
    for (int q = 0; q < 7; ++q) f[q] = fl[q];
    return 0;
  }
  if (sr <= R(0)) {
#pragma unroll
    for (int q = 0; q < 7; ++q) f[q] = fr[q];
    return 5;
  }
  const R idn = R(1) / (sr - sl);
  const R rs = (sr * ur[0] - sl * ul[0] - (fr[0] - fl[0])) * idn;
  const R fm = (sr * fl[0] - sl * fr[0] + sl * sr * (ur[0] - ul[0])) * idn;
  const R fmn = (sr * fl[1] - sl * fr[1] + sl * sr * (ur[1] - ul[1])) * idn;
  const R us = fm / rs;
  const R sq = sqrt(rs);
  const R sgn = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0));
  const R ssl = us - fabs(bn) / sq, ssr = us + fabs(bn) / sq;
  // transverse star state of one side across its fast wave (speed s)
  auto star = [&](const R* w, R s, R* t) {
    const R rho = w[0], vn = w[1];
    const R den = rho * (s - vn) * (s - us) - bn * bn;
    R vt1 = w[2], vt2 = w[3], bt1 = w[5], bt2 = w[6];
    if (fabs(den) >= Eps<R>::hlld * (rho * (s - vn) * (s - vn) + bn * bn)) {
      const R fv = bn * (us - vn) / den;
      const R fb = (rho * (s - vn) * (s - vn) - bn * bn) / den;
      vt1 = w[2] - w[5] * fv;
      vt2 = w[3] - w[6] * fv;
      bt1 = w[5] * fb;
      bt2 = w[6] * fb;
    }
    t[0] = vt1; t[1] = vt2; t[2] = bt1; t[3] = bt2;
  };
  R tl[4], tr[4];
  star(wl, sl, tl);
  star(wr, sr, tr);
  const bool right = ssl < R(0) && ssr <= R(0);
  const bool central = ssl < R(0) && ssr > R(0);
  // outer star flux of the selected side, transverse entries
  const R* uk = right ? ur : ul;
  const R* fk = right ? fr : fl;
  const R* tk = right ? tr : tl;
  const R sk = right ? sr : sl;
  R g2 = fk[2] + sk * (rs * tk[0] - uk[2]);
  R g3 = fk[3] + sk * (rs * tk[1] - uk[3]);
  R g5 = fk[5] + sk * (tk[2] - uk[5]);
  R g6 = fk[6] + sk * (tk[3] - uk[6]);
  if (central) {
    // central state between the Alfven waves (equal densities both sides)
    const R vc1 = R(0.5) * (tl[0] + tr[0]) + R(0.5) * (tr[2] - tl[2]) * sgn / sq;
    const R vc2 = R(0.5) * (tl[1] + tr[1]) + R(0.5) * (tr[3] - tl[3]) * sgn / sq;
    const R bc1 = R(0.5) * (tl[2] + tr[2]) + R(0.5) * sq * (tr[0] - tl[0]) * sgn;
    const R bc2 = R(0.5) * (tl[3] + tr[3]) + R(0.5) * sq * (tr[1] - tl[1]) * sgn;
    g2 += ssl * (rs * vc1 - rs * tl[0]);
    g3 += ssl * (rs * vc2 - rs * tl[1]);
    g5 += ssl * (bc1 - tl[2]);
    g6 += ssl * (bc2 - tl[3]);
  }
  f[0] = fm; f[1] = fmn; f[2] = g2; f[3] = g3; f[4] = R(0); f[5] = g5; f[6] = g6;
  return central ? 2 : (right ? 4 : 1);
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
