"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them:

* HLLD: physical flux on equal states (consistency); exact hydro limit = the
  textbook HLLC; exact resolution of a stationary contact with B_n != 0;
  invariance under rotations of the transverse plane.
* HLLE: consistency; upwind flux on supersonic faces; the closed-form
  Rusanov reduction on a stationary contact; mirror/rotation symmetry;
  positive density and pressure of the implied HLL state; Sod against the
  exact solution; second order of PLM + HLLE + RK2 on a smooth wave.
* Reconstruction: linear data exact (PLM, PPM); the fourth-order PPM
  interface value exact for cubic cell averages; first order at extrema.
* Corner EMF (Gardiner & Stone 2005): plane-parallel data along either
  transverse axis reduces the corner value to the face value.
* Time integrators: temporal order 3 (SSP-RK3) and 2 (SSP-RK2) at fixed
  grid on a smooth wave.
* Whole scheme: Sod shock tube (paper Sec. 5.1 set-up) against the exact
  Riemann solution; second-order convergence of the 3-D linear fast wave;
  div B at round-off; conservation to round-off; bitwise symmetry of a 1-D
  MHD Riemann problem run along x, y and z (the Liska-Wendroff property of
  Sec. 5.4).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import inputs as I
from tests import exact_riemann as ER

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def physical_flux(g, w, bn):
    """Ideal-MHD flux along the normal (Eqs. 1-4), face frame."""
    rho, vn, v1, v2, p, b1, b2 = w
    bb = bn * bn + b1 * b1 + b2 * b2
    pt = p + 0.5 * bb
    e = p / (g - 1) + 0.5 * rho * (vn * vn + v1 * v1 + v2 * v2) + 0.5 * bb
    vb = vn * bn + v1 * b1 + v2 * b2
    return np.array([rho * vn, rho * vn * vn + pt - bn * bn, rho * vn * v1 - bn * b1,
                     rho * vn * v2 - bn * b2, (e + pt) * vn - bn * vb,
                     b1 * vn - bn * v1, b2 * vn - bn * v2])


def rand_state(rng):
    return np.array([rng.uniform(0.2, 2), rng.normal(), rng.normal(), rng.normal(),
                     rng.uniform(0.1, 2), rng.normal(), rng.normal()])


# --------------------------------------------------------------------- HLLD

def test_hlld_consistency_equal_states():
    rng = np.random.default_rng(1)
    for _ in range(200):
        w = rand_state(rng)
        bn = rng.normal()
        f, _ = O.hlld(5 / 3, w, w, bn)
        np.testing.assert_allclose(f, physical_flux(5 / 3, w, bn), rtol=1e-12, atol=1e-12)


def hllc_textbook(g, wl, wr):
    """Toro's HLLC (Riemann Solvers, Sec. 10.4) with the HLLD wave-speed
    estimates S_L = min(u) - max(c), S_R = max(u) + max(c)."""
    def cons(w):
        rho, u, v, ww, p = w[:5]
        return np.array([rho, rho * u, rho * v, rho * ww,
                         p / (g - 1) + 0.5 * rho * (u * u + v * v + ww * ww)])

    def flux(w):
        rho, u, v, ww, p = w[:5]
        U = cons(w)
        return np.array([rho * u, rho * u * u + p, rho * u * v, rho * u * ww, (U[4] + p) * u])

    cl, cr = math.sqrt(g * wl[4] / wl[0]), math.sqrt(g * wr[4] / wr[0])
    sl = min(wl[1], wr[1]) - max(cl, cr)
    sr = max(wl[1], wr[1]) + max(cl, cr)
    rl, ul, pl = wl[0], wl[1], wl[4]
    rr, ur, pr = wr[0], wr[1], wr[4]
    ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))
    if sl >= 0:
        return flux(wl)
    if sr <= 0:
        return flux(wr)

    def ustar(w, s):
        rho, u, v, ww, p = w[:5]
        U = cons(w)
        fac = rho * (s - u) / (s - ss)
        return fac * np.array([1.0, ss, v, ww, U[4] / rho + (ss - u) * (ss + p / (rho * (s - u)))])

    if ss >= 0:
        return flux(wl) + sl * (ustar(wl, sl) - cons(wl))
    return flux(wr) + sr * (ustar(wr, sr) - cons(wr))


def test_hlld_hydro_limit_is_hllc():
    rng = np.random.default_rng(2)
    g = 1.4
    for _ in range(300):
        wl = rand_state(rng); wr = rand_state(rng)
        wl[5:] = 0; wr[5:] = 0
        f, _ = O.hlld(g, wl, wr, 0.0)
        np.testing.assert_allclose(f[:5], hllc_textbook(g, wl, wr), rtol=1e-11, atol=1e-12)
        assert np.all(f[5:] == 0)


def test_hlld_resolves_stationary_contact():
    # rho jumps, u = 0, p, v_t and B continuous, B_n != 0: an exact
    # stationary contact; HLLD must return zero mass flux and the exact
    # momentum/energy fluxes (no diffusion).
    wl = np.array([1.0, 0.0, 0.3, -0.2, 0.7, 0.4, 0.9])
    wr = wl.copy(); wr[0] = 0.25
    for bn in (0.8, -0.5, 0.0):
        f, _ = O.hlld(5 / 3, wl, wr, bn)
        ex = physical_flux(5 / 3, wl, bn)
        np.testing.assert_allclose(f, ex, atol=1e-13)
        assert abs(f[0]) < 1e-14


def test_hlld_transverse_rotation_invariance():
    rng = np.random.default_rng(3)
    for _ in range(100):
        wl = rand_state(rng); wr = rand_state(rng); bn = rng.normal()
        th = rng.uniform(0, 2 * math.pi)
        c, s = math.cos(th), math.sin(th)

        def rot(w):
            w = w.copy()
            w[2], w[3] = c * w[2] - s * w[3], s * w[2] + c * w[3]
            w[5], w[6] = c * w[5] - s * w[6], s * w[5] + c * w[6]
            return w

        f, _ = O.hlld(5 / 3, wl, wr, bn)
        fr, _ = O.hlld(5 / 3, rot(wl), rot(wr), bn)
        exp = f.copy()
        exp[2], exp[3] = c * f[2] - s * f[3], s * f[2] + c * f[3]
        exp[5], exp[6] = c * f[5] - s * f[6], s * f[5] + c * f[6]
        np.testing.assert_allclose(fr, exp, rtol=1e-9, atol=1e-11)


def test_hlld_mirror_symmetry():
    # reflecting x -> -x swaps L and R and flips the normal components
    rng = np.random.default_rng(4)
    for _ in range(100):
        wl = rand_state(rng); wr = rand_state(rng); bn = rng.normal()

        def mir(w):
            w = w.copy(); w[1] = -w[1]
            return w

        f, _ = O.hlld(5 / 3, wl, wr, bn)
        fm, _ = O.hlld(5 / 3, mir(wr), mir(wl), -bn)
        # mass, energy, transverse momentum flip; normal momentum stays;
        # transverse induction flux flips sign twice (v_n and B_n) -> flips
        exp = np.array([-f[0], f[1], -f[2], -f[3], -f[4], -f[5], -f[6]])
        np.testing.assert_allclose(fm, exp, rtol=1e-9, atol=1e-11)


# --------------------------------------------------------------------- HLLE

def _cons(g, w, bn):
    rho, vn, v1, v2, p, b1, b2 = w
    bb = bn * bn + b1 * b1 + b2 * b2
    e = p / (g - 1) + 0.5 * rho * (vn * vn + v1 * v1 + v2 * v2) + 0.5 * bb
    return np.array([rho, rho * vn, rho * v1, rho * v2, e, b1, b2])


def _cf(g, w, bn):
    """Fast magnetosonic speed along the normal."""
    rho, p = w[0], w[4]
    a2 = g * p / rho
    b2 = (bn * bn + w[5] ** 2 + w[6] ** 2) / rho
    s = a2 + b2
    return math.sqrt(0.5 * (s + math.sqrt(max(s * s - 4 * a2 * bn * bn / rho, 0.0))))


def test_hlle_consistency_equal_states():
    rng = np.random.default_rng(21)
    for _ in range(200):
        w = rand_state(rng)
        bn = rng.normal()
        np.testing.assert_allclose(O.hlle(5 / 3, w, w, bn), physical_flux(5 / 3, w, bn),
                                   rtol=1e-12, atol=1e-12)


def test_hlle_supersonic_faces_take_the_upwind_flux():
    rng = np.random.default_rng(22)
    for _ in range(100):
        wl = rand_state(rng); wr = rand_state(rng); bn = rng.normal()
        c = max(_cf(5 / 3, wl, bn), _cf(5 / 3, wr, bn))
        wl[1] = wr[1] = 0.0
        wl[1] += c + 0.1 + rng.uniform(0, 1); wr[1] += c + 0.1 + rng.uniform(0, 1)
        np.testing.assert_allclose(O.hlle(5 / 3, wl, wr, bn), physical_flux(5 / 3, wl, bn),
                                   rtol=1e-13, atol=1e-13)
        wl[1], wr[1] = -wl[1], -wr[1]
        np.testing.assert_allclose(O.hlle(5 / 3, wl, wr, bn), physical_flux(5 / 3, wr, bn),
                                   rtol=1e-13, atol=1e-13)


def test_hlle_stationary_contact_is_rusanov_with_the_fast_speed():
    # u = 0 on both sides, p, v_t and B continuous, rho jumps: the two
    # physical fluxes agree and S_R = -S_L = c_max, so HLLE reduces to
    # F_L - (c_max / 2)(U_R - U_L): a diffusive contact (HLLD's is exact)
    wl = np.array([1.0, 0.0, 0.3, -0.2, 0.7, 0.4, 0.9])
    wr = wl.copy(); wr[0] = 0.25
    for bn in (0.8, -0.5, 0.0):
        c = max(_cf(5 / 3, wl, bn), _cf(5 / 3, wr, bn))
        ex = physical_flux(5 / 3, wl, bn) - 0.5 * c * (_cons(5 / 3, wr, bn) - _cons(5 / 3, wl, bn))
        np.testing.assert_allclose(O.hlle(5 / 3, wl, wr, bn), ex, rtol=1e-13, atol=1e-14)
        assert O.hlle(5 / 3, wl, wr, bn)[0] > 0.1     # mass diffuses toward the light side


def test_hlle_mirror_and_rotation_symmetry():
    rng = np.random.default_rng(23)
    for _ in range(100):
        wl = rand_state(rng); wr = rand_state(rng); bn = rng.normal()

        def mir(w):
            w = w.copy(); w[1] = -w[1]
            return w

        f = O.hlle(5 / 3, wl, wr, bn)
        fm = O.hlle(5 / 3, mir(wr), mir(wl), -bn)
        np.testing.assert_allclose(fm, [-f[0], f[1], -f[2], -f[3], -f[4], -f[5], -f[6]],
                                   rtol=1e-9, atol=1e-11)
        th = rng.uniform(0, 2 * math.pi)
        c, s_ = math.cos(th), math.sin(th)

        def rot(w):
            w = w.copy()
            w[2], w[3] = c * w[2] - s_ * w[3], s_ * w[2] + c * w[3]
            w[5], w[6] = c * w[5] - s_ * w[6], s_ * w[5] + c * w[6]
            return w

        fr = O.hlle(5 / 3, rot(wl), rot(wr), bn)
        exp = f.copy()
        exp[2], exp[3] = c * f[2] - s_ * f[3], s_ * f[2] + c * f[3]
        exp[5], exp[6] = c * f[5] - s_ * f[6], s_ * f[5] + c * f[6]
        np.testing.assert_allclose(fr, exp, rtol=1e-9, atol=1e-11)


def test_hlle_hll_state_keeps_density_and_pressure_positive():
    # Einfeldt's property of HLLE with outer speed bounds: the intermediate
    # state U* = U_L + (F - F_L) / S_L implied by the flux stays physical,
    # here on strong hydro rarefactions (states moving apart)
    rng = np.random.default_rng(24)
    g = 1.4
    for _ in range(300):
        wl = rand_state(rng); wr = rand_state(rng)
        wl[5:] = wr[5:] = 0.0
        wl[1] = -abs(wl[1]) - rng.uniform(0, 3); wr[1] = abs(wr[1]) + rng.uniform(0, 3)
        f = O.hlle(g, wl, wr, 0.0)
        c = max(_cf(g, wl, 0.0), _cf(g, wr, 0.0))
        sl = min(wl[1], wr[1]) - c
        us = _cons(g, wl, 0.0) + (f - physical_flux(g, wl, 0.0)) / sl
        assert us[0] > 0
        pstar = (g - 1) * (us[4] - 0.5 * (us[1] ** 2 + us[2] ** 2 + us[3] ** 2) / us[0])
        assert pstar > 0, (wl, wr, us)


def test_sod_shock_tube_hlle_against_exact():
    errs = []
    for n in (128, 256):
        st = I.riemann_1d(0, n, I.SOD_LEFT, I.SOD_RIGHT, 1.4)
        s = _run_1d(st, 0.25, riemann=O.HLLE)
        x = st.block.centers(0)
        ex = ER.sample(x, 0.25, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
        errs.append(np.mean(np.abs(s.cons[0, 0, 0, :] - ex[0])))
    assert errs[1] < 8e-3
    order = math.log2(errs[0] / errs[1])
    assert 0.6 < order < 1.3, (errs, order)


def test_plm_hlle_rk2_fast_wave_second_order():
    # the paper's throughput combination (PLM + HLLE + RK2) on a smooth wave
    e64 = _aligned_wave_error(64, riemann=O.HLLE, integ=O.RK2)
    e128 = _aligned_wave_error(128, riemann=O.HLLE, integ=O.RK2)
    assert math.log2(e64 / e128) > 1.9, (e64, e128)


# ------------------------------------------------------------ reconstruction

@pytest.mark.parametrize("recon", [O.DONOR, O.PLM, O.PPM])
def test_recon_linear_exact(recon):
    w = 0.3 + 0.7 * np.arange(12.0)
    wl, wr = O.recon_line(recon, w)
    ok = ~np.isnan(wl)
    f = np.arange(11)[ok]
    if recon == O.DONOR:
        np.testing.assert_array_equal(wl[ok], w[f]); np.testing.assert_array_equal(wr[ok], w[f + 1])
    else:
        np.testing.assert_allclose(wl[ok], 0.3 + 0.7 * (f + 0.5), rtol=1e-14)
        np.testing.assert_allclose(wr[ok], 0.3 + 0.7 * (f + 0.5), rtol=1e-14)


def test_ppm_interface_exact_for_cubics():
    # cell averages of a monotone cubic: the fourth-order interface value is
    # its exact point value; the CW84 limiter stays inactive.
    h = 0.05
    xf = np.arange(13) * h + 0.3
    F = lambda x: 0.25 * x ** 4 + 0.5 * x ** 2     # antiderivative of x^3 + x
    avg = (F(xf[1:]) - F(xf[:-1])) / h
    wl, wr = O.recon_line(O.PPM, avg)
    exact = xf[1:-1] ** 3 + xf[1:-1]
    ok = ~np.isnan(wl)
    np.testing.assert_allclose(wl[ok], exact[ok], rtol=1e-12)
    np.testing.assert_allclose(wr[ok], exact[ok], rtol=1e-12)


@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_recon_flattens_extremum(recon):
    w = np.array([0.0, 1.0, 2.0, 3.0, 2.0, 1.0, 0.0])
    wl, wr = O.recon_line(recon, w)
    # cell 3 is a maximum: both of its face states equal its mean
    assert wl[3] == 3.0 and wr[2] == 3.0


def test_plm_harmonic_limiter_value():
    # van Leer: slope 2 d- d+ / (d- + d+) for same-sign differences
    w = np.array([0.0, 1.0, 4.0, 5.0])
    wl, wr = O.recon_line(O.PLM, w)
    d = 2 * 1.0 * 3.0 / 4.0
    assert wl[1] == pytest.approx(1.0 + 0.5 * d, rel=1e-15)
    d2 = 2 * 3.0 * 1.0 / 4.0
    assert wr[1] == pytest.approx(4.0 - 0.5 * d2, rel=1e-15)


# --------------------------------------------------------------- corner EMF

@pytest.mark.parametrize("flags", [(1, 1, 1, 1), (-1, -1, -1, -1), (0, 0, 0, 0),
                                   (1, -1, 0, 1), (-1, 1, 1, 0)])
def test_corner_emf_plane_parallel_reduction(flags):
    rng = np.random.default_rng(5)
    fa_m, fa_p, fb_m, fb_p = flags
    for _ in range(20):
        # data depending on the a-coordinate only: b-faces carry the exact
        # flux of identical states = the cell reference values of their
        # column; the corner value must equal the a-face value
        Ra = rng.normal(size=2)       # column a-1, a
        X = rng.normal()
        eref = [[Ra[0], Ra[1]], [Ra[0], Ra[1]]]
        e = O.corner_emf(X, X, Ra[0], Ra[1], eref, fa_m, fa_p, fb_m, fb_p)
        assert e == pytest.approx(X, abs=1e-14)
        # data depending on the b-coordinate only
        Rb = rng.normal(size=2)       # row b-1, b
        Y = rng.normal()
        eref = [[Rb[0], Rb[0]], [Rb[1], Rb[1]]]
        e = O.corner_emf(Rb[0], Rb[1], Y, Y, eref, fa_m, fa_p, fb_m, fb_p)
        assert e == pytest.approx(Y, abs=1e-14)


def test_corner_emf_upwind_selection():
    # with all mass fluxes positive the corner value must not depend on the
    # downwind (column a / row b) reference values
    base = dict(ea_m=0.3, ea_p=-0.1, eb_m=0.2, eb_p=0.5, fa_m=1, fa_p=1, fb_m=1, fb_p=1)
    e1 = O.corner_emf(base["ea_m"], base["ea_p"], base["eb_m"], base["eb_p"],
                      [[0.1, 0.2], [0.3, 0.4]], 1, 1, 1, 1)
    e2 = O.corner_emf(base["ea_m"], base["ea_p"], base["eb_m"], base["eb_p"],
                      [[0.1, 0.2], [0.3, 9.0]], 1, 1, 1, 1)
    assert e1 == e2
    e3 = O.corner_emf(base["ea_m"], base["ea_p"], base["eb_m"], base["eb_p"],
                      [[0.1, 0.2], [0.3, 9.0]], -1, -1, -1, -1)
    assert e3 != e1


# ---------------------------------------------------------- whole-scheme pins

def _run_1d(st, t_end, recon=O.PLM, integ=O.VL2, cfl=0.3, riemann=O.HLLD):
    b = st.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    p = O.make_params(gamma=st.gamma, recon=recon, integrator=integ, cfl=cfl,
                      mhd=bool(np.any(st.b1) or np.any(st.b2) or np.any(st.b3)), riemann=riemann)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    O.run(g, p, s, t_end=t_end)
    return s


def test_sod_star_state_satisfies_the_jump_conditions():
    # the exact solver used by the shock-tube pins, on the paper's Sod set-up
    # (Sec. 5.1: gamma = 1.4, (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1)):
    # its star state must satisfy, with nothing stored,
    # * across the right shock (Rankine-Hugoniot): the mass flux m and the
    #   shock speed S from mass and momentum, then the energy condition
    #   gamma/(gamma-1) p/rho + (u - S)^2 / 2 equal on both sides;
    # * across the left rarefaction: isentropic rho* = rho_L (p*/p_L)^(1/gamma)
    #   and the Riemann invariant u + 2c/(gamma - 1) conserved.
    # The two conditions fix (p*, u*) uniquely.
    g = 1.4
    rl, ul, pl, rr, ur, pr = 1.0, 0.0, 1.0, 0.125, 0.0, 0.1
    p, u = ER.star_state(rl, ul, pl, rr, ur, pr, g)
    m = (p - pr) / (u - ur)                  # m = rho (w) with w = u - S, shock frame
    S = ur + m / rr
    rs = m / (S - u)
    h = lambda pp, rho, w: g / (g - 1) * pp / rho + 0.5 * w * w
    assert h(pr, rr, ur - S) == pytest.approx(h(p, rs, u - S), rel=1e-10)
    rls = rl * (p / pl) ** (1 / g)
    cl, cls = math.sqrt(g * pl / rl), math.sqrt(g * p / rls)
    assert ul + 2 * cl / (g - 1) == pytest.approx(u + 2 * cls / (g - 1), rel=1e-10)
    # a shock to the right, a rarefaction to the left
    assert pr < p < pl and S > u > 0 and rs > rr


def test_exact_sod_solution_conserves_mass_momentum_energy():
    # the exact solver's sampled solution at t = 0.25 on [-0.5, 0.5], where
    # every wave stays inside: mass and energy as at t = 0, momentum grown
    # by the pressure difference of the two constant ends, (p_L - p_R) t
    # (midpoint rule on 2e5 cells; each discontinuity costs O(h))
    g, t = 1.4, 0.25
    n = 200000
    x = (np.arange(n) + 0.5) / n - 0.5
    rho, u, p = ER.sample(x, t, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g)
    h = 1.0 / n
    assert np.sum(rho) * h == pytest.approx(0.5 * 1.0 + 0.5 * 0.125, abs=2e-5)
    assert np.sum(rho * u) * h == pytest.approx((1.0 - 0.1) * t, abs=2e-5)
    E = p / (g - 1) + 0.5 * rho * u * u
    assert np.sum(E) * h == pytest.approx(0.5 / (g - 1) * (1.0 + 0.1), abs=2e-5)


def test_sod_shock_tube_against_exact():
    errs = []
    for n in (128, 256):
        st = I.riemann_1d(0, n, I.SOD_LEFT, I.SOD_RIGHT, 1.4)
        s = _run_1d(st, 0.25)
        x = st.block.centers(0)
        ex = ER.sample(x, 0.25, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
        rho = s.cons[0, 0, 0, :]
        errs.append(np.mean(np.abs(rho - ex[0])))
    # captured discontinuities: L1 error ~ N^-(0.7..1)
    assert errs[1] < 6e-3
    order = math.log2(errs[0] / errs[1])
    assert 0.6 < order < 1.3, (errs, order)


def test_sod_velocity_pressure_plateau():
    n = 256
    st = I.riemann_1d(0, n, I.SOD_LEFT, I.SOD_RIGHT, 1.4)
    s = _run_1d(st, 0.25)
    x = st.block.centers(0)
    rho = s.cons[0, 0, 0]
    u = s.cons[1, 0, 0] / rho
    # inside the star region away from the contact and the shock
    mask = (x > 0.0) & (x < 0.18)
    assert np.max(np.abs(u[mask] - 0.927453)) < 5e-3
    mask2 = (x > 0.27) & (x < 0.40)
    assert np.max(np.abs(rho[mask2] - 0.265574)) < 5e-3


@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_brio_wu_bitwise_axis_symmetry(recon):
    n = 64
    res = []
    for axis in range(3):
        st = I.brio_wu(axis, n)
        b = st.block
        g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
        p = O.make_params(gamma=2.0, recon=recon, cfl=0.3)
        s = O.State(st.cons, st.b1, st.b2, st.b3)
        O.run(g, p, s, nsteps=40)
        # rotate the result back to the x-axis frame (cyclic permutation)
        rho = s.cons[0].reshape(-1)
        e = s.cons[4].reshape(-1)
        m = [s.cons[1 + ((axis + q) % 3)].reshape(-1) for q in range(3)]
        res.append((rho, e, m))
    for axis in (1, 2):
        assert np.array_equal(res[0][0], res[axis][0])
        assert np.array_equal(res[0][1], res[axis][1])
        for q in range(3):
            assert np.array_equal(res[0][2][q], res[axis][2][q])


def _wave_error(n):
    st = I.linear_fast_wave(n)
    g = O.make_grid((n, n, n))
    p = O.make_params(gamma=st.gamma, recon=O.PLM, cfl=0.3)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    O.run(g, p, s, t_end=st.meta["period"])
    err = 0.0
    for v in range(5):
        err += np.mean(np.abs(s.cons[v] - st.cons[v])) ** 2
    for a, b0 in ((s.b1, st.b1), (s.b2, st.b2), (s.b3, st.b3)):
        err += np.mean(np.abs(a - b0)) ** 2
    return math.sqrt(err) / st.meta["amp"]


def _aligned_wave_error(n, amp=1e-6, ntrans=4, riemann=O.HLLD, integ=O.VL2, recon=O.PLM):
    """Fast wave along x in a thin 3-D periodic box (B = (1, sqrt2, 0.5),
    rho = 1, P = 1/gamma): L1 error of rho after one period."""
    g_ = 5 / 3
    lam, r = I.fast_eigenvector(g_)
    b = I.Block((n, ntrans, ntrans))
    X, _, _ = I._cell_mesh(b)
    h = 1.0 / n
    k = 2 * math.pi
    cavg = np.cos(k * X) * math.sin(k * h / 2) / (k * h / 2)
    by = math.sqrt(2.0) + amp * r[5] * cavg
    bz = 0.5 + amp * r[6] * cavg
    b1 = np.full((ntrans, ntrans, n + 1), 1.0)
    b2 = np.empty((ntrans, ntrans + 1, n)); b2[...] = by[:, :1, :]
    b3 = np.empty((ntrans + 1, ntrans, n)); b3[...] = bz[:1, :, :]
    cons = np.stack([1 + amp * r[0] * cavg, amp * r[1] * cavg, amp * r[2] * cavg, amp * r[3] * cavg,
                     (1 / g_ + amp * r[4] * cavg) / (g_ - 1) + 0.5 * (1 + by ** 2 + bz ** 2)])
    g = O.make_grid((n, ntrans, ntrans))
    p = O.make_params(riemann=riemann, integrator=integ, recon=recon)
    s = O.State(cons, b1, b2, b3)
    O.run(g, p, s, t_end=1.0 / lam)
    return np.mean(np.abs(s.cons[0] - cons[0])) / amp


def test_aligned_fast_wave_second_order():
    e64, e128 = _aligned_wave_error(64), _aligned_wave_error(128)
    assert math.log2(e64 / e128) > 1.9, (e64, e128)


@pytest.mark.slow
def test_linear_fast_wave_second_order():
    # the 32^3 diagonal wave of the benchmark set-up, refined once
    e16 = _wave_error(16)
    e32 = _wave_error(32)
    e64 = _wave_error(64)
    assert math.log2(e16 / e32) > 1.6, (e16, e32)
    assert math.log2(e32 / e64) > 1.9, (e32, e64)


def _temporal_error(integ, m, t_end, ref):
    """rho after m equal steps of the 16^3 fast wave with donor-cell states
    and HLLE: a smooth semi-discrete operator (no limiter; HLLD would switch
    between its ** states where S_M crosses zero around a fluid at rest,
    which caps the observable temporal order), against `ref`."""
    st = I.linear_fast_wave(16)
    g = O.make_grid((16, 16, 16))
    p = O.make_params(gamma=st.gamma, recon=O.DONOR, integrator=integ, riemann=O.HLLE)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    O.run(g, p, s, dts=[t_end / m] * m)
    if ref is None:
        return s.cons[0].copy()
    return float(np.mean(np.abs(s.cons[0] - ref))) / st.meta["amp"]


@pytest.mark.parametrize("integ,order", [(O.RK3, 3.0), (O.RK2, 2.0)])
def test_runge_kutta_temporal_order(integ, order):
    # same grid, step halved twice: the difference to a fine-step reference
    # falls as dt^order (a wrong stage weight drops SSP-RK3 to first or
    # second order)
    t_end = 0.25 * I.linear_fast_wave(16).meta["period"]
    ref = _temporal_error(integ, 1024, t_end, None)
    e8, e16, e32 = (_temporal_error(integ, m, t_end, ref) for m in (8, 16, 32))
    assert math.log2(e8 / e16) > order - 0.3, (e8, e16)
    assert math.log2(e16 / e32) > order - 0.3, (e16, e32)


def _random_periodic(n=12, seed=7, recon=O.PLM, integ=O.VL2, steps=6):
    st = I.smooth_random_mhd(I.Block((n, n + 2, n - 2)), seed, v_rms=0.8, b_rms=0.7,
                             B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    p = O.make_params(recon=recon, integrator=integ)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    d0 = O.diagnostics(g, p, s)
    O.run(g, p, s, nsteps=steps)
    d1 = O.diagnostics(g, p, s)
    return st, s, d0, d1, g, p


@pytest.mark.parametrize("recon,integ", [(O.PLM, O.VL2), (O.PPM, O.VL2), (O.PLM, O.RK2),
                                         (O.PLM, O.RK3)])
def test_conservation_and_divb(recon, integ):
    st, s, d0, d1, g, p = _random_periodic(recon=recon, integ=integ)
    assert d0["max_divb_rel"] < 1e-14
    assert d1["max_divb_rel"] < 1e-13
    assert abs(d1["mass"] - d0["mass"]) <= 1e-14 * abs(d0["mass"])
    assert abs(d1["energy"] - d0["energy"]) <= 1e-14 * abs(d0["energy"])
    scale = np.sum(np.abs(st.cons[1:4])) / st.cons[0].size
    for q in range(3):
        assert abs(d1["mom"][q] - d0["mom"][q]) <= 1e-14 * scale
    # periodic image faces stay consistent
    assert np.array_equal(s.b1[:, :, 0], s.b1[:, :, -1])
    assert np.array_equal(s.b2[:, 0, :], s.b2[:, -1, :])
    assert np.array_equal(s.b3[0], s.b3[-1])


def test_uniform_state_is_exactly_steady():
    # uniform flow through a uniform field: every flux difference vanishes
    n = 6
    b = I.Block((n, n, n))
    rho = np.full((n, n, n), 1.3)
    v = [np.full((n, n, n), c) for c in (0.4, -0.2, 0.7)]
    pr = np.full((n, n, n), 0.9)
    b1 = np.full((n, n, n + 1), 0.3); b2 = np.full((n, n + 1, n), -0.6); b3 = np.full((n + 1, n, n), 0.2)
    st = I._assemble(b, 5 / 3, rho, v, pr, b1, b2, b3)
    g = O.make_grid(b.n)
    p = O.make_params()
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    O.run(g, p, s, nsteps=3)
    np.testing.assert_allclose(s.cons, st.cons, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(s.b1, st.b1, rtol=1e-14)


def test_cfl_dt_closed_form():
    # uniform state: dt = C * dx / (|v_d| + c_f,d) minimised over d
    n = 4
    b = I.Block((n, n, n), hi=(1.0, 2.0, 0.5))
    rho = np.full((n, n, n), 2.0)
    vel = (0.3, -0.5, 0.1)
    v = [np.full((n, n, n), c) for c in vel]
    pr = np.full((n, n, n), 0.6)
    B = (0.4, 0.8, -0.3)
    b1 = np.full((n, n, n + 1), B[0]); b2 = np.full((n, n + 1, n), B[1]); b3 = np.full((n + 1, n, n), B[2])
    st = I._assemble(b, 5 / 3, rho, v, pr, b1, b2, b3)
    g = O.make_grid(b.n, hi=(1.0, 2.0, 0.5))
    p = O.make_params(cfl=0.3)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    g_ = 5 / 3
    a2 = g_ * 0.6 / 2.0
    bb = sum(x * x for x in B) / 2.0
    dts = []
    for d, dx in enumerate((0.25, 0.5, 0.125)):
        cf = math.sqrt(0.5 * (a2 + bb + math.sqrt((a2 + bb) ** 2 - 4 * a2 * B[d] ** 2 / 2.0)))
        dts.append(dx / (abs(vel[d]) + cf))
    assert O.compute_dt(g, p, s) == pytest.approx(0.3 * min(dts), rel=1e-13)


# ---------------------------------------------------------- spherical-polar

def _sph_grid(n):
    return O.make_grid(n, lo=(1.0, math.pi / 4, 0.0), hi=(2.0, 3 * math.pi / 4, math.pi / 2),
                       coord=O.SPH, bc=(O.OUTFLOW, O.OUTFLOW, O.PERIODIC))


@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_spherical_medium_at_rest_stays_at_rest(recon):
    # Sec. 2.7: the curvilinear sources use the same face areas and volumes
    # as the flux divergence, so a uniform medium at rest stays at rest to
    # machine precision
    n = (12, 10, 8)
    b = I.Block(n, lo=(1.0, math.pi / 4, 0.0), hi=(2.0, 3 * math.pi / 4, math.pi / 2),
                coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    rho = np.full(n[::-1], 1.3)
    v = [np.zeros(n[::-1])] * 3
    pr = np.full(n[::-1], 0.7)
    z = (np.zeros((n[2], n[1], n[0] + 1)), np.zeros((n[2], n[1] + 1, n[0])),
         np.zeros((n[2] + 1, n[1], n[0])))
    st = I._assemble(b, 5 / 3, rho, v, pr, *z)
    g = _sph_grid(n)
    p = O.make_params(recon=recon, mhd=False)
    s = O.State(st.cons, *z)
    O.run(g, p, s, nsteps=5, dts=[0.01] * 5)
    assert np.max(np.abs(s.cons[1:4])) < 1e-14
    np.testing.assert_allclose(s.cons[0], st.cons[0], rtol=1e-14)
    np.testing.assert_allclose(s.cons[4], st.cons[4], rtol=1e-14)


def test_spherical_divb_and_mass_conservation():
    n = (12, 10, 8)
    b = I.Block(n, lo=(1.0, math.pi / 4, 0.0), hi=(2.0, 3 * math.pi / 4, math.pi / 2),
                coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    st = I.smooth_random_mhd(b, 5, v_rms=0.3, b_rms=0.5)
    g = _sph_grid(n)
    p = O.make_params()
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    d0 = O.diagnostics(g, p, s)
    assert d0["max_divb_rel"] < 1e-14   # generator: B from a vector potential
    O.run(g, p, s, nsteps=5)
    d1 = O.diagnostics(g, p, s)
    assert d1["max_divb_rel"] < 1e-13     # CT keeps div B at round-off (Sec. 2.5)


def _rigid_rotation_drift(nr, recon, omega=0.5, t_end=0.02):
    """Mean drift of each conserved variable, away from the r and theta
    boundaries, of a rigidly rotating medium on a spherical wedge."""
    n = (nr, nr, 4)
    lo, hi = (1.0, math.pi / 4, 0.0), (2.0, 3 * math.pi / 4, math.pi / 2)
    b = I.Block(n, lo=lo, hi=hi, coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    R, TH, _ = I._cell_mesh(b)
    zero = np.zeros(R.shape)
    # v_phi = Omega r sin(theta) with the centrifugal balance
    # dp/dR = rho Omega^2 R (R = r sin(theta)): p = p0 + rho Omega^2 R^2 / 2
    vphi = omega * R * np.sin(TH)
    pr = 1.0 + 0.5 * omega ** 2 * (R * np.sin(TH)) ** 2
    z = (np.zeros((n[2], n[1], n[0] + 1)), np.zeros((n[2], n[1] + 1, n[0])),
         np.zeros((n[2] + 1, n[1], n[0])))
    st = I._assemble(b, 5 / 3, np.ones(R.shape), [zero, zero, vphi], pr, *z)
    g = _sph_grid(n)
    s = O.State(st.cons.copy(), *z)
    O.run(g, O.make_params(mhd=False, recon=recon), s, t_end=t_end)
    # the zero-gradient r and theta boundaries do not hold the equilibrium:
    # measure where their disturbance has not arrived
    keep = (R > 1.25) & (R < 1.75) & (TH > math.pi / 4 + 0.35) & (TH < 3 * math.pi / 4 - 0.35)
    return [float(np.mean(np.abs(s.cons[v] - st.cons[v])[keep])) for v in range(5)]


@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_spherical_rigid_rotation_is_steady_to_second_order(recon):
    # an exact steady state that exercises the velocity stresses of the
    # curvilinear sources (Eq. 12): rho v_phi^2 enters S_r through <1/r> and
    # S_theta through <cot(theta)/r>; the scheme holds it up to its
    # truncation error, which falls at second order (measured 1.9-2.4).
    # Dropping the rho v_phi^2 part of T_phiphi from both leaves a drift of
    # 7e-3 in M_r at every resolution.
    e = [_rigid_rotation_drift(nr, recon) for nr in (16, 32, 64)]
    for v in range(5):
        o1, o2 = math.log2(e[0][v] / e[1][v]), math.log2(e[1][v] / e[2][v])
        assert o1 > 1.7 and o2 > 1.7, (v, e)
    assert e[2][1] < 5e-7, e[2]


def _toroidal_field_drift(nr, recon, b0=0.3, t_end=0.02):
    """Drift of a static toroidal-field equilibrium on a spherical wedge:
    B_phi = b0 R (R = r sin(theta)) has tension B^2/R and magnetic pressure
    gradient B dB/dR, together 2 b0^2 R inward, held by p = p0 - b0^2 R^2."""
    n = (nr, nr, 4)
    lo, hi = (1.0, math.pi / 4, 0.0), (2.0, 3 * math.pi / 4, math.pi / 2)
    b = I.Block(n, lo=lo, hi=hi, coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    R, TH, _ = I._cell_mesh(b)
    zero = np.zeros(R.shape)
    pr = 1.0 - b0 ** 2 * (R * np.sin(TH)) ** 2
    rc, tc = b.centers(0), b.centers(1)
    b1 = np.zeros((n[2], n[1], n[0] + 1))
    b2 = np.zeros((n[2], n[1] + 1, n[0]))
    b3 = np.empty((n[2] + 1, n[1], n[0]))
    b3[...] = b0 * rc[None, :] * np.sin(tc)[:, None]     # phi faces: no phi dependence
    st = I._assemble(b, 5 / 3, np.ones(R.shape), [zero, zero, zero], pr, b1, b2, b3)
    g = _sph_grid(n)
    p = O.make_params(recon=recon)
    s = O.State(st.cons.copy(), b1.copy(), b2.copy(), b3.copy())
    assert O.diagnostics(g, p, s)["max_divb_rel"] == 0.0
    O.run(g, p, s, t_end=t_end)
    keep = (R > 1.25) & (R < 1.75) & (TH > math.pi / 4 + 0.35) & (TH < 3 * math.pi / 4 - 0.35)
    e = [float(np.mean(np.abs(s.cons[v] - st.cons[v])[keep])) for v in range(5)]
    e.append(float(np.mean(np.abs(s.b3[:-1] - b3[:-1])[keep])))
    return e


@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_spherical_toroidal_field_equilibrium_is_steady_to_second_order(recon):
    # the magnetic stresses of the curvilinear sources (Eq. 12, T_ij with
    # -B_i B_j and the magnetic pressure): the static equilibrium drifts by
    # the truncation error only, falling at second order (measured 2.0-2.3);
    # M_phi stays zero by symmetry.  The wrong sign on B_i B_j drifts by
    # 5e-3 in M_r at every resolution.
    e = [_toroidal_field_drift(nr, recon) for nr in (16, 32, 64)]
    for v in (0, 1, 2, 4, 5):
        o1, o2 = math.log2(e[0][v] / e[1][v]), math.log2(e[1][v] / e[2][v])
        assert o1 > 1.7 and o2 > 1.7, (v, e)
    assert max(x[3] for x in e) < 1e-15
    assert e[2][1] < 5e-7, e[2]


def _rotating_axial_mhd_drift(nr, recon, U=0.3, om=0.5, B=0.4, t_end=0.02):
    """Drift of an exact steady MHD state on a spherical wedge: rigid
    rotation Omega about the axis plus a uniform axial flow U and a uniform
    axial field B.  (v.grad)v is the centrifugal term alone, held by
    p = p0 + rho Omega^2 R^2 / 2; the EMF -v x B = -Omega R B R_hat is
    curl-free, so B stays.  In spherical components every stress T_ij and
    both EMF components of the CT are non-zero."""
    n = (nr, nr, 4)
    lo, hi = (1.0, math.pi / 4, 0.0), (2.0, 3 * math.pi / 4, math.pi / 2)
    b = I.Block(n, lo=lo, hi=hi, coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    R, TH, _ = I._cell_mesh(b)
    te = np.linspace(lo[1], hi[1], n[1] + 1)
    v = [U * np.cos(TH), -U * np.sin(TH), om * R * np.sin(TH)]
    pr = 1.0 + 0.5 * om ** 2 * (R * np.sin(TH)) ** 2
    # face averages of the uniform field B z_hat: the exact flux through
    # each face over its exact area (r faces: B (sin^2 t2 - sin^2 t1) / 2 /
    # (cos t1 - cos t2); theta faces: -B sin(theta); phi faces: 0)
    t1, t2 = te[:-1], te[1:]
    b1 = np.empty((n[2], n[1], n[0] + 1))
    b1[...] = (B * 0.5 * (np.sin(t2) ** 2 - np.sin(t1) ** 2) / (np.cos(t1) - np.cos(t2)))[None, :, None]
    b2 = np.empty((n[2], n[1] + 1, n[0]))
    b2[...] = (-B * np.sin(te))[None, :, None]
    b3 = np.zeros((n[2] + 1, n[1], n[0]))
    st = I._assemble(b, 5 / 3, np.ones(R.shape), v, pr, b1, b2, b3)
    g = _sph_grid(n)
    p = O.make_params(recon=recon)
    s = O.State(st.cons.copy(), b1.copy(), b2.copy(), b3.copy())
    assert O.diagnostics(g, p, s)["max_divb_rel"] < 1e-15
    O.run(g, p, s, t_end=t_end)
    keep = (R > 1.25) & (R < 1.75) & (TH > math.pi / 4 + 0.35) & (TH < 3 * math.pi / 4 - 0.35)
    e = [float(np.mean(np.abs(s.cons[q] - st.cons[q])[keep])) for q in range(5)]
    e.append(float(np.mean(np.abs(s.b1[..., :-1] - b1[..., :-1])[keep])))
    e.append(float(np.mean(np.abs(s.b2[:, :-1, :] - b2[:, :-1, :])[keep])))
    e.append(float(np.mean(np.abs(s.b3[:-1] - b3[:-1])[keep])))
    return e


@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_spherical_rotating_axial_flow_and_field_is_steady_to_second_order(recon):
    # pins the off-diagonal stresses of Eq. 12 (T_r theta in S_theta;
    # T_phi r and T_phi theta in S_phi) and spherical CT with a non-zero
    # EMF: every variable drifts at second order (measured 1.8-3.0); at 64
    # cells the theta and phi momenta drift by < 1e-5 (4e-6, 3e-6), where
    # dropping -T_r theta <1/r> gives 2e-4 in M_theta and a wrong sign, or a
    # dropped cot term, in S_phi gives 6e-4 to 1.2e-3 in M_phi.
    e = [_rotating_axial_mhd_drift(nr, recon) for nr in (16, 32, 64)]
    for q in range(8):
        o1, o2 = math.log2(e[0][q] / e[1][q]), math.log2(e[1][q] / e[2][q])
        assert o1 > 1.7 and o2 > 1.7, (q, e)
    assert e[2][2] < 1e-5 and e[2][3] < 1e-5, e[2]


def test_spherical_geometry_closed_forms():
    # exact volume of the whole wedge and exact outer-face area sum
    import ctypes
    n = (6, 5, 4)
    b = I.Block(n, lo=(1.0, math.pi / 4, 0.0), hi=(2.0, 3 * math.pi / 4, math.pi / 2),
                coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    rho = np.ones(n[::-1])
    v = [np.zeros(n[::-1])] * 3
    z = (np.zeros((n[2], n[1], n[0] + 1)), np.zeros((n[2], n[1] + 1, n[0])),
         np.zeros((n[2] + 1, n[1], n[0])))
    st = I._assemble(b, 5 / 3, rho, v, np.ones(n[::-1]), *z)
    g = _sph_grid(n)
    d = O.diagnostics(g, O.make_params(mhd=False), O.State(st.cons, *z))
    vol = (2 ** 3 - 1) / 3 * (math.cos(math.pi / 4) - math.cos(3 * math.pi / 4)) * math.pi / 2
    assert d["mass"] == pytest.approx(vol, rel=1e-14)
