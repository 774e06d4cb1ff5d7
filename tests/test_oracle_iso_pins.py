"""Pins of the oracle's isothermal closure (p = c_s^2 rho, Sec. 2.1) and its
solvers (isothermal HLLD of Mignone 2007, isothermal HLLE; Sec. 2.4):

* both solvers: physical flux on equal states, upwind flux on supersonic
  faces, mirror and rotation symmetry, zero energy flux;
* HLLD: the closed form at B_n = 0 (HLL mass and normal-momentum fluxes,
  transverse momentum and field carried by u* = F_rho / rho*, upwinded by
  its sign), and an isolated stationary rotational discontinuity returned
  exactly (the Alfven waves are resolved);
* whole scheme: an isothermal shock tube against the exact isothermal
  Riemann solution, second-order convergence of an isothermal sound wave,
  conservation and div B on a random isothermal MHD box.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import inputs as I
from tests import exact_riemann as ER


def iso_flux(cs, w, bn):
    """Isothermal ideal-MHD flux along the normal, face frame (energy 0)."""
    rho, vn, v1, v2, _, b1, b2 = w
    pt = cs * cs * rho + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    return np.array([rho * vn, rho * vn * vn + pt - bn * bn, rho * vn * v1 - bn * b1,
                     rho * vn * v2 - bn * b2, 0.0, b1 * vn - bn * v1, b2 * vn - bn * v2])


def iso_cons(w):
    rho, vn, v1, v2, _, b1, b2 = w
    return np.array([rho, rho * vn, rho * v1, rho * v2, 0.0, b1, b2])


def iso_cf(cs, w, bn):
    rho = w[0]
    a2 = cs * cs
    b2 = (bn * bn + w[5] ** 2 + w[6] ** 2) / rho
    s = a2 + b2
    return math.sqrt(0.5 * (s + math.sqrt(max(s * s - 4 * a2 * bn * bn / rho, 0.0))))


def rand_state(rng):
    return np.array([rng.uniform(0.2, 2), rng.normal(), rng.normal(), rng.normal(), 0.0,
                     rng.normal(), rng.normal()])


SOLVERS = [O.hlld_iso, O.hlle_iso]


@pytest.mark.parametrize("solver", SOLVERS)
def test_iso_consistency_and_zero_energy_flux(solver):
    rng = np.random.default_rng(31)
    for _ in range(200):
        w = rand_state(rng); bn = rng.normal(); cs = rng.uniform(0.3, 2)
        np.testing.assert_allclose(solver(cs, w, w, bn), iso_flux(cs, w, bn), rtol=1e-12, atol=1e-12)
        assert solver(cs, w, rand_state(rng), bn)[4] == 0.0


@pytest.mark.parametrize("solver", SOLVERS)
def test_iso_supersonic_faces_take_the_upwind_flux(solver):
    rng = np.random.default_rng(32)
    for _ in range(100):
        wl = rand_state(rng); wr = rand_state(rng); bn = rng.normal(); cs = 0.7
        c = max(iso_cf(cs, wl, bn), iso_cf(cs, wr, bn))
        wl[1] = c + 0.1 + rng.uniform(0, 1); wr[1] = c + 0.1 + rng.uniform(0, 1)
        np.testing.assert_allclose(solver(cs, wl, wr, bn), iso_flux(cs, wl, bn), rtol=1e-13, atol=1e-13)
        wl[1], wr[1] = -wl[1], -wr[1]
        np.testing.assert_allclose(solver(cs, wl, wr, bn), iso_flux(cs, wr, bn), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("solver", SOLVERS)
def test_iso_mirror_and_rotation_symmetry(solver):
    rng = np.random.default_rng(33)
    for _ in range(100):
        wl = rand_state(rng); wr = rand_state(rng); bn = rng.normal(); cs = 0.9

        def mir(w):
            w = w.copy(); w[1] = -w[1]
            return w

        f = solver(cs, wl, wr, bn)
        fm = solver(cs, mir(wr), mir(wl), -bn)
        np.testing.assert_allclose(fm, [-f[0], f[1], -f[2], -f[3], 0.0, -f[5], -f[6]],
                                   rtol=1e-9, atol=1e-11)
        th = rng.uniform(0, 2 * math.pi)
        c, s = math.cos(th), math.sin(th)

        def rot(w):
            w = w.copy()
            w[2], w[3] = c * w[2] - s * w[3], s * w[2] + c * w[3]
            w[5], w[6] = c * w[5] - s * w[6], s * w[5] + c * w[6]
            return w

        fr = solver(cs, rot(wl), rot(wr), bn)
        exp = f.copy()
        exp[2], exp[3] = c * f[2] - s * f[3], s * f[2] + c * f[3]
        exp[5], exp[6] = c * f[5] - s * f[6], s * f[5] + c * f[6]
        np.testing.assert_allclose(fr, exp, rtol=1e-9, atol=1e-11)


def test_iso_hlld_closed_form_without_normal_field():
    rng = np.random.default_rng(34)
    cs = 0.8
    for _ in range(300):
        wl = rand_state(rng); wr = rand_state(rng)
        f = O.hlld_iso(cs, wl, wr, 0.0)
        c = max(iso_cf(cs, wl, 0.0), iso_cf(cs, wr, 0.0))
        sl, sr = min(wl[1], wr[1]) - c, max(wl[1], wr[1]) + c
        if sl >= 0 or sr <= 0:
            continue
        fl, fr = iso_flux(cs, wl, 0.0), iso_flux(cs, wr, 0.0)
        ul, ur = iso_cons(wl), iso_cons(wr)
        hll = (sr * fl - sl * fr + sl * sr * (ur - ul)) / (sr - sl)
        rs = (sr * ur[0] - sl * ul[0] - (fr[0] - fl[0])) / (sr - sl)
        us = hll[0] / rs
        w, s = (wl, sl) if us >= 0 else (wr, sr)
        bt = np.array(w[5:7]) * (s - w[1]) / (s - us)
        exp = np.array([hll[0], hll[1], hll[0] * w[2], hll[0] * w[3], 0.0, us * bt[0], us * bt[1]])
        np.testing.assert_allclose(f, exp, rtol=1e-10, atol=1e-12)


def test_iso_hlld_resolves_a_stationary_rotational_discontinuity():
    # rho = 1, B_n = 1, v_n = -1: the right-going Alfven wave is at rest;
    # B_t rotates at constant magnitude and v_t jumps by -sgn(B_n) dB_t /
    # sqrt(rho) (Walen): both physical fluxes agree, and so must HLLD's
    cs = 0.7
    bn = 1.0
    wl = np.array([1.0, -1.0, 0.1, 0.2, 0.0, 0.5, 0.0])
    wr = wl.copy()
    wr[5], wr[6] = 0.0, 0.5
    wr[2] = wl[2] - (wr[5] - wl[5])
    wr[3] = wl[3] - (wr[6] - wl[6])
    np.testing.assert_allclose(iso_flux(cs, wl, bn), iso_flux(cs, wr, bn), atol=1e-15)
    np.testing.assert_allclose(O.hlld_iso(cs, wl, wr, bn), iso_flux(cs, wl, bn), atol=1e-14)
    # HLLE smears it
    assert np.max(np.abs(O.hlle_iso(cs, wl, wr, bn) - iso_flux(cs, wl, bn))) > 1e-2


def _iso_tube(n, riemann):
    left = {"rho": 1.0, "v": (0.0, 0.0, 0.0), "p": 1.0}
    right = {"rho": 0.25, "v": (0.0, 0.0, 0.0), "p": 0.25}
    st = I.riemann_1d(0, n, left, right, 5.0 / 3.0)
    b = st.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    p = O.make_params(recon=O.PLM, mhd=False, iso=True, cs=1.0, riemann=riemann)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    O.run(g, p, s, t_end=0.2)
    x = b.centers(0)
    rho_ex, _ = ER.iso_sample(x, 0.2, (1.0, 0.0), (0.25, 0.0), 1.0)
    return float(np.mean(np.abs(s.cons[0, 0, 0, :] - rho_ex)))


def test_exact_isothermal_star_state_satisfies_the_jump_conditions():
    # the exact isothermal solver used by the tube pin, on its tube
    # (rho, u) = (1, 0) | (0.25, 0), c = 1: the star state must satisfy,
    # with nothing stored,
    # * across the right shock: mass fixes the shock speed S, then momentum
    #   rho (u - S)^2 + c^2 rho is continuous;
    # * across the left rarefaction: the invariant u + c ln(rho) holds.
    c = 1.0
    rl, ul, rr, ur = 1.0, 0.0, 0.25, 0.0
    rs, us = ER.iso_star(rl, ul, rr, ur, c)
    S = (rs * us - rr * ur) / (rs - rr)
    mom = lambda r, u: r * (u - S) ** 2 + c * c * r
    assert mom(rr, ur) == pytest.approx(mom(rs, us), rel=1e-12)
    assert ul + c * math.log(rl) == pytest.approx(us + c * math.log(rs), abs=1e-12)
    assert rr < rs < rl and S > us > 0
    # the sampled solution at t = 0.2 on [-0.5, 0.5] (every wave inside)
    # keeps its mass, and its momentum grows by c^2 (rho_L - rho_R) t
    n, t = 200000, 0.2
    x = (np.arange(n) + 0.5) / n - 0.5
    rho, u = ER.iso_sample(x, t, (rl, ul), (rr, ur), c)
    assert np.sum(rho) / n == pytest.approx(0.5 * (rl + rr), abs=2e-5)
    assert np.sum(rho * u) / n == pytest.approx(c * c * (rl - rr) * t, abs=2e-5)
    # a perturbed star density breaks the pair of conditions
    rs2 = rs * (1 + 1e-6)
    us2 = ul + c * math.log(rl / rs2)
    S2 = (rs2 * us2 - rr * ur) / (rs2 - rr)
    m2 = lambda r, u: r * (u - S2) ** 2 + c * c * r
    assert abs(m2(rr, ur) / m2(rs2, us2) - 1) > 1e-7


@pytest.mark.parametrize("riemann", [O.HLLD, O.HLLE])
def test_iso_shock_tube_against_exact(riemann):
    e1, e2 = _iso_tube(128, riemann), _iso_tube(256, riemann)
    assert e2 < 6e-3, (e1, e2)
    order = math.log2(e1 / e2)
    assert 0.6 < order < 1.3, (e1, e2, order)


def _iso_sound_error(n, amp=1e-6, cs=1.0, ntrans=4):
    """Right-moving isothermal sound wave along x: rho = 1 + a cos kx,
    v_x = c_s a cos kx (exact cell averages), one period."""
    b = I.Block((n, ntrans, ntrans))
    X, _, _ = I._cell_mesh(b)
    h = 1.0 / n
    k = 2 * math.pi
    cavg = np.cos(k * X) * math.sin(k * h / 2) / (k * h / 2)
    cons = np.zeros((5,) + X.shape)
    cons[0] = 1.0 + amp * cavg
    cons[1] = cs * amp * cavg
    z = [np.zeros((ntrans, ntrans, n + 1)), np.zeros((ntrans, ntrans + 1, n)), np.zeros((ntrans + 1, ntrans, n))]
    g = O.make_grid((n, ntrans, ntrans))
    p = O.make_params(recon=O.PLM, mhd=False, iso=True, cs=cs)
    s = O.State(cons, *z)
    O.run(g, p, s, t_end=1.0 / cs)
    return float(np.mean(np.abs(s.cons[0] - cons[0]))) / amp


def test_iso_sound_wave_second_order():
    e32, e64 = _iso_sound_error(32), _iso_sound_error(64)
    assert math.log2(e32 / e64) > 1.8, (e32, e64)


def test_iso_mhd_conservation_and_divb():
    st = I.smooth_random_mhd(I.Block((12, 14, 10)), 35, v_rms=0.6, b_rms=0.7, B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    p = O.make_params(recon=O.PLM, iso=True, cs=0.8)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    d0 = O.diagnostics(g, p, s)
    O.run(g, p, s, nsteps=6)
    d1 = O.diagnostics(g, p, s)
    assert d1["max_divb_rel"] < 1e-13
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    for q in range(3):
        assert abs(d1["mom"][q] - d0["mom"][q]) < 1e-12
