"""Pins of the oracle's dual-energy formalism (Sec. 2.8): the entropy
S = p / rho^(gamma-1) advected as a sixth cell variable with the flux
(mass flux) x (S/rho of the upwind side); the pressure taken from S where
the internal energy from E is below alpha_switch times the kinetic plus
magnetic energy (E then rewritten), S resynchronised from E above
alpha_sync.

* init: S of a uniform state in closed form;
* non-interference: where every cell stays above alpha_sync, the five
  conserved variables and B are bit for bit those of the run without it;
* the entropy flux is the upwinded mass flux times S/rho: a uniform S/rho
  stays uniform to round-off and the total S is conserved while neither
  threshold acts;
* resynchronisation carries shock heating into S (Sod);
* the purpose: a cold sheared density wave advected at Mach ~800 keeps its
  uniform pressure (2%) from S, while the subtraction from E loses it
  (errors ~1000x p, floors hit).
"""
import math

import numpy as np

import oracle as O
from paper_2608_14048_gb300 import inputs as I
from tests import exact_riemann as ER

G = 5.0 / 3.0


def test_dual_init_closed_form():
    n = (4, 3, 2)
    rho, p = 2.0, 3.0
    cons = np.zeros((5, 2, 3, 4))
    cons[0] = rho
    cons[1] = rho * 0.5
    cons[4] = p / (G - 1) + 0.5 * rho * 0.25
    g = O.make_grid(n)
    prm = O.make_params(mhd=False, dual=True)
    s = O.dual_init(g, prm, O.State(cons))
    np.testing.assert_allclose(s.cons[5], p / rho ** (G - 1), rtol=1e-14)
    np.testing.assert_array_equal(s.cons[:5], cons)


def test_dual_energy_leaves_the_dynamics_alone_above_alpha_sync():
    st = I.smooth_random_mhd(I.Block((12, 10, 9)), 91, v_rms=0.5, b_rms=0.5, B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    plain = O.State(st.cons, st.b1, st.b2, st.b3)
    pd = O.make_params(recon=O.PLM, integrator=O.RK2, dual=True)
    dual = O.dual_init(g, pd, plain)
    dts = O.run(g, O.make_params(recon=O.PLM, integrator=O.RK2), plain, nsteps=4)
    O.run(g, pd, dual, dts=dts)
    np.testing.assert_array_equal(dual.cons[:5], plain.cons)
    for a, b in ((dual.b1, plain.b1), (dual.b2, plain.b2), (dual.b3, plain.b3)):
        np.testing.assert_array_equal(a, b)


def test_entropy_flux_is_upwinded_mass_flux_times_specific_entropy():
    # S = s0 rho with the thresholds disabled (no switch, no sync): S/rho
    # stays s0 everywhere and the S integral is conserved
    st = I.smooth_random_mhd(I.Block((12, 10, 9)), 92, v_rms=0.8, b_rms=0.5, B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    prm = O.make_params(recon=O.PPM, dual=True, alpha_switch=-1e300, alpha_sync=1e300)
    s = O.dual_init(g, prm, O.State(st.cons, st.b1, st.b2, st.b3))
    s0 = 0.731
    s.cons[5] = s0 * s.cons[0]
    total0 = s.cons[5].sum()
    O.run(g, prm, s, nsteps=5)
    np.testing.assert_allclose(s.cons[5] / s.cons[0], s0, rtol=1e-13)
    assert abs(s.cons[5].sum() - total0) < 1e-12 * total0


def test_resync_carries_shock_heating_into_the_entropy():
    st = I.riemann_1d(0, 256, I.SOD_LEFT, I.SOD_RIGHT, 1.4)
    b = st.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    prm = O.make_params(gamma=1.4, recon=O.PLM, mhd=False, dual=True)
    s = O.dual_init(g, prm, O.State(st.cons))
    O.run(g, prm, s, t_end=0.25)
    x = b.centers(0)
    rho = s.cons[0, 0, 0]
    u = s.cons[1, 0, 0] / rho
    p = (1.4 - 1) * (s.cons[4, 0, 0] - 0.5 * rho * u * u)
    S = s.cons[5, 0, 0]
    # post-shock plateau (between contact and shock): the advected S equals
    # the shocked gas's p / rho^(gamma-1), not the pre-shock value
    ex = ER.sample(x, 0.25, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    mask = (x > 0.27) & (x < 0.40)
    np.testing.assert_allclose(S[mask], (p / rho ** 0.4)[mask], rtol=2e-2)
    pre = 0.1 / 0.125 ** 0.4
    assert np.all(S[mask] > 1.8 * pre)
    assert np.max(np.abs(rho[mask] - ex[0][mask])) < 5e-3


def _cold_advection(dual, n=64):
    """A cold sheared density wave: rho = 1 + 0.5 cos 2 pi x, v = (10,
    10 sin 2 pi x, 0) and uniform p = 1e-4 (Mach ~800), carried once through
    a periodic box.  The exact solution keeps p uniform.  The scheme's
    dissipation of the transverse velocity turns O(h^2) of the kinetic
    energy (~50) into internal energy, far above p.  Returns the recovered
    pressure over p0 and the floor hits."""
    b = I.Block((n, 2, 2))
    X, _, _ = I._cell_mesh(b)
    h = 1.0 / n
    k = 2 * math.pi
    shape = math.sin(k * h / 2) / (k * h / 2)          # cell averages of cos/sin
    rho = 1.0 + 0.5 * np.cos(k * X) * shape
    vx, vy, p0 = 10.0, 10.0 * np.sin(k * X) * shape, 1e-4
    cons = np.stack([rho, rho * vx, rho * vy, 0 * rho,
                     p0 / (G - 1) + 0.5 * rho * (vx * vx + vy * vy)])
    g = O.make_grid(b.n)
    prm = O.make_params(recon=O.PLM, integrator=O.RK2, mhd=False, dual=dual, p_floor=1e-12)
    s = O.State(cons)
    if dual:
        s = O.dual_init(g, prm, s)
    hits = 0
    t = 0.0
    while t < 0.1 - 1e-12:
        dt = min(O.compute_dt(g, prm, s), 0.1 - t)
        hits += O.step(g, prm, dt, s)
        t += dt
    r = s.cons[0]
    ke = 0.5 * (s.cons[1] ** 2 + s.cons[2] ** 2 + s.cons[3] ** 2) / r
    if dual:
        eint = s.cons[4] - ke
        use_s = eint < prm.alpha_switch * ke
        assert use_s.all()
        p = s.cons[5] * r ** (G - 1)
    else:
        p = (G - 1) * (s.cons[4] - ke)
    return p / p0, hits


def test_cold_supersonic_advection_keeps_its_pressure_only_with_dual_energy():
    pd, hd = _cold_advection(True)
    pp, hp = _cold_advection(False)
    assert np.max(np.abs(pd - 1.0)) < 0.05, np.max(np.abs(pd - 1.0))
    assert hd == 0
    # the subtraction from E: the dissipated kinetic energy, ~1000x the
    # pressure, with floors where it went negative
    assert np.max(np.abs(pp - 1.0)) > 100.0 and hp > 0


def _roll_state(s, sh):
    """Periodic shift of a state by sh = (sx, sy, sz) cells (face arrays:
    the interior faces roll, the last face is the image of the first)."""
    sx, sy, sz = sh
    cons = np.roll(s.cons, (sz, sy, sx), axis=(1, 2, 3))

    def face(a, ax):
        inner = np.take(a, range(a.shape[ax] - 1), axis=ax)
        inner = np.roll(inner, (sz, sy, sx), axis=(0, 1, 2))
        return np.concatenate([inner, np.take(inner, [0], axis=ax)], axis=ax)

    return O.State(cons, face(s.b1, 2), face(s.b2, 1), face(s.b3, 0))


def test_dual_energy_is_translation_invariant_on_a_periodic_box():
    """A periodic shift of the input shifts the result, S included: every
    cell, the last one along each axis too, sees its current bounding faces
    in the resync."""
    st = I.smooth_random_mhd(I.Block((10, 9, 8)), 93, v_rms=0.8, b_rms=0.6, B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    prm = O.make_params(recon=O.PLM, integrator=O.RK2, dual=True)
    a = O.dual_init(g, prm, O.State(st.cons, st.b1, st.b2, st.b3))
    sh = (3, 5, 2)
    b = _roll_state(a, sh)
    dts = O.run(g, prm, a, nsteps=3)
    O.run(g, prm, b, dts=dts)
    ra = _roll_state(a, sh)
    np.testing.assert_allclose(b.cons, ra.cons, rtol=0, atol=1e-13)
    for x, y in ((b.b1, ra.b1), (b.b2, ra.b2), (b.b3, ra.b3)):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)
