"""Pins of the oracle's low-dissipation HLLD (LHLLD; Sec. 2.4 after Minoshima
& Miyoshi 2021): HLLD whose pressure dissipation at the contact is scaled by
the local Mach number.

* flux-level: HLLD bit for bit once the local Mach number reaches 1 and on
  supersonic faces; consistency; an exact stationary contact; mirror and
  rotation symmetry; the pressure dissipation of a low-Mach velocity jump
  falls in proportion to the Mach number (HLLD's stays at the sound-speed
  scale);
* whole scheme: the Taylor-Green vortex of the paper's low-Mach test
  (Sec. 5, PLM + RK2): with LHLLD the kinetic-energy decay in turnover units
  is the same at Mach 0.1 and 0.01, while HLLD's grows with 1/M; Sod still
  converges to the exact solution; conservation and div B.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import inputs as I
from tests import exact_riemann as ER
from tests.test_oracle_pins import _run_1d

G = 5.0 / 3.0


def _fast(w, bn):
    rho, p = w[0], w[4]
    a2 = G * p / rho
    b2 = (bn * bn + w[5] ** 2 + w[6] ** 2) / rho
    s = a2 + b2
    return math.sqrt(0.5 * (s + math.sqrt(max(s * s - 4 * a2 * bn * bn / rho, 0.0))))


def _rand(rng, vscale):
    return np.array([rng.uniform(0.3, 2), vscale * rng.normal(), vscale * rng.normal(),
                     vscale * rng.normal(), rng.uniform(0.3, 2), rng.normal(), rng.normal()])


def test_lhlld_equals_hlld_at_local_mach_one_and_above():
    rng = np.random.default_rng(71)
    n = 0
    while n < 200:
        wl, wr, bn = _rand(rng, 3.0), _rand(rng, 3.0), rng.normal()
        vmax = max(np.linalg.norm(wl[1:4]), np.linalg.norm(wr[1:4]))
        if vmax < max(_fast(wl, bn), _fast(wr, bn)):
            continue
        n += 1
        f0, r0 = O.hlld(G, wl, wr, bn)
        f1, r1 = O.lhlld(G, wl, wr, bn)
        assert r0 == r1
        assert np.array_equal(f0, f1)


def test_lhlld_consistency_and_stationary_contact():
    rng = np.random.default_rng(72)
    for _ in range(100):
        w = _rand(rng, 0.3); bn = rng.normal()
        np.testing.assert_array_equal(O.lhlld(G, w, w, bn)[0], O.hlld(G, w, w, bn)[0])
    # contact at rest: density jump, equal pressure, B_n = 0
    wl = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.4, 0.0])
    wr = np.array([0.2, 0.0, 0.0, 0.0, 1.0, 0.4, 0.0])
    f, _ = O.lhlld(G, wl, wr, 0.0)
    np.testing.assert_allclose(f, [0, 1.0 + 0.5 * 0.16, 0, 0, 0, 0, 0], atol=1e-15)


def test_lhlld_mirror_and_rotation_symmetry():
    rng = np.random.default_rng(73)
    for _ in range(100):
        wl, wr, bn = _rand(rng, 0.4), _rand(rng, 0.4), rng.normal()
        f, _ = O.lhlld(G, wl, wr, bn)
        # mirror x -> -x: swap sides, negate normal velocity and normal field
        m = lambda w: np.array([w[0], -w[1], w[2], w[3], w[4], w[5], w[6]])
        fm, _ = O.lhlld(G, m(wr), m(wl), -bn)
        exp = np.array([-f[0], f[1], -f[2], -f[3], -f[4], -f[5], -f[6]])
        np.testing.assert_allclose(fm, exp, rtol=1e-12, atol=1e-12)
        # rotation by 90 degrees about the normal: (t1, t2) -> (-t2, t1)
        r = lambda w: np.array([w[0], w[1], -w[3], w[2], w[4], -w[6], w[5]])
        fr, _ = O.lhlld(G, r(wl), r(wr), bn)
        np.testing.assert_allclose(fr, [f[0], f[1], -f[3], f[2], f[4], -f[6], f[5]],
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mach", [1e-2, 1e-3])
def test_lhlld_pressure_dissipation_scales_with_mach(mach):
    """A symmetric compressive velocity jump +-M c at uniform rho and p
    (c = 1, B = 0): the face is at rest (S_M = 0), so the normal-momentum
    flux is the star pressure and its excess over p is the pressure
    dissipation.  HLLD's is ~rho c dU / 2 (order M); LHLLD's is order M^2, so
    the ratio LHLLD / HLLD is the local Mach number."""
    p = 1.0 / G
    wl = np.array([1.0, mach, 0.0, 0.0, p, 0.0, 0.0])
    wr = np.array([1.0, -mach, 0.0, 0.0, p, 0.0, 0.0])
    fh, _ = O.hlld(G, wl, wr, 0.0)
    fl, _ = O.lhlld(G, wl, wr, 0.0)
    assert abs(fh[0]) < 1e-15 and abs(fl[0]) < 1e-15
    dh = fh[1] - p
    dl = fl[1] - p
    assert dh == pytest.approx(mach, rel=0.1)           # rho c dU / 2 with dU = 2 M
    assert dl / dh == pytest.approx(mach, rel=0.05)


def _tgv_decay(mach, riemann, n=16, t_end=1.0):
    """1 - K(t_end)/K(0) of the Taylor-Green vortex, time in turnover units
    (v0 = 1, box 2 pi), PLM + RK2."""
    st = I.taylor_green(n, mach)
    b = st.block
    g = O.make_grid(b.n, b.lo, b.hi)
    p = O.make_params(gamma=st.gamma, recon=O.PLM, integrator=O.RK2, mhd=False, riemann=riemann)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    kin = lambda c: float(np.mean(0.5 * (c[1] ** 2 + c[2] ** 2 + c[3] ** 2) / c[0]))
    k0 = kin(s.cons)
    O.run(g, p, s, t_end=t_end)
    return 1.0 - kin(s.cons) / k0


def test_taylor_green_dissipation_independent_of_mach_with_lhlld():
    """16^3, one turnover: LHLLD's decays at Mach 0.1 and 0.01 agree within
    10% (7% here, from the start-up acoustics of the Mach 0.1 run; the gap
    falls below 1% by the second turnover), while HLLD loses 3x more energy
    at Mach 0.01 than at 0.1 and 9x more than LHLLD at Mach 0.1."""
    d1, d2 = _tgv_decay(0.1, O.LHLLD), _tgv_decay(0.01, O.LHLLD)
    assert abs(d1 - d2) < 0.1 * d1, (d1, d2)
    h1, h2 = _tgv_decay(0.1, O.HLLD), _tgv_decay(0.01, O.HLLD)
    # HLLD's pressure dissipation grows with the sound speed
    assert h2 > 3 * h1 and h1 > 3 * d1, (h1, h2, d1)


def test_lhlld_sod_against_exact():
    errs = []
    for n in (128, 256):
        st = I.riemann_1d(0, n, I.SOD_LEFT, I.SOD_RIGHT, 1.4)
        s = _run_1d(st, 0.25, riemann=O.LHLLD)
        x = st.block.centers(0)
        ex = ER.sample(x, 0.25, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
        errs.append(np.mean(np.abs(s.cons[0, 0, 0, :] - ex[0])))
    assert errs[1] < 6e-3
    order = math.log2(errs[0] / errs[1])
    assert 0.6 < order < 1.3, (errs, order)


def test_lhlld_mhd_conservation_and_divb():
    st = I.smooth_random_mhd(I.Block((12, 14, 10)), 74, v_rms=0.3, b_rms=0.7,
                             B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    p = O.make_params(recon=O.PLM, riemann=O.LHLLD)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    d0 = O.diagnostics(g, p, s)
    O.run(g, p, s, nsteps=5)
    d1 = O.diagnostics(g, p, s)
    assert d1["max_divb_rel"] < 1e-13
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    assert abs(d1["energy"] - d0["energy"]) < 1e-12 * abs(d0["energy"])
