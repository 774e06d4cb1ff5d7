"""Pins from exact nonlinear MHD solutions (Sec. 5):

* the circularly polarised Alfven wave (the paper's test in its isothermal
  form, and the adiabatic variant): B_perp and v_perp = -B_perp / sqrt(rho)
  rotate with the wave at the Alfven speed while the total pressure stays
  uniform, so after one period the state must return to its start;
  the error falls at second order (the paper reports 2.4 for
  PLM + HLLE + RK2);
* an isolated stationary rotational (Alfven) discontinuity is returned
  exactly by the adiabatic HLLD (Miyoshi & Kusano 2005), and smeared by
  HLLE.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import inputs as I


def _cpaw(n, iso, riemann, integ, recon=O.PLM, amp=0.1, ntrans=2):
    """Wave along x on [0, 1] x thin periodic box: rho = 1, B = (1,
    amp sin 2 pi x, amp cos 2 pi x), v = (0, -amp sin, -amp cos) (right-
    moving, v_A = 1), p = 0.1 (adiabatic, gamma 5/3) or c_s = 1
    (isothermal); exact cell and face averages.  Returns the L1 error of
    the y-face field after one period."""
    g_ = 5.0 / 3.0
    b = I.Block((n, ntrans, ntrans))
    X, _, _ = I._cell_mesh(b)
    h = 1.0 / n
    k = 2 * math.pi
    sinc = math.sin(k * h / 2) / (k * h / 2)
    by = amp * np.sin(k * X) * sinc
    bz = amp * np.cos(k * X) * sinc
    cons = np.zeros((5,) + X.shape)
    cons[0] = 1.0
    cons[2] = -by
    cons[3] = -bz
    # the kinetic and magnetic energies of the exact cell averages
    cons[4] = 0.1 / (g_ - 1) + 0.5 * (by ** 2 + bz ** 2) + 0.5 * (1.0 + by ** 2 + bz ** 2)
    b1 = np.ones((ntrans, ntrans, n + 1))
    b2 = np.empty((ntrans, ntrans + 1, n)); b2[...] = by[:, :1, :]
    b3 = np.empty((ntrans + 1, ntrans, n)); b3[...] = bz[:1, :, :]
    g = O.make_grid(b.n)
    p = O.make_params(gamma=g_, recon=recon, integrator=integ, riemann=riemann, iso=iso, cs=1.0)
    s = O.State(cons, b1, b2, b3)
    b2_0 = b2.copy()
    O.run(g, p, s, t_end=1.0)
    return float(np.mean(np.abs(s.b2 - b2_0)))


@pytest.mark.parametrize("iso,riemann,integ", [(True, O.HLLE, O.RK2), (True, O.HLLD, O.RK2),
                                               (False, O.HLLD, O.VL2), (False, O.HLLE, O.RK2)])
def test_circularly_polarised_alfven_wave_second_order(iso, riemann, integ):
    # the limiter clips the wave's extrema at 16 cells per wavelength; from
    # 32 on the error falls at second order (measured 1.85-2.0, then
    # 2.0-2.4; the paper reports 2.4 for PLM + HLLE + RK2)
    e32, e64, e128 = (_cpaw(n, iso, riemann, integ) for n in (32, 64, 128))
    o1, o2 = math.log2(e32 / e64), math.log2(e64 / e128)
    assert o1 > 1.8 and o2 > 1.9, (e32, e64, e128, o1, o2)
    assert e128 < 3e-3 * 0.1, e128        # well below the 0.1 amplitude


def _physical_flux(gamma, w, bn):
    rho, vn, v1, v2, p, b1, b2 = w
    e = p / (gamma - 1) + 0.5 * rho * (vn * vn + v1 * v1 + v2 * v2) + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    pt = p + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    vb = vn * bn + v1 * b1 + v2 * b2
    return np.array([rho * vn, rho * vn * vn + pt - bn * bn, rho * vn * v1 - bn * b1,
                     rho * vn * v2 - bn * b2, (e + pt) * vn - bn * vb, b1 * vn - bn * v1,
                     b2 * vn - bn * v2])


def test_hlld_resolves_a_stationary_rotational_discontinuity_exactly():
    # rho = 1, B_n = 1, v_n = -1: the right-going Alfven wave (v_n + B_n /
    # sqrt(rho)) is at rest; B_t rotates at fixed magnitude and v_t jumps by
    # -sgn(B_n) dB_t / sqrt(rho) (Walen relation): both sides have the same
    # physical flux, which HLLD must return
    gamma = 5.0 / 3.0
    bn = 1.0
    wl = np.array([1.0, -1.0, 0.1, 0.2, 0.8, 0.6, 0.0])
    wr = wl.copy()
    wr[5], wr[6] = 0.0, 0.6
    wr[2] = wl[2] - (wr[5] - wl[5])
    wr[3] = wl[3] - (wr[6] - wl[6])
    fl, fr = _physical_flux(gamma, wl, bn), _physical_flux(gamma, wr, bn)
    np.testing.assert_allclose(fl, fr, atol=1e-15)
    f, _ = O.hlld(gamma, wl, wr, bn)
    np.testing.assert_allclose(f, fl, atol=1e-13)
    assert np.max(np.abs(O.hlle(gamma, wl, wr, bn) - fl)) > 1e-2


def test_isothermal_alfven_wave_order_matches_the_papers_figure():
    """The paper reports order 2.4 for PLM + HLLE + RK2 on this wave
    (tests/golden/cpaw_order.txt); the oracle's order between 64 and 128
    cells lies within 0.3 of it (measured 2.36)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "cpaw_order.txt")
    vals = dict(l.split() for l in open(path) if l.strip() and not l.startswith("#"))
    printed = float(vals["order_plm_hlle_rk2"])
    e64, e128 = (_cpaw(n, True, O.HLLE, O.RK2) for n in (64, 128))
    order = math.log2(e64 / e128)
    assert abs(order - printed) < 0.3, (order, printed)
