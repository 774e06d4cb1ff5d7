"""Pins of the oracle's PPM5 reconstruction (Sec. 2.4): the interface value
of each cell is the point value of the quartic through the five cell
averages centred on it, clipped into the range of the two cells it
separates, followed by the CW84 parabola limiter of PPM.

* exactness for cell averages of monotone quartics (a fact of the quartic
  interpolant, checked against analytic point values), where PPM's
  fourth-order value is not exact;
* fifth-order convergence of the interface value on smooth monotone data;
* no new extrema: face states stay inside the range of their three-cell
  neighbourhoods on random data; flattening at an extremum;
* linear data reproduced exactly;
* whole scheme: Sod against the exact solution, a second-order smooth
  wave, conservation and div B on a random MHD box.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import inputs as I
from tests import exact_riemann as ER
from tests.test_oracle_pins import _aligned_wave_error, _run_1d


def _averages(F, x0, h, n):
    """Cell averages of F' over n uniform cells starting at x0 (F is the
    antiderivative), and the face positions."""
    xf = x0 + h * np.arange(n + 1)
    return (F(xf[1:]) - F(xf[:-1])) / h, xf


def test_ppm5_exact_for_monotone_quartics():
    # f = x + 0.1 x^4 is increasing on [0, 1.3]; its antiderivative in closed form
    F = lambda x: 0.5 * x ** 2 + 0.02 * x ** 5
    f = lambda x: x + 0.1 * x ** 4
    avg, xf = _averages(F, 0.1, 1.0 / 32, 36)
    wl, wr = O.recon_line(O.PPM5, avg)
    ok = ~np.isnan(wl)
    exact = f(xf[1:-1])
    np.testing.assert_allclose(wl[ok], exact[ok], rtol=0, atol=1e-13)
    np.testing.assert_allclose(wr[ok], exact[ok], rtol=0, atol=1e-13)
    # PPM's fourth-order value misses the quartic term
    pl, _ = O.recon_line(O.PPM, avg)
    assert np.max(np.abs(pl[ok] - exact[ok])) > 1e-9


def test_ppm5_interface_value_is_fifth_order_on_smooth_data():
    # sin on a monotone stretch: the interface error falls as h^5
    errs = []
    for n in (16, 32):
        h = 1.0 / n
        avg, xf = _averages(lambda x: -np.cos(x), 0.1, h, n + 6)
        wl, wr = O.recon_line(O.PPM5, avg)
        ok = ~np.isnan(wl)
        exact = np.sin(xf[1:-1])
        errs.append(max(np.max(np.abs(wl[ok] - exact[ok])), np.max(np.abs(wr[ok] - exact[ok]))))
    order = math.log2(errs[0] / errs[1])
    assert order > 4.6, (errs, order)


def test_ppm5_linear_data_exact():
    w = 0.3 + 0.7 * np.arange(12.0)
    wl, wr = O.recon_line(O.PPM5, w)
    ok = ~np.isnan(wl)
    f = np.arange(11)[ok]
    np.testing.assert_allclose(wl[ok], 0.3 + 0.7 * (f + 0.5), rtol=1e-14)
    np.testing.assert_allclose(wr[ok], 0.3 + 0.7 * (f + 0.5), rtol=1e-14)


def test_ppm5_creates_no_new_extrema():
    rng = np.random.default_rng(5)
    for _ in range(50):
        w = rng.normal(size=40) * rng.uniform(0.1, 10)
        wl, wr = O.recon_line(O.PPM5, w)
        for f in range(len(wl)):
            if np.isnan(wl[f]):
                continue
            # left state belongs to cell f, right state to cell f + 1
            nl = w[max(f - 1, 0):f + 2]
            nr = w[f:f + 3]
            assert nl.min() - 1e-12 <= wl[f] <= nl.max() + 1e-12
            assert nr.min() - 1e-12 <= wr[f] <= nr.max() + 1e-12


def test_ppm5_flattens_extremum():
    w = np.array([0.0, 1.0, 2.0, 3.0, 2.0, 1.0, 0.0])
    wl, wr = O.recon_line(O.PPM5, w)
    assert wl[3] == 3.0 and wr[2] == 3.0


def test_ppm5_sod_against_exact():
    errs = []
    for n in (128, 256):
        st = I.riemann_1d(0, n, I.SOD_LEFT, I.SOD_RIGHT, 1.4)
        s = _run_1d(st, 0.25, recon=O.PPM5)
        x = st.block.centers(0)
        ex = ER.sample(x, 0.25, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
        errs.append(np.mean(np.abs(s.cons[0, 0, 0, :] - ex[0])))
    assert errs[1] < 6e-3
    order = math.log2(errs[0] / errs[1])
    assert 0.6 < order < 1.3, (errs, order)


def test_ppm5_smooth_wave_second_order():
    # the two-stage integrator bounds the scheme's order at 2
    e32 = _aligned_wave_error(32, integ=O.RK2, recon=O.PPM5)
    e64 = _aligned_wave_error(64, integ=O.RK2, recon=O.PPM5)
    assert math.log2(e32 / e64) > 1.8, (e32, e64)


def test_ppm5_mhd_conservation_and_divb():
    st = I.smooth_random_mhd(I.Block((12, 14, 10)), 51, v_rms=0.6, b_rms=0.7,
                             B0=(0.3, -0.2, 0.1))
    g = O.make_grid(st.block.n)
    p = O.make_params(recon=O.PPM5)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    d0 = O.diagnostics(g, p, s)
    O.run(g, p, s, nsteps=5)
    d1 = O.diagnostics(g, p, s)
    assert d1["max_divb_rel"] < 1e-13
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    assert abs(d1["energy"] - d0["energy"]) < 1e-12 * abs(d0["energy"])
