"""Isothermal gas under dust on the GPU (Sec. 2.1 isothermal closure, Sec.
2.2 dust with both drag laws) against the FP64 oracle, and the paper's
steady dusty shock (Sec. 5.8.2) held by the GPU.

* Parity, element by element with the oracle's dt sequence: isothermal
  hydro gas (isothermal HLLD) plus three species, constant stopping times
  or constant drag coefficients (t_k = rho_k / K_k), FP64 at 1e-12 and
  FP32 transport at 1e-5, FP64 and FP32 drag.  The gas energy slot takes no
  drag heating in the isothermal closure: it stays bit for bit as set.
* The steady isothermal dusty shock: Mach 2 gas carrying three species
  with drag coefficients K = 1, 3, 5 (tests/golden/dusty_shock.txt).
  Started on the stationary ODE structure (as the oracle pin does, 200
  cells of the paper's 40-unit domain), the FP64 GPU run stays at the
  oracle's state to 1e-10 over 4 time units and holds the structure: every
  density within 5e-3 of the ODE profile off the front, the front in
  place, the far-downstream compression the paper prints (16).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I
from tests.gpu_helpers import rel_l1
from tests.test_oracle_dust_pins import _SteadyDustyShock, _paper_shock_values

pytestmark = pytest.mark.gpu


def _oracle(gas, dust, ts, nsteps, law, cs):
    b = gas.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    p = O.make_params(mhd=False, iso=True, cs=cs, recon=O.PLM)
    dp = O.make_dust_params(ts, law=law)
    cons, d = gas.cons.copy(), dust.copy()
    dts = []
    for _ in range(nsteps):
        dt = O.dust_dt(g, p, dp, cons, d)
        O.dust_step(g, p, dp, dt, cons, d)
        dts.append(dt)
    return cons, d, dts


def _gpu(block, cons0, dust0, ts, dts, prec, law, cs, drag=A.DRAG_FP64, cfl=0.3):
    import torch
    cfg = A.make_config(recon=A.PLM, integrator=A.IMEX2P, precision=prec, mhd=False, t_stop=ts,
                        iso=True, cs=cs, drag_precision=drag, drag_law=law, cfl=cfl)
    sv = A.Solver(cfg, [A.make_block(block.n, block.lo, block.hi, block.coord, block.bc)],
                  stream=torch.cuda.current_stream())
    try:
        sv.set_state(0, cons0)
        for k in range(len(ts)):
            A.aeth_set_dust(sv.ctx, 0, k, np.ascontiguousarray(dust0[k]))
        for dt in dts:
            sv.step(dt)
        cons = sv.get_state(0)[0]
        d = np.empty_like(dust0)
        for k in range(len(ts)):
            buf = np.empty(dust0.shape[1:])
            A.aeth_get_dust(sv.ctx, 0, k, buf)
            d[k] = buf
        dt_dev = sv.compute_dt()
    finally:
        sv.close()
    return cons, d, dt_dev


@pytest.mark.parametrize("law", [A.DRAG_TSTOP, A.DRAG_COEFF])
@pytest.mark.parametrize("prec,drag,tol", [(A.FP64, A.DRAG_FP64, 1e-12),
                                           (A.FP32, A.DRAG_FP64, 1e-5),
                                           (A.FP32, A.DRAG_FP32, 1e-5)])
def test_isothermal_dust_parity(law, prec, drag, tol):
    cs = 1.0
    gas, dust, ts = I.dust_box(I.Block((16, 12, 10)), 91, nd=3, t_stop=[0.003, 0.05, 1.0])
    if law == A.DRAG_COEFF:
        ts = [3.0, 0.5, 0.02]      # drag coefficients K_k: t_k = rho_k / K_k
    rc, rd, dts = _oracle(gas, dust, ts, 4, O.DRAG_COEFF if law == A.DRAG_COEFF else O.DRAG_TSTOP,
                          cs)
    cons, d, dt_dev = _gpu(gas.block, gas.cons, dust, ts, dts, prec, law, cs, drag)
    errs = [rel_l1(cons[v], rc[v]) for v in range(4)]
    errs += [rel_l1(d[k, q], rd[k, q]) for k in range(3) for q in range(4)]
    assert max(errs) < tol, errs
    # no drag heating: the isothermal energy slot is carried as set (in
    # the working precision)
    e0 = gas.cons[4] if prec == A.FP64 else gas.cons[4].astype(np.float32).astype(np.float64)
    assert np.array_equal(cons[4], e0)
    # the device CFL step of the end state equals the oracle's (dust c = 0,
    # gas c_s, Cmax = 1 / lambda)
    b = gas.block
    dt_ref = O.dust_dt(O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc),
                       O.make_params(mhd=False, iso=True, cs=cs), O.make_dust_params(
                           ts, law=O.DRAG_COEFF if law == A.DRAG_COEFF else O.DRAG_TSTOP), rc, rd)
    assert abs(dt_dev - dt_ref) <= (1e-12 if prec == A.FP64 else 1e-5) * dt_ref


def test_steady_dusty_shock_on_the_gpu():
    g = _paper_shock_values()
    L, xs, nx, t_end = g["length"][0], 10.0, 200, 4.0
    s = _SteadyDustyShock(g["cs"][0], g["v_up"][0], g["dust_to_gas"], g["K"])
    sol = s.solve(xs, L)
    x = (np.arange(nx) + 0.5) * L / nx
    up = x < xs
    vd = np.where(up[None, :], s.v_up, sol.sol(np.maximum(x, xs)))
    vg = np.where(up, s.v_up, s.v_gas(vd))
    block = I.Block((nx, 1, 1), (0.0, 0.0, 0.0), (L, L / nx, L / nx),
                    bc=(I.OUTFLOW, I.PERIODIC, I.PERIODIC))
    cons = np.zeros((5, 1, 1, nx))
    cons[0, 0, 0] = s.jg / vg
    cons[1, 0, 0] = s.jg
    cons[4] = 1.0
    dust = np.zeros((3, 4, 1, 1, nx))
    for k in range(3):
        dust[k, 0, 0, 0] = s.jd[k] / vd[k]
        dust[k, 1, 0, 0] = s.jd[k]
    ref_g, ref_d = cons[0, 0, 0].copy(), dust[:, 0, 0, 0].copy()
    # the oracle's run and dt sequence
    grid = O.make_grid((nx, 1, 1), hi=(L, L / nx, L / nx), bc=(O.OUTFLOW, O.PERIODIC, O.PERIODIC))
    p = O.make_params(mhd=False, iso=True, cs=g["cs"][0], recon=O.PLM, cfl=0.4)
    dp = O.make_dust_params(g["K"], law=O.DRAG_COEFF)
    oc, od = cons.copy(), dust.copy()
    dts, t = [], 0.0
    while t < t_end - 1e-12:
        dt = min(O.dust_dt(grid, p, dp, oc, od), t_end - t)
        O.dust_step(grid, p, dp, dt, oc, od)
        dts.append(dt)
        t += dt
    gc, gd, _ = _gpu(block, cons, dust, list(g["K"]), dts, A.FP64, A.DRAG_COEFF, g["cs"][0],
                     cfl=0.4)
    assert max(rel_l1(gc[v], oc[v]) for v in range(2)) < 1e-10
    assert max(rel_l1(gd[k, q], od[k, q]) for k in range(3) for q in range(2)) < 1e-10
    keep = np.abs(np.arange(nx) - int(round(xs * nx / L))) > 4
    eg = np.sum(np.abs(gc[0, 0, 0] - ref_g)[keep]) / np.sum(ref_g[keep])
    ed = [np.sum(np.abs(gd[k, 0, 0, 0] - ref_d[k])[keep]) / np.sum(ref_d[k][keep]) for k in range(3)]
    print("steps", len(dts), "structure L1 gas", eg, "dust", ed)
    assert eg < 5e-3 and max(ed) < 5e-3, (eg, ed)
    front = x[np.argmax(gc[0, 0, 0] > 2.5)]
    assert abs(front - xs) < 0.5
    assert gc[0, 0, 0, -1] == pytest.approx(g["compression"][0], rel=1e-4)
    assert np.allclose(gd[:, 0, 0, 0, -1], g["compression"][0], rtol=1e-4)
