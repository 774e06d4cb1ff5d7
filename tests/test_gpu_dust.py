"""GPU parity of the multifluid-dust path (IMEX2P, closed-form FP64 drag,
pressureless Rusanov transport) against the FP64 oracle, element by element
with the oracle's dt sequence.  Tolerances as in test_gpu_parity: 1e-12
relative L1 per variable for the FP64 path, 1e-5 for FP32 transport."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I
from tests.gpu_helpers import rel_l1

pytestmark = pytest.mark.gpu


def _oracle(gas, dust, ts, nsteps, recon=O.PLM, riemann=O.HLLD):
    b = gas.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    p = O.make_params(gamma=gas.gamma, recon=recon, mhd=False, riemann=riemann)
    dp = O.make_dust_params(ts)
    cons = gas.cons.copy()
    d = dust.copy()
    dts = []
    for _ in range(nsteps):
        dt = O.dust_dt(g, p, dp, cons, d)
        O.dust_step(g, p, dp, dt, cons, d)
        dts.append(dt)
    return cons, d, dts


def _gpu(gas, dust, ts, dts, prec, recon=A.PLM, use_run=False, riemann=A.HLLD):
    import torch
    cfg = A.make_config(gamma=gas.gamma, recon=recon, integrator=A.IMEX2P, precision=prec,
                        mhd=False, t_stop=ts, riemann=riemann)
    b = gas.block
    sv = A.Solver(cfg, [A.make_block(b.n, b.lo, b.hi, b.coord, b.bc)],
                  stream=torch.cuda.current_stream())
    try:
        sv.set_state(0, gas.cons)
        for k in range(len(ts)):
            A.aeth_set_dust(sv.ctx, 0, k, np.ascontiguousarray(dust[k]))
        if use_run:
            sv.run(len(dts))
        else:
            for dt in dts:
                sv.step(dt)
        cons = sv.get_state(0)[0]
        d = np.empty_like(dust)
        for k in range(len(ts)):
            buf = np.empty(dust.shape[1:])
            A.aeth_get_dust(sv.ctx, 0, k, buf)
            d[k] = buf
        dt_dev = sv.compute_dt()
    finally:
        sv.close()
    return cons, d, dt_dev


def _errs(cons, d, rc, rd):
    e = [rel_l1(cons[v], rc[v]) for v in range(5)]
    for k in range(d.shape[0]):
        e += [rel_l1(d[k, q], rd[k, q]) for q in range(4)]
    return e


@pytest.mark.parametrize("prec,tol", [(A.FP64, 1e-12), (A.FP32, 1e-5), (A.FP32_P64, 1e-5)])
def test_dust_parity_three_species(prec, tol):
    gas, dust, ts = I.dust_box(I.Block((16, 12, 10)), 81, nd=3, t_stop=[0.002, 0.05, 1.0])
    rc, rd, dts = _oracle(gas, dust, ts, 4)
    cons, d, _ = _gpu(gas, dust, ts, dts, prec)
    errs = _errs(cons, d, rc, rd)
    assert max(errs) < tol, errs


def test_dust_parity_ppm5():
    # gas and dust share the reconstruction: PPM5 on both
    gas, dust, ts = I.dust_box(I.Block((14, 12, 9)), 84, nd=3, t_stop=[0.003, 0.05, 1.0])
    rc, rd, dts = _oracle(gas, dust, ts, 3, recon=O.PPM5)
    cons, d, _ = _gpu(gas, dust, ts, dts, A.FP64, recon=A.PPM5)
    assert max(_errs(cons, d, rc, rd)) < 1e-12


def test_dust_parity_lhllc_gas():
    # the gas solver of a dust run may be the low-dissipation HLLC
    gas, dust, ts = I.dust_box(I.Block((14, 12, 9)), 85, nd=2, t_stop=[0.01, 0.5])
    rc, rd, dts = _oracle(gas, dust, ts, 3, riemann=O.LHLLD)
    cons, d, _ = _gpu(gas, dust, ts, dts, A.FP64, riemann=A.LHLLD)
    assert max(_errs(cons, d, rc, rd)) < 1e-12


def test_dust_parity_eight_species_stiff():
    # the 128^3 recipe at 16^3: t_s log-spaced 1e-4..1, dt/t_s,min ~ 10
    gas, dust, ts = I.dust_box(I.Block((16, 16, 16)), 82, nd=8)
    rc, rd, dts = _oracle(gas, dust, ts, 3)
    assert dts[0] / ts[0] > 5
    cons, d, _ = _gpu(gas, dust, ts, dts, A.FP64)
    assert max(_errs(cons, d, rc, rd)) < 1e-12
    cons, d, _ = _gpu(gas, dust, ts, dts, A.FP32)
    assert max(_errs(cons, d, rc, rd)) < 1e-5


def test_dust_cfl_and_device_run():
    gas, dust, ts = I.dust_box(I.Block((12, 10, 8)), 83, nd=4)
    rc, rd, dts = _oracle(gas, dust, ts, 3)
    cons, d, dt_dev = _gpu(gas, dust, ts, dts, A.FP64, use_run=True)
    assert max(_errs(cons, d, rc, rd)) < 1e-11
    b = gas.block
    dt_ref = O.dust_dt(O.make_grid(b.n), O.make_params(mhd=False), O.make_dust_params(ts), rc, rd)
    assert abs(dt_dev - dt_ref) <= 1e-13 * dt_ref


def test_dust_fp32_drag_against_fp64_oracle():
    # is FP64 needed for the drag solve at the smallest stopping times? The
    # closed form sums positive weights only, so FP32 drag is expected to stay
    # inside the FP32 bound on the stiff 8-species case.
    import torch
    gas, dust, ts = I.dust_box(I.Block((16, 16, 16)), 84, nd=8)
    rc, rd, dts = _oracle(gas, dust, ts, 3)
    cfg = A.make_config(gamma=gas.gamma, recon=A.PLM, integrator=A.IMEX2P, precision=A.FP32,
                        mhd=False, t_stop=ts, drag_precision=A.FP32)
    sv = A.Solver(cfg, [A.make_block(gas.block.n)], stream=torch.cuda.current_stream())
    try:
        sv.set_state(0, gas.cons)
        for k in range(8):
            A.aeth_set_dust(sv.ctx, 0, k, np.ascontiguousarray(dust[k]))
        for dt in dts:
            sv.step(dt)
        cons = sv.get_state(0)[0]
        d = np.empty_like(dust)
        for k in range(8):
            buf = np.empty(dust.shape[1:])
            A.aeth_get_dust(sv.ctx, 0, k, buf)
            d[k] = buf
    finally:
        sv.close()
    assert max(_errs(cons, d, rc, rd)) < 1e-5
