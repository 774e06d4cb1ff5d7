"""GPU parity of the isothermal closure (p = c_s^2 rho, Sec. 2.1) with the
isothermal HLLD (Mignone 2007) and HLLE solvers (Sec. 2.4): the CUDA library
through its C ABI against the pinned FP64 oracle, element by element, on
seeded inputs with the oracle's dt sequence.  Tolerances as in the adiabatic
parity tests: 1e-12 relative L1 per variable in FP64, 1e-5 in FP32.
"""
import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I
from tests.gpu_helpers import compare, gpu_run, oracle_run, rel_l1

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5
CS = 0.8


def _state(n=(20, 18, 13), seed=41, mhd=True):
    return I.smooth_random_mhd(I.Block(n), seed, v_rms=0.7, b_rms=0.6,
                               B0=(0.3, -0.2, 0.1) if mhd else (0, 0, 0), mhd=mhd)


@pytest.mark.parametrize("path", [A.FUSED, A.UNFUSED])
@pytest.mark.parametrize("recon,integ,riemann", [
    ("plm", "vl2", "hlld"), ("ppm", "vl2", "hlld"), ("donor", "rk2", "hlld"),
    ("plm", "rk2", "hlle"), ("ppm", "rk3", "hlld"), ("plm", "vl2", "hlle")])
def test_iso_mhd_fp64_parity(recon, integ, riemann, path):
    st = _state()
    ref, dts = oracle_run(st, recon, integ, nsteps=5, riemann=riemann, iso=True, cs=CS)
    (out,), diag = gpu_run([st], dts, recon, integ, "fp64", path=path, riemann=riemann,
                           iso=True, cs=CS)
    errs = compare(out, ref)
    assert max(errs) < FP64_TOL, errs
    assert diag["max_divb_rel"] < 1e-12


@pytest.mark.parametrize("path", [A.FUSED, A.UNFUSED])
@pytest.mark.parametrize("riemann", ["hlld", "hlle"])
def test_iso_hydro_fp64_parity(riemann, path):
    st = _state(seed=42, mhd=False)
    ref, dts = oracle_run(st, "plm", "rk2", nsteps=5, mhd=False, riemann=riemann, iso=True,
                          cs=CS)
    (out,), _ = gpu_run([st], dts, "plm", "rk2", "fp64", mhd=False, path=path,
                        riemann=riemann, iso=True, cs=CS)
    errs = compare(out, ref, mhd=False)
    assert max(errs) < FP64_TOL, errs


@pytest.mark.parametrize("prec", ["fp32", "fp32_p64"])
@pytest.mark.parametrize("mhd,riemann", [(True, "hlld"), (True, "hlle"), (False, "hlld")])
def test_iso_fp32_parity(prec, mhd, riemann):
    st = _state(seed=43, mhd=mhd)
    ref, dts = oracle_run(st, "plm", "vl2", nsteps=5, mhd=mhd, riemann=riemann, iso=True,
                          cs=CS)
    (out,), _ = gpu_run([st], dts, "plm", "vl2", prec, mhd=mhd, riemann=riemann, iso=True,
                        cs=CS)
    errs = compare(out, ref, mhd=mhd)
    assert max(errs[:4] + errs[5:]) < FP32_TOL, errs


def test_iso_energy_slot_is_carried_unchanged():
    """No energy equation: with VL2 (stage weights 1, 0) the energy entry
    receives a zero flux divergence, so it leaves every step bit for bit
    as it came in, on both sides."""
    st = _state(seed=44)
    ref, dts = oracle_run(st, "plm", "vl2", nsteps=3, iso=True, cs=CS)
    (out,), _ = gpu_run([st], dts, "plm", "vl2", "fp64", iso=True, cs=CS)
    assert np.array_equal(out[0][4], st.cons[4])
    assert np.array_equal(ref.cons[4], st.cons[4])


def test_iso_device_cfl_matches_oracle():
    """aeth_compute_dt and the device-CFL run (graph replay) with the
    isothermal fast speed (gamma = 1, p = c_s^2 rho)."""
    import torch
    st = _state(seed=45)
    g = O.make_grid(st.block.n)
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-6)):
        p = O.make_params(iso=True, cs=CS)
        dt_ref = O.compute_dt(g, p, O.State(st.cons, st.b1, st.b2, st.b3))
        cfg = A.make_config(precision={"fp64": A.FP64, "fp32": A.FP32}[prec], iso=True, cs=CS)
        sv = A.Solver(cfg, [A.make_block(st.block.n)], stream=torch.cuda.current_stream())
        try:
            sv.set_state(0, st.cons, st.b1, st.b2, st.b3)
            dt = sv.compute_dt()
        finally:
            sv.close()
        assert abs(dt - dt_ref) <= tol * dt_ref, (prec, dt, dt_ref)
    ref, dts = oracle_run(st, "plm", "vl2", nsteps=4, iso=True, cs=CS)
    (out,), _ = gpu_run([st], dts, "plm", "vl2", "fp64", use_run=True, iso=True, cs=CS)
    errs = compare(out, ref)
    assert max(errs) < 1e-11, errs


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_iso_shock_tube_outflow_parity(axis):
    # the isothermal tube of the oracle pins (density ratio 4, c_s = 1),
    # along each axis with outflow boundaries
    left = {"rho": 1.0, "v": (0.0, 0.0, 0.0), "p": 1.0}
    right = {"rho": 0.25, "v": (0.0, 0.0, 0.0), "p": 0.25}
    st = I.riemann_1d(axis, 64, left, right, 5.0 / 3.0, ntrans=3)
    ref, dts = oracle_run(st, "plm", "vl2", nsteps=20, mhd=False, iso=True, cs=1.0)
    (out,), _ = gpu_run([st], dts, "plm", "vl2", "fp64", mhd=False, iso=True, cs=1.0)
    errs = compare(out, ref, mhd=False)
    assert all(e < FP64_TOL for e in errs if np.isfinite(e)), errs


def test_iso_uneven_blocks_one_context():
    """Several blocks of different sizes in one context (the device-table
    launch of every pass) with a ragged size along every axis."""
    sts = [_state(n=(12, 10, 9), seed=46), _state(n=(33, 8, 11), seed=47),
           _state(n=(9, 17, 5), seed=48)]
    r0, dts = oracle_run(sts[0], "ppm", "rk2", nsteps=3, iso=True, cs=CS)
    refs = [r0] + [oracle_run(s, "ppm", "rk2", dts=dts, iso=True, cs=CS)[0] for s in sts[1:]]
    outs, _ = gpu_run(sts, dts, "ppm", "rk2", "fp64", iso=True, cs=CS)
    for o, r in zip(outs, refs):
        assert max(compare(o, r)) < FP64_TOL


def test_iso_differs_from_adiabatic():
    """The closure switch reaches the kernels: the isothermal and adiabatic
    runs of the same state differ well beyond round-off."""
    st = _state(seed=49)
    _, dts = oracle_run(st, "plm", "vl2", nsteps=3)
    (a,), _ = gpu_run([st], dts, "plm", "vl2", "fp64")
    (b,), _ = gpu_run([st], dts, "plm", "vl2", "fp64", iso=True, cs=CS)
    assert max(rel_l1(a[0][v], b[0][v]) for v in range(4)) > 1e-6


@pytest.mark.parametrize("path,prec,tol", [(A.FUSED, "fp64", FP64_TOL), (A.UNFUSED, "fp64", FP64_TOL),
                                           (A.FUSED, "fp32", FP32_TOL)])
def test_iso_spherical_block_parity(path, prec, tol):
    """The isothermal closure on a spherical-polar block: the curvilinear
    sources of Eq. 12 take p = c_s^2 rho."""
    import math as _m
    blk = I.Block((16, 12, 10), lo=(1.0, _m.pi / 4, 0.0), hi=(2.0, 3 * _m.pi / 4, _m.pi / 2),
                  coord=I.SPH, bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC))
    st = I.smooth_random_mhd(blk, 50, v_rms=0.3, b_rms=0.4)
    ref, dts = oracle_run(st, "plm", "vl2", nsteps=4, iso=True, cs=CS)
    (out,), diag = gpu_run([st], dts, "plm", "vl2", prec, path=path, iso=True, cs=CS)
    errs = compare(out, ref)
    assert max(errs) < tol, errs
    assert diag["max_divb_rel"] < (1e-12 if prec == "fp64" else 1e-5)


def test_iso_rejected_combinations():
    import torch
    for kw, code in ((dict(riemann=A.MLP, precision=A.FP32), -8), (dict(cs=0.0), -1),
                     (dict(cs=float("nan")), -1), (dict(t_stop=[0.1], mhd=False), -8)):
        cfg = A.make_config(iso=True, **{"cs": CS, **kw})
        with pytest.raises(A.AethError) as e:
            A.Solver(cfg, [A.make_block((8, 8, 8))], stream=torch.cuda.current_stream())
        assert e.value.code == code, kw


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_iso_circularly_polarised_alfven_wave_parity(prec, tol):
    """The paper's isothermal Alfven-wave test (rho = 1, c_s = 1, B_x = 1,
    0.1 amplitude) along x at 32 cells, PLM + HLLE + RK2 for a quarter
    period, against the oracle with its dt sequence."""
    import math as _m
    n, amp = 32, 0.1
    b = I.Block((n, 2, 2))
    X, _, _ = I._cell_mesh(b)
    k = 2 * _m.pi
    sinc = _m.sin(k / n / 2) / (k / n / 2)
    by, bz = amp * np.sin(k * X) * sinc, amp * np.cos(k * X) * sinc
    cons = np.zeros((5,) + X.shape)
    cons[0] = 1.0
    cons[2], cons[3] = -by, -bz
    cons[4] = 1.0      # carried, unused by the isothermal closure
    b1 = np.ones((2, 2, n + 1))
    b2 = np.empty((2, 3, n)); b2[...] = by[:, :1, :]
    b3 = np.empty((3, 2, n)); b3[...] = bz[:1, :, :]
    st = I.InitialState(b, cons, b1, b2, b3, 5.0 / 3.0, {})
    g = O.make_grid(b.n)
    p = O.make_params(recon=O.PLM, integrator=O.RK2, riemann=O.HLLE, iso=True, cs=1.0)
    ref = O.State(cons, b1, b2, b3)
    dts = O.run(g, p, ref, t_end=0.25)
    (out,), diag = gpu_run([st], dts, "plm", "rk2", prec, riemann="hlle", iso=True, cs=1.0)
    errs = compare(out, ref)
    # M1 is only what the scheme's errors make of an exactly zero start:
    # its error is taken against the transverse momentum's norm
    mnorm = (np.sum(np.abs(ref.cons[2])) + np.sum(np.abs(ref.cons[3]))) / 2
    errs[1] = float(np.sum(np.abs(out[0][1] - ref.cons[1])) / mnorm)
    assert max(errs) < tol, errs
    assert diag["max_divb_rel"] < (1e-12 if prec == "fp64" else 1e-5)
