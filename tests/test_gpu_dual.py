"""GPU parity of the dual-energy formalism (Sec. 2.8): the CUDA library
through its C ABI against the pinned FP64 oracle, element by element, on
seeded inputs with the oracle's dt sequence: the five conserved variables,
the face fields and the advected entropy S.  Tolerances: 1e-12 relative L1
in FP64, 1e-5 in FP32 (as in the other parity tests)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I
from tests.gpu_helpers import RECON, INTEG, RIEMANN, PREC, rel_l1

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def _oracle(st, recon, integ, riemann="hlld", nsteps=4, dts=None, mhd=True):
    b = st.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    p = O.make_params(gamma=st.gamma, recon=RECON[recon][0], integrator=INTEG[integ][0], mhd=mhd,
                      riemann=RIEMANN[riemann][0], dual=True)
    s = O.dual_init(g, p, O.State(st.cons, st.b1, st.b2, st.b3))
    s_init = s.cons[5].copy()
    used = O.run(g, p, s, nsteps=None if dts is not None else nsteps, dts=dts)
    return s, used, s_init


def _gpu(sts, dts, recon, integ, prec, riemann="hlld", mhd=True, dual=True):
    import torch
    cfg = A.make_config(gamma=sts[0].gamma, recon=RECON[recon][1], integrator=INTEG[integ][1],
                        precision=PREC[prec], mhd=mhd, riemann=RIEMANN[riemann][1], dual=dual)
    blocks = [A.make_block(s.block.n, s.block.lo, s.block.hi, s.block.coord, s.block.bc)
              for s in sts]
    sv = A.Solver(cfg, blocks, stream=torch.cuda.current_stream())
    try:
        for i, s in enumerate(sts):
            sv.set_state(i, s.cons, s.b1, s.b2, s.b3)
        init = [sv.get_entropy(i) for i in range(len(sts))] if dual else None
        for dt in dts:
            sv.step(dt)
        out = [sv.get_state(i) for i in range(len(sts))]
        ent = [sv.get_entropy(i) for i in range(len(sts))] if dual else None
        diag = sv.diagnostics()
    finally:
        sv.close()
    return out, ent, init, diag


def _errs(out, ent, ref, mhd=True):
    cons, b1, b2, b3 = out
    e = [rel_l1(cons[v], ref.cons[v]) for v in range(5)] + [rel_l1(ent, ref.cons[5])]
    if mhd:
        e += [rel_l1(b1, ref.b1), rel_l1(b2, ref.b2), rel_l1(b3, ref.b3)]
    return e


def _box(seed, n=(20, 18, 13), mhd=True, v_rms=0.8):
    return I.smooth_random_mhd(I.Block(n), seed, v_rms=v_rms, b_rms=0.6,
                               B0=(0.3, -0.2, 0.1) if mhd else (0, 0, 0), mhd=mhd)


@pytest.mark.parametrize("recon,integ,riemann", [("plm", "vl2", "hlld"), ("ppm", "rk2", "hlle"),
                                                 ("ppm5", "rk3", "lhlld")])
def test_dual_fp64_parity_random_mhd_box(recon, integ, riemann):
    st = _box(101)
    ref, dts, s_init = _oracle(st, recon, integ, riemann)
    (out,), (ent,), (init,), diag = _gpu([st], dts, recon, integ, "fp64", riemann)
    assert rel_l1(init, s_init) < 1e-14
    errs = _errs(out, ent, ref)
    assert max(errs) < FP64_TOL, errs
    assert diag["max_divb_rel"] < 1e-12


def _cold_shear(n=64):
    """The cold sheared density wave of the oracle pins (Mach ~800, every
    cell takes its pressure from the entropy), as a 3-D state."""
    b = I.Block((n, 4, 4))
    X, _, _ = I._cell_mesh(b)
    h = 1.0 / n
    k = 2 * math.pi
    shape = math.sin(k * h / 2) / (k * h / 2)
    rho = 1.0 + 0.5 * np.cos(k * X) * shape
    vx, vy, p0 = 10.0, 10.0 * np.sin(k * X) * shape, 1e-4
    g_ = 5.0 / 3.0
    cons = np.stack([rho, rho * vx, rho * vy, 0 * rho,
                     p0 / (g_ - 1) + 0.5 * rho * (vx * vx + vy * vy)])
    z = [np.zeros((4, 4, n + 1)), np.zeros((4, 5, n)), np.zeros((5, 4, n))]
    return I.InitialState(b, cons, *z, g_, {})


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", FP32_TOL)])
def test_dual_cold_supersonic_shear_parity(prec, tol):
    """Every cell below alpha_switch: E rewritten from S at every stage.
    FP32 holds the FP32 bound here because the pressure comes from S, not
    from E minus a kinetic energy 10^6 times larger."""
    st = _cold_shear()
    ref, dts, _ = _oracle(st, "plm", "rk2", nsteps=12, mhd=False)
    (out,), (ent,), _, _ = _gpu([st], dts, "plm", "rk2", prec, mhd=False)
    errs = _errs(out, ent, ref, mhd=False)
    # M3 stays exactly zero on both sides
    assert max(errs[q] for q in (0, 1, 2, 4)) < tol, errs
    assert np.max(np.abs(out[0][3])) == 0.0
    # S starts from p = (gamma-1)(E - K) with K ~ 50 and E - K ~ 1.5e-4:
    # one rounding of K (1e-16 relative, FMA-contracted on the GPU, not in
    # the oracle) is 7e-11 of S, which the advection then carries; hence
    # 1e-10 for S in FP64 (measured 1.3e-11)
    assert errs[5] < max(tol, 1e-10), errs


def test_dual_sod_outflow_parity():
    st = I.riemann_1d(0, 128, I.SOD_LEFT, I.SOD_RIGHT, 1.4, ntrans=3)
    ref, dts, _ = _oracle(st, "plm", "vl2", nsteps=25, mhd=False)
    (out,), (ent,), _, _ = _gpu([st], dts, "plm", "vl2", "fp64", mhd=False)
    errs = _errs(out, ent, ref, mhd=False)
    assert all(e < FP64_TOL for e in errs if np.isfinite(e)), errs


def test_dual_uneven_blocks_and_spherical_block():
    sts = [_box(102, n=(12, 10, 9)), _box(103, n=(17, 8, 11)),
           I.smooth_random_mhd(I.Block((10, 12, 8), lo=(1.0, math.pi / 4, 0.0),
                                       hi=(2.0, 3 * math.pi / 4, math.pi / 2), coord=I.SPH,
                                       bc=(I.OUTFLOW, I.OUTFLOW, I.PERIODIC)),
                               104, v_rms=0.3, b_rms=0.4)]
    r0, dts, _ = _oracle(sts[0], "plm", "rk2", nsteps=3)
    refs = [r0] + [_oracle(s, "plm", "rk2", dts=dts)[0] for s in sts[1:]]
    outs, ents, _, _ = _gpu(sts, dts, "plm", "rk2", "fp64")
    for o, e, r in zip(outs, ents, refs):
        errs = _errs(o, e, r)
        assert all(x < FP64_TOL for x in errs if np.isfinite(x)), errs


def test_dual_leaves_the_dynamics_alone_above_alpha_sync():
    # same GPU, same dt: with every cell above alpha_sync the dual run's
    # conserved state and fields are those of the plain run, bit for bit
    st = _box(105, v_rms=0.5)
    ref, dts, _ = _oracle(st, "plm", "rk2")
    (a,), _, _, _ = _gpu([st], dts, "plm", "rk2", "fp64", dual=True)
    (b,), _, _, _ = _gpu([st], dts, "plm", "rk2", "fp64", dual=False)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_dual_rejected_combinations_and_entropy_without_dual():
    import torch
    blk = [A.make_block((8, 8, 8))]
    for kw in (dict(path=A.UNFUSED), dict(precision=A.FP32_P64), dict(iso=True),
               dict(mhd=False, t_stop=[0.1], integrator=A.IMEX2P),
               dict(riemann=A.MLP, precision=A.FP32)):
        with pytest.raises(A.AethError) as e:
            A.Solver(A.make_config(dual=True, **kw), blk, stream=torch.cuda.current_stream())
        assert e.value.code == -8, kw
    sv = A.Solver(A.make_config(), blk, stream=torch.cuda.current_stream())
    try:
        with pytest.raises(A.AethError) as e:
            sv.get_entropy(0)
        assert e.value.code == -7
    finally:
        sv.close()
