"""Mesh-block decomposition (Sec. 2.3): one domain split into linked blocks
on the GPU against the oracle advancing the whole domain as one block.  The
decomposition is an implementation detail of the GPU path, so the gathered
result must equal the single-domain one: 1e-12 relative L1 in FP64.  Block
sizes are uneven (ragged) along every axis, and each block exchanges faces,
edges and corners with up to 26 neighbours."""
import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I
from tests.gpu_helpers import INTEG, RECON, RIEMANN, PREC, compare, oracle_run, rel_l1

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _gather(outs, origin, splits, n):
    """Assemble per-block (cons, b1, b2, b3) into whole-domain arrays."""
    nx, ny, nz = n
    cons = np.zeros((5, nz, ny, nx))
    b1 = np.zeros((nz, ny, nx + 1))
    b2 = np.zeros((nz, ny + 1, nx))
    b3 = np.zeros((nz + 1, ny, nx))
    for (c, f1, f2, f3), (i0, j0, k0) in zip(outs, origin):
        _, bz, by, bx = c.shape
        cons[:, k0:k0 + bz, j0:j0 + by, i0:i0 + bx] = c
        b1[k0:k0 + bz, j0:j0 + by, i0:i0 + bx + 1] = f1
        b2[k0:k0 + bz, j0:j0 + by + 1, i0:i0 + bx] = f2
        b3[k0:k0 + bz + 1, j0:j0 + by, i0:i0 + bx] = f3
    return cons, b1, b2, b3


def _split_state(st, origin, descs):
    out = []
    for (i0, j0, k0), d in zip(origin, descs):
        bx, by, bz = d.nx, d.ny, d.nz
        out.append((np.ascontiguousarray(st.cons[:, k0:k0 + bz, j0:j0 + by, i0:i0 + bx]),
                    np.ascontiguousarray(st.b1[k0:k0 + bz, j0:j0 + by, i0:i0 + bx + 1]),
                    np.ascontiguousarray(st.b2[k0:k0 + bz, j0:j0 + by + 1, i0:i0 + bx]),
                    np.ascontiguousarray(st.b3[k0:k0 + bz + 1, j0:j0 + by, i0:i0 + bx])))
    return out


def _run_blocks(st, splits, dts, recon="plm", integ="vl2", prec="fp64", mhd=True,
                riemann="hlld", use_run=False, dual=False):
    import torch
    b = st.block
    descs, links, origin = A.decompose(b.n, splits, b.lo, b.hi, b.bc)
    cfg = A.make_config(gamma=st.gamma, recon=RECON[recon][1], integrator=INTEG[integ][1],
                        precision=PREC[prec], mhd=mhd, riemann=RIEMANN[riemann][1], dual=dual)
    sv = A.Solver(cfg, descs, stream=torch.cuda.current_stream(), links=links)
    try:
        for q, parts in enumerate(_split_state(st, origin, descs)):
            sv.set_state(q, *parts)
        if use_run:
            sv.run(len(dts))
        else:
            for dt in dts:
                sv.step(dt)
        outs = [sv.get_state(q) for q in range(len(descs))]
        diag = sv.diagnostics()
        dt_next = sv.compute_dt()
    finally:
        sv.close()
    return _gather(outs, origin, splits, b.n), diag, dt_next


def _box(n, seed, bc=(A.PERIODIC,) * 3):
    blk = I.Block(n, bc=bc)
    return I.smooth_random_mhd(blk, seed, v_rms=0.8, b_rms=0.6, B0=(0.3, -0.2, 0.1))


@pytest.mark.parametrize("recon,integ", [("plm", "vl2"), ("ppm", "rk2"), ("ppm5", "rk3")])
def test_periodic_domain_in_uneven_blocks_matches_single_domain(recon, integ):
    n = (24, 20, 14)
    splits = ([9, 15], [8, 5, 7], [6, 8])     # 12 blocks, ragged along every axis
    st = _box(n, 111)
    ref, dts = oracle_run(st, recon, integ, nsteps=4)
    (cons, b1, b2, b3), diag, _ = _run_blocks(st, splits, dts, recon, integ)
    errs = compare((cons, b1, b2, b3), ref)
    assert max(errs) < FP64_TOL, errs
    assert diag["max_divb_rel"] < 1e-12


def test_outflow_domain_in_blocks_matches_single_domain():
    n = (20, 16, 12)
    st = _box(n, 112, bc=(A.OUTFLOW, A.PERIODIC, A.OUTFLOW))
    ref, dts = oracle_run(st, "plm", "rk2", nsteps=4)
    (cons, b1, b2, b3), diag, _ = _run_blocks(st, ([7, 13], [16], [5, 7]), dts, "plm", "rk2")
    errs = compare((cons, b1, b2, b3), ref)
    assert max(errs) < FP64_TOL, errs


def test_blocks_device_cfl_run_and_fp32():
    n = (24, 16, 16)
    st = _box(n, 113)
    ref, dts = oracle_run(st, "plm", "vl2", nsteps=4)
    (cons, b1, b2, b3), _, dt_next = _run_blocks(st, ([12, 12], [8, 8], [8, 8]), dts, use_run=True)
    assert max(compare((cons, b1, b2, b3), ref)) < 1e-11
    g = O.make_grid(n)
    dt_ref = O.compute_dt(g, O.make_params(), ref)
    assert abs(dt_next - dt_ref) < 1e-13 * dt_ref
    (c32, f1, f2, f3), _, _ = _run_blocks(st, ([12, 12], [8, 8], [8, 8]), dts, prec="fp32")
    assert max(compare((c32, f1, f2, f3), ref)) < 1e-5


def test_blocks_with_lhlld():
    n = (16, 12, 10)
    st = _box(n, 114)
    ref, dts = oracle_run(st, "plm", "rk2", nsteps=3, riemann="lhlld")
    (cons, b1, b2, b3), _, _ = _run_blocks(st, ([8, 8], [5, 7], [10]), dts, "plm", "rk2",
                                           riemann="lhlld")
    assert max(compare((cons, b1, b2, b3), ref)) < FP64_TOL


def test_single_block_linked_to_itself_is_periodic():
    n = (12, 10, 8)
    st = _box(n, 115)
    ref, dts = oracle_run(st, "ppm", "vl2", nsteps=3)
    (cons, b1, b2, b3), _, _ = _run_blocks(st, ([12], [10], [8]), dts, "ppm", "vl2")
    assert max(compare((cons, b1, b2, b3), ref)) < FP64_TOL


def test_linked_blocks_with_dual_energy():
    """Dual energy (Sec. 2.8) across block links: the entropy is a cell
    variable that the fill copies across linked faces like the density.  The
    random MHD box in 12 ragged blocks (most cells trust E) and the cold
    Mach-800 shear in two blocks along x (every cell takes p from S, so the
    entropy crossing the link decides the result) against the dual-energy
    oracle on the whole domain."""
    from tests.test_gpu_dual import _cold_shear, _oracle as _dual_oracle
    st = _box((24, 20, 14), 116)
    ref, dts, _ = _dual_oracle(st, "plm", "vl2", nsteps=4)
    got, diag, _ = _run_blocks(st, ([9, 15], [8, 5, 7], [6, 8]), dts, dual=True)
    assert max(compare(got, ref)) < FP64_TOL
    assert diag["max_divb_rel"] < 1e-12
    sh = _cold_shear()
    ref2, dts2, _ = _dual_oracle(sh, "plm", "rk2", nsteps=12, mhd=False)
    got2, _, _ = _run_blocks(sh, ([24, 40], [4], [4]), dts2, "plm", "rk2", mhd=False, dual=True)
    errs = [rel_l1(got2[0][v], ref2.cons[v]) for v in (0, 1, 2, 4)]
    assert max(errs) < FP64_TOL, errs
