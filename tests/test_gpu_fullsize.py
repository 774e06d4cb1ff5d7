"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (fused path, FP32 bulk): the GPU advances the whole 256^3 turbulence
box one step; the oracle recomputes sampled sub-boxes.

One VL2 step moves information at most 1 (predictor flux) + 1 (EMF ring)
+ 2 (PLM stencil) + 1 (EMF ring) = 5 cells, so a sub-box cut out of the
periodic input with an 8-cell halo on every side gives the oracle exactly
the data the GPU used for its centre; the centre is compared element by
element (relative L1 <= 1e-5, the FP32 bound).  dt comes from the oracle's
CFL evaluation of the full input.

Normalisation: the five conserved variables use their own L1 norm; the face
field components use the L1 norm of the whole face field (mean over its
three components), because two of them start at exactly zero in this
workload (uniform B_x), so their own norm after one step is O(dt) and would
turn FP32 round-off of the O(1) field into a spurious large ratio.
"""
import numpy as np
import pytest

import oracle as O
from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I
from tests.gpu_helpers import rel_l1

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HALO = 8


def _cut(arr_c, b1, b2, b3, lo, size, n):
    """Periodic sub-box [lo, lo+size) (x, y, z) with its face arrays."""
    ix = [(lo[d] + np.arange(size[d])) % n for d in range(3)]
    cons = arr_c[:, ix[2]][:, :, ix[1]][:, :, :, ix[0]]
    fx = (lo[0] + np.arange(size[0] + 1)) % n
    fy = (lo[1] + np.arange(size[1] + 1)) % n
    fz = (lo[2] + np.arange(size[2] + 1)) % n
    s1 = b1[ix[2]][:, ix[1]][:, :, fx]
    s2 = b2[ix[2]][:, fy][:, :, ix[0]]
    s3 = b3[fz][:, ix[1]][:, :, ix[0]]
    return [np.ascontiguousarray(x) for x in (cons, s1, s2, s3)]


def test_turbulence_256_fp32_one_step_sampled():
    import torch
    n = 256
    st = I.turbulence_box(n=n, seed=20260816, mach=2.0, beta=1.0, gamma=1.0001)
    g = O.make_grid((n, n, n))
    p = O.make_params(gamma=st.gamma, recon=O.PLM)
    dt = O.compute_dt(g, p, O.State(st.cons, st.b1, st.b2, st.b3))
    cfg = A.make_config(gamma=st.gamma, recon=A.PLM, precision=A.FP32, path=A.FUSED)
    sv = A.Solver(cfg, [A.make_block((n, n, n))], stream=torch.cuda.current_stream())
    try:
        sv.set_state(0, st.cons, st.b1, st.b2, st.b3)
        sv.step(dt)
        gc, g1, g2, g3 = sv.get_state(0)
        diag = sv.diagnostics()
    finally:
        sv.close()
    assert diag["max_divb_rel"] < 1e-5
    rng = np.random.default_rng(7)
    corners = [(0, 0, 0), (n - 12, n - 12, n - 12)] + [tuple(rng.integers(0, n, 3)) for _ in range(2)]
    m = 24
    for c0 in corners:
        lo = tuple(int(x) - HALO for x in c0)
        size = (m + 2 * HALO,) * 3
        sub = _cut(st.cons, st.b1, st.b2, st.b3, lo, size, n)
        gs = O.make_grid(size, hi=tuple(x / n for x in size))   # same dx as the full box
        s = O.State(*sub)
        O.step(gs, p, dt, s)
        centre = _cut(gc, g1, g2, g3, tuple(int(x) for x in c0), (m,) * 3, n)
        h = slice(HALO, HALO + m)
        ref = [s.cons[:, h, h, h], s.b1[h, h, HALO:HALO + m + 1], s.b2[h, HALO:HALO + m + 1, h],
               s.b3[HALO:HALO + m + 1, h, h]]
        errs = [rel_l1(centre[0][v], ref[0][v]) for v in range(5)]
        bnorm = sum(np.sum(np.abs(ref[q])) / ref[q].size for q in (1, 2, 3)) / 3
        errs += [float(np.mean(np.abs(centre[q] - ref[q]))) / bnorm for q in (1, 2, 3)]
        assert max(errs) < 1e-5, (c0, errs)


def test_dust_128_eight_species_one_step_sampled():
    import torch
    n = 128
    gas, dust, ts = I.dust_box(I.Block((n, n, n)), 20260817, nd=8)
    g = O.make_grid((n, n, n))
    p = O.make_params(gamma=gas.gamma, recon=O.PLM, mhd=False)
    dp = O.make_dust_params(ts)
    dt = O.dust_dt(g, p, dp, gas.cons, dust)
    cfg = A.make_config(gamma=gas.gamma, recon=A.PLM, integrator=A.IMEX2P, precision=A.FP32,
                        mhd=False, t_stop=ts)
    sv = A.Solver(cfg, [A.make_block((n, n, n))], stream=torch.cuda.current_stream())
    try:
        sv.set_state(0, gas.cons)
        for k in range(8):
            A.aeth_set_dust(sv.ctx, 0, k, np.ascontiguousarray(dust[k]))
        sv.step(dt)
        gc = sv.get_state(0)[0]
        gd = np.empty_like(dust)
        for k in range(8):
            buf = np.empty(dust.shape[1:])
            A.aeth_get_dust(sv.ctx, 0, k, buf)
            gd[k] = buf
    finally:
        sv.close()
    m = 16
    for c0 in [(0, 0, 0), (60, 100, 7)]:
        lo = [x - HALO for x in c0]
        size = (m + 2 * HALO,) * 3
        ix = [(lo[d] + np.arange(size[d])) % n for d in range(3)]
        take = lambda a: np.ascontiguousarray(a[..., ix[2], :, :][..., ix[1], :][..., ix[0]])
        sc, sd = take(gas.cons), take(dust)
        O.dust_step(O.make_grid(size, hi=tuple(x / n for x in size)), p, dp, dt, sc, sd)
        h = slice(HALO, HALO + m)
        jx = [(c0[d] + np.arange(m)) % n for d in range(3)]
        cen = lambda a: a[..., jx[2], :, :][..., jx[1], :][..., jx[0]]
        errs = [rel_l1(cen(gc)[v], sc[v, h, h, h]) for v in range(5)]
        errs += [rel_l1(cen(gd)[k, q], sd[k, q, h, h, h]) for k in range(8) for q in range(4)]
        assert max(errs) < 1e-5, (c0, max(errs))
