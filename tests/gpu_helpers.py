"""Shared helpers for the GPU parity tests: run the oracle and the CUDA
library on the same seeded input with the oracle's dt sequence, and compare
element by element."""
import numpy as np

import oracle as O
from paper_2608_14048_gb300 import aether as A

RECON = {"donor": (O.DONOR, A.DONOR), "plm": (O.PLM, A.PLM), "ppm": (O.PPM, A.PPM),
         "ppm5": (O.PPM5, A.PPM5)}
INTEG = {"vl2": (O.VL2, A.VL2), "rk2": (O.RK2, A.RK2), "rk3": (O.RK3, A.RK3)}
PREC = {"fp64": A.FP64, "fp32": A.FP32, "fp32_p64": A.FP32_P64}
RIEMANN = {"hlld": (O.HLLD, A.HLLD), "hlle": (O.HLLE, A.HLLE), "lhlld": (O.LHLLD, A.LHLLD)}


def rel_l1(a, b):
    den = np.sum(np.abs(b))
    return float(np.sum(np.abs(a - b)) / den) if den > 0 else float(np.sum(np.abs(a)))


def oracle_run(st, recon="plm", integ="vl2", nsteps=4, mhd=True, dts=None, cfl=0.3,
               riemann="hlld", iso=False, cs=1.0):
    b = st.block
    g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
    p = O.make_params(gamma=st.gamma, recon=RECON[recon][0], integrator=INTEG[integ][0],
                      mhd=mhd, cfl=cfl, riemann=RIEMANN[riemann][0], iso=iso, cs=cs)
    s = O.State(st.cons, st.b1, st.b2, st.b3)
    used = O.run(g, p, s, nsteps=None if dts is not None else nsteps, dts=dts)
    return s, used


def gpu_run(states, dts, recon="plm", integ="vl2", prec="fp64", mhd=True, path=A.FUSED,
            use_run=False, cfl=0.3, riemann="hlld", iso=False, cs=1.0):
    """Advance one or several blocks (list of InitialState) with the given dt
    sequence; returns a list of (cons, b1, b2, b3) per block."""
    import torch
    cfg = A.make_config(gamma=states[0].gamma, recon=RECON[recon][1], integrator=INTEG[integ][1],
                        precision=PREC[prec], mhd=mhd, path=path, cfl=cfl,
                        riemann=RIEMANN[riemann][1], iso=iso, cs=cs)
    blocks = [A.make_block(s.block.n, s.block.lo, s.block.hi, s.block.coord, s.block.bc)
              for s in states]
    sv = A.Solver(cfg, blocks, stream=torch.cuda.current_stream())
    try:
        for i, s in enumerate(states):
            sv.set_state(i, s.cons, s.b1, s.b2, s.b3)
        if use_run:
            sv.run(len(dts))
        else:
            for dt in dts:
                sv.step(dt)
        out = [sv.get_state(i) for i in range(len(states))]
        diag = sv.diagnostics()
    finally:
        sv.close()
    return out, diag


def compare(gpu, ref, mhd=True):
    """Relative L1 per variable: rho, M1, M2, M3, E, b1, b2, b3."""
    cons, b1, b2, b3 = gpu
    errs = [rel_l1(cons[v], ref.cons[v]) for v in range(5)]
    if mhd:
        errs += [rel_l1(b1, ref.b1), rel_l1(b2, ref.b2), rel_l1(b3, ref.b3)]
    return errs
