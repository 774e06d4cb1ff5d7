"""FP64 CPU oracle of the Aether.jl finite-volume MHD step (arXiv 2608.14048).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the CUDA library and its
Python binding never import it, and it shares no code with them.

The numerics live in plain C (``mhd.c``, ``dust.c``, ``mlp.c``), compiled here
with gcc at ``-O2 -ffp-contract=off`` (no fused multiply-add, so x86 and Arm
give the same bits).  This file only marshals numpy arrays into those calls.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["mhd.c", "dust.c", "mlp.c", "learned.c"]
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

CART, SPH = 0, 1
PERIODIC, OUTFLOW = 0, 1
DONOR, PLM, PPM, PPM5 = 0, 1, 2, 3
VL2, RK2, RK3 = 0, 1, 2
HLLD, HLLE, LHLLD = 0, 1, 2
DRAG_TSTOP, DRAG_COEFF = 0, 1


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("coord", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", C.c_int * 3)]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("recon", C.c_int),
                ("integrator", C.c_int), ("cfl", C.c_double), ("mhd", C.c_int),
                ("riemann", C.c_int), ("iso", C.c_int), ("cs_iso", C.c_double),
                ("dual", C.c_int), ("alpha_switch", C.c_double), ("alpha_sync", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("mom", C.c_double * 3),
                ("energy", C.c_double), ("max_divb_rel", C.c_double),
                ("floor_hits", C.c_long)]


class DustParams(C.Structure):
    _fields_ = [("nd", C.c_int), ("t_stop", C.POINTER(C.c_double)),
                ("rho_floor_dust", C.c_double), ("gas_accel", C.c_double * 3),
                ("law", C.c_int)]


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle's C sources into ``liborc.so`` next to them."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h"),
                                                       os.path.join(_HERE, "oracle_internal.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unknown-pragmas"]
    if openmp:
        cmd.append("-fopenmp")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd += srcs + ["-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.orc_mhd_step.argtypes = [C.POINTER(Grid), C.POINTER(Params), C.c_double,
                                       dp, dp, dp, dp, C.POINTER(C.c_long)]
            L.orc_mhd_step.restype = C.c_int
            L.orc_mhd_dt.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, dp, dp, dp]
            L.orc_mhd_dt.restype = C.c_double
            L.orc_mhd_diag.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, dp, dp, dp,
                                       C.POINTER(Diag)]
            L.orc_mhd_diag.restype = None
            L.orc_hlld.argtypes = [C.c_double, dp, dp, C.c_double, dp]
            L.orc_hlld.restype = C.c_int
            L.orc_lhlld.argtypes = [C.c_double, dp, dp, C.c_double, dp]
            L.orc_lhlld.restype = C.c_int
            L.orc_dual_init.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, dp, dp, dp]
            L.orc_dual_init.restype = None
            L.orc_hlle.argtypes = [C.c_double, dp, dp, C.c_double, dp]
            L.orc_hlle.restype = None
            for fn in ("orc_hlld_iso", "orc_hlle_iso"):
                getattr(L, fn).argtypes = [C.c_double, dp, dp, C.c_double, dp]
                getattr(L, fn).restype = None
            L.orc_recon_line.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.orc_recon_line.restype = None
            L.orc_corner_emf.argtypes = [C.c_double] * 4 + [dp] + [C.c_double] * 4
            L.orc_corner_emf.restype = C.c_double
            if hasattr(L, "orc_drag_solve"):
                L.orc_drag_solve.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, dp, dp]
                L.orc_drag_solve.restype = None
                L.orc_dust_step.argtypes = [C.POINTER(Grid), C.POINTER(Params),
                                            C.POINTER(DustParams), C.c_double, dp, dp,
                                            C.POINTER(C.c_long)]
                L.orc_dust_step.restype = C.c_int
                L.orc_dust_dt.argtypes = [C.POINTER(Grid), C.POINTER(Params),
                                          C.POINTER(DustParams), dp, dp]
                L.orc_dust_dt.restype = C.c_double
            if hasattr(L, "orc_mlp_forward"):
                ip = C.POINTER(C.c_int)
                L.orc_mlp_forward.argtypes = [C.c_int, ip, dp, C.c_int, dp, dp]
                L.orc_mlp_forward.restype = None
                L.orc_mlp_grad.argtypes = [C.c_int, ip, dp, C.c_int, dp, dp, dp]
                L.orc_mlp_grad.restype = C.c_double
            if hasattr(L, "orc_learned_flux_batch"):
                ip = C.POINTER(C.c_int)
                L.orc_learned_flux_batch.argtypes = [C.c_double, C.c_int, dp, dp, dp, dp,
                                                     C.c_double, C.c_int, dp, ip, dp]
                L.orc_learned_flux_batch.restype = None
                L.orc_learned_target.argtypes = [C.c_double, dp, dp, C.c_double, dp]
                L.orc_learned_target.restype = None
                L.orc_learned_features.argtypes = [C.c_double, dp, dp, C.c_double, dp, dp]
                L.orc_learned_features.restype = None
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_grid(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), coord=CART, bc=(PERIODIC,) * 3) -> Grid:
    nx, ny, nz = n
    return Grid(nx, ny, nz, coord, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi),
                (C.c_int * 3)(*bc))


def make_params(gamma=5.0 / 3.0, recon=PLM, integrator=VL2, cfl=0.3, mhd=True,
                rho_floor=1e-12, p_floor=1e-10, riemann=HLLD, iso=False, cs=1.0, dual=False,
                alpha_switch=1e-3, alpha_sync=1e-1) -> Params:
    """iso=True: the isothermal closure p = cs^2 rho (gamma unused).
    dual=True: the dual-energy formalism (Sec. 2.8); the state's cons then
    has six variables, the sixth the entropy S (see dual_init)."""
    return Params(gamma, rho_floor, p_floor, recon, integrator, cfl, 1 if mhd else 0, riemann,
                  1 if iso else 0, cs, 1 if dual else 0, alpha_switch, alpha_sync)


class State:
    """Host FP64 state of one block: cons[5][nz][ny][nx] and the three face
    arrays with the shapes of the C interface."""

    def __init__(self, cons, b1=None, b2=None, b3=None):
        # always private copies: the oracle advances them in place
        self.cons = np.array(cons, dtype=np.float64, order="C", copy=True)
        nz, ny, nx = self.cons.shape[1:]
        z = lambda s: np.zeros(s, dtype=np.float64)
        self.b1 = np.array(b1 if b1 is not None else z((nz, ny, nx + 1)), dtype=np.float64, order="C", copy=True)
        self.b2 = np.array(b2 if b2 is not None else z((nz, ny + 1, nx)), dtype=np.float64, order="C", copy=True)
        self.b3 = np.array(b3 if b3 is not None else z((nz + 1, ny, nx)), dtype=np.float64, order="C", copy=True)

    def copy(self) -> "State":
        return State(self.cons.copy(), self.b1.copy(), self.b2.copy(), self.b3.copy())


def dual_init(grid: Grid, params: Params, s: State) -> State:
    """A copy of ``s`` with the entropy S = p / rho^(gamma-1) appended as the
    sixth cell variable (orc_dual_init), for dual-energy runs."""
    out = s.copy()
    cons6 = np.zeros((6,) + out.cons.shape[1:])
    cons6[:5] = out.cons[:5]
    out.cons = np.ascontiguousarray(cons6)
    lib().orc_dual_init(C.byref(grid), C.byref(params), _dp(out.cons), _dp(out.b1),
                        _dp(out.b2), _dp(out.b3))
    return out


def step(grid: Grid, params: Params, dt: float, s: State) -> int:
    """Advance ``s`` in place by one full step; returns the floor-hit count."""
    hits = C.c_long(0)
    rc = lib().orc_mhd_step(C.byref(grid), C.byref(params), float(dt), _dp(s.cons),
                            _dp(s.b1), _dp(s.b2), _dp(s.b3), C.byref(hits))
    if rc != 0:
        raise RuntimeError(f"orc_mhd_step failed: {rc}")
    return hits.value


def compute_dt(grid: Grid, params: Params, s: State) -> float:
    return lib().orc_mhd_dt(C.byref(grid), C.byref(params), _dp(s.cons), _dp(s.b1),
                            _dp(s.b2), _dp(s.b3))


def diagnostics(grid: Grid, params: Params, s: State) -> dict:
    d = Diag()
    lib().orc_mhd_diag(C.byref(grid), C.byref(params), _dp(s.cons), _dp(s.b1), _dp(s.b2),
                       _dp(s.b3), C.byref(d))
    return {"mass": d.mass, "mom": list(d.mom), "energy": d.energy,
            "max_divb_rel": d.max_divb_rel}


def hlld(gamma: float, wl, wr, bn: float):
    """Face-frame HLLD flux; returns (flux[7], region)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(7)
    reg = lib().orc_hlld(float(gamma), _dp(wl), _dp(wr), float(bn), _dp(f))
    return f, reg


def lhlld(gamma: float, wl, wr, bn: float):
    """Face-frame low-dissipation HLLD flux (orc_lhlld); returns (flux[7], region)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(7)
    reg = lib().orc_lhlld(float(gamma), _dp(wl), _dp(wr), float(bn), _dp(f))
    return f, reg


def hlld_iso(cs: float, wl, wr, bn: float):
    """Face-frame isothermal HLLD flux[7] (orc_hlld_iso; energy entry 0)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(7)
    lib().orc_hlld_iso(float(cs), _dp(wl), _dp(wr), float(bn), _dp(f))
    return f


def hlle_iso(cs: float, wl, wr, bn: float):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(7)
    lib().orc_hlle_iso(float(cs), _dp(wl), _dp(wr), float(bn), _dp(f))
    return f


def hlle(gamma: float, wl, wr, bn: float):
    """Face-frame HLLE flux[7] (orc_hlle)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(7)
    lib().orc_hlle(float(gamma), _dp(wl), _dp(wr), float(bn), _dp(f))
    return f


def recon_line(recon: int, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = w.size
    wl = np.zeros(max(n - 1, 0))
    wr = np.zeros(max(n - 1, 0))
    lib().orc_recon_line(recon, n, _dp(w), _dp(wl), _dp(wr))
    return wl, wr


def corner_emf(ea_m, ea_p, eb_m, eb_p, eref, fa_m, fa_p, fb_m, fb_p) -> float:
    r = np.ascontiguousarray(np.asarray(eref, dtype=np.float64).reshape(4))
    return lib().orc_corner_emf(ea_m, ea_p, eb_m, eb_p, _dp(r), fa_m, fa_p, fb_m, fb_p)


def run(grid: Grid, params: Params, s: State, nsteps: int = None, t_end: float = None,
        dts=None):
    """Advance with the CFL step of Eq. 11 (or a given dt sequence); returns
    the list of dt values used."""
    used = []
    t = 0.0
    k = 0
    while True:
        if dts is not None:
            if k >= len(dts):
                break
            dt = dts[k]
        else:
            if nsteps is not None and k >= nsteps:
                break
            dt = compute_dt(grid, params, s)
            if t_end is not None:
                if t >= t_end * (1 - 1e-14):
                    break
                dt = min(dt, t_end - t)
        step(grid, params, dt, s)
        used.append(dt)
        t += dt
        k += 1
    return used


# ---- multifluid dust (dust.c) ------------------------------------------

def make_dust_params(t_stop, rho_floor_dust=1e-20, gas_accel=(0.0, 0.0, 0.0), law=DRAG_TSTOP):
    """Dust parameters (Sec. 2.2).  ``t_stop`` holds the stopping times t_k
    (law DRAG_TSTOP) or the drag coefficients K_k of the constant-coefficient
    law t_k = rho_k / K_k (law DRAG_COEFF)."""
    ts = np.ascontiguousarray(t_stop, dtype=np.float64)
    dp = DustParams(len(ts), _dp(ts), rho_floor_dust, (C.c_double * 3)(*gas_accel), law)
    dp._keep = ts
    return dp


def drag_solve(h, rho_g, v_g, rho_d, v_d, t_stop):
    """One implicit drag solve of one velocity component; returns (v_g', v_d')."""
    rd = np.ascontiguousarray(rho_d, dtype=np.float64)
    vd = np.array(v_d, dtype=np.float64)
    ts = np.ascontiguousarray(t_stop, dtype=np.float64)
    vg = C.c_double(v_g)
    lib().orc_drag_solve(len(rd), float(h), float(rho_g), _dp(rd), _dp(ts), C.byref(vg), _dp(vd))
    return vg.value, vd


def dust_step(grid, params, dparams, dt, cons, dust) -> int:
    """One IMEX2P step of gas (hydro) + dust, in place on the numpy arrays
    cons[5][nz][ny][nx] and dust[nd][4][nz][ny][nx]."""
    hits = C.c_long(0)
    rc = lib().orc_dust_step(C.byref(grid), C.byref(params), C.byref(dparams), float(dt),
                             _dp(cons), _dp(dust), C.byref(hits))
    if rc != 0:
        raise RuntimeError(f"orc_dust_step failed: {rc}")
    return hits.value


def dust_dt(grid, params, dparams, cons, dust) -> float:
    return lib().orc_dust_dt(C.byref(grid), C.byref(params), C.byref(dparams), _dp(cons), _dp(dust))


# ---- learned-flux MLP reference (mlp.c) --------------------------------

def mlp_forward(dims, params, x):
    """FP64 forward pass; x[n][dims[0]] -> y[n][dims[-1]]."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    y = np.zeros((n, dims[-1]))
    lib().orc_mlp_forward(len(dims) - 1, d.ctypes.data_as(C.POINTER(C.c_int)), _dp(p), n,
                          _dp(x), _dp(y))
    return y


def mlp_grad(dims, params, x, target):
    """(loss, gradient) of 0.5/n sum |y - t|^2 by backpropagation."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64)
    g = np.zeros_like(p)
    loss = lib().orc_mlp_grad(len(dims) - 1, d.ctypes.data_as(C.POINTER(C.c_int)), _dp(p),
                              x.shape[0], _dp(x), _dp(t), _dp(g))
    return loss, g


def mlp_param_count(dims):
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def learned_flux(gamma, wl, wr, bn, params, tau=0.25, mhd=True, info=False):
    """The learned face flux (learned.c) of n face-frame states: wl, wr
    [n][7], bn [n], the 14-128-128-128-7 network params (packed W then b per
    layer).  Returns (flux [n][7], accepted [n] bool) and, with info=True,
    the per-face record [n][24] (candidate F, J, k, the two margins, y)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64).reshape(-1, 7)
    wr = np.ascontiguousarray(wr, dtype=np.float64).reshape(-1, 7)
    bn = np.ascontiguousarray(bn, dtype=np.float64).reshape(-1)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    n = wl.shape[0]
    flux = np.zeros((n, 7))
    acc = np.zeros(n, dtype=np.int32)
    rec = np.zeros((n, 24)) if info else None
    lib().orc_learned_flux_batch(float(gamma), n, _dp(wl), _dp(wr), _dp(bn), _dp(prm),
                                 float(tau), 1 if mhd else 0, _dp(flux),
                                 acc.ctypes.data_as(C.POINTER(C.c_int)),
                                 _dp(rec) if info else None)
    return (flux, acc.astype(bool), rec) if info else (flux, acc.astype(bool))


def learned_target(gamma, wl, wr, bn):
    """The network's training target y = (F_HLLD - F_E) / (k J) of one face."""
    y = np.zeros(7)
    lib().orc_learned_target(float(gamma), _dp(np.ascontiguousarray(wl, dtype=np.float64)),
                             _dp(np.ascontiguousarray(wr, dtype=np.float64)), float(bn), _dp(y))
    return y


def learned_features(gamma, wl, wr, bn):
    """The 14 features and the 7 flux scales k of one face."""
    x, k = np.zeros(14), np.zeros(7)
    lib().orc_learned_features(float(gamma), _dp(np.ascontiguousarray(wl, dtype=np.float64)),
                               _dp(np.ascontiguousarray(wr, dtype=np.float64)), float(bn),
                               _dp(x), _dp(k))
    return x, k
