"""Thin Python binding of the C ABI in include/aether_gb.h.

Argument marshalling only: every step of the MHD update runs in the CUDA
library libaether_gb.so.  The functions keep the C names (aeth_create,
aeth_step, ...); `Solver` is a small convenience wrapper over them.

PyTorch is used only for device memory and streams: a torch CUDA tensor can
serve as the library's arena (aeth_bind_arena) and the current torch stream
can be bound (aeth_bind_stream).  If the library is missing this module
raises at import of the library (no CPU fallback exists).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaether_gb.so")

AETH_OK = 0
STATUS = {0: "AETH_OK", -1: "AETH_ERR_ARG", -2: "AETH_ERR_OOM", -3: "AETH_ERR_CUDA",
          -4: "AETH_ERR_NONFINITE", -5: "AETH_ERR_FLOOR", -6: "AETH_ERR_TIMEOUT",
          -7: "AETH_ERR_STATE", -8: "AETH_ERR_UNSUPPORTED"}
EOS_MHD, EOS_HYDRO, EOS_ISO_MHD, EOS_ISO_HYDRO = 0, 1, 2, 3
DONOR, PLM, PPM, PPM5 = 0, 1, 2, 3
HLLD, HLLE, MLP, LHLLD = 0, 1, 2, 3
TCGEN05, MMA_SYNC = 0, 1          # tensor-core engine of the learned flux
VL2, RK2, IMEX2P, RK3 = 0, 1, 2, 3
FP64, FP32, FP32_P64, FP32_SEL64 = 0, 1, 2, 3
DRAG_FP64, DRAG_FP32, DRAG_SEL64 = 0, 1, 2      # drag_precision
DRAG_TSTOP, DRAG_COEFF = 0, 1                    # drag_law
CART, SPH = 0, 1
PERIODIC, OUTFLOW = 0, 1
FUSED, UNFUSED = 0, 1

# every symbol include/aether_gb.h declares
EXPORTS = ["aeth_create", "aeth_bind_stream", "aeth_bind_arena", "aeth_add_block", "aeth_plan",
           "aeth_finalize", "aeth_set_state", "aeth_get_state", "aeth_set_state_async",
           "aeth_get_state_async", "aeth_state_doubles", "aeth_set_state_all_async",
           "aeth_get_state_all_async", "aeth_compute_dt", "aeth_step",
           "aeth_run", "aeth_sync", "aeth_diagnostics", "aeth_set_dust", "aeth_get_dust",
           "aeth_load_mlp", "aeth_mlp_infer", "aeth_mlp_infer_tc", "aeth_mlp_face_flux", "aeth_selftest_wait_timeout", "aeth_mlp_collect", "aeth_mlp_work_floats", "aeth_mlp_grad",
           "aeth_mlp_adam", "aeth_profile", "aeth_profile_read", "aeth_autotune",
           "aeth_set_flux_tile", "aeth_get_flux_tile",
           "aeth_cfl_dt_noalloc", "aeth_get_entropy", "aeth_link_blocks", "aeth_probe_fma",
           "aeth_last_error", "aeth_destroy"]


class AethError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class aeth_config(C.Structure):
    _fields_ = [("eos", C.c_int), ("gamma", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("recon", C.c_int), ("riemann", C.c_int),
                ("integrator", C.c_int), ("cfl", C.c_double), ("precision", C.c_int),
                ("path", C.c_int), ("strict_floors", C.c_int), ("n_dust", C.c_int),
                ("t_stop", C.POINTER(C.c_double)), ("drag_precision", C.c_int),
                ("mlp_tau", C.c_double), ("mlp_engine", C.c_int), ("cs_iso", C.c_double),
                ("dual_energy", C.c_int), ("alpha_switch", C.c_double),
                ("alpha_sync", C.c_double), ("p64_ratio", C.c_double),
                ("drag_ratio", C.c_double), ("drag_law", C.c_int)]


class aeth_block_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("coord", C.c_int),
                ("x1min", C.c_double), ("x1max", C.c_double), ("x2min", C.c_double),
                ("x2max", C.c_double), ("x3min", C.c_double), ("x3max", C.c_double),
                ("bc", C.c_int * 3)]


class aeth_diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("mom", C.c_double * 3), ("energy", C.c_double),
                ("max_divb_rel", C.c_double), ("floor_hits", C.c_longlong),
                ("mlp_fallbacks", C.c_longlong)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libaether_gb.so (built by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    sig = {
        "aeth_create": ([C.POINTER(aeth_config), C.POINTER(P)], C.c_int),
        "aeth_bind_stream": ([P, P], C.c_int),
        "aeth_bind_arena": ([P, P, C.c_size_t], C.c_int),
        "aeth_add_block": ([P, C.POINTER(aeth_block_desc), C.POINTER(C.c_int)], C.c_int),
        "aeth_plan": ([P, C.POINTER(C.c_size_t)], C.c_int),
        "aeth_finalize": ([P, C.POINTER(C.c_size_t)], C.c_int),
        "aeth_set_state": ([P, C.c_int, P, P, P, P], C.c_int),
        "aeth_get_state": ([P, C.c_int, P, P, P, P], C.c_int),
        "aeth_set_state_async": ([P, C.c_int, P, P, P, P], C.c_int),
        "aeth_get_state_async": ([P, C.c_int, P, P, P, P], C.c_int),
        "aeth_state_doubles": ([P, P], C.c_int),
        "aeth_set_state_all_async": ([P, P], C.c_int),
        "aeth_get_state_all_async": ([P, P], C.c_int),
        "aeth_compute_dt": ([P, dp], C.c_int),
        "aeth_step": ([P, C.c_double], C.c_int),
        "aeth_run": ([P, C.c_int], C.c_int),
        "aeth_sync": ([P], C.c_int),
        "aeth_diagnostics": ([P, C.POINTER(aeth_diag)], C.c_int),
        "aeth_set_dust": ([P, C.c_int, C.c_int, P], C.c_int),
        "aeth_get_dust": ([P, C.c_int, C.c_int, P], C.c_int),
        "aeth_load_mlp": ([P, P, C.c_size_t], C.c_int),
        "aeth_mlp_infer": ([P, P, P, C.c_int], C.c_int),
        "aeth_mlp_infer_tc": ([P, P, P, C.c_int], C.c_int),
        "aeth_mlp_face_flux": ([P, P, P, P, C.c_int], C.c_int),
        "aeth_selftest_wait_timeout": ([P], C.c_int),
        "aeth_mlp_collect": ([P, C.c_int, P, P, C.c_longlong, C.POINTER(C.c_longlong)], C.c_int),
        "aeth_mlp_work_floats": ([C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "aeth_mlp_grad": ([P, P, P, C.c_int, P, P, C.c_size_t, P, P], C.c_int),
        "aeth_mlp_adam": ([P, P, P, P, C.c_longlong, C.c_int, C.c_float, C.c_float, C.c_float,
                           C.c_float, P], C.c_int),
        "aeth_profile": ([P, C.c_int], C.c_int),
        "aeth_profile_read": ([P, dp, C.POINTER(C.c_longlong), dp, C.POINTER(C.c_longlong)],
                              C.c_int),
        "aeth_autotune": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "aeth_set_flux_tile": ([P, C.c_int, C.c_int], C.c_int),
        "aeth_get_flux_tile": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "aeth_cfl_dt_noalloc": ([P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_int, P, P], C.c_int),
        "aeth_last_error": ([P], C.c_char_p),
        "aeth_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(a):
    """Host pointer of a numpy array or a (CPU, pinned or not) torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "need C-contiguous float64"
        return a.ctypes.data_as(C.c_void_p)
    import torch  # noqa: WPS433 (only when a tensor is passed)
    assert isinstance(a, torch.Tensor) and a.dtype == torch.float64 and a.is_contiguous()
    assert a.device.type == "cpu", "state arrays are host buffers"
    return C.c_void_p(a.data_ptr())


# ---- C names -------------------------------------------------------------

def aeth_create(cfg: aeth_config):
    h = C.c_void_p()
    _check(None, load_library().aeth_create(C.byref(cfg), C.byref(h)))
    return h


def aeth_bind_stream(ctx, stream_ptr: int):
    _check(ctx, load_library().aeth_bind_stream(ctx, C.c_void_p(stream_ptr)))


def aeth_bind_arena(ctx, dev_ptr: int, nbytes: int):
    _check(ctx, load_library().aeth_bind_arena(ctx, C.c_void_p(dev_ptr), nbytes))


def aeth_add_block(ctx, desc: aeth_block_desc) -> int:
    bid = C.c_int(-1)
    _check(ctx, load_library().aeth_add_block(ctx, C.byref(desc), C.byref(bid)))
    return bid.value


def aeth_plan(ctx) -> int:
    n = C.c_size_t(0)
    _check(ctx, load_library().aeth_plan(ctx, C.byref(n)))
    return n.value


def aeth_finalize(ctx) -> int:
    n = C.c_size_t(0)
    _check(ctx, load_library().aeth_finalize(ctx, C.byref(n)))
    return n.value


def aeth_set_state(ctx, block, cons, b1=None, b2=None, b3=None):
    _check(ctx, load_library().aeth_set_state(ctx, block, _ptr(cons), _ptr(b1), _ptr(b2), _ptr(b3)))


def aeth_get_state(ctx, block, cons, b1=None, b2=None, b3=None):
    _check(ctx, load_library().aeth_get_state(ctx, block, _ptr(cons), _ptr(b1), _ptr(b2), _ptr(b3)))


def aeth_set_state_async(ctx, block, cons, b1=None, b2=None, b3=None):
    """Enqueue the state upload on the context's stream (page-locked host
    arrays, e.g. torch pin_memory(); keep them unchanged until the stream
    has passed the call)."""
    _check(ctx, load_library().aeth_set_state_async(ctx, block, _ptr(cons), _ptr(b1), _ptr(b2),
                                                     _ptr(b3)))


def aeth_state_doubles(ctx) -> int:
    """Length (doubles) of the packed state of every block."""
    n = C.c_size_t(0)
    _check(ctx, load_library().aeth_state_doubles(ctx, C.byref(n)))
    return n.value


def aeth_set_state_all_async(ctx, packed):
    """Enqueue the upload of every block's state from one packed,
    page-locked host array (block after block: cons, then b1, b2, b3)."""
    _check(ctx, load_library().aeth_set_state_all_async(ctx, _ptr(packed)))


def aeth_get_state_all_async(ctx, packed):
    """Enqueue the read-back of every block's state into one packed,
    page-locked host array."""
    _check(ctx, load_library().aeth_get_state_all_async(ctx, _ptr(packed)))


def pack_states(states, mhd=True, dust=None):
    """The packed host layout of aeth_set_state_all_async from per-block
    (cons, b1, b2, b3) arrays (numpy, FP64), with each block's dust species
    [nd][4][nz][ny][nx] after it when `dust` (one array per block) is given."""
    parts = []
    for q, st in enumerate(states):
        parts.append(np.ascontiguousarray(st[0], dtype=np.float64).ravel())
        if mhd:
            parts += [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in st[1:4]]
        if dust is not None:
            parts.append(np.ascontiguousarray(dust[q], dtype=np.float64).ravel())
    return np.concatenate(parts)


def aeth_get_state_async(ctx, block, cons, b1=None, b2=None, b3=None):
    """Enqueue the state read-back on the context's stream (page-locked host
    arrays; valid once the stream has passed the call)."""
    _check(ctx, load_library().aeth_get_state_async(ctx, block, _ptr(cons), _ptr(b1), _ptr(b2),
                                                     _ptr(b3)))


def aeth_probe_fma(precision) -> float:
    """Measured FMA throughput (FLOP/s) of the current device, FP32 or FP64."""
    f = C.c_double(0)
    _check(None, load_library().aeth_probe_fma(int(precision), C.byref(f)))
    return f.value


def aeth_link_blocks(ctx, lo, axis, hi):
    _check(ctx, load_library().aeth_link_blocks(ctx, int(lo), int(axis), int(hi)))


def decompose(n, splits, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(PERIODIC,) * 3):
    """Split the box [lo, hi] of n = (nx, ny, nz) cells into blocks with
    splits[d] = the cell counts along axis d (summing to n[d]).  Returns the
    block descriptors (x fastest), their links (lo, axis, hi) -- periodic
    axes wrap around -- and each block's first cell (i0, j0, k0)."""
    assert all(sum(splits[d]) == n[d] for d in range(3))
    dx = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    starts = [np.concatenate([[0], np.cumsum(splits[d])[:-1]]).astype(int) for d in range(3)]
    nb = [len(splits[d]) for d in range(3)]
    descs, origin = [], []
    idx = lambda a, b, c: (c * nb[1] + b) * nb[0] + a
    for c in range(nb[2]):
        for b in range(nb[1]):
            for a in range(nb[0]):
                p = (a, b, c)
                cnt = [splits[d][p[d]] for d in range(3)]
                o = [int(starts[d][p[d]]) for d in range(3)]
                l3 = [lo[d] + o[d] * dx[d] for d in range(3)]
                h3 = [lo[d] + (o[d] + cnt[d]) * dx[d] for d in range(3)]
                descs.append(make_block(tuple(cnt), tuple(l3), tuple(h3), CART, bc))
                origin.append(tuple(o))
    links = []
    for c in range(nb[2]):
        for b in range(nb[1]):
            for a in range(nb[0]):
                p = [a, b, c]
                for d in range(3):
                    q = list(p)
                    q[d] += 1
                    if q[d] == nb[d]:
                        if bc[d] != PERIODIC:
                            continue
                        q[d] = 0
                    links.append((idx(*p), d, idx(*q)))
    return descs, links, origin


def aeth_get_entropy(ctx, block, S):
    _check(ctx, load_library().aeth_get_entropy(ctx, block, _ptr(S)))


def aeth_compute_dt(ctx) -> float:
    dt = C.c_double(0)
    _check(ctx, load_library().aeth_compute_dt(ctx, C.byref(dt)))
    return dt.value


def aeth_step(ctx, dt: float):
    _check(ctx, load_library().aeth_step(ctx, float(dt)))


def aeth_run(ctx, nsteps: int):
    _check(ctx, load_library().aeth_run(ctx, int(nsteps)))


def aeth_sync(ctx):
    _check(ctx, load_library().aeth_sync(ctx))


def aeth_diagnostics(ctx) -> dict:
    d = aeth_diag()
    _check(ctx, load_library().aeth_diagnostics(ctx, C.byref(d)))
    return {"mass": d.mass, "mom": list(d.mom), "energy": d.energy,
            "max_divb_rel": d.max_divb_rel, "floor_hits": d.floor_hits,
            "mlp_fallbacks": d.mlp_fallbacks}


def aeth_set_dust(ctx, block, k, rho_mom):
    _check(ctx, load_library().aeth_set_dust(ctx, block, k, _ptr(rho_mom)))


def aeth_get_dust(ctx, block, k, rho_mom):
    _check(ctx, load_library().aeth_get_dust(ctx, block, k, _ptr(rho_mom)))


def aeth_load_mlp(ctx, params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, load_library().aeth_load_mlp(ctx, p.ctypes.data_as(C.c_void_p), p.size))


MLP_DIMS = [14, 128, 128, 128, 7]
MLP_NPARAM = sum(MLP_DIMS[l + 1] * MLP_DIMS[l] + MLP_DIMS[l + 1] for l in range(4))


def aeth_mlp_infer(ctx, d_X: int, d_Y: int, n: int):
    _check(ctx, load_library().aeth_mlp_infer(ctx, C.c_void_p(d_X), C.c_void_p(d_Y), int(n)))


def aeth_mlp_infer_tc(ctx, d_X: int, d_Y: int, n: int):
    _check(ctx, load_library().aeth_mlp_infer_tc(ctx, C.c_void_p(d_X), C.c_void_p(d_Y), int(n)))


def aeth_mlp_face_flux(ctx, d_states: int, d_flux: int, d_accept: int, n: int):
    """Learned face flux (network + checks + HLLD fallback) of n face-frame
    states d_states[n][15] into d_flux[n][7] and d_accept[n] (device
    pointers); asynchronous on the bound stream."""
    _check(ctx, load_library().aeth_mlp_face_flux(ctx, C.c_void_p(d_states), C.c_void_p(d_flux),
                                                  C.c_void_p(d_accept), int(n)))


def aeth_selftest_wait_timeout(ctx) -> int:
    """Status code of the bounded-wait self-test (AETH_ERR_TIMEOUT expected)."""
    return int(load_library().aeth_selftest_wait_timeout(ctx))


def aeth_mlp_collect(ctx, stride: int, d_X: int, d_Y: int, capacity: int) -> int:
    n = C.c_longlong(0)
    _check(ctx, load_library().aeth_mlp_collect(ctx, int(stride), C.c_void_p(d_X), C.c_void_p(d_Y),
                                                int(capacity), C.byref(n)))
    return n.value


def aeth_mlp_work_floats(n: int) -> int:
    w = C.c_size_t(0)
    _check(None, load_library().aeth_mlp_work_floats(int(n), C.byref(w)))
    return w.value


def aeth_mlp_grad(d_params, d_X, d_Y, n, d_grad, d_work, work_floats, d_loss, stream=0):
    _check(None, load_library().aeth_mlp_grad(C.c_void_p(d_params), C.c_void_p(d_X),
                                              C.c_void_p(d_Y), int(n), C.c_void_p(d_grad),
                                              C.c_void_p(d_work), int(work_floats),
                                              C.c_void_p(d_loss), C.c_void_p(stream)))


def aeth_mlp_adam(d_params, d_grad, d_m, d_v, n, step, lr, beta1=0.9, beta2=0.999, eps=1e-8,
                  stream=0):
    _check(None, load_library().aeth_mlp_adam(C.c_void_p(d_params), C.c_void_p(d_grad),
                                              C.c_void_p(d_m), C.c_void_p(d_v), int(n), int(step),
                                              float(lr), float(beta1), float(beta2), float(eps),
                                              C.c_void_p(stream)))


def aeth_profile(ctx, enable: bool):
    _check(ctx, load_library().aeth_profile(ctx, 1 if enable else 0))


def aeth_profile_read(ctx):
    """(total device ms, launches, algorithmic bytes) of the timed dominant-
    kernel launches, and the count of all kernels launched since enable."""
    ms = C.c_double(0)
    n = C.c_longlong(0)
    b = C.c_double(0)
    al = C.c_longlong(0)
    _check(ctx, load_library().aeth_profile_read(ctx, C.byref(ms), C.byref(n), C.byref(b),
                                                 C.byref(al)))
    return ms.value, n.value, b.value, al.value


def aeth_autotune(ctx):
    """Time the flux pass's tile candidates (widths 32 / 16 / band tiles,
    z-chunks 8..64) on the current state (which it advances) and keep the
    fastest; returns (flux_tx, kchunk), flux_tx 0 for band tiles."""
    tx, kc = C.c_int(0), C.c_int(0)
    _check(ctx, load_library().aeth_autotune(ctx, C.byref(tx), C.byref(kc)))
    return tx.value, kc.value


def aeth_set_flux_tile(ctx, flux_tx: int, kchunk: int):
    _check(ctx, load_library().aeth_set_flux_tile(ctx, int(flux_tx), int(kchunk)))


def aeth_get_flux_tile(ctx):
    tx, kc = C.c_int(0), C.c_int(0)
    _check(ctx, load_library().aeth_get_flux_tile(ctx, C.byref(tx), C.byref(kc)))
    return tx.value, kc.value


def tile_cache_key(cfg, descs, device=""):
    """Key of a tuned flux-tile shape: the configuration fields that change
    the flux pass, the block sizes (as a multiset) and the device name."""
    import hashlib
    import json
    blocks = {}
    for d in descs:
        k = f"{d.nx}x{d.ny}x{d.nz}:{d.coord}"
        blocks[k] = blocks.get(k, 0) + 1
    body = {"eos": cfg.eos, "precision": cfg.precision, "recon": cfg.recon,
            "riemann": cfg.riemann, "integrator": cfg.integrator, "path": cfg.path,
            "dual": cfg.dual_energy, "n_dust": cfg.n_dust,
            "blocks": sorted(blocks.items()), "device": device}
    return hashlib.sha256(json.dumps(body, sort_keys=True).encode()).hexdigest()[:24], body


def default_tile_cache():
    """JSON file of tuned flux-tile shapes ($AETHER_TILE_CACHE, else
    ~/.cache/aether_gb/flux_tiles.json)."""
    return os.environ.get("AETHER_TILE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "aether_gb", "flux_tiles.json")


def load_tile_cache(path):
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_tile_cache(path, key, entry):
    """Add one entry to the cache file (written to a temporary file, then
    moved into place, so a concurrent reader never sees half a file)."""
    import json
    import tempfile
    d = load_tile_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def aeth_cfl_dt_noalloc(d_cons, d_b1, d_b2, d_b3, n, dx, gamma, rho_floor, p_floor, cfl, mhd,
                        d_dt, stream_ptr=0):
    """Allocation-free CFL step of one Cartesian block: all pointers are
    device addresses (ints) the caller owns; the result lands in d_dt."""
    nx, ny, nz = n
    rc = load_library().aeth_cfl_dt_noalloc(
        C.c_void_p(d_cons), C.c_void_p(d_b1), C.c_void_p(d_b2), C.c_void_p(d_b3), nx, ny, nz,
        float(dx[0]), float(dx[1]), float(dx[2]), float(gamma), float(rho_floor), float(p_floor),
        float(cfl), 1 if mhd else 0, C.c_void_p(d_dt), C.c_void_p(stream_ptr))
    if rc != AETH_OK:
        raise AethError(rc, "aeth_cfl_dt_noalloc")


def aeth_last_error(ctx) -> str:
    r = load_library().aeth_last_error(ctx)
    return r.decode() if r else ""


def aeth_destroy(ctx):
    if ctx:
        load_library().aeth_destroy(ctx)


def _check(ctx, rc):
    if rc != AETH_OK:
        msg = aeth_last_error(ctx) if ctx else ""
        raise AethError(rc, msg)


# ---- convenience wrapper ---------------------------------------------------

def make_config(gamma=5.0 / 3.0, recon=PLM, integrator=VL2, cfl=0.3, precision=FP64, mhd=True,
                path=FUSED, rho_floor=1e-12, p_floor=1e-10, strict_floors=0, t_stop=None,
                riemann=HLLD, drag_precision=FP64, mlp_tau=0.0, mlp_engine=TCGEN05, iso=False,
                cs=1.0, dual=False, alpha_switch=0.0, alpha_sync=0.0, p64_ratio=0.0,
                drag_ratio=0.0, drag_law=0):
    """iso=True selects the isothermal closure p = cs^2 rho (gamma unused);
    dual=True the dual-energy formalism (alpha_* <= 0: the defaults);
    p64_ratio / drag_ratio: thresholds of FP32_SEL64 / DRAG_SEL64 (<= 0: the
    defaults, 4 and 1)."""
    cfg = aeth_config()
    if iso:
        cfg.eos = EOS_ISO_MHD if mhd else EOS_ISO_HYDRO
    else:
        cfg.eos = EOS_MHD if mhd else EOS_HYDRO
    cfg.cs_iso = cs
    cfg.dual_energy = 1 if dual else 0
    cfg.alpha_switch, cfg.alpha_sync = alpha_switch, alpha_sync
    cfg.p64_ratio, cfg.drag_ratio, cfg.drag_law = p64_ratio, drag_ratio, drag_law
    cfg.gamma, cfg.rho_floor, cfg.p_floor = gamma, rho_floor, p_floor
    cfg.recon, cfg.riemann, cfg.integrator, cfg.cfl = recon, riemann, integrator, cfl
    cfg.precision, cfg.path, cfg.strict_floors = precision, path, strict_floors
    cfg.drag_precision = drag_precision
    cfg.mlp_tau = mlp_tau
    cfg.mlp_engine = mlp_engine
    if t_stop is not None and len(t_stop) > 0:
        arr = (C.c_double * len(t_stop))(*t_stop)
        cfg.n_dust = len(t_stop)
        cfg.t_stop = C.cast(arr, C.POINTER(C.c_double))
        cfg._keep = arr
    else:
        cfg.n_dust = 0
        cfg.t_stop = None
    return cfg


def make_block(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), coord=CART, bc=(PERIODIC,) * 3):
    d = aeth_block_desc()
    d.nx, d.ny, d.nz = n
    d.coord = coord
    d.x1min, d.x2min, d.x3min = lo
    d.x1max, d.x2max, d.x3max = hi
    d.bc = (C.c_int * 3)(*bc)
    return d


class Solver:
    """One library context with its blocks.  `arena="torch"` allocates the
    device arena as a torch uint8 tensor; `stream` binds a torch stream."""

    def __init__(self, cfg: aeth_config, blocks, arena: str = "torch", stream=None, links=()):
        self.ctx = aeth_create(cfg)
        self.cfg = cfg
        self.blocks = []
        self._arena = None
        try:
            if stream is not None:
                aeth_bind_stream(self.ctx, stream.cuda_stream)
            for b in blocks:
                self.blocks.append(aeth_add_block(self.ctx, b))
            for lo_b, axis, hi_b in links:
                aeth_link_blocks(self.ctx, lo_b, axis, hi_b)
            self.descs = list(blocks)
            if arena == "torch":
                import torch
                nbytes = aeth_plan(self.ctx)
                self._arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
                base = self._arena.data_ptr()
                aligned = (base + 255) // 256 * 256
                aeth_bind_arena(self.ctx, aligned, nbytes)
            self.bytes = aeth_finalize(self.ctx)
        except Exception:
            aeth_destroy(self.ctx)
            self.ctx = None
            raise

    def close(self):
        if self.ctx:
            aeth_destroy(self.ctx)
            self.ctx = None
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shapes(self, b):
        d = self.descs[b]
        nx, ny, nz = d.nx, d.ny, d.nz
        return (5, nz, ny, nx), (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)

    def set_state(self, b, cons, b1=None, b2=None, b3=None):
        aeth_set_state(self.ctx, b, cons, b1, b2, b3)

    def get_state(self, b):
        s = self.shapes(b)
        out = [np.empty(x) for x in s]
        aeth_get_state(self.ctx, b, *out)
        return out

    def get_entropy(self, b):
        d = self.descs[b]
        out = np.empty((d.nz, d.ny, d.nx))
        aeth_get_entropy(self.ctx, b, out)
        return out

    def compute_dt(self):
        return aeth_compute_dt(self.ctx)

    def tune_tiles(self, cache=None, device=""):
        """Flux-tile shape for this context: taken from the JSON cache when
        the same configuration, block sizes and device were tuned before,
        else timed with aeth_autotune (which ADVANCES the state: load the
        real state afterwards) and stored.  Returns (flux_tx, kchunk,
        "cache" | "tuned")."""
        path = cache or default_tile_cache()
        key, body = tile_cache_key(self.cfg, self.descs, device)
        e = load_tile_cache(path).get(key)
        if e is not None:
            try:
                aeth_set_flux_tile(self.ctx, e["flux_tx"], e["kchunk"])
                return e["flux_tx"], e["kchunk"], "cache"
            except (AethError, KeyError, TypeError):
                pass   # a stale or foreign entry: tune again
        tx, kc = aeth_autotune(self.ctx)
        store_tile_cache(path, key, {"flux_tx": tx, "kchunk": kc, "what": body})
        return tx, kc, "tuned"

    def step(self, dt):
        aeth_step(self.ctx, dt)

    def run(self, nsteps):
        aeth_run(self.ctx, nsteps)

    def sync(self):
        aeth_sync(self.ctx)

    def diagnostics(self):
        return aeth_diagnostics(self.ctx)
