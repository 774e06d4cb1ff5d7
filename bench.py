"""Benchmark of the GB300 MHD step: cell-updates/s on one GPU (replicas on N).

Default workload: 3-D decaying MHD turbulence, 256^3 periodic, FP32 bulk,
PLM + HLLD + CT + VL2, CFL 0.3 (rho = 1, beta = 1 uniform B_x, solenoidal
Gaussian velocity with P(k) ~ k^-2 on 2 <= k <= 8, rms Mach 2, gamma =
1.0001).  One "step" is one full VL2 step (both stages, CFL dt computed on
the device), counted once per cell (zone-cycles).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--prec fp32|fp64|fp32_p64|fp32_sel64] [--recon plm|ppm|ppm5] [--n 256]
                  [--workload turb256|batched512|dust128|wave32|learned512|wave512|tgv128]
                  [--iso] [--dual] [--block-size N] [--hydro] [--riemann lhlld|hlld]

Prints ONE JSON line (rank 0).  With --gpus N > 1 (torchrun) every rank
advances its own independent replica (weak scaling, no cross-GPU exchange
in the step); value = all ranks' cell-updates / max time.  `e2e` is the same
metric with every step's state copied in from, and read back into, pinned
host memory through the public API: --e2e-contexts (default 3) contexts on
as many streams, so that one context's copies overlap another's step (1:
the synchronous calls on one context, also reported as e2e.serial_value).

--impl reference times the FP64 CPU oracle instead, on the host cores: W
untimed and K timed steps of a bounded sample of the same workload (64^3 of
its generator, smaller when K + W steps would take more than a few
minutes); rank 0 alone runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s on 1 GB300 (FP32/learned vs FP64 plain) at stated L1; % HBM roofline"
UNIT = "cell-updates/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=None, choices=["fp32", "fp64", "fp32_p64", "fp32_sel64"],
                    help="working precision (default: fp64 for wave512, the paper's, else fp32)")
    ap.add_argument("--recon", default="plm", choices=["plm", "ppm", "ppm5"])
    ap.add_argument("--path", default="fused", choices=["fused", "unfused"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--e2e-contexts", type=int, default=3,
                    help="contexts (streams) of the end-to-end measurement; 1: the synchronous calls")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="turb256", choices=WORKLOADS)
    ap.add_argument("--drag", default="fp64", choices=["fp64", "fp32", "sel"],
                    help="dust128: drag solve in FP64, FP32, or FP64 only for the stiff species")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--train-on", default="c2", choices=["c2", "c5"],
                    help="learned512: the network's training states: the 256^3 Mach-2 "
                         "turbulence (held out from the benchmark) or the benchmarked generator")
    ap.add_argument("--l1-steps", type=int, default=None,
                    help="steps of the L1 statement against the FP64 GPU path (default: the "
                         "configuration's own step count: 100 for turb256, 50 for dust128, "
                         "20 otherwise; 0: skip)")
    ap.add_argument("--mlp-engine", default="tcgen05", choices=["tcgen05", "mma_sync"])
    ap.add_argument("--hydro", action="store_true", help="wave512: the hydro column (B = 0)")
    ap.add_argument("--riemann", default="lhlld", choices=["lhlld", "hlld"],
                    help="tgv128: the gas solver (LHLLC / HLLC in hydro)")
    ap.add_argument("--block-size", type=int, default=0,
                    help="turb256/wave512/tgv128: run the domain as linked blocks of this many "
                         "cells per axis (the paper's mesh-block decomposition), 0: one block")
    ap.add_argument("--dual", action="store_true",
                    help="turb256: dual-energy formalism (entropy-based pressure where the "
                         "internal energy is untrusted), FP32 or FP64")
    ap.add_argument("--iso", action="store_true",
                    help="turb256: isothermal closure p = cs^2 rho with cs = 1 (the sound "
                         "speed of the generator) and the isothermal HLLD")
    a = ap.parse_args(argv)
    a.argv = list(sys.argv[1:] if argv is None else argv)
    if a.steps < 1 or a.warmup < 0:
        ap.error("--steps must be >= 1 and --warmup >= 0")
    if a.prec is None:
        a.prec = "fp64" if a.workload == "wave512" else "fp32"
    if a.l1_steps is None:
        a.l1_steps = {"turb256": 100, "dust128": 50}.get(a.workload, 20)
    if a.iso and a.workload != "turb256":
        ap.error("--iso applies to the turb256 workload")
    if a.block_size and a.workload not in ("turb256", "wave512", "tgv128"):
        ap.error("--block-size applies to turb256, wave512 and tgv128")
    if a.dual and (a.workload != "turb256" or a.iso or a.prec in ("fp32_p64", "fp32_sel64")):
        ap.error("--dual applies to the adiabatic turb256 workload in fp32 or fp64")
    return a


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOADS = ("turb256", "batched512", "dust128", "wave32", "learned512", "wave512", "tgv128")
# the paper's single-device throughput table (Sec. 6.1): PLM + HLLE + RK2,
# FP64, 3-D linear wave at 512 x 512 x 256, NVIDIA A100 40 GB, in cells per
# second per device
PAPER_WAVE512 = {"mhd": 300e6, "hydro": 709e6}


def flux_tile_record(A, current, tuned):
    """The flux pass's tile shape in the bench line: width x height x
    z-chunk, and whether the autotuner timed it now or its cache gave it."""
    tx, kc = current
    shape = {"tx": tx, "ty": 128 // tx} if tx else {"tx": "band", "ty": "256 / (n_x + 2) rows"}
    return {**shape, "kchunk": kc, "source": tuned[2] if tuned else "default (no autotune)"}


def learned_n(a):
    """Grid of the learned-flux workload: 512^3 unless --n is given."""
    return a.n if any(x == "--n" or x.startswith("--n=") for x in a.argv) else 512


def workload_config(a):
    cfg = _workload_config(a)
    if a.block_size:
        n = cfg["grid"]
        nb = [g // a.block_size for g in n]
        cfg["workload"] += f"_blocks{a.block_size}"
        cfg["blocks"] = (f"{nb[0] * nb[1] * nb[2]} linked blocks of {a.block_size}^3 "
                         f"({nb[0]}x{nb[1]}x{nb[2]}), ghost cells exchanged through the fill")
    return cfg


def _workload_config(a):
    if a.workload == "batched512":
        return {"workload": "batched_512_uneven_mhd_boxes", "blocks": 512,
                "sides": [16, 24, 32, 48, 64], "spherical_every": 3, "recon": a.recon.upper(),
                "riemann": "HLLD", "ct": "upwind corner EMF (GS05)", "integrator": "VL2",
                "cfl": 0.3, "gamma": 5.0 / 3.0, "precision": a.prec, "path": a.path,
                "seed": 20260818, "launch": "one launch per pass over all blocks",
                "l2": "inputs larger than L2 (2.5e7 cells x 8 vars x 2 registers)"}
    if a.workload == "dust128":
        return {"workload": "multifluid_dust_128^3_8_species", "grid": [128, 128, 128],
                "species": 8, "t_stop": "log-spaced 1e-4..1", "integrator": "IMEX2P",
                "recon": a.recon.upper(), "gas": "adiabatic hydro gamma 5/3, HLLD (=HLLC)",
                "drag": f"closed-form arrowhead, {a.drag.upper()}", "precision": a.prec,
                "seed": 20260817,
                "l2": "inputs larger than L2 (128^3 x 37 vars x 2 registers)"}
    if a.workload == "learned512":
        n = learned_n(a)
        return {"workload": f"learned_flux_mhd_turbulence_{n}^3", "grid": [n, n, n],
                "riemann": f"BF16 MLP 14-128-128-128-7 ({a.mlp_engine}) + HLLD fallback",
                "recon": "PLM", "integrator": "VL2", "mach_rms": 4.0,
                "beta": "0.1..10 (log10 beta = sin 2 pi y)", "gamma": 1.0001,
                "precision": "fp32 state, bf16 network", "seed": 20260820,
                "training": ("~1e8 interface states of the 256^3 Mach-2 turbulence "
                             "(another configuration), HLLD targets"
                             if a.train_on == "c2" else
                             "interface states of a 128^3 HLLD run of the same generator"),
                "l2": "inputs larger than L2"}
    if a.workload == "wave512":
        kind = "hydro" if a.hydro else "mhd"
        return {"workload": f"linear_wave_512x512x256_{kind}", "grid": [512, 512, 256],
                "box": [2.0, 2.0, 1.0], "recon": "PLM", "riemann": "HLLE", "integrator": "RK2",
                "ct": "upwind corner EMF (GS05)" if not a.hydro else None, "cfl": 0.3,
                "gamma": 5.0 / 3.0, "precision": a.prec, "path": a.path, "amplitude": 1e-6,
                "blocks": "one 512x512x256 block (the paper tiles it into 128^3 blocks)",
                "paper_reference": f"{PAPER_WAVE512[kind] / 1e6:.0f} Mzcps, NVIDIA A100 40GB, FP64 "
                                   "(paper Sec. 6.1 table)",
                "l2": "inputs larger than L2"}
    if a.workload == "tgv128":
        return {"workload": "taylor_green_128^3_mach0.01", "grid": [128, 128, 128],
                "box": "[0, 2 pi]^3", "recon": "PLM", "riemann": f"{a.riemann.upper()} (hydro)",
                "integrator": "RK2", "cfl": 0.3, "gamma": 5.0 / 3.0, "mach": 0.01,
                "precision": a.prec, "path": a.path,
                "paper_test": "low-Mach Taylor-Green vortex (Sec. 5): 128^3, PLM + RK2, "
                              "HLLC vs LHLLC at Mach 0.1 / 0.01",
                "l2": "inputs larger than L2 (128^3 x 5 vars x 2 registers x fp32 = 84 MB "
                      "state + 170 MB scratch)"}
    if a.workload == "wave32":
        return {"workload": "linear_fast_wave_32^3", "grid": [32, 32, 32], "recon": "PLM",
                "riemann": "HLLD", "integrator": "VL2", "cfl": 0.3, "precision": a.prec,
                "amplitude": 1e-6,
                "l2": "inputs smaller than L2; L2 is flushed between timed steps"}
    if a.iso:
        return {"workload": f"mhd_decaying_turbulence_{a.n}^3_isothermal",
                "grid": [a.n, a.n, a.n], "recon": a.recon.upper(),
                "riemann": "isothermal HLLD (Mignone 2007)", "ct": "upwind corner EMF (GS05)",
                "integrator": "VL2", "cfl": 0.3, "eos": "isothermal, c_s = 1", "mach_rms": 2.0,
                "beta": 1.0, "precision": a.prec, "path": a.path, "seed": 20260816,
                "l2": f"inputs larger than L2 (state {a.n}^3 x 8 vars x 2 registers)"}
    if a.dual:
        return {"workload": f"mhd_decaying_turbulence_{a.n}^3_dual_energy",
                "grid": [a.n, a.n, a.n], "recon": a.recon.upper(), "riemann": "HLLD",
                "ct": "upwind corner EMF (GS05)", "integrator": "VL2", "cfl": 0.3,
                "gamma": 1.0001, "mach_rms": 2.0, "beta": 1.0,
                "dual_energy": "entropy S advected; alpha_switch 1e-3, alpha_sync 1e-1",
                "precision": a.prec, "path": a.path, "seed": 20260816,
                "l2": f"inputs larger than L2 (state {a.n}^3 x 9 vars x 2 registers)"}
    return {"workload": f"mhd_decaying_turbulence_{a.n}^3", "grid": [a.n, a.n, a.n],
            "recon": a.recon.upper(), "riemann": "HLLD", "ct": "upwind corner EMF (GS05)",
            "integrator": "VL2", "cfl": 0.3, "gamma": 1.0001, "mach_rms": 2.0, "beta": 1.0,
            "precision": a.prec, "path": a.path, "seed": 20260816,
            "l2": f"inputs larger than L2 (state {a.n}^3 x 8 vars x 2 registers)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("flux3.cuh", "common.cuh", "stage.cuh")


def nvtx_push(name):
    import torch
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    import torch
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def kernel_source_hash():
    """Hash of the dominant (flux) kernel's sources, comments and blank
    lines left out: a committed traffic figure is only reported while the
    code is unchanged."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, "paper_2608_14048_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        code = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln.strip()).encode())
    return h.hexdigest()[:16]


def ncu_figure(kernel_key, field):
    """A per-launch figure of the dominant kernel (DRAM bytes, warp
    instructions) from the committed ncu summary, or None if absent or
    taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p) or kernel_key is None:
        return None
    d = json.load(open(p))
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get(field)


def ncu_traffic(kernel_key):
    return ncu_figure(kernel_key, "bytes_per_launch")


def issue_roofline(kernel_key, kernel_ms, sm_mhz, sms=152):
    """The flux pass is bound by instruction issue, not by HBM or an FP
    pipe: its warp instructions per launch (ncu) over its live launch time,
    against 4 issue slots per SM per cycle at the sampled SM clock."""
    inst = ncu_figure(kernel_key, "warp_inst_per_launch")
    if not inst or not kernel_ms or not sm_mhz:
        return None
    achieved = inst / (kernel_ms * 1e-3) / 1e12
    peak = 4.0 * sms * sm_mhz * 1e6 / 1e12
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "T warp-inst/s",
            "frac": achieved / peak, "warp_inst_per_launch": inst,
            "peak_kind": f"4 issue slots x {sms} SMs x sampled SM clock"}


def alu_peaks(A):
    """Measured FP32 and FP64 FMA throughput of this GPU (TFLOP/s)."""
    try:
        return {"fp32_tflops": A.aeth_probe_fma(A.FP32) / 1e12,
                "fp64_tflops": A.aeth_probe_fma(A.FP64) / 1e12,
                "how": "aeth_probe_fma: 8 independent FMA chains per thread, 8 CTAs x 256 per SM"}
    except Exception as e:   # reported, not fatal
        return {"error": str(e)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


TRAIN_SOURCES = {
    # the 256^3 decaying turbulence (Mach 2, beta = 1, gamma = 1.0001): a
    # configuration other than the one the learned flux is measured on, two
    # snapshots of every face, ~1e8 interface states
    "c2": dict(n=256, seed=20260816, mach=2.0, beta=1.0, beta_modulated=False, stride=1,
               snapshots=2, gap=20),
    # the benchmarked generator itself (Mach 4, beta 0.1..10) on a 128^3 box
    "c5": dict(n=128, seed=20260821, mach=4.0, beta=1.0, beta_modulated=True, stride=2,
               snapshots=3, gap=10),
}


def train_learned_flux(A, I, torch, dev, source="c2", steps=4000, batch=8192, lr=2e-3):
    """Train the learned flux on interface states of an HLLD run (the
    project's own collection and training kernels).  source "c2": the
    256^3 Mach-2 turbulence configuration, so the 512^3 Mach-4 benchmark
    measures the network on a configuration it was not trained on; "c5":
    a 128^3 box of the benchmarked generator.  The gas is the same
    (gamma = 1.0001) in both: the network has no gamma input."""
    import math
    t0 = time.perf_counter()
    src = TRAIN_SOURCES[source]
    n = src["n"]
    st = I.turbulence_box(n=n, seed=src["seed"], mach=src["mach"], beta=src["beta"],
                          beta_modulated=src["beta_modulated"], gamma=1.0001)
    cfg = A.make_config(gamma=st.gamma, precision=A.FP32)
    sv = A.Solver(cfg, [A.make_block((n, n, n))], stream=torch.cuda.current_stream(dev))
    per = 3 * n ** 3 // src["stride"] + 3 * n ** 2 * 8
    cap = per * src["snapshots"]
    X = torch.zeros((cap, 16), dtype=torch.float32, device=dev)
    Y = torch.zeros((cap, 8), dtype=torch.float32, device=dev)
    got = 0
    sv.set_state(0, st.cons, st.b1, st.b2, st.b3)
    for _ in range(src["snapshots"]):
        got += A.aeth_mlp_collect(sv.ctx, src["stride"], X[got:].data_ptr(), Y[got:].data_ptr(),
                                  cap - got)
        sv.run(src["gap"])
    sv.close()
    X, Y = X[:got], Y[:got]
    p = torch.from_numpy(I.mlp_init_params(13)).to(dev)
    m, v, g = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    wf = A.aeth_mlp_work_floats(batch)
    work = torch.zeros(wf, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(13)
    s = torch.cuda.current_stream(dev).cuda_stream
    losses = []
    for it in range(1, steps + 1):
        idx = torch.randint(0, got, (batch,), device=dev, generator=gen)
        xb, yb = X[idx].contiguous(), Y[idx].contiguous()
        A.aeth_mlp_grad(p.data_ptr(), xb.data_ptr(), yb.data_ptr(), batch, g.data_ptr(),
                        work.data_ptr(), wf, loss.data_ptr(), s)
        lr_t = 5e-5 + 0.5 * (lr - 5e-5) * (1 + math.cos(math.pi * it / steps))
        A.aeth_mlp_adam(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(), it,
                        lr_t, stream=s)
        if it == 1 or it == steps:
            torch.cuda.synchronize(dev)
            losses.append(loss.item())
    return {"params": p.cpu().numpy(), "samples": got, "losses": losses,
            "seconds": time.perf_counter() - t0, "source": source}


def split_into_blocks(A, st, bs):
    """The whole-domain state as linked blocks of bs cells per axis: the
    per-block states (cell and face arrays cut out of the domain's), their
    descriptors and the links."""
    import numpy as np

    from paper_2608_14048_gb300 import inputs as I
    n = st.block.n
    if any(x % bs for x in n):
        raise SystemExit(f"--block-size {bs} does not divide the grid {n}")
    splits = tuple([bs] * (x // bs) for x in n)
    descs, links, origin = A.decompose(n, splits, st.block.lo, st.block.hi, st.block.bc)
    parts = []
    for (i0, j0, k0), d in zip(origin, descs):
        bx, by, bz = d.nx, d.ny, d.nz
        blk = I.Block((bx, by, bz), (d.x1min, d.x2min, d.x3min), (d.x1max, d.x2max, d.x3max),
                      st.block.coord, st.block.bc)
        cut = lambda arr, ex: np.ascontiguousarray(
            arr[..., k0:k0 + bz + ex[2], j0:j0 + by + ex[1], i0:i0 + bx + ex[0]])
        parts.append(I.InitialState(blk, cut(st.cons, (0, 0, 0)), cut(st.b1, (1, 0, 0)),
                                    cut(st.b2, (0, 1, 0)), cut(st.b3, (0, 0, 1)), st.gamma,
                                    st.meta))
    return parts, descs, links


def make_input(a):
    from paper_2608_14048_gb300 import inputs as I
    return I.turbulence_box(n=a.n, seed=20260816, mach=2.0, beta=1.0, gamma=1.0001)


SAMPLE_PROBE = {"dust128": 32, "wave32": 32}   # other workloads: 64


def _oracle_sample(a, n):
    """The FP64 oracle's bounded sample of the workload at linear size n: the
    same generator on a smaller box (n x n x n/2 of the 2 x 2 x 1 box for
    the linear wave; for the 512 uneven boxes, the first 8 (n/64)^3 of them
    with one global dt).  Returns (step, cells, description): step() runs
    one step of the sample with its initial CFL dt."""
    import oracle as O
    from paper_2608_14048_gb300 import inputs as I

    def gas_step(g, p, s):
        if getattr(a, "dual", False):
            s = O.dual_init(g, p, s)
        dt = O.compute_dt(g, p, s)
        return lambda: O.step(g, p, dt, s)

    if a.workload == "dust128":
        gas, dust, ts = I.dust_box(I.Block((n, n, n)), 20260817, nd=8)
        g = O.make_grid((n, n, n))
        p = O.make_params(gamma=gas.gamma, recon=O.PLM, mhd=False)
        dp = O.make_dust_params(ts)
        cons, d = gas.cons.copy(), dust.copy()
        dt = O.dust_dt(g, p, dp, cons, d)
        return (lambda: O.dust_step(g, p, dp, dt, cons, d)), n ** 3, \
            f"{n}^3 gas + 8 dust species of the same generator (IMEX2P, FP64 drag)"
    if a.workload == "batched512":
        m = max(1, round(8 * (n / 64) ** 3))
        boxes = I.batched_boxes(m, 20260818, gl=2)
        runs = []
        for st in boxes:
            b = st.block
            g = O.make_grid(b.n, b.lo, b.hi, b.coord, b.bc)
            p = O.make_params(gamma=st.gamma, recon=O.PLM)
            runs.append((g, p, O.State(st.cons, st.b1, st.b2, st.b3)))
        dt = min(O.compute_dt(g, p, s) for g, p, s in runs)

        def step():
            for g, p, s in runs:
                O.step(g, p, dt, s)
        cells = sum(math.prod(st.block.n) for st in boxes)
        return step, cells, f"the first {m} of the 512 uneven boxes ({cells} cells, one dt)"
    if a.workload == "wave32":
        st = I.linear_fast_wave(n)
        g = O.make_grid((n, n, n))
        p = O.make_params(gamma=st.gamma, recon=O.PLM)
        return gas_step(g, p, O.State(st.cons, st.b1, st.b2, st.b3)), n ** 3, \
            f"fast wave {n}^3 (PLM + HLLD + VL2)"
    if a.workload == "wave512":
        shape = (n, n, max(2, n // 2))
        st = I.linear_wave_box(shape, (2.0, 2.0, 1.0), mhd=not a.hydro)
        g = O.make_grid(shape, hi=(2.0, 2.0, 1.0))
        p = O.make_params(gamma=st.gamma, recon=O.PLM, integrator=O.RK2, riemann=O.HLLE,
                          mhd=not a.hydro)
        what = (f"{'hydro' if a.hydro else 'MHD'} linear wave {shape[0]}x{shape[1]}x{shape[2]} "
                f"(PLM+HLLE+RK2)")
        return gas_step(g, p, O.State(st.cons, st.b1, st.b2, st.b3)), \
            shape[0] * shape[1] * shape[2], what
    if a.workload == "tgv128":
        st = I.taylor_green(n, 0.01)
        g = O.make_grid((n, n, n), hi=(2 * math.pi,) * 3)
        p = O.make_params(gamma=st.gamma, recon=O.PLM, integrator=O.RK2, mhd=False,
                          riemann=O.LHLLD if a.riemann == "lhlld" else O.HLLD)
        return gas_step(g, p, O.State(st.cons, st.b1, st.b2, st.b3)), n ** 3, \
            f"Taylor-Green vortex {n}^3 at Mach 0.01 (PLM + {solver_label(a)} + RK2)"
    if a.workload == "learned512":
        # the oracle has no learned flux: HLLD on the same Mach-4 input
        st = I.turbulence_box(n=n, seed=20260820, mach=4.0, beta_modulated=True, gamma=1.0001)
        g = O.make_grid((n, n, n))
        p = O.make_params(gamma=st.gamma, recon=O.PLM)
        return gas_step(g, p, O.State(st.cons, st.b1, st.b2, st.b3)), n ** 3, \
            f"{n}^3 box of the same Mach-4 generator, HLLD (the oracle has no learned flux)"
    st = I.turbulence_box(n=n, seed=20260816, mach=2.0, beta=1.0, gamma=1.0001)
    g = O.make_grid((n, n, n))
    p = O.make_params(gamma=st.gamma, recon={"plm": O.PLM, "ppm": O.PPM, "ppm5": O.PPM5}[a.recon],
                      iso=a.iso, cs=1.0, dual=a.dual)
    what = f"{n}^3 box of the same turbulence generator" + (", isothermal" if a.iso else "")
    if a.dual:
        what += ", dual energy"
    return gas_step(g, p, O.State(st.cons, st.b1, st.b2, st.b3)), n ** 3, what


def _host_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def _oracle_rate(a, n, seconds):
    """Cell-updates/s of the oracle on the workload's sample at linear size
    n, stepped for about `seconds` after one untimed step."""
    step, cells, what = _oracle_sample(a, n)
    t0 = time.perf_counter()
    step()
    one = time.perf_counter() - t0
    k = max(1, min(20, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    el = time.perf_counter() - t0
    return {"value": cells * k / el, "steps": k, "seconds": el, "what": what}


def single_thread_rate(a, n, seconds=5.0):
    """The same measurement on one host thread, in a child process started
    with OMP_NUM_THREADS=1 (the OpenMP team size is fixed per process)."""
    code = ("import json, sys; import bench; a = bench.parse(json.loads(sys.argv[1])); "
            "print(json.dumps(bench._oracle_rate(a, int(sys.argv[2]), float(sys.argv[3]))))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code, json.dumps(a.argv), str(n), str(seconds)],
                       cwd=os.path.dirname(os.path.abspath(__file__)), env=env,
                       capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(a, st_full):
    """The FP64 oracle, as it stands, on a bounded sample of the workload
    (64^3 or its equivalent), stepped until ~10 s of CPU work over all host
    threads; beside it the rate on one thread, on the half-size sample."""
    n = SAMPLE_PROBE.get(a.workload, 64)
    r = _oracle_rate(a, n, 10.0)
    cores = _host_threads()
    one = single_thread_rate(a, max(8, n // 2))
    base = {"value": r["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {r['what']}, {r['steps']} steps ({r['seconds']:.1f} s), "
                      f"OpenMP over {cores} host threads"}
    if "value" in one:
        base["single_thread"] = {"value": one["value"], "unit": UNIT,
                                 "sample": f"{one['what']}, {one['steps']} steps "
                                           f"({one['seconds']:.1f} s), 1 thread"}
    else:
        base["single_thread"] = one
    return base


def reference_sample_size(t_probe, n_probe, steps, budget_s=150.0):
    """Linear size of the oracle's sample box so that `steps` steps take
    about budget_s, from one measured step of t_probe seconds at n_probe
    (the step's cost grows with the cell count, n^3); at most n_probe,
    a multiple of 8, at least 16."""
    if steps * t_probe <= budget_s:
        return n_probe
    n = n_probe * (budget_s / (steps * t_probe)) ** (1.0 / 3.0)
    return max(16, int(n) // 8 * 8)


def solver_label(a):
    if a.workload == "learned512":
        return "face-state dump"
    if a.workload == "wave512":
        return "HLLE"
    if a.workload == "tgv128":
        return "LHLLC" if a.riemann == "lhlld" else "HLLC"
    if a.dual:
        return "HLLD + entropy flux (dual energy)"
    return "isothermal HLLD" if a.iso else "HLLD"


def vs_paper(a, value):
    """value / the paper's number for this exact workload, metric and
    precision (only the FP64 linear-wave benchmark has one), else None."""
    if a.workload == "wave512" and a.prec == "fp64":
        return value / PAPER_WAVE512["hydro" if a.hydro else "mhd"]
    return None


def bytes_per_cell_update(a):
    """HBM bytes per cell-update of the two-stage step at the state's
    precision: 40 words for MHD, 25 for hydro, ~185 for 8 dust species, +4
    with dual energy."""
    hydro = (a.workload == "wave512" and a.hydro) or a.workload == "tgv128"
    words = 185.0 if a.workload == "dust128" else (25.0 if hydro else 40.0)
    if getattr(a, "dual", False):
        words += 4.0   # the entropy read and written in each of the two stages
    return words * (8.0 if a.prec == "fp64" else 4.0)



def workload_cfg(a, A, gamma, prec, riemann=None, drag=None, t_stop=None):
    """The library configuration of the workload at working precision
    `prec` (riemann / drag override the solver and the drag precision)."""
    rec = {"plm": A.PLM, "ppm": A.PPM, "ppm5": A.PPM5}[a.recon]
    path = A.FUSED if a.path == "fused" else A.UNFUSED
    if a.workload == "batched512":
        return A.make_config(gamma=5.0 / 3.0, recon=rec, integrator=A.VL2, cfl=0.3,
                             precision=prec, path=path)
    if a.workload == "dust128":
        d = drag if drag is not None else {"fp64": A.DRAG_FP64, "fp32": A.DRAG_FP32,
                                           "sel": A.DRAG_SEL64}[a.drag]
        return A.make_config(gamma=gamma, recon=rec, integrator=A.IMEX2P, cfl=0.3,
                             precision=prec, mhd=False, t_stop=t_stop, drag_precision=d)
    if a.workload == "learned512":
        return A.make_config(gamma=gamma, recon=A.PLM, integrator=A.VL2, cfl=0.3,
                             precision=prec, path=path,
                             riemann=A.MLP if riemann is None else riemann,
                             mlp_engine=A.TCGEN05 if a.mlp_engine == "tcgen05" else A.MMA_SYNC)
    if a.workload == "wave512":
        return A.make_config(gamma=gamma, recon=A.PLM, integrator=A.RK2, cfl=0.3,
                             precision=prec, path=path, riemann=A.HLLE, mhd=not a.hydro)
    if a.workload == "tgv128":
        return A.make_config(gamma=gamma, recon=A.PLM, integrator=A.RK2, cfl=0.3,
                             precision=prec, path=path, mhd=False,
                             riemann=A.LHLLD if a.riemann == "lhlld" else A.HLLD)
    if a.workload == "wave32":
        return A.make_config(gamma=gamma, recon=A.PLM, integrator=A.VL2, cfl=0.3,
                             precision=prec, path=path)
    return A.make_config(gamma=gamma, recon=rec, integrator=A.VL2, cfl=0.3, precision=prec,
                         path=path, iso=a.iso, cs=1.0, dual=a.dual)



def _l1_sums(out, ref, mhd, gamma, iso, acc):
    """Accumulate |q - q_ref| and |q_ref| sums per variable of one block
    into acc (host FP64 arrays (cons, b1, b2, b3))."""
    import numpy as np
    names = ["rho", "M1", "M2", "M3", "E"]
    pairs = [(out[0][v], ref[0][v]) for v in range(5)]
    if mhd:
        names += ["B1f", "B2f", "B3f"]
        pairs += [(out[q], ref[q]) for q in (1, 2, 3)]
    if not iso:
        def pres(st):
            c = st[0]
            e = c[4] - 0.5 * (c[1] ** 2 + c[2] ** 2 + c[3] ** 2) / c[0]
            if mhd:
                e = e - 0.5 * ((0.5 * (st[1][..., :-1] + st[1][..., 1:])) ** 2
                               + (0.5 * (st[2][..., :-1, :] + st[2][..., 1:, :])) ** 2
                               + (0.5 * (st[3][:-1] + st[3][1:])) ** 2)
            return (gamma - 1.0) * e
        names.append("p")
        pairs.append((pres(out), pres(ref)))
    for nm, (x, y) in zip(names, pairs):
        d, r = acc.setdefault(nm, [0.0, 0.0])
        acc[nm] = [d + float(np.sum(np.abs(x - y))), r + float(np.sum(np.abs(y)))]


def _l1_finish(acc):
    """Relative L1 per variable; momentum and face-field components are
    taken against their vector field's mean component norm (a component
    that starts at exactly zero, like B_y of a uniform B_x, has an O(dt)
    norm of its own)."""
    out = {}
    groups = {"M": ["M1", "M2", "M3"], "B": ["B1f", "B2f", "B3f"]}
    for nm, (d, r) in acc.items():
        g = next((k for k, v in groups.items() if nm in v), None)
        den = sum(acc[m][1] for m in groups[g]) / 3.0 if g else r
        out[nm] = d / den if den > 0 else d
    return out


def l1_statement(a, A, torch, stream, states, dust, t_stop, blocks, links, mlp_params):
    """Relative L1 per variable of the benchmarked configuration against the
    FP64 GPU path of the same configuration (held by the parity tests to
    1e-12 of the FP64 oracle), from the same initial state, every step with
    the FP64 run's CFL dt; for the learned flux also plain FP32 HLLD and
    FP32 HLLE (the method without the network) against FP64 HLLD."""
    if a.prec == "fp64":
        return {"vs": None, "steps": 0,
                "note": "FP64 line: the FP64 path is held to 1e-12 relative L1 of the FP64 "
                        "oracle by the parity tests"}
    t0 = time.perf_counter()
    gamma = states[0].gamma
    prec = {"fp32": A.FP32, "fp32_p64": A.FP32_P64, "fp32_sel64": A.FP32_SEL64}[a.prec]
    learned = a.workload == "learned512"
    mhd = not (a.workload in ("dust128", "tgv128") or (a.workload == "wave512" and a.hydro))
    cfgs = {"fp64": workload_cfg(a, A, gamma, A.FP64, t_stop=t_stop, drag=A.FP64,
                                 riemann=A.HLLD if learned else None),
            "bench": workload_cfg(a, A, gamma, prec, t_stop=t_stop)}
    if learned:
        cfgs["hlld_fp32"] = workload_cfg(a, A, gamma, A.FP32, riemann=A.HLLD)
        cfgs["hlle_fp32"] = workload_cfg(a, A, gamma, A.FP32, riemann=A.HLLE)
    n = a.l1_steps
    marks = {n} if learned else ({s for s in (1, 2, 5, 10, 20, 50, 100, 200) if s < n} | {n})
    svs = {}
    try:
        for name, cfg in cfgs.items():
            sv = A.Solver(cfg, blocks, stream=stream, links=links)
            svs[name] = sv
            if name == "bench" and learned:
                A.aeth_load_mlp(sv.ctx, mlp_params)
            for q, s_ in enumerate(states):
                sv.set_state(q, s_.cons, s_.b1, s_.b2, s_.b3)
            if dust is not None:
                import numpy as np
                for k in range(dust.shape[0]):
                    A.aeth_set_dust(sv.ctx, 0, k, np.ascontiguousarray(dust[k]))
        curve, final = [], {}
        for step in range(1, n + 1):
            dt = svs["fp64"].compute_dt()
            for sv in svs.values():
                sv.step(dt)
            if step not in marks:
                continue
            refs = [svs["fp64"].get_state(q) for q in range(len(states))]
            per = {}
            for name, sv in svs.items():
                if name == "fp64":
                    continue
                acc = {}
                for q in range(len(states)):
                    _l1_sums(sv.get_state(q), refs[q], mhd, gamma, a.iso, acc)
                if dust is not None:
                    import numpy as np
                    worst = {}
                    for k in range(dust.shape[0]):
                        x = np.empty(dust.shape[1:])
                        y = np.empty(dust.shape[1:])
                        A.aeth_get_dust(sv.ctx, 0, k, x)
                        A.aeth_get_dust(svs["fp64"].ctx, 0, k, y)
                        for v, nm in enumerate(("rho_d", "M1_d", "M2_d", "M3_d")):
                            r = float(np.sum(np.abs(y[v])))
                            e = float(np.sum(np.abs(x[v] - y[v]))) / r if r > 0 else 0.0
                            worst[nm] = max(worst.get(nm, 0.0), e)
                per[name] = _l1_finish(acc)
                if dust is not None:
                    per[name].update({k + "_max_species": v for k, v in worst.items()})
            curve.append([step, max(v for k, v in per["bench"].items() if k != "p")])
            final = per
        diag = svs["fp64"].diagnostics()
    finally:
        for sv in svs.values():
            sv.close()
    out = {"vs": "FP64 GPU path of the same configuration"
                 + (" with HLLD" if learned else "")
                 + " (1e-12 of the FP64 oracle in the parity tests)",
           "steps": n, "dt": "the FP64 run's CFL dt, every step",
           "norm": "relative L1 per variable; momentum and face-field components against "
                   "their vector field's mean component norm; p = (gamma - 1) (E - kinetic - "
                   "magnetic) from the cell averages",
           "final": final.get("bench"), "max_final": curve[-1][1] if curve else None,
           "curve_max_over_variables": curve, "fp64_floor_hits": diag["floor_hits"],
           "seconds": time.perf_counter() - t0}
    if learned:
        out["hlld_fp32"] = final.get("hlld_fp32")
        out["hlle_fp32"] = final.get("hlle_fp32")
    return out


def max_over_ranks(x, ws, device=None):
    """The maximum over all ranks of a per-rank float (the slowest rank sets
    a multi-GPU time); the value itself at one rank."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Whole-job throughput: the units every rank processed over the
    (max-over-ranks) time."""
    return units_per_rank * ws / seconds


def run_reference(a):
    """The reference arm: the FP64 oracle as it stands, on the host cores,
    W untimed and K timed steps of a bounded sample of the workload (64^3,
    smaller when K + W steps of it would take more than a few minutes)."""
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    n0 = SAMPLE_PROBE.get(a.workload, 64)
    step, cells, what = _oracle_sample(a, n0)
    t0 = time.perf_counter()
    step()                                    # first warm-up step, also the size probe
    n = reference_sample_size(time.perf_counter() - t0, n0, a.steps + a.warmup)
    if n != n0:
        step, cells, what = _oracle_sample(a, n)
        step()
    for _ in range(a.warmup - 1):
        step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    el = time.perf_counter() - t0
    cores = _host_threads()
    base = {"value": cells * a.steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {what}, {max(1, a.warmup)} untimed + {a.steps} timed steps "
                      f"({el:.1f} s), OpenMP over {cores} host threads"}
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": el / a.steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a), "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch

    from paper_2608_14048_gb300 import aether as A

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # CPU baseline first (rank 0, N = 1), before the GPU work starts
    base = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        base = cpu_baseline(a, None)

    prec = {"fp32": A.FP32, "fp64": A.FP64, "fp32_p64": A.FP32_P64,
            "fp32_sel64": A.FP32_SEL64}[a.prec]
    dust = None
    learned = None
    if a.workload == "batched512":
        from paper_2608_14048_gb300 import inputs as I
        states = I.batched_boxes(512, 20260818, gl=2, workers=min(16, os.cpu_count() or 1))
    elif a.workload == "dust128":
        from paper_2608_14048_gb300 import inputs as I
        gas, dust, ts = I.dust_box(I.Block((128, 128, 128)), 20260817, nd=8)
        states = [gas]
    elif a.workload == "learned512":
        from paper_2608_14048_gb300 import inputs as I
        n = learned_n(a)
        learned = train_learned_flux(A, I, torch, dev, source=a.train_on)
        states = [I.turbulence_box(n=n, seed=20260820, mach=4.0, beta_modulated=True,
                                   gamma=1.0001)]
    elif a.workload == "wave512":
        from paper_2608_14048_gb300 import inputs as I
        states = [I.linear_wave_box((512, 512, 256), (2.0, 2.0, 1.0), mhd=not a.hydro)]
    elif a.workload == "tgv128":
        from paper_2608_14048_gb300 import inputs as I
        states = [I.taylor_green(128, 0.01)]
    elif a.workload == "wave32":
        from paper_2608_14048_gb300 import inputs as I
        states = [I.linear_fast_wave(32)]
    else:
        states = [make_input(a)]
    t_stop = ts if dust is not None else None
    cfg = workload_cfg(a, A, states[0].gamma, prec, t_stop=t_stop)
    links = ()
    if a.block_size:
        states, blocks, links = split_into_blocks(A, states[0], a.block_size)
    else:
        blocks = [A.make_block(s_.block.n, s_.block.lo, s_.block.hi, s_.block.coord, s_.block.bc)
                  for s_ in states]
    stream = torch.cuda.current_stream(dev)
    sv = A.Solver(cfg, blocks, stream=stream, links=links)
    mhd_run = a.workload not in ("dust128", "tgv128") and not (a.workload == "wave512" and a.hydro)
    if a.workload == "learned512":
        A.aeth_load_mlp(sv.ctx, learned["params"])

    def upload(host=None, host_dust=None):
        for q, s_ in enumerate(states):
            if host is None:
                sv.set_state(q, s_.cons, s_.b1, s_.b2, s_.b3)
            else:
                A.aeth_set_state(sv.ctx, q, *host[q])
        if dust is not None:
            for k in range(dust.shape[0]):
                A.aeth_set_dust(sv.ctx, 0, k, np.ascontiguousarray(dust[k]) if host_dust is None
                                else host_dust[k])

    upload()
    tile = None
    if not a.no_autotune and a.workload not in ("dust128", "learned512"):
        # tile shape chosen by the autotuner on this workload's own state
        # (or its cached choice for this configuration, block sizes and
        # GPU), then the state is reloaded (the autotuner advances it)
        tile = sv.tune_tiles(device=torch.cuda.get_device_name(dev))
        upload()
    cells = sum(int(np.prod(s_.block.n)) for s_ in states)
    flush = None
    if a.workload == "wave32":
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(a.warmup):
        sv.run(1)
    sv.sync()

    # the timed region runs the product path: aeth_run's CUDA-graph replay
    # of the CFL-driven step, with no profiling events inside it
    clk = ClockSampler(local)
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # NVTX range "timed" around the timed steps: a profiler capture can be
    # restricted to them (ncu --nvtx --nvtx-include timed/)
    nvtx_push("timed")
    if flush is None:
        e0.record(stream)
        sv.run(a.steps)
        e1.record(stream)
    else:
        # small working set: flush L2 before every timed step and time the
        # steps only (events around each step)
        ms_acc = 0.0
        for _ in range(a.steps):
            flush.zero_()
            e0.record(stream)
            sv.run(1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms_acc += e0.elapsed_time(e1)
    torch.cuda.synchronize(dev)
    nvtx_pop()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) if flush is None else ms_acc
    clocks = clk.stop()
    diag = sv.diagnostics()   # counters of the timed steps
    # a second, untimed pass of the same K steps launched eagerly with CUDA
    # events around every launch of the dominant kernel: its per-launch time
    # for the roofline, and the count of the library's kernels per step (the
    # graph replays exactly these launches)
    A.aeth_profile(sv.ctx, True)
    if flush is None:
        sv.run(a.steps)
    else:
        for _ in range(a.steps):
            flush.zero_()
            sv.run(1)
    kms, klaunch, kbytes, all_launches = A.aeth_profile_read(sv.ctx)
    A.aeth_profile(sv.ctx, False)
    sv.sync()
    peaks_alu = alu_peaks(A) if rank == 0 else None
    extra = {}
    if a.workload == "learned512":
        # the same input and step count with plain HLLD, and with the other
        # tensor-core engine, on the same GPU
        def other(cfg_o, params=None):
            svh = A.Solver(cfg_o, blocks, stream=stream)
            if params is not None:
                A.aeth_load_mlp(svh.ctx, params)
            svh.set_state(0, states[0].cons, states[0].b1, states[0].b2, states[0].b3)
            for _ in range(a.warmup):
                svh.run(1)
            svh.sync()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            svh.run(a.steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms_o = e0.elapsed_time(e1)
            svh.close()
            return ms_o

        ms_h = other(workload_cfg(a, A, states[0].gamma, A.FP32, riemann=A.HLLD))
        other_engine = "mma_sync" if a.mlp_engine == "tcgen05" else "tcgen05"
        cfg_e = workload_cfg(a, A, states[0].gamma, A.FP32)
        cfg_e.mlp_engine = A.TCGEN05 if other_engine == "tcgen05" else A.MMA_SYNC
        ms_e = other(cfg_e, learned["params"])
        faces = 3 * (states[0].block.n[0] + 1) * (states[0].block.n[1] + 2) * \
            (states[0].block.n[2] + 2) * 2 * a.steps
        # the flux pass (state dump + three tensor-core MLP launches + HLLD
        # fallbacks) against the sustained BF16 peak: 2 (16*128 + 2*128^2 +
        # 128*8) = 71680 flop per face
        nn = states[0].block.n
        flops_pass = 3 * (nn[0] + 1) * (nn[1] + 2) * (nn[2] + 2) * 71680.0
        tf = flops_pass * klaunch / (kms * 1e-3) / 1e12 if kms > 0 else None
        peak_t = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"] \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1700.0
        extra = {"roofline_tensor": {"bound": "tensor", "achieved": tf, "peak": peak_t,
                                     "unit": "TFLOP/s", "frac": tf / peak_t if tf else None,
                                     "kernel": f"learned-flux pass ({a.mlp_engine} BF16)",
                                     "flop_per_face": 71680},
                 "learned": {"hlld_value": cells * a.steps / (ms_h * 1e-3),
                             "speedup_vs_hlld": ms_h / ms,
                             "engine": a.mlp_engine,
                             f"{other_engine}_value": cells * a.steps / (ms_e * 1e-3),
                             "fallback_fraction": diag["mlp_fallbacks"] / faces,
                             "train_samples": learned["samples"],
                             "train_source": learned["source"],
                             "train_loss": learned["losses"], "train_s": learned["seconds"]}}

    ms = max_over_ranks(ms, ws, device=dev)
    value = whole_job_rate(cells * a.steps, ws, ms * 1e-3)

    # end to end through the public API with host buffers: every step copies
    # the state in from pinned host memory and reads it back
    ke = a.e2e_steps or min(a.steps, 10)
    hin = [[torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
            for x in (s_.cons, s_.b1, s_.b2, s_.b3)] for s_ in states]
    hout = [[torch.empty(shp, dtype=torch.float64).pin_memory() for shp in sv.shapes(q)]
            for q in range(len(states))]
    if not mhd_run:
        hin = [[h[0], None, None, None] for h in hin]
        hout = [[h[0], None, None, None] for h in hout]
    nbytes = lambda lst: sum(x.numel() * 8 for h in lst for x in h if x is not None)
    h2d, d2h = nbytes(hin), nbytes(hout)
    hdust = None
    if dust is not None:
        h2d += dust.nbytes
        d2h += dust.nbytes
        hdust = [torch.from_numpy(np.ascontiguousarray(dust[k])).pin_memory()
                 for k in range(dust.shape[0])]
        dbuf = [torch.empty(dust.shape[1:], dtype=torch.float64).pin_memory()
                for _ in range(dust.shape[0])]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(ke):
        upload(hin, hdust)
        sv.run(1)
        for q in range(len(states)):
            A.aeth_get_state(sv.ctx, q, *hout[q])
        if dust is not None:
            for k in range(dust.shape[0]):
                A.aeth_get_dust(sv.ctx, 0, k, dbuf[k])
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, device=dev)
    e2e_serial = whole_job_rate(cells * ke, ws, e2e_s)
    e2e_val, e2e_how = e2e_serial, ("one context: aeth_set_state, aeth_run(1), aeth_get_state per "
                                    "step, each call synchronous")
    e2e_steps = ke
    sv_tile = A.aeth_get_flux_tile(sv.ctx)
    if a.e2e_contexts > 1:
        # the same copies through the asynchronous calls on several contexts
        # and streams: the copy engines move one context's state while
        # another steps, and the host link carries both directions at once
        more = []
        try:
            for _ in range(a.e2e_contexts - 1):
                s_q = torch.cuda.Stream(dev)
                sv_q = A.Solver(cfg, blocks, stream=s_q, links=links)
                more.append((sv_q, s_q))
                if learned is not None:
                    A.aeth_load_mlp(sv_q.ctx, learned["params"])
                A.aeth_set_flux_tile(sv_q.ctx, *sv_tile)
        except (A.AethError, torch.cuda.OutOfMemoryError):
            pass   # device memory: as many contexts as fit
        # the whole mesh's state in one packed, pinned array (one transfer
        # per direction and step, whatever the number of blocks)
        packed_in = torch.from_numpy(A.pack_states(
            [[x.numpy() for x in h if x is not None] for h in hin], mhd=mhd_run,
            dust=None if dust is None else [dust])).pin_memory()
        ctxs = [(sv, stream, torch.empty_like(packed_in).pin_memory())] + [
            (sv_q, s_q, torch.empty_like(packed_in).pin_memory()) for sv_q, s_q in more]
        try:
            if len(ctxs) > 1:
                # the uploads of the contexts follow one another, and so do
                # the read-backs (events across the streams): each direction
                # of the link carries one copy at a time, at its full rate,
                # while the other direction and the steps run beside it
                chain = {"up": None, "down": None}

                def round_():
                    for svq, sq, hq in ctxs:
                        if chain["up"] is not None:
                            sq.wait_event(chain["up"])
                        A.aeth_set_state_all_async(svq.ctx, packed_in)
                        chain["up"] = torch.cuda.Event()
                        chain["up"].record(sq)
                        svq.run(1)
                        if chain["down"] is not None:
                            sq.wait_event(chain["down"])
                        A.aeth_get_state_all_async(svq.ctx, hq)
                        chain["down"] = torch.cuda.Event()
                        chain["down"].record(sq)

                round_()   # captures the other contexts' step graphs
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                for _ in range(ke):
                    round_()
                torch.cuda.synchronize(dev)
                e2e_p = max_over_ranks(time.perf_counter() - t0, ws, device=dev)
                e2e_steps = len(ctxs) * ke
                e2e_val = whole_job_rate(cells * e2e_steps, ws, e2e_p)
                e2e_how = (f"{len(ctxs)} contexts on {len(ctxs)} streams, {ke} steps each: per step, "
                           "aeth_set_state_all_async from a pinned host array of every block's "
                           "state (gas and dust), aeth_run(1), aeth_get_state_all_async into a "
                           "pinned host array; one context's copies overlap another's step (the "
                           "contexts' uploads follow one another, and so do their read-backs)")
        finally:
            for sv_q, _ in more:
                sv_q.close()
    sv.close()
    l1 = None
    if rank == 0 and a.l1_steps > 0:
        l1 = l1_statement(a, A, torch, stream, states, dust, t_stop, blocks, links,
                          learned["params"] if learned else None)

    hbm, peak_kind = peaks()
    # the dominant kernel's algorithmic bytes per launch follow the per
    # cell-update figure of the two-stage step (each stage reads its input
    # state once and writes its output once): half of it per stage launch,
    # times the interior cells; the flux pass's own outputs (fluxes, face
    # and reference EMFs written for the later passes) are implementation
    # bytes, reported beside it
    algo_launch = bytes_per_cell_update(a) / 2.0 * cells
    kms_launch = kms / max(klaunch, 1)
    achieved = algo_launch / (kms_launch * 1e-3) / 1e9 if kms > 0 else None
    impl_launch = kbytes / max(klaunch, 1)
    # the committed ncu figures hold for the 256^3 default grid only
    kernel_key = (f"{a.path}_{a.prec}_{a.recon}" + ("_iso" if a.iso else "")
                  + ("_dual" if a.dual else "") + (f"_b{a.block_size}" if a.block_size else "")
                  if a.workload == "turb256" and a.n == 256 else None)
    traffic = ncu_traffic(kernel_key) if kernel_key else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": vs_paper(a, value),
        "dtype": {"fp32": "f32", "fp64": "f64", "fp32_p64": "f32+f64",
                  "fp32_sel64": "f32+f64"}[a.prec],
        "data": "synthetic", "config": workload_config(a),
        "l1": l1,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                     "traffic_over_algo": (traffic / algo_launch) if traffic else None,
                     "kernel": (f"k_flux3 (fused prim + reconstruction + {solver_label(a)}, "
                                "3 directions)") if a.path == "fused" else "k_flux",
                     "peak_kind": peak_kind,
                     "algo_bytes_per_launch": algo_launch,
                     "algo_bytes_rule": f"{bytes_per_cell_update(a) / 2.0:g} B per interior "
                                        "cell per stage (half the two-stage step's bytes per "
                                        "cell-update)",
                     "impl_bytes_per_launch": impl_launch,
                     "impl_frac": (impl_launch / (kms_launch * 1e-3) / 1e9 / hbm)
                     if kms > 0 else None,
                     "kernel_ms_per_launch": kms_launch,
                     "kernel_timing": "CUDA events around each launch in an eager pass of the "
                                      "same K steps right after the graph-timed region",
                     "kernel_share_of_step": (kms / ms) if ms > 0 else None,
                     "cell_rate_hbm_frac": value / ws * bytes_per_cell_update(a) / (hbm * 1e9)},
        "roofline_issue": issue_roofline(kernel_key, kms / max(klaunch, 1),
                                         clocks.get("sm_mhz") if isinstance(clocks, dict) else None,
                                         torch.cuda.get_device_properties(dev).multi_processor_count),
        "alu_peaks": peaks_alu,
        "cpu_baseline": base,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "how": e2e_how,
                "serial_value": e2e_serial},
        "clocks": clocks,
        "gpu_launches": all_launches,
        "gpu_launches_how": "the library's launch counter over an eager pass of the same K "
                            "steps; the timed CUDA graph replays the same launches",
        "diag_after": {"max_divb_rel": diag["max_divb_rel"], "floor_hits": diag["floor_hits"]},
        "flux_tile": flux_tile_record(A, sv_tile, tile),
        **extra,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
