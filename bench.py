#!/usr/bin/env python
"""Throughput of the NS-PNP fractional step on GB300: cell-steps/s.

Workload (one step = one full RK3 step = explicit terms, y-implicit solves,
pressure projection and potential solve, three substages): turbulent-Couette
configuration 256 x 193 x 256 (Nx x Ny face nodes x Nz; 12,582,912 cells),
box 2 pi x 2 x pi, tanh-stretched y (gamma 2.5), Re 3000, Debye length 0.01,
Sc 1, wall potential 2 (V-hat = 4), beta 0.5, dt 0.004, Gouy-Chapman ions
plus seeded 0.1 velocity noise.  The working set (~2 GB) is far larger than
the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 NumPy oracle on
the host cores instead (bounded slab samples of the same workload).
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WL = dict(nx=256, ny=193, nz=256, Lx=2 * math.pi, Lz=math.pi, stretch=2.5, Re=3000.0, lam=0.01, Sc=1.0, V=2.0,
          beta=0.5, dt=0.004, seed=1702, amp=0.1)
WL_NAME = "turbulent Couette 256x193x256, Re 3000, lambda_D/h 0.01, Sc 1, V 2 (V-hat 4), dt 0.004"
METRIC = "NS-PNP cell-steps/s on 1 GB300 (mixed vs FP64 @ stated err); % HBM roofline"
UNIT = "cell-steps/s"


def cells(wl=WL):
    return wl["nx"] * (wl["ny"] - 1) * wl["nz"]


# --------------------------------------------------------------------------
# Algorithmic cost per cell per substage of each launch site: bytes every
# input read once and every output written once, and FP64-pipe instructions
# (FP64 arithmetic and FP64<->FP32 conversions), counted from the kernel
# sources.  ``half`` = spectral points per real point ((Nx/2+1)/Nx).
# --------------------------------------------------------------------------
# dram__bytes_read.sum + dram__bytes_write.sum per launch, turbulent Couette
# 256x193x256, from the one-pass ncu capture summarised under profiles/
# (shape = the stencil's tuned launch code the capture ran with)
# DRAM bytes (read + write) of all 45 launches of one step of that workload, from the
# one-pass ncu capture summarised under profiles/ (cold cache: ncu flushes L2 before
# each kernel), per cell-step, for the launch shapes the capture ran with
STEP_NCU = {"mixed": {"bytes_per_cell_step": 839.6, "cells": 12582912, "shape": [64, 64, 32, 16],
                     "note": "45 launches, 582 B read + at least 257 B written per cell-step (writes still in L2 "
                             "at a kernel's end are not counted)"}}

# Algorithmic bytes per cell-step of the whole step (every input read once, every
# output written once per phase; the phases the method's synchronisation points
# separate): 268 B per substage in the mixed path, 352 in FP64
STEP_BYTES = {"mixed": 804.0, "fp64": 1056.0}
NOMINAL_HBM_GBS = 7900.0

NCU_TRAFFIC = {
    # mean of three consecutive launches (one per RK3 substage) of the stencil with
    # the fused CN forward elimination, launch code 0 / 64
    ("mixed", "rhs"): {"kernel": "k_rhs_mixed_tile<64, 4, 2, false, 2> (fused CN forward elimination)",
                       "shape": (0, 64), "cells": 12582912, "bytes": 913655040},
}


def site_cost(site, precision, launch_cfg=None, fused=True):
    half = (WL["nx"] // 2 + 1) / WL["nx"]
    # mixed CN: the back substitution after the stencil's fused forward elimination
    # (the default) and the shared-memory line tiles (launch code 32) move 76 B per
    # cell (d in, state in and out); the unfused line kernels also write and re-read d (116 B)
    cn_tiled = fused or (launch_cfg is not None and launch_cfg[1] == 32)
    if precision == "fp64":
        table = {
            "rhs": (176, 220), "cn_thomas": (200, 20),
            "p_fftx": (24 + 16 * half, 30), "p_fftz": (32 * half, 20), "p_thomas": (80 * half, 10 * half),
            "p_ifftz": (32 * half, 20), "p_ifftx": (16 * half + 8, 22), "project": (72, 8),
            "e_fftx": (16 + 16 * half, 24), "e_fftz": (32 * half, 20), "e_thomas": (80 * half, 10 * half),
            "e_ifftz": (32 * half, 20), "e_ifftx": (16 * half + 8, 22),
        }
    else:
        table = {
            # stencil: 28 B of inputs and 20 B of right-hand sides per cell, plus the
            # previous H (20 B) when zeta != 0 and the new H (20 B) except in the
            # last substage: 68, 88, 68 B over the three substages
            "rhs": (224 / 3, 0), "cn_thomas": (76 if cn_tiled else 116, 0),
            "p_fftx": (12 + 8 * half, 0), "p_fftz": (16 * half, 0), "p_thomas": (64 * half, 0),
            "p_ifftz": (16 * half, 0), "p_ifftx": (8 * half + 4, 0), "project": (36, 0),
            "e_fftx": (8 + 8 * half, 0), "e_fftz": (16 * half, 0), "e_thomas": (64 * half, 0),
            "e_ifftz": (16 * half, 0), "e_ifftx": (8 * half + 4, 0.25),
        }
    b, f = table[site]
    return {"bytes": b, "fp64_ops": f}


# --------------------------------------------------------------------------
# Ensemble workload: 48 cases on two grids, Re x Debye length x wall potential.
# Per case: the smallest tanh stretching that keeps the Gouy-Chapman potential
# drop across the wall cell <= 1 (flagged when even g = 6 cannot), and dt from
# the explicit limits: advection CFL 0.5, wall-normal migration CFL 0.5 and the
# dielectric relaxation rate D (c+ + c-)_wall / (2 lam^2) (RK3 real-axis bound).
# --------------------------------------------------------------------------
def stable_dt(nx, ny, Re, lam, V, stretch, Lx=2 * math.pi):
    """dt from the explicit limits: advection CFL 0.5 (wall speed 1), wall-normal
    migration CFL 0.5 across the wall cell under the Gouy-Chapman wall field,
    and the dielectric relaxation rate (RK3 real-axis bound); also returns the
    potential drop across the wall cell."""
    import math as m
    bq = 2 * lam * (m.cosh(V / 2) - 1)
    sq = 0.5 * (-bq + m.sqrt(bq * bq + 4))
    cb = sq * sq
    dphi_w = 2 * m.sqrt(cb) * m.sinh(V / 2) / lam
    dy0 = 1 - m.tanh(stretch * (1 - 2.0 / (ny - 1))) / m.tanh(stretch) if stretch > 0 else 2.0 / (ny - 1)
    D = 1.0 / Re
    dt = 0.5 * Lx / nx
    if V > 0:
        dt = min(dt, 0.5 * dy0 / (D * dphi_w))
    cwall = cb * (m.exp(V) + m.exp(-V))
    dt = min(dt, 2.0 / (D * cwall / (2 * lam * lam)))
    return dt, dphi_w * dy0


def run_mlp(args, B, torch):
    """Throughput of the wall model's network on its tcgen05 kernels: inference
    (the fused kernel: 180 B of input and output per row for 110 kFLOP, so bound by
    the tensor cores and the on-chip epilogues, not by HBM) and the training step
    (layer by layer: every z is stored for the backward pass, 64 FLOPs per byte at
    the 128-wide layers, so HBM-bound) on 65,536 rows (the training batch; a
    coupled step of the 128x49x128 grid feeds 32,768)."""
    import ctypes as C

    import numpy as np

    from paper_1701_02005_gb300 import wallmodel as wm

    rows, reps = 65536, 50
    net = wm.MLP(rows, seed=7)
    net.set_normalization(np.zeros(40), np.ones(40), np.zeros(5), np.ones(5))
    g = torch.Generator(device="cuda").manual_seed(1707)
    X = torch.randn((rows, 40), device="cuda", generator=g)
    T = torch.randn((rows, 5), device="cuda", generator=g)
    Y = torch.empty((rows, 5), device="cuda")
    torch.cuda.synchronize()
    fwd = lambda: B.check(B.pnp_mlp_forward(net.m, C.c_void_p(X.data_ptr()), rows, C.c_void_p(Y.data_ptr())),
                          "pnp_mlp_forward")
    trn = lambda: B.check(B.pnp_mlp_train_step(net.m, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), rows,
                                               1e-6, None), "pnp_mlp_train_step")

    def timed(fn):
        for _ in range(5):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        net.stream.synchronize()
        e0.record(net.stream)
        for _ in range(reps):
            fn()
        e1.record(net.stream)
        net.stream.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    t_f, t_t = timed(fwd), timed(trn)
    macs = 40 * 128 + 3 * 128 * 128 + 128 * 5
    flops_f = 2.0 * rows * macs
    # the fused inference kernel reads each input row and writes its outputs, nothing else
    bytes_f = 4.0 * rows * (40 + 5)
    # the training step's forward stores every layer's z for the backward pass: FP32 values
    # read + written per row: input scaling 40 + 40, layers (40 + 128) + 3 (128 + 128) + (128 + 5)
    bytes_train_fwd = 4.0 * rows * (80 + 168 + 3 * 256 + 133)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    out = {"rows": rows, "forward_us": t_f * 1e6, "train_step_us": t_t * 1e6,
           "forward_tflops": flops_f / t_f / 1e12, "train_step_tflops": 3 * flops_f / t_t / 1e12,
           "forward_gbs": bytes_f / t_f / 1e9,
           "roofline_forward": {"bound": "tensor", "achieved": flops_f / t_f / 1e12, "peak": bf16,
                                "unit": "TFLOP/s", "frac": flops_f / t_f / 1e12 / bf16,
                                "per_unit": f"2 x {macs} FLOPs per row x {rows} rows (180 B per row: "
                                            f"{bytes_f / t_f / 1e9:.0f} GB/s, {bytes_f / t_f / 1e9 / hbm:.3f} of HBM)",
                                "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)"},
           "train_step_forward_bytes_per_row": bytes_train_fwd / rows, "status": net.status()}
    net.close()
    return out


def ensemble_cases():
    import math as m
    out = []
    grids = [(64, 65, 64), (128, 97, 128)]
    idx = 0
    for (nx, ny, nz) in grids:
        for Re in (1000.0, 3000.0):
            for lam in (0.005, 0.0158, 0.05):
                for V in (0.0, 2.0, 5.0, 10.0):
                    bq = 2 * lam * (m.cosh(V / 2) - 1)
                    sq = 0.5 * (-bq + m.sqrt(bq * bq + 4))
                    cb = sq * sq
                    dphi_w = 2 * m.sqrt(cb) * m.sinh(V / 2) / lam
                    chosen, dy0 = None, None
                    for g in (1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0):
                        d0 = 1 - m.tanh(g * (1 - 2.0 / (ny - 1))) / m.tanh(g)
                        if dphi_w * d0 <= 1.0:
                            chosen, dy0 = g, d0
                            break
                    flagged = chosen is None
                    if flagged:
                        chosen = 6.0
                        dy0 = 1 - m.tanh(chosen * (1 - 2.0 / (ny - 1))) / m.tanh(chosen)
                    dt, _ = stable_dt(nx, ny, Re, lam, V, chosen)
                    out.append(dict(nx=nx, ny=ny, nz=nz, Re=Re, lam=lam, V=V, stretch=chosen, dt=dt,
                                    dphi_wall_cell=dphi_w * dy0, flagged=flagged, seed=1703 + idx))
                    idx += 1
    return out


def run_ensemble(args, B, Solver, torch):
    from paper_1701_02005_gb300 import autotune
    from paper_1701_02005_gb300.ensemble import Ensemble

    cases = ensemble_cases()
    prec = B.PNP_MIXED if args.precision == "mixed" else B.PNP_FP64
    solvers, tuned = [], {}
    for c in cases:
        s = Solver(c["nx"], c["ny"], c["nz"], 2 * math.pi, math.pi, stretch=c["stretch"], precision=prec)
        s.set_params(c["Re"], c["lam"], 1.0, c["V"], 0.5)
        cfg, _ = autotune.tune(s, c["dt"])
        tuned[f'{c["nx"]}x{c["ny"]}x{c["nz"]}'] = cfg
        s.init_state(B.PNP_IC_PB, c["seed"], 0.1)
        solvers.append(s)
    ens = Ensemble(solvers)
    dts = [c["dt"] for c in cases]
    Ke, We = args.ensemble_steps, 3
    ens.step(We, dts)
    ens.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ens.stream)
    ens.step(Ke, dts)
    e1.record(ens.stream)
    ens.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    ncells = sum(c["nx"] * (c["ny"] - 1) * c["nz"] for c in cases)
    bad = []
    for c, s in zip(cases, solvers):
        d = s.diagnostics()
        if d["status"] != 0:
            bad.append(c["seed"])
    ens.close()
    for s in solvers:
        s.close()
    return {"cases": len(cases), "cells": ncells, "steps": Ke, "value": ncells * Ke / t, "unit": UNIT,
            "ms_per_step": 1e3 * t / Ke, "graph_launches_per_step": 1, "precision": args.precision,
            "autotuned": tuned, "flagged_under_resolved": [c["seed"] for c in cases if c["flagged"]],
            "nonfinite_or_negative": bad,
            "recipe": "2 grids (64x65x64, 128x97x128) x Re {1000,3000} x lambda {0.005,0.0158,0.05} x "
                      "V {0,2,5,10}; Gouy-Chapman ions + 0.1 noise; per-case stretching and dt"}


# --------------------------------------------------------------------------
# Large single case: 1024 x 385 x 512 (201,326,592 cells), Re 1e4, Debye length
# 0.005, V 5, tanh stretching 3; mixed precision against the all-FP64 path
# from the same initial state.
# --------------------------------------------------------------------------
C4 = dict(nx=1024, ny=385, nz=512, Lx=2 * math.pi, Lz=math.pi, stretch=3.0, Re=1.0e4, lam=0.005, Sc=1.0, V=5.0,
          beta=0.5, seed=1704, amp=0.1)


def run_large(args, B, Solver, torch):
    from paper_1701_02005_gb300.solver import FIELD_NAMES

    c = C4
    dt, dphi_cell = stable_dt(c["nx"], c["ny"], c["Re"], c["lam"], c["V"], c["stretch"])
    mk = lambda prec: Solver(c["nx"], c["ny"], c["nz"], c["Lx"], c["Lz"], stretch=c["stretch"], precision=prec)
    s64 = mk(B.PNP_FP64)
    s64.set_params(c["Re"], c["lam"], c["Sc"], c["V"], c["beta"])
    s64.init_state(B.PNP_IC_PB, c["seed"], c["amp"])
    smx = mk(B.PNP_MIXED)
    smx.set_params(c["Re"], c["lam"], c["Sc"], c["V"], c["beta"])
    for nm in ("u", "v", "w", "p", "cp", "cm", "Phi"):   # the same initial state, copied on the device
        t = torch.empty(s64.shape(nm), dtype=torch.float64, device=s64.device)
        s64.synchronize()
        B.check(B.pnp_get_state(s64.ctx, FIELD_NAMES[nm], t.data_ptr(), 1), "pnp_get_state")
        s64.synchronize()
        smx.set_device(nm, t)
        del t
    d0 = s64.diagnostics()
    K = args.large_steps
    out = {"workload": "1024x385x512, Re 1e4, lambda_D/h 0.005, Sc 1, V 5 (V-hat 10), tanh stretching 3, "
                       "Gouy-Chapman ions + 0.1 noise, seed 1704",
           "cells": c["nx"] * (c["ny"] - 1) * c["nz"], "dt": dt, "dphi_wall_cell": dphi_cell, "steps": K}
    for name, s in (("fp64", s64), ("mixed", smx)):
        s.step(1, dt)   # graph capture
        s.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(K, dt)
        e1.record(s.stream)
        s.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[name] = {"value": out["cells"] * K / t, "unit": UNIT, "ms_per_step": 1e3 * t / K}
    um64, ummx = s64.mean_profile("u"), smx.mean_profile("u")
    d64, dmx = s64.diagnostics(), smx.diagnostics()
    import numpy as np
    out.update({"speedup": out["mixed"]["value"] / out["fp64"]["value"],
                "mean_u_abs_err": float(np.max(np.abs(ummx - um64))),
                "tau_w_rel_err": float(max(abs(dmx["tau_bot"] - d64["tau_bot"]) / abs(d64["tau_bot"]),
                                           abs(dmx["tau_top"] - d64["tau_top"]) / abs(d64["tau_top"]))),
                "n_plus_rel_drift_mixed": float(abs(dmx["n_plus"] - d0["n_plus"]) / d0["n_plus"]),
                "n_plus_rel_drift_fp64": float(abs(d64["n_plus"] - d0["n_plus"]) / d0["n_plus"]),
                "status": [d64["status"], dmx["status"]], "cfl": dmx["cfl"], "max_dphi": dmx["max_dphi"],
                "tolerance": 1e-4, "launch_config": "built-in defaults (not autotuned)"})
    s64.close()
    smx.close()
    return out


# The step under the options beyond the headline scheme, each against the default
# step on the same solver and state (256x193x256 mixed, built-in launch shapes).
# AF: the periodic x/z sweeps of the approximate factorisation run inside the CN
# site, on the stencil's forward values (the fused path): their own time is that
# site under AF less the same site without them.  At this workload's taps they
# run as one pass of circulant convolutions (x and z together) that reads and
# writes each of the five FP32 arrays once: 40 B per cell and substage.
AF_SWEEP_BYTES = 5 * 8


def run_next_rows(args, B, Solver, torch):
    import numpy as np

    from paper_1701_02005_gb300.solver import profile

    s = Solver(WL["nx"], WL["ny"], WL["nz"], WL["Lx"], WL["Lz"], stretch=WL["stretch"], precision=B.PNP_MIXED)
    try:   # the solver's device memory is released whatever happens below
        return _next_rows(args, B, s, torch, np, profile)
    finally:
        s.close()


def _next_rows(args, B, s, torch, np, profile):
    s.set_params(WL["Re"], WL["lam"], WL["Sc"], WL["V"], WL["beta"])
    s.init_state(B.PNP_IC_PB, WL["seed"], WL["amp"])
    dt, K, n = WL["dt"], args.next_steps, cells()

    def timed(fn, k=K):
        fn(1)   # a changed configuration captures its graph on its first step
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        e0.record(s.stream)
        out = fn(k)
        e1.record(s.stream)
        s.synchronize()
        ms = e0.elapsed_time(e1) / k
        r = {"ms_per_step": ms, "value": n / (ms * 1e-3), "unit": UNIT, "host_ms_per_step":
             1e3 * (time.perf_counter() - h0) / k, "status": s.diagnostics()["status"]}
        return r, out

    step = lambda k: s.step(k, dt)
    base, _ = timed(step)
    nprof = 3
    cn_default = profile(s, nprof, dt)[0]["cn_thomas"] / (3 * nprof)
    B.check(B.pnp_set_scheme(s.ctx, B.PNP_SCHEME_AF), "pnp_set_scheme")
    af, _ = timed(step)
    cn_af = profile(s, nprof, dt)[0]["cn_thomas"] / (3 * nprof)
    B.check(B.pnp_set_fusion(s.ctx, 0), "pnp_set_fusion")
    af_unfused, _ = timed(step)
    B.check(B.pnp_set_fusion(s.ctx, 1), "pnp_set_fusion")
    B.check(B.pnp_set_scheme(s.ctx, B.PNP_SCHEME_CN), "pnp_set_scheme")
    sweep_ms = cn_af - cn_default
    gbs = AF_SWEEP_BYTES * n / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else None
    af.update({"vs_default_ms": af["ms_per_step"] - base["ms_per_step"],
               "unfused_ms_per_step": af_unfused["ms_per_step"],
               "cn_site_ms": {"default": cn_default, "af": cn_af},
               "sweeps": {"ms_per_substage": sweep_ms, "bytes_per_cell": AF_SWEEP_BYTES, "achieved_gbs": gbs,
                          "note": "the CN site under AF less the same site without the sweeps (both fused); the x "
                                  "and z sweeps of u, v, w, c+, c- in one pass (each FP32 array read and written "
                                  "once)"}})
    # wall potentials varying along the walls (the lift added in the inverse x-transforms)
    x = (np.arange(WL["nx"]) + 0.5) * WL["Lx"] / WL["nx"]
    z = (np.arange(WL["nz"]) + 0.5) * WL["Lz"] / WL["nz"]
    pat = np.outer(np.cos(2 * np.pi * z / WL["Lz"]), np.sin(2 * np.pi * x / WL["Lx"]))
    s.set_wall_potential(-WL["V"] + 0.5 * pat, WL["V"] + 0.5 * pat[::-1])
    wp, _ = timed(step)
    wp.update({"vs_default_ms": wp["ms_per_step"] - base["ms_per_step"],
               "map": "Phi_wall = -+V + 0.5 cos(2 pi z / Lz) sin(2 pi x / Lx) (top mirrored in z)"})
    s.set_wall_potential(None, None)
    # adaptive dt: limits read every 10 steps (each check synchronises), at most twice the fixed dt
    ad, dts = timed(lambda k: s.step_adaptive(k, 2 * dt, 0.5, 10))
    dts = np.asarray(dts)
    ad.update({"dt": {"min": float(dts.min()), "mean": float(dts.mean()), "max": float(dts.max())},
               "check_every": 10, "cfl": 0.5, "dt_max": 2 * dt,
               "time_units_per_s": float(dts.sum()) / (1e-3 * ad["host_ms_per_step"] * len(dts)),
               "time_units_per_s_fixed_dt": dt / (1e-3 * base["ms_per_step"])})
    return {"workload": WL_NAME + " (mixed, built-in launch shapes)", "steps": K, "default": base,
            "approximate_factorisation": af, "wall_potential_map": wp, "adaptive_dt": ad}


# --------------------------------------------------------------------------
# Learned wall model at the workload's scale: the turbulent flow at V = 5
# resolved on 256x193x256 (mixed precision) is the truth; the coarse grid keeps
# every 4th y-face and every 2nd x/z cell (128x49x128).  Training pairs the
# coarse run's near-wall features with the fine run's filtered labels over
# consecutive windows of the fine run (pass 0: coarse run alone; passes 1, 2:
# coarse run coupled to the previous network, dataset aggregation); a later,
# unseen window judges c_f against the fine run, and times fine and coarse.
WM = dict(V=5.0, rx=2, ry=4, window=1000, every=2, spinup=8000, layer_steps=1000, passes=3, iters=3000,
          batch=65536, chunk=20, mode=3, relax=1.0, potential_gain=0.3, flux_gain=0.3, seed=1705, amp=0.05,
          residual=True)


def vortices_and_streaks(yf, nz, Lz, A=0.15, Bs=0.4, m=1):
    """Streamwise vortices (a y-z streamfunction psi on the y-face x z-face nodes,
    zero on the walls) and the streaks they lift up, the structures that carry
    plane Couette flow into turbulence: v = d_z psi on the y-faces and w = -d_y psi
    on the z-faces, differenced from psi so that the discrete divergence is zero
    exactly; u' = Bs (1 - y^2) cos(2 pi m z / Lz).  Arrays over [y][z] (uniform in x)."""
    import numpy as np

    dy = np.diff(yf)
    yc = 0.5 * (yf[1:] + yf[:-1])
    dz = Lz / nz
    zf = np.arange(nz) * dz
    zc = zf + 0.5 * dz
    psi = A * (1.0 - yf[:, None] ** 2) ** 2 * np.sin(2 * np.pi * m * zf[None, :] / Lz)
    v = (np.roll(psi, -1, axis=1) - psi) / dz
    w = -(psi[1:] - psi[:-1]) / dy[:, None]
    u = Bs * (1.0 - yc[:, None] ** 2) * np.cos(2 * np.pi * m * zc[None, :] / Lz)
    return u, v, w


# The regime the wall model is for: a coarse grid that does not resolve the wall
# layers.  Walls set in motion at t = 0 under fluid at rest (Stokes layers) on a fine
# 32x65x32 grid (FP64, Re 500, lambda_D/h 0.05, V 2, tanh gamma 2) and on its 16x17x16
# coarsening (every 4th y-face: the first coarse cell spans a third of the double
# layer's thickness, the Stokes layer two cells early on); training as in the large
# block (three windows, the later two coupled), judged on another seed.
WMR = dict(nx=32, ny=65, nz=32, stretch=2.0, Re=500.0, lam=0.05, V=2.0, ry=4, rx=2, dt=0.002, steps=200, every=2,
           iters=3000, passes=3, chunk=10, mode=2, potential_gain=0.3, flux_gain=0.3, seed_train=31, seed_judge=32,
           amp=0.02, net_seed=33, residual=True)


def run_wallmodel_reduced(args, B, Solver, torch):
    import numpy as np

    from paper_1701_02005_gb300 import wallmodel as wm

    c = dict(WMR)
    if args.wm_residual is not None:
        c["residual"] = bool(args.wm_residual)
    skip = wm.PHI_SKIP if c["residual"] else None
    yf = np.tanh(c["stretch"] * (np.arange(c["ny"]) * 2.0 / (c["ny"] - 1) - 1.0)) / math.tanh(c["stretch"])
    yf[0], yf[-1] = -1.0, 1.0
    yc = 0.5 * (yf[1:] + yf[:-1])
    yfc = yf[::c["ry"]].copy()
    ncx, ncz = c["nx"] // c["rx"], c["nz"] // c["rx"]

    def mk(n, m, k, faces):
        s_ = Solver(n, m, k, 2 * math.pi, math.pi, precision=B.PNP_FP64, y_faces=faces)
        s_.set_params(c["Re"], c["lam"], 1.0, c["V"], 0.5)
        return s_

    def impulsive(s_, seed):   # the seeded, projected noise minus the Couette profile
        s_.init_state(B.PNP_IC_PB, seed, c["amp"])
        s_.set("u", s_.get("u") - yc[:, None, None])

    def couple(s_):
        wm.set_coupling(s_, c["mode"], 1.0, c["potential_gain"], c["flux_gain"])

    sf, sc = mk(c["nx"], c["ny"], c["nz"], yf), mk(ncx, len(yfc), ncz, yfc)
    t0 = time.perf_counter()
    Xs, Ts, net, losses = [], [], None, []
    for p in range(c["passes"]):
        impulsive(sf, c["seed_train"])
        wm.restrict(sf, sc)
        couple(sc)
        for n in range(c["steps"] // c["every"]):
            Xs.append(wm.features(sc, 8))
            Ts.append(wm.labels(sf, sc))
            sf.step(c["every"], c["dt"])
            if net is None:
                sc.step(c["every"], c["dt"])
            else:
                wm.step_with_model(sc, net, c["every"], c["dt"])
        wm.set_slip(sc, None, None)
        wm.clear_edl(sc)
        X, T = torch.cat(Xs), torch.cat(Ts)
        if net is None:
            R = wm.residual_targets(T, X, skip)   # what the network's own outputs learn
            xs, ts = X.double().mean(0), R.double().mean(0)
            xsd = torch.maximum(X.double().std(0), 1e-2 * torch.clamp(xs.abs(), min=1e-2))
            tsd = torch.maximum(R.double().std(0), 1e-2 * torch.clamp(ts.abs(), min=1e-4))
            net = wm.MLP(c["steps"] // c["every"] * c["passes"] * 2 * ncz * ncx, seed=c["net_seed"])
            net.set_normalization(xs.cpu().numpy(), (1.0 / xsd).cpu().numpy(), ts.cpu().numpy(),
                                  (1.0 / tsd).cpu().numpy())
            if skip is not None:
                net.set_skip(*skip)
        lr0, lr1 = (2e-3, 5e-4) if p == 0 else (1e-3, 3e-4)
        l0 = net.train_step(X, T, lr0, want_loss=True)
        for it in range(c["iters"]):
            net.train_step(X, T, lr0 if it < c["iters"] // 2 else lr1)
        losses.append([l0, net.train_step(X, T, lr1, want_loss=True)])
    train_s = time.perf_counter() - t0
    sm = mk(ncx, len(yfc), ncz, yfc)
    impulsive(sf, c["seed_judge"])
    wm.restrict(sf, sc)
    wm.restrict(sf, sm)
    couple(sm)
    N0 = sm.diagnostics()["n_plus"]
    cf = {"fine": [], "plain": [], "coupled": []}
    phi = {"plain": [], "coupled": []}
    for n in range(c["steps"] // c["chunk"]):
        sf.step(c["chunk"], c["dt"])
        sc.step(c["chunk"], c["dt"])
        wm.step_with_model(sm, net, c["chunk"], c["dt"])
        for k, s_ in (("fine", sf), ("plain", sc), ("coupled", sm)):
            cf[k].append(s_.diagnostics()["cf"])
        pf = wm.labels(sf, sc)[:, 2].cpu().numpy()
        for k, s_ in (("plain", sc), ("coupled", sm)):   # the total first-cell potential
            pc = wm.first_cell_potential(s_, c["V"], 0.5 * (yfc[1:] + yfc[:-1]))
            phi[k].append(float(np.mean(np.abs(pc - pf)) / np.mean(np.abs(pf))))
    f = np.array(cf["fine"])
    err = lambda a: float(np.mean(np.abs(np.array(a) - f) / f))
    out = {"workload": f"fine {c['nx']}x{c['ny']}x{c['nz']} (FP64) -> coarse {ncx}x{len(yfc)}x{ncz}, Re {c['Re']:g}, "
                       f"lambda_D/h {c['lam']}, V {c['V']:g}, dt {c['dt']}, walls set in motion at t = 0, "
                       f"{c['passes']} training runs of {c['steps']} steps (seed {c['seed_train']}), judged on seed "
                       f"{c['seed_judge']}",
           "coupling": {k: c[k] for k in ("mode", "potential_gain", "flux_gain", "residual")},
           "training": {"rows": int(X.shape[0]), "loss_first_last": losses, "seconds": train_s},
           "cf_err": {k: err(cf[k]) for k in ("plain", "coupled")},
           "first_cell_phi_err": {k: float(np.mean(v)) for k, v in phi.items()},
           "ion_number_drift_coupled": abs(sm.diagnostics()["n_plus"] - N0) / N0,
           "mlp_status": net.status()}
    for s_ in (sf, sc, sm):
        s_.close()
    net.close()
    return out


def run_wallmodel(args, B, Solver, torch):
    import numpy as np

    from paper_1701_02005_gb300 import wallmodel as wm

    c = dict(WM)
    if args.wm_edl is not None:
        c["potential_gain"], c["flux_gain"] = args.wm_edl
    if args.wm_residual is not None:
        c["residual"] = bool(args.wm_residual)
    skip = wm.PHI_SKIP if c["residual"] else None
    nx, ny, nz, st = WL["nx"], WL["ny"], WL["nz"], WL["stretch"]
    dt = stable_dt(nx, ny, WL["Re"], WL["lam"], c["V"], st)[0]
    yf = np.tanh(st * (np.arange(ny) * 2.0 / (ny - 1) - 1.0)) / math.tanh(st)
    yf[0], yf[-1] = -1.0, 1.0
    mk = lambda n, m, k, faces: Solver(n, m, k, WL["Lx"], WL["Lz"], precision=B.PNP_MIXED, y_faces=faces)
    fine = mk(nx, ny, nz, yf)
    # turbulence first, at V = 0 with the adaptive dt (at most the advective one; about
    # 20 time units), then the walls charged to V and the double layers formed over
    # layer_steps at the V-limited dt
    dt0 = stable_dt(nx, ny, WL["Re"], WL["lam"], 0.0, st)[0]
    fine.set_params(WL["Re"], WL["lam"], WL["Sc"], 0.0, WL["beta"])
    fine.init_state(B.PNP_IC_PB, c["seed"], c["amp"])
    du, dv, dw = vortices_and_streaks(yf, nz, WL["Lz"])
    for name, d in (("u", du), ("v", dv), ("w", dw)):
        fine.set(name, fine.get(name) + d[:, :, None])
    ncx, ncy, ncz = nx // c["rx"], (ny - 1) // c["ry"] + 1, nz // c["rx"]
    yfc = yf[::c["ry"]].copy()

    def coarse():
        s = mk(ncx, ncy, ncz, yfc)
        s.set_params(WL["Re"], WL["lam"], WL["Sc"], c["V"], WL["beta"])
        return s

    def couple(s):
        wm.set_coupling(s, c["mode"], c["relax"], c["potential_gain"], c["flux_gain"])

    t0 = time.perf_counter()
    cf_spin, t_spin = [], 0.0
    log = lambda *a: print("wallmodel:", *a, file=sys.stderr, flush=True)
    for n in range(10):   # dt from the state's limits (CFL 0.5), at most the advective dt
        t_spin += float(np.sum(fine.step_adaptive(c["spinup"] // 10, dt0, 0.5, 20)))
        d = fine.diagnostics()
        cf_spin.append(d["cf"])
        log(f"spin-up {n}: t {t_spin:.2f} cf {d['cf']:.6g} status {d['status']}")
    cf_spun = cf_spin[-1]
    fine.set_params(WL["Re"], WL["lam"], WL["Sc"], c["V"], WL["beta"])
    fine.step(c["layer_steps"], dt)
    fine.synchronize()
    spin_s = time.perf_counter() - t0
    rows = 2 * ncz * ncx
    net, Xs, Ts, losses, good = None, [], [], [], None
    sc = coarse()
    for p in range(c["passes"]):
        wm.restrict(fine, sc)
        if net is not None:
            couple(sc)
        for n in range(c["window"] // c["every"]):
            if n % 50 == 49 and sc.diagnostics()["status"] != 0:
                break   # a coupled run that left the valid states ends its window early
            Xs.append(wm.features(sc, 8))
            Ts.append(wm.labels(fine, sc))
            fine.step(c["every"], dt)
            if net is None:
                sc.step(c["every"], dt)
            else:
                wm.step_with_model(sc, net, c["every"], dt)
        wm.set_slip(sc, None, None)
        wm.clear_edl(sc)
        X, T = torch.cat(Xs), torch.cat(Ts)
        R = wm.residual_targets(T, X, skip)   # what the network's own outputs learn
        ok = torch.isfinite(X).all(1) & torch.isfinite(T).all(1)   # rows of a run gone non-finite stay out
        if net is not None:   # and rows far outside the first pass's spread
            ok &= (((X.double() - xs) / xsd).abs() < 20).all(1) & (((R.double() - ts) / tsd).abs() < 20).all(1)
        X, T, R = X[ok].contiguous(), T[ok].contiguous(), R[ok]
        log(f"pass {p}: {len(Xs)} snapshots, {int(ok.sum())} of {ok.numel()} rows kept, coarse cf "
            f"{sc.diagnostics()['cf']:.6g}")
        if X.shape[0] == 0:
            break
        if net is None:
            xs, ts = X.mean(0).double(), R.mean(0).double()
            xsd = torch.maximum(X.double().std(0), 1e-2 * torch.clamp(xs.abs(), min=1e-2))
            tsd = torch.maximum(R.double().std(0), 1e-2 * torch.clamp(ts.abs(), min=1e-4))
            net = wm.MLP(max(c["batch"], rows), seed=c["seed"])
            net.set_normalization(xs.cpu().numpy(), (1.0 / xsd).cpu().numpy(), ts.cpu().numpy(),
                                  (1.0 / tsd).cpu().numpy())
            if skip is not None:
                net.set_skip(*skip)
        del R
        lr0, lr1 = (2e-3, 5e-4) if p == 0 else (1e-3, 3e-4)
        nb = max(1, X.shape[0] // c["batch"])
        gen = torch.Generator(device=X.device).manual_seed(c["seed"] + p)
        perm = torch.randperm(X.shape[0], device=X.device, generator=gen)
        Xp, Tp = X[perm].contiguous(), T[perm].contiguous()
        l0 = net.train_step(Xp[:c["batch"]], Tp[:c["batch"]], lr0, want_loss=True)
        for it in range(c["iters"]):
            b = it % nb
            net.train_step(Xp[b * c["batch"]:(b + 1) * c["batch"]], Tp[b * c["batch"]:(b + 1) * c["batch"]],
                           lr0 if it < c["iters"] // 2 else lr1)
        l1 = net.train_step(Xp[:c["batch"]], Tp[:c["batch"]], lr1, want_loss=True)
        losses.append([l0, l1])
        log(f"pass {p}: loss {l0:.4g} -> {l1:.4g}")
        del Xp, Tp, perm
        if not math.isfinite(l1):   # a pass that failed to train: back to the last good network
            if good is not None:
                net.set_params(good)
            break
        good = net.params()
    train_s = time.perf_counter() - t0
    if net is None:
        for s_ in (fine, sc):
            s_.close()
        return {"error": "no finite training rows", "spinup_cf": cf_spin, "spinup_time_units": t_spin}
    # the judged window: fine truth, coarse alone, and the coarse run coupled to the
    # network in two ways: the double layer only (the solver's own wall shear, mode 3)
    # and the double layer with the plane-mean predicted wall stress (mode 2)
    sp = coarse()
    cpl = {"coupled_edl": coarse(), "coupled_shear": coarse()}
    wm.restrict(fine, sp)
    for k, s_ in cpl.items():
        wm.restrict(fine, s_)
        wm.set_coupling(s_, 3 if k == "coupled_edl" else 2, c["relax"], c["potential_gain"], c["flux_gain"])
    runs = {"plain": sp, **cpl}
    cf = {"fine": [], **{k: [] for k in runs}}
    phi_err = {k: [] for k in runs}
    for n in range(c["window"] // c["chunk"]):
        fine.step(c["chunk"], dt)
        sp.step(c["chunk"], dt)
        for s_ in cpl.values():
            wm.step_with_model(s_, net, c["chunk"], dt)
        cf["fine"].append(fine.diagnostics()["cf"])
        phi_f = wm.labels(fine, sp)[:, 2].cpu().numpy()
        for k, s_ in runs.items():
            cf[k].append(s_.diagnostics()["cf"])
            phi_c = wm.first_cell_potential(s_, c["V"], 0.5 * (yfc[1:] + yfc[:-1]))   # offsets included
            phi_err[k].append(float(np.mean(np.abs(phi_c - phi_f)) / np.mean(np.abs(phi_f))))
    f = np.array(cf["fine"])
    err = lambda a: float(np.mean(np.abs(np.array(a) - f) / f))
    merr = lambda a: float(abs(np.mean(a) - np.mean(f)) / np.mean(f))
    # <u>(y) at the end of the window: the fine profile averaged onto the coarse cells
    dyf = np.diff(yf)
    uf = fine.mean_profile("u")
    ufc = (uf * dyf).reshape(-1, c["ry"]).sum(1) / dyf.reshape(-1, c["ry"]).sum(1)
    u_err = {k: float(np.max(np.abs(s_.mean_profile("u") - ufc))) for k, s_ in runs.items()}
    sm = cpl["coupled_edl"]

    # time per step: fine, coarse alone, coarse with the model
    def timed(fn, s, n=100):
        fn(10)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        fn(n)
        e1.record(s.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms_f = timed(lambda n: fine.step(n, dt), fine)
    ms_p = timed(lambda n: sp.step(n, dt), sp)
    ms_c = timed(lambda n: wm.step_with_model(sm, net, n, dt), sm)
    out = {"workload": f"fine {nx}x{ny}x{nz} (mixed) -> coarse {ncx}x{ncy}x{ncz}, Re {WL['Re']:g}, "
                       f"lambda_D/h {WL['lam']}, V {c['V']:g}, dt {dt:.4g}, {c['spinup']} spin-up steps at V 0, "
                       f"{c['passes']} training windows + 1 judged window of {c['window']} steps",
           "coupling": {**{k: c[k] for k in ("mode", "relax", "potential_gain", "flux_gain", "residual")},
                        "note": "training passes coupled in this mode; judged in mode 3 (coupled_edl) and mode 2 "
                                "(coupled_shear)"},
           "spinup": {"steps_at_V0": c["spinup"], "dt_max_V0": dt0, "time_units": t_spin, "cf_after": cf_spun,
                      "cf_laminar": 2.0 / WL["Re"],
                      "cf_series": [round(x, 7) for x in cf_spin], "turbulent": bool(cf_spun > 2.0 * 2.0 / WL["Re"]),
                      "layer_steps_at_V": c["layer_steps"], "seconds": spin_s},
           "training": {"rows": int(X.shape[0]), "snapshots": len(Xs), "iters_per_pass": c["iters"],
                        "batch": c["batch"], "loss_first_last": losses, "seconds": train_s - spin_s},
           "cf_err": {k: err(cf[k]) for k in runs}, "mean_cf_err": {k: merr(cf[k]) for k in runs},
           "first_cell_phi_err": {k: float(np.mean(v)) for k, v in phi_err.items()},
           "mean_cf": {k: float(np.mean(v)) for k, v in cf.items()},
           "mean_u_max_err": u_err,
           "cf_series": {k: [round(x, 6) for x in v[::5]] for k, v in cf.items()},
           "ms_per_step": {"fine": ms_f, "coarse": ms_p, "coarse_with_model": ms_c},
           "speedup_coarse_with_model_over_fine": ms_f / ms_c, "mlp_status": net.status(),
           "status": {"fine": fine.diagnostics()["status"], **{k: s_.diagnostics()["status"] for k, s_ in cpl.items()}}}
    for s_ in (fine, sc, sp, *cpl.values()):
        s_.close()
    net.close()
    return out


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = str(index)
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        # nvidia-smi's own start-up (driver initialisation) can hold up the launches of
        # this process for a moment: let it finish before the timed region opens
        t0 = time.time()
        while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9 or p[0] != self.index:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# The FP64 oracle on the host cores: the workload split into z-slabs (each an
# independent problem of the same x/y grid and parameters, periodic in z over
# its own extent), one slab per process, all processes timed together from a
# common barrier.  Processes are spawned (never forked after the GPU is in use).
# --------------------------------------------------------------------------
def _oracle_slab(wl, nz):
    from oracle import pnp_oracle as o

    g = o.Grid(wl["nx"], wl["ny"], nz, wl["Lx"], wl["Lz"] * nz / wl["nz"], stretch=wl["stretch"])
    prm = o.Params(Re=wl["Re"], lam=wl["lam"], Sc=wl["Sc"], V=wl["V"], beta=wl["beta"])
    return o, g, prm, o.initial_state(g, prm, o.IC_PB, seed=wl["seed"], amp=wl["amp"])


def _oracle_worker(wl, nz, warmup, steps, barrier, results):
    os.environ["OMP_NUM_THREADS"] = "1"
    o, g, prm, st = _oracle_slab(wl, nz)
    for _ in range(warmup):
        st = o.step(g, prm, st, wl["dt"], 1)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = o.step(g, prm, st, wl["dt"], 1)
    results.put((g.nx * g.nyc * g.nz * steps, time.perf_counter() - t0))


def oracle_on_host_cores(wl, warmup, steps, cores=None):
    """Cell-steps/s of the oracle over all host cores (one z-slab per process)."""
    import multiprocessing as mp

    cores = cores or os.cpu_count() or 1
    nproc = 1
    while nproc * 2 <= min(cores, wl["nz"] // 2):
        nproc *= 2
    nz = wl["nz"] // nproc
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(nproc), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(wl, nz, warmup, steps, barrier, results)) for _ in range(nproc)]
    for p in procs:
        p.start()
    out = [results.get() for _ in procs]
    for p in procs:
        p.join()
    cell_steps = sum(c for c, _ in out)
    t = max(t for _, t in out)
    return {"value": cell_steps / t, "unit": UNIT, "cores": nproc, "host_cpus": os.cpu_count(),
            "threads_per_process": 1, "kind": "oracle", "seconds": t,
            "sample": f"{nproc} processes x {steps} steps of a {wl['nx']}x{wl['ny']}x{nz} z-slab of the workload "
                      f"({nproc * nz} of its {wl['nz']} z-planes in all; each slab periodic over its own z extent, "
                      f"same x/y grid and parameters); NumPy FP64, one thread per process"}


def cpu_baseline(nsteps=3):
    """The FP64 oracle as it stands on all host cores (the workload's full cell
    count per step, a few steps), plus the small 32x33x32 configuration's 200
    steps on one core."""
    out = oracle_on_host_cores(WL, 0, nsteps)
    from oracle import pnp_oracle as o

    g = o.Grid(32, 33, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=1701, amp=1e-3)
    t0 = time.perf_counter()
    o.step(g, prm, st, 0.01, 200)
    t = time.perf_counter() - t0
    out["small_case"] = {"value": g.nx * g.nyc * g.nz * 200 / t, "unit": UNIT, "cores": 1, "steps": 200,
                         "workload": "32x33x32, Re 400, lambda_D/h 0.05, V 2, dt 0.01 (the parity configuration)"}
    return out


def run_reference(args):
    """--impl reference: the oracle on all host cores, each step the whole
    workload's cell count as independent z-slabs (one per process)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    K, W = args.steps, args.warmup
    cb = oracle_on_host_cores(WL, W, K)
    v = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * cb["seconds"] / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WL_NAME, "sample": cb["sample"], "precision": "fp64"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
def reduce_times(t, dist):
    """Max of the per-rank timed-region durations (every rank runs its own replica)."""
    if dist is None:
        return t
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(cells_per_rank, steps, world, t_max):
    """Cell-steps/s of all ranks together: every rank advances its own case."""
    return world * cells_per_rank * steps / t_max


# --------------------------------------------------------------------------
# Mixed precision (both solve policies) against the FP64 path from one initial
# state: plane-mean <u>(y) and wall-shear errors every `every` steps, and the
# time per step of each path (CUDA events over the first `timed` steps).
# --------------------------------------------------------------------------
def compare_precisions(B, Solver, torch, wl, V, dt, nsteps, every, launch_cfg=None, seed=None, device=0, tol=1e-4,
                       timed=None):
    import numpy as np

    from paper_1701_02005_gb300.solver import FIELD_NAMES

    mk = lambda prec: Solver(wl["nx"], wl["ny"], wl["nz"], wl["Lx"], wl["Lz"], stretch=wl["stretch"], precision=prec,
                             device=device)
    s64 = mk(B.PNP_FP64)
    s64.set_params(wl["Re"], wl["lam"], wl["Sc"], V, wl["beta"])
    s64.init_state(B.PNP_IC_PB, wl["seed"] if seed is None else seed, wl["amp"])
    mixed = {}
    for name, pol in (("default", B.PNP_POLICY_DEFAULT), ("fp64_solves", B.PNP_POLICY_FP64_SOLVES)):
        sm = mk(B.PNP_MIXED)
        sm.set_params(wl["Re"], wl["lam"], wl["Sc"], V, wl["beta"])
        sm.set_policy(pol)
        if launch_cfg is not None:
            import ctypes as C
            B.check(B.pnp_set_launch_config(sm.ctx, (C.c_int * 4)(*launch_cfg)), "pnp_set_launch_config")
        for nm in ("u", "v", "w", "p", "cp", "cm", "Phi"):   # the same initial state, copied on the device
            t = torch.empty(s64.shape(nm), dtype=torch.float64, device=s64.device)
            s64.synchronize()
            B.check(B.pnp_get_state(s64.ctx, FIELD_NAMES[nm], t.data_ptr(), 1), "pnp_get_state")
            s64.synchronize()
            sm.set_device(nm, t)
        mixed[name] = sm
    d0 = s64.diagnostics()
    cells_ = wl["nx"] * (wl["ny"] - 1) * wl["nz"]
    timed = timed or every
    ms = {}
    curve = []
    done = 0
    horizon = {k: None for k in mixed}
    while done < nsteps:
        n = min(every, nsteps - done)
        for name, s in [("fp64", s64)] + list(mixed.items()):
            if done == 0 and n > 1:   # time the first block (graph captured by its first step)
                s.step(1, dt)
                s.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s.stream)
                s.step(n - 1, dt)
                e1.record(s.stream)
                s.synchronize()
                ms[name] = e0.elapsed_time(e1) / (n - 1)
            else:
                s.step(n, dt)
        done += n
        um64 = s64.mean_profile("u")
        d64 = s64.diagnostics()
        point = {"step": done}
        for name, s in mixed.items():
            dm = s.diagnostics()
            eu = float(np.max(np.abs(s.mean_profile("u") - um64)))
            et = float(max(abs(dm["tau_bot"] - d64["tau_bot"]) / abs(d64["tau_bot"]),
                           abs(dm["tau_top"] - d64["tau_top"]) / abs(d64["tau_top"])))
            point[name] = {"mean_u_abs_err": eu, "tau_w_rel_err": et,
                           "n_plus_rel_drift": float(abs(dm["n_plus"] - d0["n_plus"]) / d0["n_plus"])}
            if horizon[name] is None and max(eu, et) > tol:
                horizon[name] = done
        curve.append(point)
        if all(h is not None for h in horizon.values()):
            break
    last = curve[-1]
    out = {"V": V, "dt": dt, "steps": done, "tolerance": tol,
           "fp64_ms_per_step": ms.get("fp64"), "fp64_value": cells_ / (ms["fp64"] * 1e-3) if "fp64" in ms else None,
           "mean_u_abs_err": last["default"]["mean_u_abs_err"], "tau_w_rel_err": last["default"]["tau_w_rel_err"],
           "n_plus_rel_drift": last["default"]["n_plus_rel_drift"],
           "fp64_solves": {"ms_per_step": ms.get("fp64_solves"),
                           "value": cells_ / (ms["fp64_solves"] * 1e-3) if "fp64_solves" in ms else None,
                           **last["fp64_solves"]},
           "default_ms_per_step_here": ms.get("default"),
           "tolerance_lost_at_step": horizon, "curve": curve}
    s64.close()
    for s in mixed.values():
        s.close()
    return out


def run_sweep(args):
    """A reduced version of the paper's drag-vs-voltage experiment (Results):
    plane Couette at Re 3000 on 64 x 65 x 64 (box 2 pi x 2 x pi), Debye length
    0.0158, Sc 1, wall potentials V = 0, 0.5, 1, 1.5, 2 (V-hat = 2 V) from one
    seeded perturbed state, all cases in one ensemble (one graph launch per
    step, a common dt); time statistics after a spin-up.  Context only: the
    grid is coarse and the averaging window short."""
    import numpy as np
    import torch

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.ensemble import Ensemble
    from paper_1701_02005_gb300.solver import Solver

    nx, ny, nz, Re, lam = 64, 65, 64, 3000.0, 0.0158
    Vs = (0.0, 0.5, 1.0, 1.5, 2.0)
    cases = []
    for V in Vs:
        chosen = 6.0
        for gm in (1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0):
            if stable_dt(nx, ny, Re, lam, V, gm)[1] <= 1.0:
                chosen = gm
                break
        cases.append((V, chosen))
    stretch = max(g for _, g in cases)   # one grid for all: the finest wall cell any case needs
    dt = min(stable_dt(nx, ny, Re, lam, V, stretch)[0] for V in Vs)
    solvers = []
    for V, _ in cases:
        s = Solver(nx, ny, nz, 2 * math.pi, math.pi, stretch=stretch, precision=B.PNP_MIXED)
        s.set_params(Re, lam, 1.0, V, 0.5)
        s.init_state(B.PNP_IC_PB, 1706, args.sweep_amp)
        solvers.append(s)
    ens = Ensemble(solvers)
    spin, avg, every = args.sweep_spinup, args.sweep_steps, 10
    t0 = time.perf_counter()
    ens.step(spin, [dt] * len(solvers))
    ens.synchronize()
    for s in solvers:
        s.stats_reset()
    cf_hist = [[] for _ in solvers]
    for _ in range(avg // every):
        ens.step(every, [dt] * len(solvers))
        ens.synchronize()
        for i, s in enumerate(solvers):
            s.stats_sample()
            cf_hist[i].append(s.diagnostics()["cf"])
    wall = time.perf_counter() - t0
    out = {"workload": f"{nx}x{ny}x{nz}, Re {Re:g}, lambda_D/h {lam}, Sc 1, tanh stretching {stretch}, dt {dt:.4g}, "
                       f"{spin} spin-up + {avg} averaged steps, noise {args.sweep_amp}, seed 1706",
           "wall_seconds": wall, "cases": []}
    cf0 = None
    for (V, _), s, hist in zip(cases, solvers, cf_hist):
        st, cf, n = s.stats()
        d = s.diagnostics()
        um = st["u"][0]
        tau = 0.5 * cf
        ut = math.sqrt(max(tau, 0.0))
        g = s   # plane data in wall units near the bottom wall
        yf = np.tanh(stretch * (np.arange(ny) * 2.0 / (ny - 1) - 1.0)) / math.tanh(stretch)
        yc = 0.5 * (yf[1:] + yf[:-1])
        yplus = (yc + 1.0) * Re * ut
        uplus = (um + 1.0) / ut if ut > 0 else um * 0
        if cf0 is None:
            cf0 = cf
        out["cases"].append({"V": V, "V_hat": 2 * V, "cf": cf, "cf_over_cf0": cf / cf0 if cf0 else None,
                             "re_tau": Re * ut, "cf_laminar": 2.0 / Re, "samples": n, "status": d["status"],
                             "cf_series_first_last": [hist[0], hist[-1]],
                             "u_plus_at_y_plus": [[round(float(a), 3), round(float(b), 3)]
                                                  for a, b in zip(yplus[:12:2], uplus[:12:2])],
                             "rms_cplus_max": float(np.max(st["cp"][1])), "rms_cminus_max": float(np.max(st["cm"][1])),
                             "rms_phi_max": float(np.max(st["Phi"][1]))})
    ens.close()
    for s in solvers:
        s.close()
    print(json.dumps(out), flush=True)
    return 0


def run_curve(args):
    """Mixed (both solve policies) against FP64 on the workload at V = 0, 2, 5:
    <u>(y) and wall-shear errors every 100 steps up to --curve-steps or until
    both policies have lost the 1e-4 tolerance."""
    import torch

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    out = {"workload": WL_NAME, "curves": {}}
    for V in (0.0, 2.0, 5.0):
        dtV = WL["dt"] if V <= 2.0 else stable_dt(WL["nx"], WL["ny"], WL["Re"], WL["lam"], V, WL["stretch"])[0]
        out["curves"][str(V)] = compare_precisions(B, Solver, torch, WL, V, dtV, args.curve_steps, 100)
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import FIELD_NAMES, Solver, profile

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    prec = B.PNP_MIXED if args.precision == "mixed" else B.PNP_FP64
    s = Solver(WL["nx"], WL["ny"], WL["nz"], WL["Lx"], WL["Lz"], stretch=WL["stretch"], precision=prec, device=local)
    s.set_params(WL["Re"], WL["lam"], WL["Sc"], WL["V"], WL["beta"])
    if args.no_fusion:
        B.check(B.pnp_set_fusion(s.ctx, 0), "pnp_set_fusion")
    dt = WL["dt"]
    launch_cfg = None
    if not args.no_autotune:
        from paper_1701_02005_gb300 import autotune
        launch_cfg, _ = autotune.tune(s, dt)   # before the state: tuning overwrites the workspace
    s.init_state(B.PNP_IC_PB, WL["seed"] + rank, WL["amp"])
    K, W = args.steps, args.warmup
    s.step(W, dt)
    s.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clk = ClockSampler(local)
    barrier()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(K, dt)
    e1.record(s.stream)
    s.synchronize()
    barrier()
    clocks = clk.stop()
    t = reduce_times(e0.elapsed_time(e1) / 1e3, dist)
    # repeat the timed block (after a longer warm-up) and report the median of the
    # repeats beside the contract's single timed run
    reps = []
    if args.repeats > 0:
        s.step(max(0, 10 - W), dt)
        for _ in range(args.repeats):
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(s.stream)
            s.step(K, dt)
            r1.record(s.stream)
            s.synchronize()
            reps.append(r0.elapsed_time(r1) / K)
    diag = s.diagnostics()
    n_cells = cells()
    value = whole_job_value(n_cells, K, world, t)

    # per-launch-site timing with CUDA events on the library's stream
    nprof = max(2, min(5, K))
    ms, lps = profile(s, nprof, dt)
    per_launch = {k: v / (3 * nprof) for k, v in ms.items()}
    total = sum(per_launch.values())
    # the dominant kernel: a site's time per kernel launch (the mixed CN site is
    # two kernels, ions and velocities; the potential y-solve site the FP64 mean
    # mode and the df lines)
    kernels_per_site = {"cn_thomas": 2, "e_thomas": 2} if prec == B.PNP_MIXED else {}
    dom = max(per_launch, key=lambda k: per_launch[k] / kernels_per_site.get(k, 1))
    pname = "fp64" if prec == B.PNP_FP64 else "mixed"
    fp64_peak = max(s.fp64_peak(), s.fp64_peak())   # measured now, at working clocks
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    sites = {}
    for k, v in per_launch.items():
        cst = site_cost(k, pname, launch_cfg, not args.no_fusion)
        d = v * 1e-3
        gbs = cst["bytes"] * n_cells / d / 1e9
        tf = 2.0 * cst["fp64_ops"] * n_cells / d / 1e12   # FP64 ops counted as FMA-equivalent flops
        sites[k] = {"ms": round(v, 4), "share": round(v / total, 4), "hbm_frac": round(gbs / hbm_peak, 4),
                    "fp64_frac": round(tf / (fp64_peak / 1e12), 4)}
    cst = site_cost(dom, pname, launch_cfg, not args.no_fusion)
    dur = per_launch[dom] * 1e-3
    hbm_gbs = cst["bytes"] * n_cells / dur / 1e9
    alu_tf = 2.0 * cst["fp64_ops"] * n_cells / dur / 1e12
    if alu_tf / (fp64_peak / 1e12) > hbm_gbs / hbm_peak:
        roof = {"bound": "alu", "achieved": alu_tf, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                "frac": alu_tf / (fp64_peak / 1e12), "traffic": None, "kernel": dom,
                "peak_source": "FP64 FMA throughput measured live in this run (pnp_fp64_peak)",
                "per_unit": f"{cst['fp64_ops']} FP64-pipe instructions per cell x {n_cells} cells per launch"}
    else:
        roof = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
                "traffic": None, "kernel": dom, "peak_source": hbm_src,
                "per_unit": f"{cst['bytes']:.1f} B per cell x {n_cells} cells per launch"}
    roof["share"] = per_launch[dom] / total
    # DRAM bytes (read + write) per launch of the dominant kernel from the committed
    # one-pass ncu capture of this workload (profiles/, DRAM traffic summary), valid
    # only for the kernel and launch shape that capture measured
    nt = NCU_TRAFFIC.get((pname, dom))
    if nt and nt["bytes"] and nt["cells"] == n_cells and (nt["shape"] is None or (launch_cfg and launch_cfg[0] in nt["shape"])):
        roof["traffic"] = nt["bytes"]
        roof["traffic_kernel"] = nt["kernel"]

    # the whole step against the HBM roofline: algorithmic bytes and, where a capture of
    # this workload and launch shape is committed, the bytes ncu counted
    step_roof = {"algorithmic_bytes_per_cell_step": STEP_BYTES[pname],
                 "achieved_gbs": STEP_BYTES[pname] * n_cells * K / t / 1e9}
    step_roof["frac_of_measured"] = step_roof["achieved_gbs"] / hbm_peak
    step_roof["frac_of_nominal"] = step_roof["achieved_gbs"] / NOMINAL_HBM_GBS
    sn = STEP_NCU.get(pname)
    if sn and sn["cells"] == n_cells and (sn["shape"] is None or (launch_cfg and list(launch_cfg) == sn["shape"])):
        g_ncu = sn["bytes_per_cell_step"] * n_cells * K / t / 1e9
        step_roof.update({"ncu_bytes_per_cell_step": sn["bytes_per_cell_step"], "ncu_gbs": g_ncu,
                          "ncu_frac_of_measured": g_ncu / hbm_peak, "ncu_frac_of_nominal": g_ncu / NOMINAL_HBM_GBS,
                          "ncu_note": sn["note"]})
    else:
        step_roof.update({"ncu_bytes_per_cell_step": None, "ncu_gbs": None, "ncu_frac_of_measured": None,
                          "ncu_frac_of_nominal": None})
    step_roof["peaks"] = {"measured_gbs": hbm_peak, "nominal_gbs": NOMINAL_HBM_GBS}

    # the FP64 path on the same workload, and the mixed-vs-FP64 error from one initial state
    cmp = None
    if prec == B.PNP_MIXED and not args.no_fp64_compare:
        cmp = compare_precisions(B, Solver, torch, WL, WL["V"], dt, args.compare_steps, args.compare_every,
                                 launch_cfg=launch_cfg, seed=WL["seed"] + rank, device=local)
        cmp["speedup"] = (value / world) / cmp["fp64_value"]
        cmp["other_voltages"] = {}
        for V in (0.0, 5.0):   # shorter curves at the workload's other wall potentials
            dtV = dt if V <= WL["V"] else stable_dt(WL["nx"], WL["ny"], WL["Re"], WL["lam"], V, WL["stretch"])[0]
            r = compare_precisions(B, Solver, torch, WL, V, dtV, args.compare_steps // 2, args.compare_every,
                                   launch_cfg=launch_cfg, seed=WL["seed"] + rank, device=local)
            cmp["other_voltages"][str(V)] = {k: r[k] for k in ("dt", "steps", "mean_u_abs_err", "tau_w_rel_err",
                                                                "fp64_solves", "tolerance_lost_at_step", "curve")}

    # end to end through the public API with pinned host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        names = ["u", "v", "w", "p", "cp", "cm", "Phi", "Hu", "Hv", "Hw", "Hcp", "Hcm"]
        host = {}
        for nm in names:
            a = s.get(nm)
            pin = torch.empty(a.shape, dtype=torch.float64).pin_memory()
            pin.numpy()[...] = a
            host[nm] = pin
        Ke = max(1, min(args.e2e_steps, K))
        state_bytes = sum(h.numel() * 8 for h in host.values())

        def e2e_run(pipelined):
            # no collection pause of the Python heap inside the timed region
            gc.collect()
            gc.disable()
            try:
                return e2e_timed(pipelined)
            finally:
                gc.enable()

        def e2e_timed(pipelined):
            torch.cuda.synchronize()
            u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            u0.record(s.stream)
            for nm in names:
                B.check(B.pnp_set_state(s.ctx, FIELD_NAMES[nm], host[nm].data_ptr(), 0), "pnp_set_state")
            u1.record(s.stream)
            s.synchronize()
            t1 = time.perf_counter()
            if pipelined:
                # the diagnostics of every step are read one step behind (pinned records,
                # an event per post), so the host never stalls the stream
                raws = [s.diag_buffer(), s.diag_buffer()]
                evs = [torch.cuda.Event(), torch.cuda.Event()]
                for k in range(Ke):
                    s.step(1, dt)
                    s.diagnostics_post(raws[k % 2])
                    evs[k % 2].record(s.stream)
                    if k > 0:
                        evs[(k - 1) % 2].synchronize()
                        s.diagnostics_read(raws[(k - 1) % 2])
                evs[(Ke - 1) % 2].synchronize()
                last = s.diagnostics_read(raws[(Ke - 1) % 2])
            else:
                for k in range(Ke):
                    s.step(1, dt)
                    last = s.diagnostics()
            t2 = time.perf_counter()
            out = torch.empty(host["u"].shape, dtype=torch.float64).pin_memory()
            B.check(B.pnp_get_state(s.ctx, B.PNP_U, out.data_ptr(), 0), "pnp_get_state")
            t3 = time.perf_counter()
            return {"value": n_cells * Ke / (t3 - t0), "set_state_s": t1 - t0,
                    "set_state_device_s": u0.elapsed_time(u1) / 1e3, "steps_s": t2 - t1,
                    "ms_per_step_in_loop": 1e3 * (t2 - t1) / Ke, "get_state_s": t3 - t2,
                    "d2h": out.numel() * 8, "status": last["status"]}

        r_sync = e2e_run(False)
        runs = sorted((e2e_run(True) for _ in range(3)), key=lambda q: q["value"])
        r = runs[1]   # the median of three
        # device time of one diagnostics pass (reductions + record copy) on its own
        raw = s.diag_buffer()
        s.diagnostics_post(raw)
        s.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(s.stream)
        for _ in range(20):
            s.diagnostics_post(raw)
        q1.record(s.stream)
        s.synchronize()
        diag_ms = q0.elapsed_time(q1) / 20
        e2e = {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": state_bytes / Ke,
               "d2h_bytes_per_step": 128 + r["d2h"] / Ke, "steps": Ke, "last_step_status": r["status"],
               "phases": {**{k: r[k] for k in ("set_state_s", "set_state_device_s", "steps_s", "ms_per_step_in_loop",
                                               "get_state_s")},
                          "diagnostics_ms_alone": diag_ms},
               "runs": [q["value"] for q in runs],
               "runs_set_state_s": [[q["set_state_s"], q["set_state_device_s"]] for q in runs],
               "synchronous_diagnostics": {k: r_sync[k] for k in ("value", "set_state_s", "ms_per_step_in_loop")},
               "note": "set_state of all 12 fields from pinned host, then per step pnp_step + "
                       "pnp_diagnostics_post (D2H of the step's diagnostics into a pinned record, read one step "
                       "behind), then get_state(u) to pinned host; the median of three such runs; the same with "
                       "pnp_diagnostics (synchronising every step) beside it"}

    ensemble = None
    if not args.no_ensemble:
        ensemble = run_ensemble(args, B, Solver, torch)

    large = None
    if not args.no_large:
        large = run_large(args, B, Solver, torch)

    next_rows = None
    if rank == 0 and not args.no_next:
        try:
            next_rows = run_next_rows(args, B, Solver, torch)
        except Exception as exc:  # noqa: BLE001
            next_rows = {"error": f"{type(exc).__name__}: {exc}"}

    mlp = None
    if rank == 0 and not args.no_wallmodel:
        try:
            mlp = run_mlp(args, B, torch)
        except Exception as exc:  # noqa: BLE001
            mlp = {"error": f"{type(exc).__name__}: {exc}"}

    wallmodel = None
    if rank == 0 and not args.no_wallmodel:
        try:   # a side experiment: its failure must not cost the headline line
            wallmodel = run_wallmodel(args, B, Solver, torch)
        except Exception as exc:  # noqa: BLE001
            wallmodel = {"error": f"{type(exc).__name__}: {exc}"}
        try:
            wallmodel["reduced"] = run_wallmodel_reduced(args, B, Solver, torch)
        except Exception as exc:  # noqa: BLE001
            wallmodel["reduced"] = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * t / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if pname == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": WL_NAME, "grid": [WL["nx"], WL["ny"], WL["nz"]], "cells": n_cells,
                   "precision": pname, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (working set ~2 GB vs 129 MB), no flush"},
        "roofline": roof,
        "step_roofline": step_roof,
        "mixed_vs_fp64": cmp,
        "ensemble": ensemble,
        "large_case": large,
        "next_rows": next_rows,
        "wallmodel": wallmodel,
        "wallmodel_network": mlp,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "launch_config": launch_cfg,
        "repeats": {"n": len(reps), "steps_each": K, "ms_per_step": [round(x, 4) for x in reps],
                    "median_ms_per_step": statistics.median(reps) if reps else None,
                    "median_value": n_cells * world / (statistics.median(reps) * 1e-3) if reps else None,
                    "note": "after 10 warm-up steps in all; the contract's value is the first timed run"},
        "gpu_launches": lps * K if lps > 0 else None,
        "gpu_launches_per_step": lps if lps > 0 else None,
        "clocks": clocks,
        "sites": sites,
        "status": diag["status"],
        "check": {"max_div": diag["max_div"], "n_plus": diag["n_plus"], "tau_bot": diag["tau_bot"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--compare-steps", type=int, default=200)
    ap.add_argument("--compare-every", type=int, default=20)
    ap.add_argument("--curve", action="store_true",
                    help="only the mixed-vs-FP64 error curves at V = 0, 2, 5 over --curve-steps steps")
    ap.add_argument("--curve-steps", type=int, default=2000)
    ap.add_argument("--sweep", action="store_true", help="only the reduced drag-vs-voltage sweep (ensemble)")
    ap.add_argument("--sweep-spinup", type=int, default=4000)
    ap.add_argument("--sweep-steps", type=int, default=4000)
    ap.add_argument("--sweep-amp", type=float, default=0.3)
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--repeats", type=int, default=5, help="extra timed repeats of the K steps (median reported)")
    ap.add_argument("--no-fusion", action="store_true",
                    help="store the CN right-hand sides instead of fusing the forward elimination into the stencil")
    ap.add_argument("--ensemble-steps", type=int, default=20)
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-wallmodel", action="store_true")
    ap.add_argument("--wallmodel", action="store_true", help="only the learned wall-model block (fine 256x193x256 "
                    "at V = 5 against coarse 128x49x128 with and without the network)")
    ap.add_argument("--wm-edl", type=float, nargs=2, default=None, metavar=("POTENTIAL_GAIN", "FLUX_GAIN"))
    ap.add_argument("--wm-residual", type=int, choices=(0, 1), default=None,
                    help="the network's first-cell potential as the coarse feature plus its own value (1) or "
                         "absolute (0)")
    ap.add_argument("--mlp", action="store_true", help="only the wall-model network's forward / training throughput")
    ap.add_argument("--large-steps", type=int, default=20)
    ap.add_argument("--no-next", action="store_true",
                    help="skip the approximate-factorisation, wall-potential-map and adaptive-dt block")
    ap.add_argument("--next-steps", type=int, default=40)
    ap.add_argument("--next", action="store_true", help="only that block")
    ap.add_argument("--grid", default=None,
                    help="NX,NY,NZ override of the workload grid (small cases for profiler captures only)")
    args = ap.parse_args()
    if args.grid:
        nx, ny, nz = (int(x) for x in args.grid.split(","))
        WL.update(nx=nx, ny=ny, nz=nz)
        global WL_NAME
        WL_NAME = WL_NAME.replace("256x193x256", f"{nx}x{ny}x{nz}") + " (grid override)"
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.curve:
        return run_curve(args)
    if args.sweep:
        return run_sweep(args)
    if args.mlp:
        import torch

        from paper_1701_02005_gb300 import binding as B

        print(json.dumps({"mlp": run_mlp(args, B, torch)}), flush=True)
        return 0
    if args.wallmodel:
        import torch

        from paper_1701_02005_gb300 import binding as B
        from paper_1701_02005_gb300.solver import Solver

        w = run_wallmodel(args, B, Solver, torch)
        w["reduced"] = run_wallmodel_reduced(args, B, Solver, torch)
        print(json.dumps({"wallmodel": w}), flush=True)
        return 0
    if args.next:
        import torch

        from paper_1701_02005_gb300 import binding as B
        from paper_1701_02005_gb300.solver import Solver

        print(json.dumps({"next_rows": run_next_rows(args, B, Solver, torch)}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
