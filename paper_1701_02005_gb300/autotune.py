"""Launch-shape autotuning with a JSON cache.

pnp_autotune (C++) times candidate launch shapes on a context's grid, site by
site and then on whole steps; the result is cached per (device, grid, precision) so later contexts reuse it via
pnp_set_launch_config.  Tuning overwrites the workspace, so it runs before the
state is initialised.
"""
from __future__ import annotations

import ctypes as C
import json
import os

from . import binding as B
from .build import BUILD

DEFAULT_CACHE = os.environ.get("PNP_AUTOTUNE_CACHE", os.path.join(BUILD, "autotune_cache.json"))


# bumped whenever the set of candidate kernels behind a launch-shape code changes
KERNEL_REV = 5


def _key(solver):
    name = solver.torch.cuda.get_device_name(solver.device)
    prec = "fp64" if solver.precision == B.PNP_FP64 else "mixed"
    return f"{name}|{solver.nx}x{solver.ny}x{solver.nz}|{prec}|rev{KERNEL_REV}"


def tune(solver, dt, cache_path=DEFAULT_CACHE, force=False):
    """Apply the cached launch shapes for this grid, or autotune and cache them.
    Call after set_params and before init_state / set_state."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    key = _key(solver)
    if key in cache and not force:
        cfg = (C.c_int * 4)(*cache[key]["config"])
        B.check(B.pnp_set_launch_config(solver.ctx, cfg), "pnp_set_launch_config")
        return list(cfg), None
    cfg = (C.c_int * 4)()
    ms = (C.c_double * 4)()
    B.check(B.pnp_autotune(solver.ctx, float(dt), cfg, ms), "pnp_autotune")
    cache[key] = {"config": list(cfg), "best_ms": list(ms)}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return list(cfg), list(ms)
