"""Ensemble of independent NS-PNP cases advanced by one CUDA graph launch per
step (pnp_ensemble_* in include/pnp.h)."""
from __future__ import annotations

import ctypes as C

from . import binding as B


class Ensemble:
    """Borrow a list of ``solver.Solver`` cases; each keeps its own stream."""

    def __init__(self, solvers):
        import torch

        self.torch = torch
        self.solvers = list(solvers)
        self.stream = torch.cuda.Stream(device=self.solvers[0].device)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        e = C.c_void_p()
        B.check(B.pnp_ensemble_create(C.byref(e), arr, len(self.solvers), C.c_void_p(self.stream.cuda_stream)),
                "pnp_ensemble_create")
        self.ens = e

    def step(self, nsteps, dts):
        if len(dts) != len(self.solvers):
            raise ValueError("one dt per case")
        arr = (C.c_double * len(dts))(*[float(d) for d in dts])
        B.check(B.pnp_ensemble_step(self.ens, int(nsteps), arr), "pnp_ensemble_step")

    def synchronize(self):
        self.stream.synchronize()
        for s in self.solvers:
            s.synchronize()

    def close(self):
        if getattr(self, "ens", None):
            B.pnp_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
