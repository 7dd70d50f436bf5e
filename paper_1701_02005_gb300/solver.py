"""A context of libpnp with torch-owned device memory and stream.

PyTorch supplies the device workspace (one uint8 tensor) and a CUDA stream;
every computation runs in libpnp's kernels through the C ABI.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B

FIELD_NAMES = {"u": B.PNP_U, "v": B.PNP_V, "w": B.PNP_W, "p": B.PNP_P, "cp": B.PNP_CP, "cm": B.PNP_CM,
               "Phi": B.PNP_PHI, "Hu": B.PNP_HU, "Hv": B.PNP_HV, "Hw": B.PNP_HW, "Hcp": B.PNP_HCP,
               "Hcm": B.PNP_HCM}


class Solver:
    """One NS-PNP case on one GPU.

    nx, nz: periodic sizes (powers of two); ny: y face nodes (ny - 1 cells).
    precision: binding.PNP_FP64 or binding.PNP_MIXED.
    """

    def __init__(self, nx, ny, nz, Lx, Lz, stretch=0.0, precision=B.PNP_FP64, device=0, stream=None,
                 y_faces=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libpnp needs a CUDA device")
        B.load()
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nyc = ny - 1
        self.precision = precision
        nbytes = C.c_size_t()
        B.check(B.pnp_workspace_bytes(nx, ny, nz, precision, C.byref(nbytes)), "pnp_workspace_bytes")
        self.ws = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        # the workspace is used on the library's stream from here on: order that stream
        # after the torch work still queued on the memory the allocator handed out (a
        # block freed a moment ago may still be read there), and keep torch from
        # handing the block out again before the library's stream is done with it
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.ws.record_stream(self.stream)
        ctx = C.c_void_p()
        B.check(B.pnp_init_grid(C.byref(ctx), nx, ny, nz, float(Lx), float(Lz), float(stretch), precision,
                                C.c_void_p(base + off), C.c_size_t(int(nbytes.value)),
                                C.c_void_p(self.stream.cuda_stream)), "pnp_init_grid")
        self.ctx = ctx
        if y_faces is not None:
            self.set_yfaces(y_faces)

    # -- set-up --
    def set_yfaces(self, yf):
        a = np.ascontiguousarray(yf, dtype=np.float64)
        B.check(B.pnp_set_yfaces(self.ctx, a.ctypes.data_as(C.POINTER(C.c_double)), a.size), "pnp_set_yfaces")

    def set_params(self, Re, debye, Sc=1.0, V=0.0, beta=0.5, Uw=1.0):
        B.check(B.pnp_set_params(self.ctx, Re, debye, Sc, V, beta), "pnp_set_params")
        B.check(B.pnp_set_wall_velocity(self.ctx, Uw), "pnp_set_wall_velocity")

    def init_state(self, ic=B.PNP_IC_PB, seed=1701, amp=0.0):
        B.check(B.pnp_init_state(self.ctx, ic, C.c_uint64(seed), amp), "pnp_init_state")

    # -- fields --
    def shape(self, name):
        f = FIELD_NAMES[name]
        ny = self.ny if f in (B.PNP_V, B.PNP_HV) else self.nyc
        return (ny, self.nz, self.nx)

    def set(self, name, array):
        a = np.ascontiguousarray(array, dtype=np.float64)
        if a.shape != self.shape(name):
            raise ValueError(f"{name}: shape {a.shape} != {self.shape(name)}")
        B.check(B.pnp_set_state(self.ctx, FIELD_NAMES[name], a.ctypes.data_as(C.c_void_p), 0), "pnp_set_state")
        self.stream.synchronize()

    def set_device(self, name, tensor):
        t = tensor.contiguous().to(dtype=self.torch.float64)
        self.torch.cuda.synchronize(self.device)
        B.check(B.pnp_set_state(self.ctx, FIELD_NAMES[name], C.c_void_p(t.data_ptr()), 1), "pnp_set_state")
        self.stream.synchronize()

    def get(self, name):
        a = np.empty(self.shape(name), dtype=np.float64)
        B.check(B.pnp_get_state(self.ctx, FIELD_NAMES[name], a.ctypes.data_as(C.c_void_p), 0), "pnp_get_state")
        return a

    def set_state(self, st):
        """Load an oracle-style state object (attributes u, v, w, p, cp, cm, Phi, H*)."""
        for name in FIELD_NAMES:
            self.set(name, getattr(st, name))

    # -- stepping --
    def step(self, nsteps, dt):
        B.check(B.pnp_step(self.ctx, int(nsteps), float(dt)), "pnp_step")

    def step_adaptive(self, nsteps, dt_max, cfl=0.5, check_every=10):
        """nsteps steps with dt from the state's explicit limits (pnp_step_adaptive);
        returns the dt of every step."""
        dts = np.zeros(int(nsteps), dtype=np.float64)
        B.check(B.pnp_step_adaptive(self.ctx, int(nsteps), float(dt_max), float(cfl), int(check_every),
                                    dts.ctypes.data_as(C.POINTER(C.c_double))), "pnp_step_adaptive")
        return dts

    def synchronize(self):
        self.stream.synchronize()

    _STATUS_CODES = (B.PNP_OK, B.PNP_ERR_NONFINITE, B.PNP_ERR_NEGATIVE_C, B.PNP_ERR_TIMEOUT, B.PNP_ERR_CFL,
                     B.PNP_ERR_DPHI)

    def diagnostics(self):
        d = B.pnp_diag()
        code = B.pnp_diagnostics(self.ctx, C.byref(d))
        if code not in self._STATUS_CODES:
            B.check(code, "pnp_diagnostics")
        return d.as_dict()

    def diag_buffer(self):
        """A pinned host record for diagnostics_post / diagnostics_read."""
        return self.torch.empty(B.PNP_DIAG_RAW_BYTES, dtype=self.torch.uint8).pin_memory()

    def diagnostics_post(self, raw):
        """Queue the diagnostics of the current state into raw (diag_buffer()); returns at once."""
        B.check(B.pnp_diagnostics_post(self.ctx, C.c_void_p(raw.data_ptr())), "pnp_diagnostics_post")

    def diagnostics_read(self, raw):
        """The diagnostics of a completed post (after an event or a synchronisation)."""
        d = B.pnp_diag()
        code = B.pnp_diagnostics_read(self.ctx, C.c_void_p(raw.data_ptr()), C.byref(d))
        if code not in self._STATUS_CODES:
            B.check(code, "pnp_diagnostics_read")
        return d.as_dict()

    def set_wall_potential(self, bottom=None, top=None):
        """Wall potentials along the walls ([nz][nx] arrays, units of V_T); None restores the uniform walls."""
        if bottom is None and top is None:
            B.check(B.pnp_set_wall_potential(self.ctx, None, None), "pnp_set_wall_potential")
            return
        b = np.ascontiguousarray(bottom, dtype=np.float64).reshape(self.nz, self.nx)
        t = np.ascontiguousarray(top, dtype=np.float64).reshape(self.nz, self.nx)
        B.check(B.pnp_set_wall_potential(self.ctx, b.ctypes.data_as(C.POINTER(C.c_double)),
                                         t.ctypes.data_as(C.POINTER(C.c_double))), "pnp_set_wall_potential")

    # -- time statistics --
    STAT_FIELDS = ("u", "v", "w", "cp", "cm", "Phi")

    def stats_reset(self):
        B.check(B.pnp_stats_reset(self.ctx), "pnp_stats_reset")

    def stats_sample(self):
        B.check(B.pnp_stats_sample(self.ctx), "pnp_stats_sample")

    def stats(self):
        """Time-and-plane means and RMS fluctuations per field (arrays over y),
        the time-averaged c_f and the number of samples."""
        mean = np.zeros((6, self.ny))
        rms = np.zeros((6, self.ny))
        cf = C.c_double()
        n = C.c_longlong()
        B.check(B.pnp_stats_get(self.ctx, mean.ctypes.data_as(C.POINTER(C.c_double)),
                                rms.ctypes.data_as(C.POINTER(C.c_double)), C.byref(cf), C.byref(n)), "pnp_stats_get")
        out = {}
        for q, name in enumerate(self.STAT_FIELDS):
            k = self.ny if name == "v" else self.nyc
            out[name] = (mean[q, :k].copy(), rms[q, :k].copy())
        return out, cf.value, n.value

    def set_policy(self, policy):
        """Solve precision of a mixed context: binding.PNP_POLICY_DEFAULT or PNP_POLICY_FP64_SOLVES."""
        B.check(B.pnp_set_policy(self.ctx, int(policy)), "pnp_set_policy")

    def set_limits(self, cfl_max=3 ** 0.5, dphi_max=2.0):
        """Limits of the device checks reported as PNP_ERR_CFL / PNP_ERR_DPHI."""
        B.check(B.pnp_set_limits(self.ctx, float(cfl_max), float(dphi_max)), "pnp_set_limits")

    def mean_profile(self, name):
        n = self.shape(name)[0]
        out = np.empty(n, dtype=np.float64)
        B.check(B.pnp_mean_profile(self.ctx, FIELD_NAMES[name], out.ctypes.data_as(C.POINTER(C.c_double))),
                "pnp_mean_profile")
        return out

    def poisson(self, rhs, bc):
        """Separable Poisson solve of a host array (FP64) through the C ABI."""
        t = self.torch.as_tensor(np.ascontiguousarray(rhs, dtype=np.float64)).to(self.device)
        out = self.torch.empty_like(t)
        self.torch.cuda.synchronize(self.device)
        B.check(B.pnp_poisson(self.ctx, bc, C.c_void_p(t.data_ptr()), C.c_void_p(out.data_ptr())), "pnp_poisson")
        self.stream.synchronize()
        return out.cpu().numpy()

    def status(self):
        """Device error word: PNP_OK, a field check (NaN, negative c) or a copy timeout."""
        return int(B.pnp_status(self.ctx))

    def eval_explicit(self):
        B.check(B.pnp_eval_explicit(self.ctx), "pnp_eval_explicit")
        self.stream.synchronize()

    def fp64_peak(self):
        v = C.c_double()
        B.check(B.pnp_fp64_peak(self.ctx, C.byref(v)), "pnp_fp64_peak")
        return v.value

    def close(self):
        if getattr(self, "ctx", None):
            B.pnp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def timeline(solver, dt, in_graph=False, cap=64):
    """One traced step via pnp_timeline (eager, or as one CUDA graph): a list of
    (site, stream, ms) in launch order; site is a PROFILE_SITES name or "start",
    stream "main" or "aux"."""
    site = (C.c_int * cap)()
    stream = (C.c_int * cap)()
    t = (C.c_double * cap)()
    n = C.c_int()
    B.check(B.pnp_timeline(solver.ctx, float(dt), int(bool(in_graph)), cap, site, stream, t, C.byref(n)),
            "pnp_timeline")
    return [(B.PROFILE_SITES[site[i]] if site[i] >= 0 else "start", "aux" if stream[i] else "main", t[i])
            for i in range(n.value)]


def profile(solver, nsteps, dt):
    """Per-launch-site milliseconds (summed) and launches per step via pnp_profile."""
    n = len(B.PROFILE_SITES)
    ms = (C.c_double * n)()
    lps = C.c_int()
    B.check(B.pnp_profile(solver.ctx, int(nsteps), float(dt), ms, n, C.byref(lps)), "pnp_profile")
    return dict(zip(B.PROFILE_SITES, list(ms))), lps.value
