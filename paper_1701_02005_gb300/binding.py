"""ctypes binding of libpnp (include/pnp.h): same names, argument marshalling only.

Every function here forwards to the C ABI; no step of the method runs in
Python.  Importing this module raises if the library has not been built, so
a missing extension fails loudly instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

PNP_OK = 0
PNP_DIAG_RAW_BYTES = 256
PNP_ERR_ARG = -1
PNP_ERR_GRID = -2
PNP_ERR_WORKSPACE = -3
PNP_ERR_CUDA = -4
PNP_ERR_STATE = -5
PNP_ERR_NONFINITE = -6
PNP_ERR_NEGATIVE_C = -7
PNP_ERR_UNSUPPORTED = -8
PNP_ERR_TOO_LARGE = -9
PNP_ERR_TIMEOUT = -10
PNP_ERR_CFL = -11
PNP_ERR_DPHI = -12
PNP_POLICY_DEFAULT = 0
PNP_POLICY_FP64_SOLVES = 1
PNP_SCHEME_CN = 0
PNP_SCHEME_AF = 1

PNP_FP64 = 0
PNP_MIXED = 1

PNP_U, PNP_V, PNP_W, PNP_P, PNP_CP, PNP_CM, PNP_PHI = range(7)
PNP_HU, PNP_HV, PNP_HW, PNP_HCP, PNP_HCM = range(7, 12)
PNP_NFIELDS = 12

PNP_IC_LAMINAR = 0
PNP_IC_PB = 1

PNP_NEUMANN = 0
PNP_DIRICHLET = 1

PROFILE_SITES = ("rhs", "cn_thomas", "p_fftx", "p_fftz", "p_thomas", "p_ifftz", "p_ifftx", "project",
                 "e_fftx", "e_fftz", "e_thomas", "e_ifftz", "e_ifftx")


class pnp_diag(C.Structure):
    _fields_ = [
        ("tau_bot", C.c_double), ("tau_top", C.c_double), ("cf", C.c_double), ("re_tau", C.c_double),
        ("n_plus", C.c_double), ("n_minus", C.c_double), ("net_charge", C.c_double),
        ("wall_flux", C.c_double), ("max_div", C.c_double), ("ke", C.c_double), ("time", C.c_double),
        ("nstep", C.c_longlong), ("status", C.c_int), ("precision", C.c_int),
        ("cfl", C.c_double), ("max_dphi", C.c_double), ("flux_plus", C.c_double), ("flux_minus", C.c_double),
        ("dt_cfl", C.c_double), ("dt_migration", C.c_double), ("dt_dielectric", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = {
    # name: (restype, argtypes)
    "pnp_workspace_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "pnp_init_grid": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "pnp_set_yfaces": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int]),
    "pnp_set_params": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
    "pnp_set_wall_velocity": (C.c_int, [C.c_void_p, C.c_double]),
    "pnp_init_state": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_double]),
    "pnp_set_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "pnp_get_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "pnp_field_size": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]),
    "pnp_step": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "pnp_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(pnp_diag)]),
    "pnp_diagnostics_post": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pnp_diagnostics_read": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(pnp_diag)]),
    "pnp_mean_profile": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "pnp_poisson": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "pnp_poisson_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double),
                                      C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pnp_eval_explicit": (C.c_int, [C.c_void_p]),
    "pnp_set_limits": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "pnp_set_policy": (C.c_int, [C.c_void_p, C.c_int]),
    "pnp_set_fusion": (C.c_int, [C.c_void_p, C.c_int]),
    "pnp_set_scheme": (C.c_int, [C.c_void_p, C.c_int]),
    "pnp_stats_reset": (C.c_int, [C.c_void_p]),
    "pnp_stats_sample": (C.c_int, [C.c_void_p]),
    "pnp_stats_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_longlong)]),
    "pnp_set_wall_potential": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pnp_step_adaptive": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int,
                                    C.POINTER(C.c_double)]),
    "pnp_status": (C.c_int, [C.c_void_p]),
    "pnp_clear_status": (C.c_int, [C.c_void_p]),
    "pnp_selftest_wait_timeout": (C.c_int, [C.c_void_p, C.c_double]),
    "pnp_fp64_peak": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "pnp_profile": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double), C.c_int,
                              C.POINTER(C.c_int)]),
    "pnp_timeline": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "pnp_autotune": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "pnp_set_launch_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "pnp_get_launch_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "pnp_ensemble_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "pnp_ensemble_step": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "pnp_ensemble_destroy": (None, [C.c_void_p]),
    "pnp_mlp_param_count": (C.c_int, [C.POINTER(C.c_size_t)]),
    "pnp_mlp_workspace_bytes": (C.c_int, [C.c_int, C.POINTER(C.c_size_t)]),
    "pnp_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, C.c_uint64]),
    "pnp_mlp_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_size_t]),
    "pnp_mlp_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_size_t]),
    "pnp_mlp_set_normalization": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                            C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "pnp_mlp_set_skip": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "pnp_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pnp_mlp_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_float),
                                   C.POINTER(C.c_float)]),
    "pnp_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.POINTER(C.c_float)]),
    "pnp_mlp_status": (C.c_int, [C.c_void_p]),
    "pnp_mlp_destroy": (None, [C.c_void_p]),
    "pnp_wall_features": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "pnp_restrict_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pnp_wall_labels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pnp_set_wall_slip": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pnp_step_wallmodel": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double]),
    "pnp_set_wall_stress": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pnp_set_wallmodel_coupling": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "pnp_set_wallmodel_edl": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "pnp_set_wall_edl": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "pnp_correct_wall_flux": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    "pnp_error_string": (C.c_char_p, [C.c_int]),
    "pnp_destroy": (None, [C.c_void_p]),
}

_lib = None


def load(path: str | None = None):
    """Load libpnp.so (built by ``paper_1701_02005_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise ImportError(f"libpnp not built ({path} missing): run paper_1701_02005_gb300.build.build_library()")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PNPError(RuntimeError):
    def __init__(self, code, where):
        msg = load().pnp_error_string(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code, where):
    if code != PNP_OK:
        raise PNPError(code, where)
    return code


def _fwd(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


pnp_workspace_bytes = _fwd("pnp_workspace_bytes")
pnp_init_grid = _fwd("pnp_init_grid")
pnp_set_yfaces = _fwd("pnp_set_yfaces")
pnp_set_params = _fwd("pnp_set_params")
pnp_set_wall_velocity = _fwd("pnp_set_wall_velocity")
pnp_init_state = _fwd("pnp_init_state")
pnp_set_state = _fwd("pnp_set_state")
pnp_get_state = _fwd("pnp_get_state")
pnp_field_size = _fwd("pnp_field_size")
pnp_step = _fwd("pnp_step")
pnp_diagnostics = _fwd("pnp_diagnostics")
pnp_diagnostics_post = _fwd("pnp_diagnostics_post")
pnp_diagnostics_read = _fwd("pnp_diagnostics_read")
pnp_mean_profile = _fwd("pnp_mean_profile")
pnp_poisson = _fwd("pnp_poisson")
pnp_poisson_noalloc = _fwd("pnp_poisson_noalloc")
pnp_eval_explicit = _fwd("pnp_eval_explicit")
pnp_set_limits = _fwd("pnp_set_limits")
pnp_set_policy = _fwd("pnp_set_policy")
pnp_set_fusion = _fwd("pnp_set_fusion")
pnp_set_scheme = _fwd("pnp_set_scheme")
pnp_stats_reset = _fwd("pnp_stats_reset")
pnp_stats_sample = _fwd("pnp_stats_sample")
pnp_stats_get = _fwd("pnp_stats_get")
pnp_set_wall_potential = _fwd("pnp_set_wall_potential")
pnp_step_adaptive = _fwd("pnp_step_adaptive")
pnp_status = _fwd("pnp_status")
pnp_clear_status = _fwd("pnp_clear_status")
pnp_selftest_wait_timeout = _fwd("pnp_selftest_wait_timeout")
pnp_fp64_peak = _fwd("pnp_fp64_peak")
pnp_profile = _fwd("pnp_profile")
pnp_timeline = _fwd("pnp_timeline")
pnp_autotune = _fwd("pnp_autotune")
pnp_set_launch_config = _fwd("pnp_set_launch_config")
pnp_get_launch_config = _fwd("pnp_get_launch_config")
pnp_ensemble_create = _fwd("pnp_ensemble_create")
pnp_ensemble_step = _fwd("pnp_ensemble_step")
pnp_ensemble_destroy = _fwd("pnp_ensemble_destroy")
pnp_mlp_param_count = _fwd("pnp_mlp_param_count")
pnp_mlp_workspace_bytes = _fwd("pnp_mlp_workspace_bytes")
pnp_mlp_create = _fwd("pnp_mlp_create")
pnp_mlp_get_params = _fwd("pnp_mlp_get_params")
pnp_mlp_set_params = _fwd("pnp_mlp_set_params")
pnp_mlp_set_normalization = _fwd("pnp_mlp_set_normalization")
pnp_mlp_set_skip = _fwd("pnp_mlp_set_skip")
pnp_mlp_forward = _fwd("pnp_mlp_forward")
pnp_mlp_gradient = _fwd("pnp_mlp_gradient")
pnp_mlp_train_step = _fwd("pnp_mlp_train_step")
pnp_mlp_status = _fwd("pnp_mlp_status")
pnp_mlp_destroy = _fwd("pnp_mlp_destroy")
pnp_wall_features = _fwd("pnp_wall_features")
pnp_restrict_state = _fwd("pnp_restrict_state")
pnp_wall_labels = _fwd("pnp_wall_labels")
pnp_set_wall_slip = _fwd("pnp_set_wall_slip")
pnp_step_wallmodel = _fwd("pnp_step_wallmodel")
pnp_set_wall_stress = _fwd("pnp_set_wall_stress")
pnp_set_wallmodel_coupling = _fwd("pnp_set_wallmodel_coupling")
pnp_set_wallmodel_edl = _fwd("pnp_set_wallmodel_edl")
pnp_set_wall_edl = _fwd("pnp_set_wall_edl")
pnp_correct_wall_flux = _fwd("pnp_correct_wall_flux")
pnp_error_string = _fwd("pnp_error_string")
pnp_destroy = _fwd("pnp_destroy")
