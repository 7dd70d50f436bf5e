"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol declared in include/pnp.h; argument validation needs no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_02005_gb300.build import build_library
    from paper_1701_02005_gb300 import binding as B

    build_library()
    return B.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "pnp.h")).read()
    return sorted(set(re.findall(r"\b(pnp_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    from paper_1701_02005_gb300 import binding as B

    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in B.EXPORTS, n


def test_workspace_and_grid_validation(lib):
    from paper_1701_02005_gb300 import binding as B

    n = C.c_size_t()
    assert B.pnp_workspace_bytes(256, 193, 256, B.PNP_FP64, C.byref(n)) == B.PNP_OK
    fp64 = n.value
    assert B.pnp_workspace_bytes(256, 193, 256, B.PNP_MIXED, C.byref(n)) == B.PNP_OK
    assert n.value < fp64
    # the C2 grid fits easily: ~2.3 GB in FP64
    assert 1.5e9 < fp64 < 3.5e9
    assert B.pnp_workspace_bytes(100, 33, 32, B.PNP_FP64, C.byref(n)) == B.PNP_ERR_GRID
    assert B.pnp_workspace_bytes(32, 2, 32, B.PNP_FP64, C.byref(n)) == B.PNP_ERR_GRID
    assert B.pnp_workspace_bytes(32, 33, 32, 7, C.byref(n)) == B.PNP_ERR_ARG
    assert B.pnp_error_string(B.PNP_ERR_GRID).startswith(b"invalid grid")


def test_null_context_is_rejected(lib):
    from paper_1701_02005_gb300 import binding as B

    assert B.pnp_step(None, 1, 0.01) == B.PNP_ERR_ARG
    assert B.pnp_set_params(None, 1.0, 0.1, 1.0, 0.0, 0.5) == B.PNP_ERR_ARG
    d = B.pnp_diag()
    assert B.pnp_diagnostics(None, C.byref(d)) == B.PNP_ERR_ARG


def test_tracing_and_tuning_validate_arguments(lib):
    from paper_1701_02005_gb300 import binding as B

    site, stream, n = (C.c_int * 8)(), (C.c_int * 8)(), C.c_int()
    t = (C.c_double * 8)()
    assert B.pnp_timeline(None, 0.01, 0, 8, site, stream, t, C.byref(n)) == B.PNP_ERR_ARG
    cfg, ms = (C.c_int * 4)(), (C.c_double * 4)()
    assert B.pnp_autotune(None, 0.01, cfg, ms) == B.PNP_ERR_ARG
    assert B.pnp_set_launch_config(None, cfg) == B.PNP_ERR_ARG
    out = (C.c_double * 13)()
    lps = C.c_int()
    assert B.pnp_profile(None, 1, 0.01, out, 13, C.byref(lps)) == B.PNP_ERR_ARG


def test_no_device_fails_loudly(lib):
    import torch

    from paper_1701_02005_gb300 import binding as B

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    ws = C.create_string_buffer(1024)
    rc = B.pnp_init_grid(C.byref(ctx), 8, 9, 8, 1.0, 1.0, 0.0, B.PNP_FP64, C.cast(ws, C.c_void_p), 1024, None)
    assert rc in (B.PNP_ERR_CUDA, B.PNP_ERR_WORKSPACE)
