"""pnp_poisson_noalloc: the separable Poisson solve for callers that cannot
allocate device memory (a plug-in inside a framework that owns every device
allocation, or a latency-critical path where cudaMalloc may synchronise or
fail).  Its scratch is a static device array inside libpnp; the tests call it
through the C ABI and compare each result with the context-based pnp_poisson
at the Poisson parity tolerance (1e-12 relative): two calls in a row with a
synchronisation between them, and two calls on different grids queued on one
stream with none (the second call's grid constants must not reach the first
call's kernels).  This file is collected last so that a failure here stops a
-x run only after every other test has run.
"""
import ctypes as C
import math

import numpy as np
import pytest

from tests import seeded

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _call(B, g, bc, r, x, stream):
    yf = np.ascontiguousarray(g.yf, dtype=np.float64)
    return B.pnp_poisson_noalloc(g.nx, g.ny, g.nz, g.Lx, g.Lz, yf.ctypes.data_as(C.POINTER(C.c_double)), bc,
                                 C.c_void_p(r.data_ptr()), C.c_void_p(x.data_ptr()), C.c_void_p(stream.cuda_stream))


def _reference(g, rhs, bc):
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, y_faces=g.yf)
    ref = s.poisson(rhs, bc)
    s.close()
    return ref


def test_noalloc_poisson_matches_context_solve_twice():
    import torch

    from oracle import pnp_oracle as o
    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(32, 17, 16, 2 * math.pi, math.pi, stretch=2.2)
    stream = torch.cuda.Stream()
    for call, (bc, seed) in enumerate([(B.PNP_NEUMANN, 41), (B.PNP_DIRICHLET, 42)]):
        rhs = seeded.field(seed, (g.nyc, g.nz, g.nx))
        ref = _reference(g, rhs, bc)
        r = torch.as_tensor(rhs).to("cuda")
        x = torch.full_like(r, float("nan"))
        torch.cuda.synchronize()
        rc = _call(B, g, bc, r, x, stream)
        assert rc == B.PNP_OK, (call, rc)
        stream.synchronize()
        got = x.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert _rel(got, ref) <= TOL, (call, _rel(got, ref))


def test_noalloc_calls_queued_back_to_back_on_one_stream():
    import torch

    from oracle import pnp_oracle as o
    from paper_1701_02005_gb300 import binding as B

    ga = o.Grid(32, 17, 16, 2 * math.pi, math.pi, stretch=2.2)
    gb = o.Grid(16, 25, 32, 3.0, 1.5, stretch=1.4)
    cases = [(ga, B.PNP_NEUMANN, 51), (gb, B.PNP_DIRICHLET, 52)]
    rhs = [seeded.field(seed, (g.nyc, g.nz, g.nx)) for g, _, seed in cases]
    refs = [_reference(g, r, bc) for (g, bc, _), r in zip(cases, rhs)]
    stream = torch.cuda.Stream()
    ins = [torch.as_tensor(r).to("cuda") for r in rhs]
    outs = [torch.full_like(r, float("nan")) for r in ins]
    torch.cuda.synchronize()
    for (g, bc, _), r, x in zip(cases, ins, outs):
        rc = _call(B, g, bc, r, x, stream)   # no host synchronisation between the two calls
        assert rc == B.PNP_OK, rc
    stream.synchronize()
    for i, (x, ref) in enumerate(zip(outs, refs)):
        got = x.cpu().numpy()
        assert np.all(np.isfinite(got)), i
        assert _rel(got, ref) <= TOL, (i, _rel(got, ref))


def test_noalloc_poisson_rejects_grids_beyond_its_scratch():
    from paper_1701_02005_gb300 import binding as B

    ny = 193
    yf = np.linspace(-1, 1, ny)
    rc = B.pnp_poisson_noalloc(256, ny, 256, 1.0, 1.0, yf.ctypes.data_as(C.POINTER(C.c_double)), B.PNP_NEUMANN,
                               C.c_void_p(16), C.c_void_p(16), None)
    assert rc == B.PNP_ERR_TOO_LARGE
    assert b"static scratch" in B.pnp_error_string(rc)
    yf2 = np.linspace(-1, 1, 2050)
    rc = B.pnp_poisson_noalloc(4, 2050, 4, 1.0, 1.0, yf2.ctypes.data_as(C.POINTER(C.c_double)), B.PNP_NEUMANN,
                               C.c_void_p(16), C.c_void_p(16), None)
    assert rc == B.PNP_ERR_TOO_LARGE
