"""pnp_poisson_noalloc: the separable Poisson solve for callers that cannot
allocate device memory (a plug-in inside a framework that owns every device
allocation, or a latency-critical path where cudaMalloc may synchronise or
fail).  Its scratch is a static device array inside libpnp; the test calls it
through the C ABI twice in a row and compares each result with the
context-based pnp_poisson at the Poisson parity tolerance (1e-12 relative).
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes as C
import math

import numpy as np
import pytest

from tests import seeded

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_noalloc_poisson_matches_context_solve_twice():
    import torch

    from oracle import pnp_oracle as o
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(32, 17, 16, 2 * math.pi, math.pi, stretch=2.2)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, y_faces=g.yf)
    yf = np.ascontiguousarray(g.yf, dtype=np.float64)
    stream = torch.cuda.Stream()
    for call, (bc, seed) in enumerate([(B.PNP_NEUMANN, 41), (B.PNP_DIRICHLET, 42)]):
        rhs = seeded.field(seed, (g.nyc, g.nz, g.nx))
        ref = s.poisson(rhs, bc)
        r = torch.as_tensor(rhs).to("cuda")
        x = torch.full_like(r, float("nan"))
        torch.cuda.synchronize()
        rc = B.pnp_poisson_noalloc(g.nx, g.ny, g.nz, g.Lx, g.Lz, yf.ctypes.data_as(C.POINTER(C.c_double)), bc,
                                   C.c_void_p(r.data_ptr()), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(stream.cuda_stream))
        assert rc == B.PNP_OK, (call, rc)
        stream.synchronize()
        got = x.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert _rel(got, ref) <= 1e-12, (call, _rel(got, ref))
    s.close()


def test_noalloc_poisson_rejects_grids_beyond_its_scratch():
    from paper_1701_02005_gb300 import binding as B

    ny = 193
    yf = np.linspace(-1, 1, ny)
    rc = B.pnp_poisson_noalloc(256, ny, 256, 1.0, 1.0, yf.ctypes.data_as(C.POINTER(C.c_double)), B.PNP_NEUMANN,
                               C.c_void_p(16), C.c_void_p(16), None)
    assert rc == B.PNP_ERR_TOO_LARGE
    assert b"static scratch" in B.pnp_error_string(rc)
