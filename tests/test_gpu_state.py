"""Checkpoint / resume and failure detection on the GPU.

* N steps == K steps + get_state of every field + a new context + set_state +
  (N - K) steps, bitwise (FP64).
* An unstable time step drives the state non-finite; the device status word
  reports it (PNP_ERR_NONFINITE) through pnp_diagnostics / pnp_status, the
  context stays usable, and nothing faults.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o

pytestmark = pytest.mark.gpu

NAMES = ("u", "v", "w", "p", "cp", "cm", "Phi", "Hu", "Hv", "Hw", "Hcp", "Hcm")


def _new(g, prm):
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    return s


def test_checkpoint_resume_bitwise():
    g = o.Grid(32, 17, 16, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.1, V=2.0)
    a = _new(g, prm)
    a.init_state(1, 77, 0.05)
    a.step(10, 0.01)
    b = _new(g, prm)
    b.init_state(1, 77, 0.05)
    b.step(4, 0.01)
    ckpt = {n: b.get(n) for n in NAMES}
    b.close()
    c = _new(g, prm)
    for n in NAMES:
        c.set(n, ckpt[n])
    c.step(6, 0.01)
    for n in NAMES:
        assert np.array_equal(a.get(n), c.get(n)), n
    a.close()
    c.close()


def test_unstable_step_is_reported_not_faulted():
    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(16, 17, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, V=5.0)
    s = _new(g, prm)
    s.init_state(1, 3, 0.1)
    assert s.diagnostics()["status"] == B.PNP_OK
    s.step(20, 5.0)   # far beyond every explicit stability limit
    d = s.diagnostics()
    assert d["status"] in (B.PNP_ERR_NONFINITE, B.PNP_ERR_NEGATIVE_C)
    assert B.pnp_status(s.ctx) == d["status"]
    # the context is still usable: a fresh state steps cleanly
    s.init_state(1, 3, 0.1)
    s.step(2, 0.001)
    assert s.diagnostics()["status"] == B.PNP_OK
    s.close()


def test_copy_wait_timeout_is_reported_and_cleared():
    # the bounded mbarrier wait of the TMA stencil, run on a barrier no copy
    # completes: it gives up after the limit, records PNP_ERR_TIMEOUT, and the
    # context keeps working once the status is cleared
    import math

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(32, 33, 32, 2 * math.pi, math.pi, stretch=2.0, precision=B.PNP_MIXED)
    s.set_params(400.0, 0.05, 1.0, 2.0, 0.5)
    s.init_state(B.PNP_IC_PB, 3, 1e-2)
    s.step(2, 0.01)
    assert s.status() == 0
    assert B.pnp_selftest_wait_timeout(s.ctx, 0.05) == B.PNP_ERR_TIMEOUT
    assert s.status() == B.PNP_ERR_TIMEOUT          # sticky until cleared
    assert s.diagnostics()["status"] == B.PNP_ERR_TIMEOUT
    B.check(B.pnp_clear_status(s.ctx), "pnp_clear_status")
    s.step(2, 0.01)
    assert s.status() == 0 and s.diagnostics()["status"] == 0
    s.close()
