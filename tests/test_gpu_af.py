"""Approximate factorisation (x/z viscous and diffusive terms implicit,
periodic x/z sweeps before the wall-normal solve) against the oracle's
factored step, FP64 at the parity tolerance and mixed at the mixed path's;
and at a dt beyond the explicit x/z diffusion limit, where only the factored
scheme is stable.  The sweeps run as one pass of truncated circulant
convolutions where a few taps reach the arithmetic's rounding (here: the FP64
32x33x32 case and the mixed cases at Re 300 and 3000) and as cyclic Thomas
sweeps otherwise (the 16x13x8 case, whose 8 z-cells are too few for the taps,
and the Re 1 cases, whose kernels decay slowly)."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded

pytestmark = pytest.mark.gpu


def _solver(g, prm, precision):
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta, prm.Uw)
    B.check(B.pnp_set_scheme(s.ctx, B.PNP_SCHEME_AF), "pnp_set_scheme")
    return s


def _rel(a, b, floor=1e-300):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor))


@pytest.mark.parametrize("shape,nsteps", [((16, 13, 8), 4), ((32, 33, 32), 20)])
def test_af_fp64_matches_the_oracle(shape, nsteps):
    nx, ny, nz = shape
    g = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5, af=True)
    st = o.initial_state(g, prm, o.IC_PB, seed=41, amp=0.05)
    shp = (g.nyc, g.nz, g.nx)
    st.cp = st.cp * seeded.positive_field(42, shp, 0.97, 1.03)
    st.cm = st.cm * seeded.positive_field(43, shp, 0.97, 1.03)
    st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
    s = _solver(g, prm, 0)
    s.set_state(st)
    s.step(nsteps, 0.01)
    ref = o.step(g, prm, st, 0.01, nsteps)
    errs = {n: _rel(s.get(n), getattr(ref, n)) for n in ("u", "v", "w", "p", "cp", "cm", "Phi")}
    assert all(e <= 1e-10 for e in errs.values()), errs
    assert s.diagnostics()["status"] == 0
    s.close()


@pytest.mark.parametrize("fusion", [1, 0])
def test_af_mixed_matches_the_oracle(fusion):
    """Fused: the x/z sweeps act on the stencil's forward values, between the
    stencil and the back substitution (the y-elimination and the sweeps are
    linear maps along different axes and commute); unfused: on the stored
    right-hand sides, before the y-solves."""
    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(64, 41, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5, af=True)
    st = o.initial_state(g, prm, o.IC_PB, seed=44, amp=0.1)
    s = _solver(g, prm, 1)
    B.check(B.pnp_set_fusion(s.ctx, fusion), "pnp_set_fusion")
    s.set_state(st)
    s.step(5, 0.005)
    ref = o.step(g, prm, st, 0.005, 5)
    for n in ("u", "v", "w", "cp", "cm", "Phi"):
        r = getattr(ref, n)
        e = _rel(s.get(n), r, 1.0 if n in ("u", "v", "w") else 1e-300)
        assert e <= 1e-5, (n, e)
    assert s.diagnostics()["status"] == 0
    s.close()


def test_af_mixed_larger_grid_matches_the_oracle():
    """The convolution pass with 128-thread rows, 48 planes per family and both
    velocity and ion families, at Re 3000."""
    g = o.Grid(128, 49, 64, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=3000.0, lam=0.02, Sc=1.0, V=2.0, beta=0.5, af=True)
    st = o.initial_state(g, prm, o.IC_PB, seed=46, amp=0.1)
    s = _solver(g, prm, 1)
    s.set_state(st)
    s.step(3, 0.004)
    ref = o.step(g, prm, st, 0.004, 3)
    for n in ("u", "v", "w", "cp", "cm", "Phi"):
        r = getattr(ref, n)
        e = _rel(s.get(n), r, 1.0 if n in ("u", "v", "w") else 1e-300)
        assert e <= 1e-5, (n, e)
    assert s.diagnostics()["status"] == 0
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_af_is_stable_beyond_the_explicit_diffusion_limit(precision):
    # Re = 1, 32 cells over 2 pi: nu dt / dx^2 = 2.6 at dt = 0.1, far past the
    # explicit x/z diffusion bound of the RK3 (about 0.6); the factored scheme
    # damps every mode, as the oracle's factored step does
    g = o.Grid(32, 17, 16, 2 * math.pi, math.pi, stretch=1.5)
    prm = o.Params(Re=1.0, lam=0.2, Sc=1.0, V=1.0, beta=0.5, af=True)
    st = o.initial_state(g, prm, o.IC_PB, seed=45, amp=0.2)
    s = _solver(g, prm, precision)
    s.set_state(st)
    s.step(10, 0.1)
    ref = o.step(g, prm, st, 0.1, 10)
    tol = 1e-10 if precision == 0 else 1e-5
    for n in ("u", "v", "w", "cp", "cm"):
        r = getattr(ref, n)
        e = _rel(s.get(n), r, 1.0)
        assert e <= tol, (n, e)
    assert np.max(np.abs(ref.v)) < 0.2   # the noise decays
    assert s.diagnostics()["status"] == 0
    s.close()
