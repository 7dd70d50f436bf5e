"""GPU parity: libpnp (through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs.

Tolerance for the FP64 path: relative 1e-10 in the max norm of each field
(difference / max|oracle field|).  The two sides differ only in rounding
order (own FFT vs numpy's, reciprocal-multiply vs divide), so agreement is
expected near 1e-13; 1e-10 leaves room for growth over 200 steps.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _solver(g, prm=None, precision=0):
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    if prm is not None:
        s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta, prm.Uw)
    return s


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


FIELDS = ("u", "v", "w", "p", "cp", "cm", "Phi")


def _assert_state(s, ref, tol=TOL, names=FIELDS):
    errs = {n: _rel(s.get(n), getattr(ref, n)) for n in names}
    bad = {n: e for n, e in errs.items() if not e <= tol}
    assert not bad, errs
    return errs


# every register-transform length in x (Nx/2 = 16 .. 512) and z (16 .. 512) in FP64,
# and the shared-memory transforms of the smallest grids
@pytest.mark.parametrize("shape", [(8, 9, 4), (32, 17, 16), (64, 33, 32), (128, 5, 64), (256, 5, 128),
                                   (512, 5, 256), (1024, 5, 512)])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_poisson_parity(shape, bc):
    from paper_1701_02005_gb300 import binding as B

    nx, ny, nz = shape
    g = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=2.2)
    s = _solver(g)
    rhs = seeded.field(7 + nx, (g.nyc, g.nz, g.nx))
    got = s.poisson(rhs, B.PNP_NEUMANN if bc == "neumann" else B.PNP_DIRICHLET)
    ref = o.poisson_solve(g, rhs, o.NEUMANN if bc == "neumann" else o.DIRICHLET)
    assert _rel(got, ref) <= 1e-12
    s.close()


def _random_state(g, prm, seed):
    st = o.initial_state(g, prm, o.IC_PB, seed=seed, amp=0.1)
    shp = (g.nyc, g.nz, g.nx)
    st.p = seeded.field(seed + 1, shp, 0.01)
    st.cp = st.cp * seeded.positive_field(seed + 2, shp, 0.9, 1.1)
    st.cm = st.cm * seeded.positive_field(seed + 3, shp, 0.9, 1.1)
    st.Phi = st.Phi + seeded.field(seed + 4, shp, 0.05)
    st.Hu = seeded.field(seed + 5, shp, 0.1)
    st.Hv = seeded.wall_zero_faces(seed + 6, (g.ny, g.nz, g.nx), 0.1)
    st.Hw = seeded.field(seed + 7, shp, 0.1)
    st.Hcp = seeded.field(seed + 8, shp, 0.1)
    st.Hcm = seeded.field(seed + 9, shp, 0.1)
    return st


@pytest.mark.parametrize("shape", [(8, 9, 4), (32, 21, 16)])
def test_explicit_terms_parity(shape):
    nx, ny, nz = shape
    g = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.1, Sc=1.5, V=2.0, beta=0.5)
    st = _random_state(g, prm, 100 + nx)
    s = _solver(g, prm)
    s.set_state(st)
    s.eval_explicit()
    H = o.explicit_terms(g, prm, st)
    for name, ref in zip(("Hu", "Hv", "Hw", "Hcp", "Hcm"), H):
        assert _rel(s.get(name), ref) <= 1e-12, name
    s.close()


def test_initial_state_parity():
    g = o.Grid(32, 17, 16, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    ref = o.initial_state(g, prm, o.IC_PB, seed=1701, amp=1e-3)
    s = _solver(g, prm)
    s.init_state(1, 1701, 1e-3)
    _assert_state(s, ref, 1e-12)
    s.close()


@pytest.mark.parametrize("nsteps", [1, 4])
def test_step_parity_small(nsteps):
    g = o.Grid(16, 13, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5)
    st = _random_state(g, prm, 11)
    s = _solver(g, prm)
    s.set_state(st)
    s.step(nsteps, 0.01)
    ref = o.step(g, prm, st, 0.01, nsteps)
    _assert_state(s, ref, 1e-11, FIELDS)
    for name in ("Hu", "Hv", "Hw", "Hcp", "Hcm"):
        assert _rel(s.get(name), getattr(ref, name)) <= 1e-11, name
    s.close()


def test_c1_200_steps_fp64():
    # 32x33x32, box 2pi x 2 x pi, tanh y (gamma 2), Re 400, lambda 0.05, Sc 1, V 2, PB + 1e-3 noise
    g = o.Grid(32, 33, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st0 = o.initial_state(g, prm, o.IC_PB, seed=1701, amp=1e-3)
    s = _solver(g, prm)
    s.set_state(st0)
    s.step(200, 0.01)
    ref = o.step(g, prm, st0, 0.01, 200)
    errs = _assert_state(s, ref, TOL)
    d = s.diagnostics()
    d0 = o.diagnostics(g, prm, st0)
    assert d["status"] == 0
    assert abs(d["n_plus"] - d0["n_plus"]) <= 1e-12 * d0["n_plus"]
    assert abs(d["net_charge"] - d0["net_charge"]) <= 1e-11
    assert d["max_div"] <= 1e-11
    dr = o.diagnostics(g, prm, ref)
    assert abs(d["tau_bot"] - dr["tau_bot"]) <= 1e-10 * abs(dr["tau_bot"])
    print("C1 200-step rel errors:", errs)
    s.close()


def test_laminar_couette_gpu():
    g = o.Grid(32, 33, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=0.0, beta=0.5)
    s = _solver(g, prm)
    s.init_state(0, 1, 0.0)
    s.step(50, 0.01)
    u = s.get("u")
    assert np.max(np.abs(u - g.yc[:, None, None])) <= 1e-13
    d = s.diagnostics()
    assert abs(d["tau_bot"] - 1 / 400) <= 1e-14 and abs(d["cf"] - 2 / 400) <= 1e-14
    s.close()


def test_mean_profile_and_diagnostics_match_oracle():
    g = o.Grid(16, 17, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=2.0)
    st = o.initial_state(g, prm, o.IC_PB, seed=3, amp=0.05)
    s = _solver(g, prm)
    s.set_state(st)
    for name in ("u", "cp", "Phi"):
        assert np.max(np.abs(s.mean_profile(name) - o.mean_profile(getattr(st, name)))) <= 1e-13
    d = s.diagnostics()
    dr = o.diagnostics(g, prm, st)
    for k in ("tau_bot", "tau_top", "n_plus", "n_minus", "ke"):
        assert abs(d[k] - dr[k]) <= 1e-12 * max(abs(dr[k]), 1e-30), k
    assert abs(d["max_div"] - dr["max_div"]) <= 1e-13
    s.close()
