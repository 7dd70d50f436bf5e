"""Wall potentials that vary along the walls, and in time (the paper's walls
may carry any potential): the GPU potential and the stepped state against the
oracle, which solves Eq. (4) with the same Dirichlet wall data."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded

pytestmark = pytest.mark.gpu


def _maps(g, V, seed, amp=0.4):
    xc = (np.arange(g.nx) + 0.5) * g.dx
    zc = (np.arange(g.nz) + 0.5) * g.dz
    bot = -V + amp * np.cos(2 * math.pi * xc / g.Lx)[None, :] * np.ones((g.nz, 1)) + 0.1 * seeded.field(seed, (g.nz, g.nx))
    top = V + 0.5 * amp * np.sin(4 * math.pi * zc / g.Lz)[:, None] * np.ones((1, g.nx))
    return bot, top


def _rel(a, b, floor=1e-300):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor))


@pytest.mark.parametrize("precision", [0, 1])
def test_wall_potential_maps_match_the_oracle(precision):
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(16, 25, 8, 2 * math.pi, math.pi, stretch=1.8)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=4, amp=0.05)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    s.set_state(st)
    tol_phi = 1e-12 if precision == 0 else 1e-6
    tol = 1e-10 if precision == 0 else 1e-5
    dt = 0.01
    for stage, seed in enumerate((7, 8)):   # two different wall maps in turn (time-varying walls)
        bot, top = _maps(g, prm.V, seed, amp=0.4 + 0.2 * stage)
        prm = o.Params(Re=prm.Re, lam=prm.lam, Sc=prm.Sc, V=prm.V, beta=prm.beta, wall=(bot, top))
        s.set_wall_potential(bot, top)
        st = st.copy()
        st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
        assert _rel(s.get("Phi"), st.Phi) <= tol_phi, (stage, _rel(s.get("Phi"), st.Phi))
        s.step(3, dt)
        st = o.step(g, prm, st, dt, 3)
        for n in ("u", "v", "w", "cp", "cm", "Phi"):
            ref = getattr(st, n)
            e = _rel(s.get(n), ref, 1.0 if (precision == 1 and n in ("u", "v", "w")) else 1e-300)
            assert e <= tol, (stage, n, e)
        assert s.diagnostics()["status"] == 0
    # back to the uniform walls of pnp_set_params
    s.set_wall_potential(None, None)
    prm0 = o.Params(Re=prm.Re, lam=prm.lam, Sc=prm.Sc, V=prm.V, beta=prm.beta)
    phi0 = o.potential_from_ions(g, prm0, s.get("cp"), s.get("cm"))
    assert _rel(s.get("Phi"), phi0) <= tol_phi
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_parameters_changed_mid_run_give_the_potential_of_the_present_ions(precision):
    """pnp_set_params with a state present (walls charged mid-run, as the wall-model
    benchmark does): the potential is solved again for the present ions under the
    new wall potential, and stepping on from there follows the oracle."""
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(16, 25, 8, 2 * math.pi, math.pi, stretch=1.8)
    prm0 = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=0.0, beta=0.5)
    st = o.initial_state(g, prm0, o.IC_PB, seed=9, amp=0.05)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm0.Re, prm0.lam, prm0.Sc, prm0.V, prm0.beta)
    s.set_state(st)
    s.step(2, 0.01)
    st = o.step(g, prm0, st, 0.01, 2)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=1.5, beta=0.5)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
    tol_phi = 1e-12 if precision == 0 else 1e-5   # mixed: the ions of two mixed steps
    assert _rel(s.get("Phi"), st.Phi) <= tol_phi
    s.step(3, 0.01)
    st = o.step(g, prm, st, 0.01, 3)
    tol = 1e-10 if precision == 0 else 1e-5
    for n in ("u", "v", "w", "cp", "cm", "Phi"):
        e = _rel(s.get(n), getattr(st, n), 1.0 if (precision == 1 and n in ("u", "v", "w")) else 1e-300)
        assert e <= tol, (n, e)
    s.close()
