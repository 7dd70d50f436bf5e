"""Adaptive time step: the explicit limits of the state (advective CFL, ion
drift across a cell, dielectric relaxation) reported by pnp_diagnostics, and
pnp_step_adaptive's dt ladder.  An adaptive run is a sequence of ordinary
steps, so the oracle replayed with the same dt sequence must match it at the
FP64 parity tolerance."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o

pytestmark = pytest.mark.gpu


def _limits(g, prm, st):
    """dt at which each explicit number reaches 1, from the definitions."""
    uc = 0.5 * (st.u + np.roll(st.u, -1, axis=2))
    vc = 0.5 * (st.v[:-1] + st.v[1:])
    wc = 0.5 * (st.w + np.roll(st.w, -1, axis=1))
    ra = np.max(np.abs(uc) / g.dx + np.abs(vc) / g.dy[:, None, None] + np.abs(wc) / g.dz)
    P = st.Phi
    dpx = np.abs(np.roll(P, -1, axis=2) - P)
    dpz = np.abs(np.roll(P, -1, axis=1) - P)
    dpy = np.zeros_like(P)
    dpy[:-1] = np.abs(P[1:] - P[:-1]) / (g.h[1:-1] * g.dy[:-1])[:, None, None]
    rm = prm.D * np.max(dpx / g.dx ** 2 + dpy + dpz / g.dz ** 2)
    rd = prm.D * prm.q * np.max(st.cp + st.cm)
    return 1.0 / ra, 1.0 / rm, 1.0 / rd


def _setup(precision=0):
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(16, 33, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=4.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=12, amp=0.05)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    s.set_state(st)
    return g, prm, st, s


def test_reported_limits_match_their_definitions():
    g, prm, st, s = _setup()
    d = s.diagnostics()
    want = _limits(g, prm, st)
    for k, w in zip(("dt_cfl", "dt_migration", "dt_dielectric"), want):
        assert abs(d[k] - w) <= 1e-12 * w, (k, d[k], w)
    s.close()


def test_adaptive_run_is_the_oracle_with_the_same_dt_sequence():
    g, prm, st, s = _setup()
    dt_max, cfl = 0.05, 0.5
    lim = min(cfl * x if i < 2 else 4 * cfl * x for i, x in enumerate(_limits(g, prm, st)))
    k0 = max(0, math.ceil(8 * math.log2(dt_max / lim) - 1e-12))
    dts = s.step_adaptive(24, dt_max, cfl, check_every=6)
    assert dts[0] == dt_max * 2.0 ** (-k0 / 8), (dts[0], k0)
    rungs = -8 * np.log2(dts / dt_max)
    assert np.allclose(rungs, np.round(rungs), atol=1e-9)
    assert all(b >= a - 1 - 1e-9 for a, b in zip(rungs[::6], rungs[6::6]))   # growth: one rung per check at most
    ref = st
    for dt in dts:
        ref = o.step(g, prm, ref, float(dt), 1)
    for n in ("u", "v", "w", "cp", "cm", "Phi"):
        r = getattr(ref, n)
        err = np.max(np.abs(s.get(n) - r)) / np.max(np.abs(r))
        assert err <= 1e-10, (n, err)
    d = s.diagnostics()
    assert d["status"] == 0 and d["nstep"] == 24
    assert d["cfl"] <= cfl * 1.2
    s.close()


def test_adaptive_mixed_run_stays_within_its_limits():
    g, prm, st, s = _setup(precision=1)
    dts = s.step_adaptive(30, 0.05, 0.5, check_every=5)
    assert np.all(dts > 0) and np.all(dts <= 0.05)
    d = s.diagnostics()
    assert d["status"] == 0
    assert d["cfl"] <= 0.6 and dts[-1] * d["dt_migration"] ** -1 <= 0.6
    s.close()
