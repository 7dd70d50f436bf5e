"""Time statistics (mean profiles, RMS fluctuations, time-averaged c_f) of a
run against the same averages of the oracle's states, step by step."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o

pytestmark = pytest.mark.gpu

NAMES = ("u", "v", "w", "cp", "cm", "Phi")


def _oracle_stats(g, prm, st, dt, nsteps):
    acc = {n: [0.0, 0.0] for n in NAMES}
    for _ in range(nsteps):
        st = o.step(g, prm, st, dt, 1)
        for n in NAMES:
            q = getattr(st, n)
            acc[n][0] = acc[n][0] + q.mean(axis=(1, 2))
            acc[n][1] = acc[n][1] + (q * q).mean(axis=(1, 2))
    out = {}
    for n in NAMES:
        m, m2 = acc[n][0] / nsteps, acc[n][1] / nsteps
        out[n] = (m, np.sqrt(np.maximum(m2 - m * m, 0.0)))
    um = out["u"][0]
    cf = (prm.nu * (um[0] + prm.Uw) / g.h[0] + prm.nu * (prm.Uw - um[-1]) / g.h[-1]) / prm.Uw ** 2
    return out, cf


@pytest.mark.parametrize("precision", [0, 1])
def test_time_statistics_match_the_oracle(precision):
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(16, 21, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=31, amp=0.2)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    s.set_state(st)
    s.stats_reset()
    n, dt = 6, 0.01
    for _ in range(n):
        s.step(1, dt)
        s.stats_sample()
    got, cf, ns = s.stats()
    ref, cf_ref = _oracle_stats(g, prm, st, dt, n)
    assert ns == n
    tol = 1e-11 if precision == 0 else 2e-5
    for name in NAMES:
        scale = max(np.max(np.abs(ref[name][0])), 1.0)
        assert np.max(np.abs(got[name][0] - ref[name][0])) <= tol * scale, name
        # RMS of the fluctuations: an absolute bound in the field's scale (the
        # difference of two averages of squares)
        assert np.max(np.abs(got[name][1] - ref[name][1])) <= (1e-7 if precision == 0 else 3e-3) * scale, name
    assert abs(cf - cf_ref) <= (1e-10 if precision == 0 else 1e-4) * abs(cf_ref)
    s.stats_reset()
    _, _, ns = s.stats()
    assert ns == 0
    s.close()
