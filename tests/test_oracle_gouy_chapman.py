"""Electrokinetic validation of the oracle (Numerical methods, the
one-dimensional run with quiescent walls; Fig. 2): march from uniform ions
to the steady state, which must be the discrete Poisson-Boltzmann state (the
stationary solution of Eqs. (1)-(4)) and converge to the Gouy-Chapman closed
form at second order.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pnp_oracle as o

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "e2_double_layer.json")))


def _march(ny, dt, V, lam=0.1, stretch=1.5, nmax=6000, tol=1e-13):
    g = o.Grid(1, ny, 1, 1.0, 1.0, stretch=stretch)
    prm = o.Params(Re=1.0, lam=lam, Sc=GOLDEN["Sc"], V=V, beta=0.5, Uw=GOLDEN["wall_velocity"])
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    n0 = o.diagnostics(g, prm, st)
    for _ in range(nmax):
        st = o.step(g, prm, st, dt)
        c, P = st.cp[:, 0, 0], st.Phi[:, 0, 0]
        F = (c[1:] - c[:-1]) + 0.5 * (c[1:] + c[:-1]) * (P[1:] - P[:-1])
        if np.max(np.abs(F)) < tol:
            break
    return g, prm, st, n0


@pytest.fixture(scope="module")
def e2_state():
    V = 0.5 * GOLDEN["V_hat"]
    return _march(33, 8e-3, V)


def test_steady_state_is_discrete_boltzmann(e2_state):
    g, prm, st, _ = e2_state
    for s, c3 in ((1.0, st.cp), (-1.0, st.cm)):
        c, P = c3[:, 0, 0], st.Phi[:, 0, 0]
        dP = P[1:] - P[:-1]
        ratio = c[1:] / c[:-1]
        assert np.max(np.abs(ratio - (2 - s * dP) / (2 + s * dP))) <= 1e-11


def test_steady_state_statements_of_fig2(e2_state):
    g, prm, st, n0 = e2_state
    cp, cm, Phi = st.cp[:, 0, 0], st.cm[:, 0, 0], st.Phi[:, 0, 0]
    # symmetric about the centre: c+(y) = c-(-y), Phi(-y) = -Phi(y)
    assert np.max(np.abs(cp - cm[::-1])) <= 1e-10
    assert np.max(np.abs(Phi + Phi[::-1])) <= 1e-10
    # ion quantity conserved
    d = o.diagnostics(g, prm, st)
    assert abs(d["n_plus"] - n0["n_plus"]) <= 1e-12 * n0["n_plus"]
    assert abs(d["net_charge"]) <= 1e-12
    # phi = Phi - V y reaches -V y (Phi -> 0, neutral bulk) a few Debye lengths from the walls
    bulk = np.abs(g.yc) < 1 - 5 * prm.lam
    assert np.max(np.abs(Phi[bulk])) <= 0.05 * prm.V
    assert np.max(np.abs(cp[bulk] - cm[bulk])) <= 0.05
    # exponential decay on the Debye scale: counter-ion excess drops by >e^3 over 3 lam
    cb = o.gouy_chapman_bulk(prm.lam, prm.V)
    near = np.argmin(np.abs(g.yc - (-1 + 0.5 * prm.lam)))
    far = np.argmin(np.abs(g.yc - (-1 + 3.5 * prm.lam)))
    assert (cp[near] - cb) / (cp[far] - cb) > math.exp(2.5)
    # walls at rest: no flow is generated
    assert np.max(np.abs(st.u)) <= 1e-14 and np.max(np.abs(st.v)) <= 1e-14


def test_osmotic_balance_at_rest(e2_state):
    # p - K (c+ + c-) is constant at the discrete steady state (pins the force sign)
    g, prm, st, _ = e2_state
    q = (st.p - prm.K * (st.cp + st.cm))[:, 0, 0]
    assert np.max(np.abs(q - q.mean())) <= 1e-10 * prm.K * np.max(st.cp + st.cm)


def test_converges_to_gouy_chapman_second_order():
    errs = []
    for ny, dt in ((33, 8e-3), (65, 4e-3)):
        g, prm, st, _ = _march(ny, dt, V=1.0)
        Pgc, cb = o.gouy_chapman_potential(g.yc, prm.lam, prm.V)
        errs.append((np.max(np.abs(st.cp[:, 0, 0] - cb * np.exp(-Pgc))),
                     np.max(np.abs(st.Phi[:, 0, 0] - Pgc))))
    order_c = math.log2(errs[0][0] / errs[1][0])
    order_p = math.log2(errs[0][1] / errs[1][1])
    assert order_c > 1.8 and order_p > 1.8, (errs, order_c, order_p)
    assert errs[1][0] < 2e-3
