"""Pins of the oracle's approximate factorisation (x/z viscous and diffusive
terms implicit, (I - s L_x)(I - s L_z)(I - s L_y) dq = r): the cyclic
tridiagonal solve against a dense solve and against the closed-form kernel of
the symmetric operator's inverse, laminar Couette still an exact steady
state, the closed-form amplification of a pure-diffusion ion mode, and the
factored step's agreement with the unfactored one as dt -> 0."""
import math

import numpy as np

from oracle import pnp_oracle as o
from tests import seeded


def test_periodic_solve_against_a_dense_solve():
    for n in (3, 4, 7, 16):
        lo, di, up = -0.3, 1.9, -0.45
        A = np.zeros((n, n))
        for i in range(n):
            A[i, (i - 1) % n] += lo
            A[i, i] += di
            A[i, (i + 1) % n] += up
        r = seeded.field(n, (3, n, 2))
        got = o.periodic_solve(lo, di, up, r, axis=1)
        want = np.einsum("ij,ajb->aib", np.linalg.inv(A), r)
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want)), n


def test_periodic_solve_of_the_symmetric_operator_has_the_closed_form_kernel():
    """(I - s L) on a uniform periodic line, lo = up = -beta, di = 1 + 2 beta: the
    response to e_0 is g_k = (rho^k + rho^(n-k)) / ((1 - rho^n) beta (1/rho - rho)),
    rho the smaller root of beta rho^2 - (1 + 2 beta) rho + beta = 0 (the free-space
    kernel rho^|k| / (beta (1/rho - rho)) summed over the periodic images).  The
    kernel is symmetric and decays geometrically, so a few taps reproduce the cyclic
    solve to rounding where beta is small."""
    for n, beta in ((16, 0.05), (64, 0.3), (256, 5e-4), (32, 4.0)):
        e0 = np.zeros((n, 1))
        e0[0, 0] = 1.0
        g = o.periodic_solve(-beta, 1.0 + 2.0 * beta, -beta, e0, axis=0)[:, 0]
        # the roots' product is 1 and their difference sqrt(d^2 - 4 beta^2) / beta:
        # rho and beta (1/rho - rho) without cancellation at small beta
        d = 1.0 + 2.0 * beta
        disc = math.sqrt(d * d - 4.0 * beta * beta)
        rho = 2.0 * beta / (d + disc)
        k = np.arange(n)
        want = (rho ** k + rho ** (n - k)) / ((1.0 - rho ** n) * disc)
        assert np.max(np.abs(g - want)) <= 1e-13 * np.max(np.abs(want)), (n, beta)
        assert np.max(np.abs(g[1:] - g[1:][::-1])) <= 1e-14 * g[0]   # g_k = g_(n-k)
    # at the 256x193x256 workload's x-operator (beta ~ 5e-4) three taps past the
    # centre leave a tail below 2^-27 of the kernel's sum
    n, beta = 256, 5e-4
    e0 = np.zeros((n, 1))
    e0[0, 0] = 1.0
    g = np.abs(o.periodic_solve(-beta, 1.0 + 2.0 * beta, -beta, e0, axis=0)[:, 0])
    assert g[4:n - 3].sum() <= 2.0 ** -27 * g.sum()
    assert g[3:n - 2].sum() > 2.0 ** -54 * g.sum()   # and FP64 needs more of them


def test_af_keeps_laminar_couette_exact():
    g = o.Grid(8, 17, 4, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=50.0, lam=0.1, V=0.0, af=True)
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    st = o.step(g, prm, st, 0.05, 20)
    assert np.max(np.abs(st.u - g.yc[:, None, None])) <= 1e-13
    assert np.max(np.abs(st.v)) <= 1e-14 and np.max(np.abs(st.w)) <= 1e-14


def _neumann_mode(g, my):
    return np.cos(my * math.pi * (np.arange(g.nyc) + 0.5) / g.nyc)


def test_af_amplification_of_a_diffusing_ion_mode():
    # u = 0, V = 0, c+ = c- = 1 + eps cos(kx x) cos(m pi (j + 1/2) / N): no
    # charge, no flow, pure diffusion; per substage the factored CN update
    # multiplies the mode by 1 + alp dt D lam / ((1 - s lx)(1 - s lz)(1 - s ly)),
    # lam = lx + ly + lz the discrete eigenvalues, s = alp dt D / 2
    g = o.Grid(16, 9, 4, 2 * math.pi, 1.0)
    prm = o.Params(Re=4.0, lam=0.3, V=0.0, Uw=0.0, af=True)
    mx, my = 2, 3
    xc = (np.arange(g.nx) + 0.5) * g.dx
    mode = np.broadcast_to(np.cos(2 * math.pi * mx * xc / g.Lx)[None, None, :] * _neumann_mode(g, my)[:, None, None],
                           (g.nyc, g.nz, g.nx)).copy()
    eps = 1e-3
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    st.u[...] = 0.0
    st.cp = 1.0 + eps * mode
    st.cm = st.cp.copy()
    dt = 0.2
    lx = -(2 - 2 * math.cos(2 * math.pi * mx / g.nx)) / g.dx ** 2
    lz = 0.0
    ly = -(2 - 2 * math.cos(my * math.pi / g.nyc)) / g.dy[0] ** 2
    amp = 1.0
    for l in range(3):
        alp = o.RK3_GAMMA[l] + o.RK3_ZETA[l]
        s = 0.5 * alp * dt * prm.D
        amp *= 1 + alp * dt * prm.D * (lx + ly + lz) / ((1 - s * lx) * (1 - s * lz) * (1 - s * ly))
    out = o.step(g, prm, st, dt, 1)
    got = (out.cp - 1.0) / eps
    assert np.max(np.abs(got - amp * mode)) <= 1e-10, (np.max(np.abs(got - amp * mode)), amp)


def test_af_step_approaches_the_unfactored_step_as_dt_shrinks():
    # the factorisation error is O(dt^2) per substage: both schemes agree to a
    # shrinking difference, falling by about 8x per halving of dt (two steps
    # of half the size each reaching the same time)
    g = o.Grid(16, 13, 8, 2 * math.pi, math.pi, stretch=1.8)
    base = dict(Re=100.0, lam=0.1, V=1.0, beta=0.5)
    st = o.initial_state(g, o.Params(**base), o.IC_PB, seed=5, amp=0.1)
    diffs = []
    for k in range(3):
        dt, n = 0.02 / 2 ** k, 2 ** k
        a = o.step(g, o.Params(**base, af=True), st, dt, n)
        b = o.step(g, o.Params(**base), st, dt, n)
        diffs.append(np.max(np.abs(a.u - b.u)))
    rates = [diffs[i] / diffs[i + 1] for i in range(2)]
    assert all(r > 3.0 for r in rates), (diffs, rates)
