"""Pins of the oracle's time step (Numerical methods: RK3 fractional step,
Crank-Nicolson y-implicit terms, projection, potential split).

* Laminar Couette flow is an exact discrete steady state; tau_w = 1/Re and
  c_f = 2/Re (friction definitions of the Numerical-methods section).
* Discretely divergence-free velocity after every substage (Eq. (2)).
* Exact conservation of N+, N- and the net charge (zero wall flux, Fig. 1).
* Closed-form amplification of discrete Fourier/eigen modes through the
  three RK3-CN substages (pins the coefficients and the CN factor).
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o


def test_laminar_couette_is_exact_steady_state():
    g = o.Grid(8, 17, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=0.0)
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    st = o.step(g, prm, st, 0.02, 30)
    assert np.max(np.abs(st.u - g.yc[:, None, None])) <= 1e-13
    assert np.max(np.abs(st.v)) <= 1e-14 and np.max(np.abs(st.w)) <= 1e-14
    d = o.diagnostics(g, prm, st)
    assert abs(d["tau_bot"] - 1 / 400) <= 1e-14 and abs(d["tau_top"] - 1 / 400) <= 1e-14
    assert abs(d["cf"] - 2 / 400) <= 1e-14
    assert abs(d["re_tau"] - math.sqrt(400)) <= 1e-9


def _noisy_case(V=2.0, amp=0.05):
    g = o.Grid(16, 17, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=V)
    st = o.initial_state(g, prm, o.IC_PB, seed=1701, amp=amp)
    return g, prm, st


def test_divergence_free_after_every_substage():
    g, prm, st = _noisy_case()
    for l in (0, 1, 2, 0, 1, 2):
        st = o.substage(g, prm, st, 0.01, l)
        assert np.max(np.abs(o.divergence(g, st.u, st.v, st.w))) <= 1e-12
        assert np.all(st.v[0] == 0.0) and np.all(st.v[-1] == 0.0)


def test_ion_number_and_charge_conserved():
    g, prm, st = _noisy_case()
    d0 = o.diagnostics(g, prm, st)
    st = o.step(g, prm, st, 0.01, 20)
    d1 = o.diagnostics(g, prm, st)
    for k in ("n_plus", "n_minus"):
        assert abs(d1[k] - d0[k]) <= 1e-12 * d0[k]
    assert abs(d1["net_charge"] - d0["net_charge"]) <= 1e-12 * d0["n_plus"]
    # the flow actually moved ions around
    assert np.max(np.abs(st.cp - o.initial_state(g, prm, o.IC_PB, 1701, 0.05).cp)) > 1e-6


def _mode_recursion(mu_x, lam_y, diff, dt, nsteps):
    """Scalar amplitude of a mode with explicit eigenvalue mu_x (already times
    the diffusivity) and implicit eigenvalue lam_y of L_y (times ``diff``)."""
    a_prev, a = 0.0, 1.0
    for _ in range(nsteps):
        for l in range(3):
            gam, zet = o.RK3_GAMMA[l], o.RK3_ZETA[l]
            alp = gam + zet
            r = dt * (gam * mu_x * a + zet * mu_x * a_prev) + dt * alp * diff * lam_y * a
            da = r / (1.0 - 0.5 * alp * dt * diff * lam_y)
            a_prev, a = a, a + da
    return a


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 2), (2, 3)])
def test_ion_mode_amplification_closed_form(mx, my):
    # c+ = c- = 1 + eps cos(2 pi mx x / Lx) cos(my pi (j+1/2)/N): rho = 0, Phi = 0, u = 0.
    N = 12
    g = o.Grid(8, N + 1, 4, 2.0, 1.0, stretch=0.0)
    prm = o.Params(Re=5.0, lam=1.0, Sc=2.0, V=0.0, Uw=0.0)
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    xc = (np.arange(g.nx) + 0.5) * g.dx
    fy = np.cos(my * math.pi * (np.arange(N) + 0.5) / N)
    f = fy[:, None, None] * np.cos(2 * math.pi * mx * xc / g.Lx)[None, None, :] * np.ones((1, g.nz, 1))
    eps = 1e-2
    st.cp = 1 + eps * f
    st.cm = 1 + eps * f
    dt, nsteps = 0.05, 4
    st = o.step(g, prm, st, dt, nsteps)
    mu_x = -prm.D * (2 - 2 * math.cos(2 * math.pi * mx / g.nx)) / g.dx ** 2
    lam_y = -(2 - 2 * math.cos(my * math.pi / N)) / g.dy[0] ** 2
    amp = _mode_recursion(mu_x, lam_y, prm.D, dt, nsteps)
    assert np.max(np.abs(st.cp - (1 + eps * amp * f))) <= 1e-14
    assert np.max(np.abs(st.u)) <= 1e-15
    assert 0.0 < amp < 1.0


def test_momentum_mode_amplification_closed_form():
    # u = y + eps sin(m pi (j+1/2)/N) cos(2 pi z / Lz): advection and pressure vanish,
    # explicit z-viscous + implicit y-viscous (Dirichlet half-cell walls).
    N, m = 16, 3
    g = o.Grid(4, N + 1, 8, 2.0, 1.5, stretch=0.0)
    prm = o.Params(Re=10.0, lam=1.0, Sc=1.0, V=0.0)
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    zc = (np.arange(g.nz) + 0.5) * g.dz
    fy = np.sin(m * math.pi * (np.arange(N) + 0.5) / N)
    f = fy[:, None, None] * np.cos(2 * math.pi * zc / g.Lz)[None, :, None] * np.ones((1, 1, g.nx))
    eps = 1e-3
    st.u = st.u + eps * f
    dt, nsteps = 0.02, 5
    st = o.step(g, prm, st, dt, nsteps)
    mu_x = -prm.nu * (2 - 2 * math.cos(2 * math.pi / g.nz)) / g.dz ** 2
    lam_y = -(2 - 2 * math.cos(m * math.pi / N)) / g.dy[0] ** 2
    amp = _mode_recursion(mu_x, lam_y, prm.nu, dt, nsteps)
    assert np.max(np.abs(st.u - g.yc[:, None, None] - eps * amp * f)) <= 1e-15
    assert np.max(np.abs(st.v)) <= 1e-16 and np.max(np.abs(st.w)) <= 1e-16
    assert np.max(np.abs(st.p)) <= 1e-12


def test_rk3_coefficients_are_third_order():
    # the mode recursion with small dt reproduces exp(mu t) to O(dt^3)
    errs = []
    for n in (10, 20):
        dt = 1.0 / n
        a = _mode_recursion(-1.0, 0.0, 1.0, dt, n)
        errs.append(abs(a - math.exp(-1.0)))
    assert 2.7 < math.log2(errs[0] / errs[1]) < 3.3
    # the three substages span alpha-sum = 1
    assert abs(sum(g + z for g, z in zip(o.RK3_GAMMA, o.RK3_ZETA)) - 1.0) <= 1e-15


def test_initial_state_is_consistent():
    g, prm, st = _noisy_case()
    assert np.max(np.abs(o.divergence(g, st.u, st.v, st.w))) <= 1e-12
    # Phi satisfies Eq. (4) with Phi = +-V on the walls
    a, b, c, wlo, whi = o.ly_centre(g, o.DIRICHLET)
    lap = o.lap_xz(g, st.Phi) + o.apply_rows(a, b, c, st.Phi, wlo, -prm.V, whi, prm.V)
    res = lap + prm.q * (st.cp - st.cm)
    assert np.max(np.abs(res)) <= 1e-9 * prm.q * np.max(np.abs(st.cp - st.cm))
    # ions: Gouy-Chapman counter-ions enriched at the negative (bottom) wall
    assert st.cp[0].mean() > st.cp[g.nyc // 2].mean() > st.cp[-1].mean()
