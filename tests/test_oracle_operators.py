"""Pins of the oracle's explicit operators (Eqs. (1), (3), Fig. 1).

Invariants and closed forms that a dropped term, wrong sign or wrong index
breaks: discrete kinetic-energy and momentum conservation of the advection
operator, exact ion-number conservation of the flux form, the zero-flux
discrete Boltzmann equilibrium (the stationary state of Eqs. (1)-(4) is
Poisson-Boltzmann), the osmotic balance fixing the Coulomb-force sign, and
the centred-difference symbol of advection and diffusion on Fourier modes.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded


def _grid():
    return o.Grid(8, 13, 6, 2 * math.pi, math.pi, stretch=2.0)


def _divfree(g, seed):
    shp = (g.nyc, g.nz, g.nx)
    u = seeded.field(seed, shp)
    v = seeded.wall_zero_faces(seed + 1, (g.ny, g.nz, g.nx))
    w = seeded.field(seed + 2, shp)
    u, v, w, _ = o.project(g, u, v, w, 1.0)
    return u, v, w


def test_projection_makes_divergence_free():
    g = _grid()
    u, v, w = _divfree(g, 1)
    assert np.max(np.abs(o.divergence(g, u, v, w))) <= 1e-12
    assert np.all(v[0] == 0) and np.all(v[-1] == 0)


def test_advection_conserves_kinetic_energy():
    g = _grid()
    u, v, w = _divfree(g, 21)
    Au = o.advection_u(g, u, v, w)
    Av = o.advection_v(g, u, v, w)
    Aw = o.advection_w(g, u, v, w)
    dy = g.dy[:, None, None]
    hh = g.h[:, None, None]
    prod = np.sum(u * Au * dy) + np.sum(v * Av * hh) + np.sum(w * Aw * dy)
    scale = np.sum(np.abs(u * Au * dy)) + np.sum(np.abs(v * Av * hh)) + np.sum(np.abs(w * Aw * dy))
    assert abs(prod) <= 1e-13 * scale


def test_advection_energy_conservation_detects_divergence():
    # sanity of the pin itself: a non-solenoidal field does not conserve energy
    g = _grid()
    shp = (g.nyc, g.nz, g.nx)
    u = seeded.field(31, shp)
    v = seeded.wall_zero_faces(32, (g.ny, g.nz, g.nx))
    w = seeded.field(33, shp)
    dy = g.dy[:, None, None]
    prod = (np.sum(u * o.advection_u(g, u, v, w) * dy)
            + np.sum(v * o.advection_v(g, u, v, w) * g.h[:, None, None])
            + np.sum(w * o.advection_w(g, u, v, w) * dy))
    assert abs(prod) > 1e-3


def test_advection_conserves_streamwise_and_spanwise_momentum():
    g = _grid()
    shp = (g.nyc, g.nz, g.nx)
    u = seeded.field(41, shp)
    v = seeded.wall_zero_faces(42, (g.ny, g.nz, g.nx))
    w = seeded.field(43, shp)
    dy = g.dy[:, None, None]
    assert abs(np.sum(o.advection_u(g, u, v, w) * dy)) <= 1e-11
    assert abs(np.sum(o.advection_w(g, u, v, w) * dy)) <= 1e-11


def test_uniform_flow_is_steady_under_advection():
    g = _grid()
    shp = (g.nyc, g.nz, g.nx)
    u = np.full(shp, 0.7)
    v = np.zeros((g.ny, g.nz, g.nx))
    w = np.full(shp, -0.3)
    for A in (o.advection_u(g, u, v, w), o.advection_v(g, u, v, w), o.advection_w(g, u, v, w)):
        assert np.max(np.abs(A)) <= 1e-14


def test_scalar_advection_symbol():
    # c = 1 + eps sin(k x) carried by uniform u: -div(u c) = -U (c_{i+1}-c_{i-1})/(2 dx)
    # = -U eps cos(k x_i) sin(k dx)/dx (centred-difference symbol); D -> 0.
    g = o.Grid(16, 5, 4, 2.0, 1.0, stretch=0.0)
    prm = o.Params(Re=1e300, lam=1.0, Sc=1.0)
    shp = (g.nyc, g.nz, g.nx)
    U, eps = 0.8, 0.1
    k = 2 * math.pi * 3 / g.Lx
    xc = (np.arange(g.nx) + 0.5) * g.dx
    c = 1 + eps * np.sin(k * xc)[None, None, :] * np.ones(shp)
    H = o.ion_explicit(g, prm, 1.0, c, np.full(shp, U), np.zeros((g.ny, g.nz, g.nx)),
                       np.zeros(shp), np.zeros(shp))
    expect = -U * eps * np.cos(k * xc) * math.sin(k * g.dx) / g.dx
    assert np.max(np.abs(H - expect[None, None, :])) <= 1e-13


def test_scalar_diffusion_symbol_xz():
    g = o.Grid(16, 5, 8, 2.0, 1.5, stretch=0.0)
    prm = o.Params(Re=2.0, lam=1.0, Sc=3.0)
    shp = (g.nyc, g.nz, g.nx)
    xc = (np.arange(g.nx) + 0.5) * g.dx
    zc = (np.arange(g.nz) + 0.5) * g.dz
    kx, kz = 2 * math.pi * 2 / g.Lx, 2 * math.pi * 1 / g.Lz
    f = np.cos(kx * xc)[None, None, :] * np.sin(kz * zc)[None, :, None] * np.ones(shp)
    H = o.ion_explicit(g, prm, 1.0, 1 + 0.1 * f, np.zeros(shp), np.zeros((g.ny, g.nz, g.nx)),
                       np.zeros(shp), np.zeros(shp))
    mu = -(2 - 2 * math.cos(kx * g.dx)) / g.dx ** 2 - (2 - 2 * math.cos(kz * g.dz)) / g.dz ** 2
    assert np.max(np.abs(H - prm.D * mu * 0.1 * f)) <= 1e-13
    # momentum viscous x/z term has the same symbol
    assert np.max(np.abs(prm.nu * o.lap_xz(g, f) - prm.nu * mu * f)) <= 1e-12


def test_ion_explicit_conserves_ion_number():
    g = _grid()
    prm = o.Params(Re=50.0, lam=0.1, Sc=1.0, V=2.0)
    shp = (g.nyc, g.nz, g.nx)
    c = seeded.positive_field(51, shp)
    u = seeded.field(52, shp)
    v = seeded.wall_zero_faces(53, (g.ny, g.nz, g.nx))
    w = seeded.field(54, shp)
    Phi = seeded.field(55, shp)
    for s in (1.0, -1.0):
        H = o.ion_explicit(g, prm, s, c, u, v, w, Phi)
        assert abs(np.sum(H * g.dy[:, None, None])) <= 1e-11 * np.sum(np.abs(H))


def _boltzmann_column(g, seed, s):
    """1-D c with zero discrete y-face flux: c_j / c_{j-1} = (2 - s dPhi)/(2 + s dPhi)."""
    Phi = 0.3 * np.cumsum(seeded.field(seed, g.nyc))
    c = np.empty(g.nyc)
    c[0] = 1.3
    for j in range(1, g.nyc):
        d = Phi[j] - Phi[j - 1]
        c[j] = c[j - 1] * (2 - s * d) / (2 + s * d)
    return c, Phi


@pytest.mark.parametrize("s", [1.0, -1.0])
def test_discrete_boltzmann_profile_has_zero_flux(s):
    # migration (explicit) + y-diffusion (implicit Neumann operator) cancel cell by cell
    g = o.Grid(4, 17, 4, 1.0, 1.0, stretch=1.7)
    prm = o.Params(Re=3.0, lam=0.1, Sc=2.0)
    c1, Phi1 = _boltzmann_column(g, 61, s)
    shp = (g.nyc, g.nz, g.nx)
    c = c1[:, None, None] * np.ones(shp)
    Phi = Phi1[:, None, None] * np.ones(shp)
    H = o.ion_explicit(g, prm, s, c, np.zeros(shp), np.zeros((g.ny, g.nz, g.nx)), np.zeros(shp), Phi)
    a, b, cc, _, _ = o.ly_centre(g, o.NEUMANN)
    total = H + prm.D * o.apply_rows(a, b, cc, c)
    assert np.max(np.abs(total)) <= 1e-12 * np.max(np.abs(H))
    assert np.max(np.abs(H)) > 1e-3  # the migration term itself is not trivial


def test_osmotic_balance_fixes_force_sign():
    # With both ions in discrete Boltzmann equilibrium, the Coulomb force on the
    # v-faces is exactly the gradient of K (c+ + c-): p = K (c+ + c-) balances it.
    g = o.Grid(4, 17, 4, 1.0, 1.0, stretch=1.7)
    prm = o.Params(Re=7.0, lam=0.2, Sc=1.0, beta=0.5)
    Phi1 = 0.3 * np.cumsum(seeded.field(71, g.nyc))
    shp = (g.nyc, g.nz, g.nx)
    cols = {}
    for s in (1.0, -1.0):
        c = np.empty(g.nyc)
        c[0] = 1.0
        for j in range(1, g.nyc):
            d = Phi1[j] - Phi1[j - 1]
            c[j] = c[j - 1] * (2 - s * d) / (2 + s * d)
        cols[s] = c[:, None, None] * np.ones(shp)
    Phi = Phi1[:, None, None] * np.ones(shp)
    fu, fv, fw = o.body_force(g, prm, cols[1.0], cols[-1.0], Phi)
    gp = o.grad_y(g, prm.K * (cols[1.0] + cols[-1.0]))
    assert np.max(np.abs(fv - gp)) <= 1e-12 * np.max(np.abs(gp))
    assert np.max(np.abs(fu)) == 0.0 and np.max(np.abs(fw)) == 0.0


def test_coulomb_force_direction():
    # positive charge in a field E = -grad Phi pointing in +x is pushed to +x
    g = o.Grid(8, 5, 4, 1.0, 1.0)
    prm = o.Params(Re=1.0, lam=1.0)
    shp = (g.nyc, g.nz, g.nx)
    xc = (np.arange(g.nx) + 0.5) * g.dx
    Phi = -np.sin(2 * math.pi * xc)[None, None, :] * np.ones(shp)  # E_x = 2 pi cos(...)
    cp = np.full(shp, 2.0)
    cm = np.full(shp, 1.0)
    fu, _, _ = o.body_force(g, prm, cp, cm, Phi)
    xf = np.arange(g.nx) * g.dx
    Ex = 2 * math.pi * np.cos(2 * math.pi * xf)
    assert np.all(np.sign(fu[0, 0]) == np.sign(Ex)) or np.allclose(Ex[np.sign(fu[0, 0]) != np.sign(Ex)], 0)


def test_splitmix64_published_vectors():
    # First outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; the
    # widely reproduced reference outputs of the generator)
    out = o.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_pm1_range_and_moments():
    x = o.uniform_pm1(1701, 0, (200000,))
    assert x.min() >= -1.0 and x.max() < 1.0
    assert abs(x.mean()) < 0.01 and abs(np.var(x) - 1 / 3) < 0.01
    y = o.uniform_pm1(1701, 1, (200000,))
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.01


@pytest.mark.parametrize("lam,V", [(0.05, 2.0), (0.01, 2.0), (0.01, 5.0), (0.1, 1.0)])
def test_gouy_chapman_bulk_balances_ion_number(lam, V):
    # numerically integrate the superposed profile: total c+ + c- over [-1,1] is 4
    y = np.linspace(-1, 1, 400001)
    Phi, cb = o.gouy_chapman_potential(y, lam, V)
    tot = np.trapezoid(cb * (np.exp(-Phi) + np.exp(Phi)), y)
    assert abs(tot - 4.0) <= 2e-6


def test_gouy_chapman_solves_poisson_boltzmann():
    # Phi'' = c_b sinh(Phi) / lam^2 (stationary state of Eqs. (3)-(4))
    lam, V = 0.1, 2.0
    y = np.linspace(0.2, 0.99, 2001)
    hh = 1e-4
    Phi, cb = o.gouy_chapman_potential(y, lam, V)
    Pp, _ = o.gouy_chapman_potential(y + hh, lam, V)
    Pm, _ = o.gouy_chapman_potential(y - hh, lam, V)
    d2 = (Pp - 2 * Phi + Pm) / hh ** 2
    assert np.max(np.abs(d2 - cb * np.sinh(Phi) / lam ** 2)) <= 1e-4 * np.max(np.abs(d2))
    # wall values: +-V up to the other wall's tail, 4 tanh(V/4) exp(-2 kappa)
    P1, _ = o.gouy_chapman_potential(np.array([1.0, -1.0]), lam, V)
    tail = 4 * math.tanh(V / 4) * math.exp(-2 * math.sqrt(cb) / lam)
    assert abs(P1[0] - V) <= 1.01 * tail and abs(P1[1] + V) <= 1.01 * tail
