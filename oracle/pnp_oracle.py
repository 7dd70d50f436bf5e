"""Plain FP64 NumPy oracle of the NS-PNP fractional step (TEST INFRASTRUCTURE ONLY).

This module is the parity authority for the CUDA library.  It is slow on
purpose: every operator is written out as the finite-volume formula it
stands for, on whole arrays, with no blocking, fusion or reordering.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import it; the product path never does.

What it computes (paper: "Controlling turbulent drag across electrolytes
using electric fields", arXiv:1701.02005):

* Eq. (1)  momentum with the Coulomb body force, Eq. (2) incompressibility,
  Eq. (3)  Nernst-Planck for univalent c+ and c-, Eq. (4) Poisson for Phi,
  nondimensionalised with h, U, h/U, c0, V_T and rho_w U^2 (Numerical
  methods, the control parameters lambda_D/h, beta, Sc, V, Re).
* Plane Couette geometry: walls at y = -1, +1 moving at -Uw, +Uw, periodic
  x and z (Numerical methods, geometry paragraph).
* Staggered second-order finite volumes of Fig. 1: c+-, Phi and p at cell
  centres; u, v, w and the ion fluxes on the cell faces; zero total ion
  flux through the wall faces (Fig. 1 caption).
* Low-storage RK3 for the explicit terms with a Crank-Nicolson y-implicit
  viscous / ion-diffusion term and a projection step (Numerical methods,
  the AFiD paragraph; coefficient reading: Rai & Moin 1991).
* Separable Poisson solves: FFT in x and z, Thomas in y per wavenumber,
  Neumann for the pressure correction and Dirichlet for the potential
  perturbation phi with Phi = V y + phi (Numerical methods, potential
  paragraph).

Readings of the paper where it is silent or ambiguous (the same readings
the CUDA path implements):

* Body-force sign: the Coulomb force is -rho grad Phi (Eq. (4) with Eq. (3)
  fix the sign; Eq. (1) prints +rho grad Phi).  K = beta / (2 Re^2 Sc lam^2).
* Advection in divergence (flux) form.  Momentum: arithmetic averages of the
  advected component; the advecting velocity interpolated to a v-face is the
  cell-volume-weighted mean of the two cells (discrete kinetic-energy
  conservation on the stretched y-grid).  Ions: face velocity times the
  arithmetic face mean of c.
* "Adams-Bashforth for viscous terms" read as Crank-Nicolson in y per
  substage; x and z viscous / diffusive terms explicit, or (Params.af) also
  Crank-Nicolson, approximately factorised into periodic x and z sweeps.
* Pressure update p <- p + Phi_p.  The singular (0,0) Neumann mode is pinned
  by replacing its bottom-row equation with Phi_p(0,0,j=0) = 0.
* Modified wavenumbers (2 - 2 cos(2 pi m / N)) / dx^2: the solver inverts
  the discrete 3-point operator exactly.
* y-grid: Ny face nodes, tanh stretching yf_j = tanh(g (2 j/(Ny-1) - 1)) /
  tanh(g), or faces given explicitly.

Parity: every public function is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, dense linear algebra or brute force.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Low-storage RK3 coefficients (Rai & Moin 1991); alpha = gamma + zeta.
RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)

NEUMANN = "neumann"
DIRICHLET = "dirichlet"

IC_LAMINAR = 0  # uniform ions
IC_PB = 1       # superposed Gouy-Chapman double layers


# --------------------------------------------------------------------------
# Grid and parameters
# --------------------------------------------------------------------------
class Grid:
    """Staggered grid of Fig. 1.  Arrays are indexed [y][z][x].

    ``ny`` counts y face nodes (walls included); there are ``nyc = ny - 1``
    cells in y.  Centre fields have shape (nyc, nz, nx); v lives on the y
    faces and has shape (ny, nz, nx) with zero wall planes.
    """

    def __init__(self, nx, ny, nz, Lx, Lz, stretch=0.0, y_faces=None):
        if ny < 3:
            raise ValueError("need at least two cells in y")
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.nyc = self.ny - 1
        self.Lx, self.Lz = float(Lx), float(Lz)
        if y_faces is None:
            s = np.arange(self.ny, dtype=np.float64) * 2.0 / (self.ny - 1) - 1.0
            if stretch == 0.0:
                yf = s.copy()
            else:
                yf = np.tanh(stretch * s) / math.tanh(stretch)
        else:
            yf = np.array(y_faces, dtype=np.float64)
            if yf.shape != (self.ny,):
                raise ValueError("y_faces must have ny entries")
        yf[0], yf[-1] = -1.0, 1.0
        self.yf = yf
        self.dy = yf[1:] - yf[:-1]                  # cell heights, nyc
        self.yc = 0.5 * (yf[:-1] + yf[1:])          # cell centres, nyc
        h = np.empty(self.ny)                       # centre-to-centre spacing per face
        h[0] = 0.5 * self.dy[0]
        h[1:-1] = self.yc[1:] - self.yc[:-1]
        h[-1] = 0.5 * self.dy[-1]
        self.h = h
        self.dx = self.Lx / self.nx
        self.dz = self.Lz / self.nz

    def cell_volume(self):
        return self.dx * self.dz * self.dy[:, None, None]


@dataclass
class Params:
    """Control parameters of the Numerical-methods section.

    Re = rho_w U h / eta, lam = lambda_D / h, Sc = eta / (rho_w D),
    V = wall potential in units of V_T (so the paper's V-hat = 2 V),
    beta = eps V_T^2 / (eta D), Uw = wall speed in units of U.
    """

    Re: float
    lam: float
    Sc: float = 1.0
    V: float = 0.0
    beta: float = 0.5
    Uw: float = 1.0
    # optional wall potentials (Phi_bottom, Phi_top), each (nz, nx) values on the
    # wall faces above / below the cell columns; None = the uniform -V, +V
    wall: tuple | None = None
    # approximate factorisation: x/z viscous and ion-diffusion terms implicit
    # as well, (I - s L_x)(I - s L_z)(I - s L_y) dq = r (periodic x, z sweeps)
    af: bool = False

    @property
    def nu(self):            # momentum diffusivity 1/Re
        return 1.0 / self.Re

    @property
    def D(self):             # ion diffusivity 1/(Re Sc)
        return 1.0 / (self.Re * self.Sc)

    @property
    def K(self):             # Coulomb-force coefficient
        return self.beta / (2.0 * self.Re ** 2 * self.Sc * self.lam ** 2)

    @property
    def q(self):             # charge-to-Laplacian factor 1/(2 lam^2) of Eq. (4)
        return 1.0 / (2.0 * self.lam ** 2)


@dataclass
class State:
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    p: np.ndarray
    cp: np.ndarray
    cm: np.ndarray
    Phi: np.ndarray
    Hu: np.ndarray
    Hv: np.ndarray
    Hw: np.ndarray
    Hcp: np.ndarray
    Hcm: np.ndarray
    t: float = 0.0
    nstep: int = 0

    def copy(self):
        kw = {k: (getattr(self, k).copy() if isinstance(getattr(self, k), np.ndarray)
                  else getattr(self, k)) for k in self.__dataclass_fields__}
        return State(**kw)


# --------------------------------------------------------------------------
# Periodic shifts in x (axis 2) and z (axis 1)
# --------------------------------------------------------------------------
def _xm(a):
    return np.roll(a, 1, axis=2)      # a[..., i-1]


def _xp(a):
    return np.roll(a, -1, axis=2)     # a[..., i+1]


def _zm(a):
    return np.roll(a, 1, axis=1)      # a[:, k-1, :]


def _zp(a):
    return np.roll(a, -1, axis=1)     # a[:, k+1, :]


def _col(a):
    return a[:, None, None]


# --------------------------------------------------------------------------
# Staggered operators (Fig. 1)
# --------------------------------------------------------------------------
def divergence(g, u, v, w):
    """D.u at cell centres: finite-volume form of Eq. (2)."""
    return (_xp(u) - u) / g.dx + (v[1:] - v[:-1]) / _col(g.dy) + (_zp(w) - w) / g.dz


def grad_x(g, p):
    """d p / dx at the x-faces (u points)."""
    return (p - _xm(p)) / g.dx


def grad_z(g, p):
    """d p / dz at the z-faces (w points)."""
    return (p - _zm(p)) / g.dz


def grad_y(g, p):
    """d p / dy at the interior y-faces (v points); zero on the wall planes."""
    out = np.zeros((g.ny,) + p.shape[1:])
    out[1:-1] = (p[1:] - p[:-1]) / _col(g.h[1:-1])
    return out


def lap_xz(g, q):
    """Explicit x and z second differences (periodic)."""
    return (_xp(q) - 2.0 * q + _xm(q)) / g.dx ** 2 + (_zp(q) - 2.0 * q + _zm(q)) / g.dz ** 2


def advection_u(g, u, v, w):
    """div(u u_x) at the u points, divergence form of the u.grad u term of Eq. (1)."""
    ub_p = 0.5 * (u + _xp(u))
    ub_m = 0.5 * (_xm(u) + u)
    ax = (ub_p * ub_p - ub_m * ub_m) / g.dx
    vf = 0.5 * (_xm(v) + v)                       # v at (x-face, y-face)
    uf = np.zeros_like(vf)
    uf[1:-1] = 0.5 * (u[:-1] + u[1:])
    fy = vf * uf
    ay = (fy[1:] - fy[:-1]) / _col(g.dy)
    wf = 0.5 * (_xm(w) + w)                       # w at (x-face, z-face)
    fz = wf * 0.5 * (_zm(u) + u)
    az = (_zp(fz) - fz) / g.dz
    return ax + ay + az


def advection_v(g, u, v, w):
    """div(u u_y) at the interior v points; zero on the wall planes."""
    dyl = _col(g.dy[:-1])
    dyu = _col(g.dy[1:])
    hh = _col(g.h[1:-1])
    vi = v[1:-1]
    uv = (dyl * u[:-1] + dyu * u[1:]) / (2.0 * hh)   # u at (x-face, y-face), volume weighted
    fx = uv * 0.5 * (_xm(vi) + vi)
    ax = (_xp(fx) - fx) / g.dx
    vb = 0.5 * (v[:-1] + v[1:])                      # v at the cell centres
    ay = (vb[1:] * vb[1:] - vb[:-1] * vb[:-1]) / hh
    wv = (dyl * w[:-1] + dyu * w[1:]) / (2.0 * hh)   # w at (y-face, z-face), volume weighted
    fz = wv * 0.5 * (_zm(vi) + vi)
    az = (_zp(fz) - fz) / g.dz
    out = np.zeros_like(v)
    out[1:-1] = ax + ay + az
    return out


def advection_w(g, u, v, w):
    """div(u u_z) at the w points."""
    wb_p = 0.5 * (w + _zp(w))
    wb_m = 0.5 * (_zm(w) + w)
    az = (wb_p * wb_p - wb_m * wb_m) / g.dz
    vf = 0.5 * (_zm(v) + v)                       # v at (y-face, z-face)
    wf = np.zeros_like(vf)
    wf[1:-1] = 0.5 * (w[:-1] + w[1:])
    fy = vf * wf
    ay = (fy[1:] - fy[:-1]) / _col(g.dy)
    uf = 0.5 * (_zm(u) + u)                       # u at (x-face, z-face)
    fx = uf * 0.5 * (_xm(w) + w)
    ax = (_xp(fx) - fx) / g.dx
    return ax + ay + az


def body_force(g, prm, cp, cm, Phi):
    """Coulomb force -K rho grad(Phi) at the u, v, w points (Eq. (1), sign reading)."""
    rho = cp - cm
    fu = -prm.K * 0.5 * (_xm(rho) + rho) * (Phi - _xm(Phi)) / g.dx
    fv = np.zeros((g.ny,) + rho.shape[1:])
    fv[1:-1] = -prm.K * 0.5 * (rho[:-1] + rho[1:]) * (Phi[1:] - Phi[:-1]) / _col(g.h[1:-1])
    fw = -prm.K * 0.5 * (_zm(rho) + rho) * (Phi - _zm(Phi)) / g.dz
    return fu, fv, fw


def ion_explicit(g, prm, s, c, u, v, w, Phi, xz_diffusion=True):
    """Explicit part of Eq. (3) for the ion of valence s = +1 / -1.

    Face flux F = u c_face - D grad c - s D c_face grad Phi (advective,
    diffusive, migrative), staggered on the faces as in Fig. 1.  The
    y-diffusive part is implicit and left out here.  Wall-face fluxes are
    zero (no penetration, Fig. 1 caption).  Returns -div F.
    """
    D = prm.D
    Dd = D if xz_diffusion else 0.0   # x/z diffusion explicit (CN in y) or implicit (AF)
    cx = 0.5 * (_xm(c) + c)
    Fx = u * cx - Dd * (c - _xm(c)) / g.dx - s * D * cx * (Phi - _xm(Phi)) / g.dx
    cz = 0.5 * (_zm(c) + c)
    Fz = w * cz - Dd * (c - _zm(c)) / g.dz - s * D * cz * (Phi - _zm(Phi)) / g.dz
    Fy = np.zeros((g.ny,) + c.shape[1:])
    cy = 0.5 * (c[:-1] + c[1:])
    Fy[1:-1] = v[1:-1] * cy - s * D * cy * (Phi[1:] - Phi[:-1]) / _col(g.h[1:-1])
    return -((_xp(Fx) - Fx) / g.dx + (Fy[1:] - Fy[:-1]) / _col(g.dy) + (_zp(Fz) - Fz) / g.dz)


# --------------------------------------------------------------------------
# Wall-normal second-difference operators as tridiagonal rows
# --------------------------------------------------------------------------
def ly_centre(g, bc):
    """Rows (a, b, c) of d2/dy2 for a cell-centred quantity, plus the wall
    couplings (wlo, whi) multiplying a Dirichlet wall value.

    (L q)_j = a_j q_{j-1} + b_j q_j + c_j q_{j+1}  [+ wlo q_bot at j=0, + whi q_top at j=n-1].
    Dirichlet: the wall value sits on the wall face, half a cell from the centre.
    Neumann: zero flux through the wall faces.
    """
    n = g.nyc
    a = np.zeros(n)
    b = np.zeros(n)
    c = np.zeros(n)
    for j in range(n):
        lo = 1.0 / (g.h[j] * g.dy[j])
        hi = 1.0 / (g.h[j + 1] * g.dy[j])
        if j > 0:
            a[j] = lo
            b[j] -= lo
        elif bc == DIRICHLET:
            b[j] -= lo
        if j < n - 1:
            c[j] = hi
            b[j] -= hi
        elif bc == DIRICHLET:
            b[j] -= hi
    wlo = 1.0 / (g.h[0] * g.dy[0]) if bc == DIRICHLET else 0.0
    whi = 1.0 / (g.h[n] * g.dy[n - 1]) if bc == DIRICHLET else 0.0
    return a, b, c, wlo, whi


def ly_face(g):
    """Rows (a, b, c) of d2/dy2 for v on the interior faces 1..nyc-1 (v = 0 on walls)."""
    n = g.nyc - 1
    a = np.zeros(n)
    b = np.zeros(n)
    c = np.zeros(n)
    for idx in range(n):
        j = idx + 1
        lo = 1.0 / (g.dy[j - 1] * g.h[j])
        hi = 1.0 / (g.dy[j] * g.h[j])
        if idx > 0:
            a[idx] = lo
        if idx < n - 1:
            c[idx] = hi
        b[idx] = -lo - hi
    return a, b, c


def apply_rows(a, b, c, q, wlo=0.0, qbot=0.0, whi=0.0, qtop=0.0):
    """Apply tridiagonal rows along axis 0 of q, with Dirichlet wall values."""
    out = _col(b) * q
    out[1:] += _col(a[1:]) * q[:-1]
    out[:-1] += _col(c[:-1]) * q[1:]
    out[0] += wlo * qbot
    out[-1] += whi * qtop
    return out


def thomas(a, b, c, d):
    """Thomas algorithm along axis 0: a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j.

    a, b, c broadcast against d; d may be complex.
    """
    n = d.shape[0]
    cpr = [None] * n
    dpr = [None] * n
    cpr[0] = c[0] / b[0]
    dpr[0] = d[0] / b[0]
    for j in range(1, n):
        m = b[j] - a[j] * cpr[j - 1]
        cpr[j] = c[j] / m
        dpr[j] = (d[j] - a[j] * dpr[j - 1]) / m
    x = np.empty(np.broadcast(b, d).shape if np.ndim(b) > np.ndim(d) else d.shape,
                 dtype=np.result_type(d, b))
    x[n - 1] = dpr[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dpr[j] - cpr[j] * x[j + 1]
    return x


def cn_solve(a, b, c, s, r):
    """Solve (I - s L) x = r for L given by rows (a, b, c) along axis 0."""
    return thomas(_col(-s * a), _col(1.0 - s * b), _col(-s * c), r)


def periodic_solve(lo, di, up, r, axis):
    """Solve the cyclic tridiagonal system lo x_{i-1} + di x_i + up x_{i+1} = r_i
    (indices modulo n, constant coefficients) along ``axis``: the Thomas
    algorithm on the system with its corners removed and the diagonal changed
    at both ends, plus the Sherman-Morrison correction for the rank-one rest
    (A = T + u v^T, u = (gam, 0, ..., 0, up), v = (1, 0, ..., 0, lo / gam),
    gam = -di)."""
    rr = np.moveaxis(r, axis, 0)
    n = rr.shape[0]
    gam = -di
    a = np.full(n, lo)
    b = np.full(n, di)
    c = np.full(n, up)
    a[0] = 0.0
    c[-1] = 0.0
    b[0] = di - gam
    b[-1] = di - lo * up / gam
    u = np.zeros(n)
    u[0] = gam
    u[-1] = up
    shape = (n,) + (1,) * (rr.ndim - 1)
    y = thomas(a.reshape(shape), b.reshape(shape), c.reshape(shape), rr)
    q = thomas(a, b, c, u)
    f = (y[0] + (lo / gam) * y[-1]) / (1.0 + q[0] + (lo / gam) * q[-1])
    x = y - f[None] * q.reshape(shape)
    return np.moveaxis(x, 0, axis)


def xz_factors_solve(g, s, r):
    """(I - s L_z)^-1 (I - s L_x)^-1 r with the periodic second differences."""
    bx, bz = s / g.dx ** 2, s / g.dz ** 2
    t = periodic_solve(-bx, 1.0 + 2.0 * bx, -bx, r, axis=2)
    return periodic_solve(-bz, 1.0 + 2.0 * bz, -bz, t, axis=1)


# --------------------------------------------------------------------------
# Separable Poisson solver (Numerical methods, potential paragraph)
# --------------------------------------------------------------------------
def modified_wavenumbers(g):
    """Eigenvalues of the periodic 3-point second difference in x and z."""
    m = np.arange(g.nx // 2 + 1)
    n = np.arange(g.nz)
    kx2 = (2.0 - 2.0 * np.cos(2.0 * np.pi * m / g.nx)) / g.dx ** 2
    kz2 = (2.0 - 2.0 * np.cos(2.0 * np.pi * n / g.nz)) / g.dz ** 2
    return kx2, kz2


def poisson_solve(g, rhs, bc):
    """Solve (delta_xx + delta_zz + L_y) x = rhs: real FFT in x and z, then
    one Thomas solve in y per wavenumber pair.  ``bc`` = NEUMANN (pressure
    correction; mode (0,0) pinned at its bottom cell) or DIRICHLET (phi = 0
    on the walls)."""
    a, b, c, _, _ = ly_centre(g, bc)
    kx2, kz2 = modified_wavenumbers(g)
    rh = np.fft.rfft2(rhs, axes=(1, 2))
    k2 = kz2[:, None] + kx2[None, :]
    A = np.broadcast_to(_col(a), rh.shape).copy()
    B = _col(b) - k2[None, :, :]
    C = np.broadcast_to(_col(c), rh.shape).copy()
    if bc == NEUMANN:
        B[0, 0, 0] = 1.0
        C[0, 0, 0] = 0.0
        rh[0, 0, 0] = 0.0
    sol = thomas(A, B, C, rh)
    return np.fft.irfft2(sol, s=(g.nz, g.nx), axes=(1, 2))


# --------------------------------------------------------------------------
# Time step
# --------------------------------------------------------------------------
def explicit_terms(g, prm, st):
    """H for u, v, w, c+, c- at the current level: advection, explicit
    x/z diffusion, Coulomb force, Nernst-Planck drift (Eqs. (1), (3))."""
    fu, fv, fw = body_force(g, prm, st.cp, st.cm, st.Phi)
    nxz = 0.0 if prm.af else prm.nu   # x/z viscous terms: explicit (CN in y) or implicit (AF)
    Hu = -advection_u(g, st.u, st.v, st.w) + nxz * lap_xz(g, st.u) + fu
    Hv = -advection_v(g, st.u, st.v, st.w) + nxz * lap_xz(g, st.v) + fv
    Hv[0] = 0.0
    Hv[-1] = 0.0
    Hw = -advection_w(g, st.u, st.v, st.w) + nxz * lap_xz(g, st.w) + fw
    Hcp = ion_explicit(g, prm, +1.0, st.cp, st.u, st.v, st.w, st.Phi, not prm.af)
    Hcm = ion_explicit(g, prm, -1.0, st.cm, st.u, st.v, st.w, st.Phi, not prm.af)
    return Hu, Hv, Hw, Hcp, Hcm


def wall_lift(g, prm):
    """Phi_0: the wall potentials carried into the gap linearly in y,
    Phi_0 = (1 - y)/2 Phi_bottom(x, z) + (1 + y)/2 Phi_top(x, z); V y for the
    uniform walls (-V, +V).  The finite-volume y-operator with the wall value
    on the wall face is exact on it, so only its x/z curvature is left."""
    if prm.wall is None:
        return np.broadcast_to(prm.V * _col(g.yc), (g.nyc, g.nz, g.nx)).copy()
    Pb, Pt = (np.asarray(a, dtype=np.float64).reshape(g.nz, g.nx) for a in prm.wall)
    return _col(0.5 * (1.0 - g.yc)) * Pb[None] + _col(0.5 * (1.0 + g.yc)) * Pt[None]


def potential_from_ions(g, prm, cp, cm):
    """Eq. (4): L Phi = -(c+ - c-) / (2 lam^2) with Phi given on the walls (the
    paper's walls carry any potential): Phi = Phi_0 + phi, phi = 0 on the walls,
    L phi = -(c+ - c-) / (2 lam^2) - (delta_xx + delta_zz) Phi_0."""
    Phi0 = wall_lift(g, prm)
    phi = poisson_solve(g, -(cp - cm) * prm.q - lap_xz(g, Phi0), DIRICHLET)
    return Phi0 + phi


def project(g, u, v, w, scale):
    """Projection-correction: solve L Phi_p = D.u / scale (Neumann), subtract
    scale * grad(Phi_p).  Returns the corrected velocity and Phi_p."""
    phip = poisson_solve(g, divergence(g, u, v, w) / scale, NEUMANN)
    u = u - scale * grad_x(g, phip)
    v = v - scale * grad_y(g, phip)
    w = w - scale * grad_z(g, phip)
    return u, v, w, phip


def substage(g, prm, st, dt, l):
    """One RK3 substage l = 0, 1, 2 (Numerical methods, AFiD paragraph)."""
    gam, zet = RK3_GAMMA[l], RK3_ZETA[l]
    alp = gam + zet
    nu, D = prm.nu, prm.D
    Hu, Hv, Hw, Hcp, Hcm = explicit_terms(g, prm, st)

    au, bu, cu, wlo, whi = ly_centre(g, DIRICHLET)
    av, bv, cv = ly_face(g)
    an, bn, cn, _, _ = ly_centre(g, NEUMANN)

    ru = dt * (gam * Hu + zet * st.Hu - alp * grad_x(g, st.p)
               + alp * nu * apply_rows(au, bu, cu, st.u, wlo, -prm.Uw, whi, prm.Uw))
    rv = dt * (gam * Hv[1:-1] + zet * st.Hv[1:-1] - alp * grad_y(g, st.p)[1:-1]
               + alp * nu * apply_rows(av, bv, cv, st.v[1:-1]))
    rw = dt * (gam * Hw + zet * st.Hw - alp * grad_z(g, st.p)
               + alp * nu * apply_rows(au, bu, cu, st.w, wlo, 0.0, whi, 0.0))
    rcp = dt * (gam * Hcp + zet * st.Hcp + alp * D * apply_rows(an, bn, cn, st.cp))
    rcm = dt * (gam * Hcm + zet * st.Hcm + alp * D * apply_rows(an, bn, cn, st.cm))

    su = 0.5 * alp * dt * nu
    sc = 0.5 * alp * dt * D
    if prm.af:
        # approximate factorisation: the x/z second differences join L_y on the
        # right-hand side (explicit half) and in the factored operator
        ru = ru + dt * alp * nu * lap_xz(g, st.u)
        rv = rv + dt * alp * nu * lap_xz(g, st.v[1:-1])
        rw = rw + dt * alp * nu * lap_xz(g, st.w)
        rcp = rcp + dt * alp * D * lap_xz(g, st.cp)
        rcm = rcm + dt * alp * D * lap_xz(g, st.cm)
        ru, rv, rw = (xz_factors_solve(g, su, r) for r in (ru, rv, rw))
        rcp, rcm = (xz_factors_solve(g, sc, r) for r in (rcp, rcm))
    uh = st.u + cn_solve(au, bu, cu, su, ru)
    vh = st.v.copy()
    vh[1:-1] += cn_solve(av, bv, cv, su, rv)
    wh = st.w + cn_solve(au, bu, cu, su, rw)
    cp = st.cp + cn_solve(an, bn, cn, sc, rcp)
    cm = st.cm + cn_solve(an, bn, cn, sc, rcm)

    u, v, w, phip = project(g, uh, vh, wh, alp * dt)
    p = st.p + phip
    Phi = potential_from_ions(g, prm, cp, cm)
    return State(u, v, w, p, cp, cm, Phi, Hu, Hv, Hw, Hcp, Hcm,
                 t=st.t + alp * dt, nstep=st.nstep)


def step(g, prm, st, dt, nsteps=1):
    """``nsteps`` full RK3 steps of size dt."""
    for _ in range(nsteps):
        for l in range(3):
            st = substage(g, prm, st, dt, l)
        st.nstep += 1
    return st


# --------------------------------------------------------------------------
# Initial condition
# --------------------------------------------------------------------------
_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def splitmix64(seed, counters):
    """SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
    output n of the stream seeded with ``seed`` is mix(seed + (n+1) * gamma)."""
    with np.errstate(over="ignore"):
        x = (np.uint64(seed & _MASK) + (counters.astype(np.uint64) + np.uint64(1)) * np.uint64(_SM_GAMMA))
        x = (x ^ (x >> np.uint64(30))) * np.uint64(_SM_M1)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(_SM_M2)
        return x ^ (x >> np.uint64(31))


def uniform_pm1(seed, field_id, shape):
    """Uniform numbers in [-1, 1) for counters (field_id << 40) + flat index."""
    n = int(np.prod(shape))
    ctr = (np.uint64(field_id) << np.uint64(40)) + np.arange(n, dtype=np.uint64)
    bits = splitmix64(seed, ctr) >> np.uint64(11)
    return (bits.astype(np.float64) * 2.0 ** -53 * 2.0 - 1.0).reshape(shape)


def gouy_chapman_bulk(lam, V):
    """Bulk concentration c_b left when two Gouy-Chapman layers form from c = 1:
    c_b + 2 lam sqrt(c_b) (cosh(V/2) - 1) = 1 (ion-number balance)."""
    beta = 2.0 * lam * (math.cosh(0.5 * V) - 1.0)
    s = 0.5 * (-beta + math.sqrt(beta * beta + 4.0))
    return s * s


def gouy_chapman_potential(y, lam, V):
    """Superposed Gouy-Chapman potentials of the walls at y = -1 (-V) and
    y = +1 (+V) with screening length lam / sqrt(c_b)."""
    cb = gouy_chapman_bulk(lam, V)
    kap = math.sqrt(cb) / lam
    t = math.tanh(0.25 * V)
    return (4.0 * np.arctanh(t * np.exp(-(1.0 - y) * kap))
            - 4.0 * np.arctanh(t * np.exp(-(1.0 + y) * kap))), cb


def initial_state(g, prm, kind=IC_PB, seed=1701, amp=0.0):
    """Couette profile u = Uw y plus seeded noise of amplitude ``amp`` damped
    by (1 - y^2), projected to be divergence free; ions uniform (IC_LAMINAR)
    or Gouy-Chapman (IC_PB); Phi from Eq. (4); p = H = 0."""
    shp = (g.nyc, g.nz, g.nx)
    u = np.broadcast_to(prm.Uw * _col(g.yc), shp).copy()
    v = np.zeros((g.ny, g.nz, g.nx))
    w = np.zeros(shp)
    if amp != 0.0:
        u += amp * _col(1.0 - g.yc ** 2) * uniform_pm1(seed, 0, shp)
        v += amp * _col(1.0 - g.yf ** 2) * uniform_pm1(seed, 1, v.shape)
        w += amp * _col(1.0 - g.yc ** 2) * uniform_pm1(seed, 2, shp)
        u, v, w, _ = project(g, u, v, w, 1.0)
    if kind == IC_PB and prm.V != 0.0:
        phigc, cb = gouy_chapman_potential(g.yc, prm.lam, prm.V)
        cp = np.broadcast_to(_col(cb * np.exp(-phigc)), shp).copy()
        cm = np.broadcast_to(_col(cb * np.exp(phigc)), shp).copy()
    else:
        cp = np.ones(shp)
        cm = np.ones(shp)
    Phi = potential_from_ions(g, prm, cp, cm)
    z = np.zeros
    return State(u, v, w, z(shp), cp, cm, Phi, z(shp), z(v.shape), z(shp), z(shp), z(shp))


# --------------------------------------------------------------------------
# Diagnostics (Numerical methods: tau_w, c_f, Re_tau; Fig. 1: wall flux)
# --------------------------------------------------------------------------
def mean_profile(q):
    return q.mean(axis=(1, 2))


def diagnostics(g, prm, st):
    um = mean_profile(st.u)
    tau_bot = prm.nu * (um[0] + prm.Uw) / g.h[0]
    tau_top = prm.nu * (prm.Uw - um[-1]) / g.h[-1]
    vol = g.cell_volume()
    n_plus = float(np.sum(st.cp * vol))
    n_minus = float(np.sum(st.cm * vol))
    tau = 0.5 * (tau_bot + tau_top)
    ke = 0.5 * g.dx * g.dz * (np.sum(st.u ** 2 * _col(g.dy)) + np.sum(st.v ** 2 * _col(g.h))
                              + np.sum(st.w ** 2 * _col(g.dy)))
    return dict(
        tau_bot=float(tau_bot), tau_top=float(tau_top),
        cf=float(2.0 * tau / max(prm.Uw, 1e-300) ** 2) if prm.Uw != 0 else 0.0,
        re_tau=float(prm.Re * math.sqrt(max(tau, 0.0))),
        n_plus=n_plus, n_minus=n_minus, net_charge=n_plus - n_minus,
        max_div=float(np.max(np.abs(divergence(g, st.u, st.v, st.w)))),
        ke=float(ke),
    )
