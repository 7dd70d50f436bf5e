"""Pins of the oracle's linear algebra: Thomas, the y-operators and the
separable Poisson solver (Numerical methods, potential paragraph).

Each check compares the oracle with something other than itself: dense
LAPACK solves, brute-force operators assembled from ``divergence`` and the
gradients, closed-form discrete eigenfunctions, and continuous manufactured
solutions with their observed order.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded


def _dense(a, b, c):
    n = len(b)
    M = np.diag(b)
    M[np.arange(1, n), np.arange(n - 1)] = a[1:]
    M[np.arange(n - 1), np.arange(1, n)] = c[:-1]
    return M


@pytest.mark.parametrize("n", [2, 3, 17, 64])
@pytest.mark.parametrize("cplx", [False, True])
def test_thomas_vs_dense(n, cplx):
    a, b, c, d = seeded.diag_dominant_rows(100 + n, n, complex_rhs=cplx)
    x = o.thomas(a[:, None], b[:, None], c[:, None], d)
    ref = np.linalg.solve(_dense(a, b, c), d)
    assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def _grid(n=24, stretch=2.0, nx=8, nz=4):
    return o.Grid(nx, n + 1, nz, 2 * math.pi, math.pi, stretch=stretch)


@pytest.mark.parametrize("bc", [o.NEUMANN, o.DIRICHLET])
def test_ly_centre_self_adjoint_in_cell_volumes(bc):
    # diag(dy) L is symmetric: the finite-volume operator is a weighted Laplacian.
    g = _grid()
    a, b, c, _, _ = o.ly_centre(g, bc)
    W = np.diag(g.dy) @ _dense(a, b, c)
    assert np.max(np.abs(W - W.T)) <= 1e-12 * np.max(np.abs(W))
    # definiteness: Neumann has exactly one zero eigenvalue, Dirichlet none
    ev = np.linalg.eigvalsh(0.5 * (W + W.T))
    assert np.all(ev < 1e-9 * np.max(np.abs(ev)))
    nzero = np.sum(np.abs(ev) < 1e-9 * np.max(np.abs(ev)))
    assert nzero == (1 if bc == o.NEUMANN else 0)


def test_ly_centre_neumann_conserves():
    g = _grid()
    a, b, c, _, _ = o.ly_centre(g, o.NEUMANN)
    q = seeded.field(3, (g.nyc, 2, 3))
    Lq = o.apply_rows(a, b, c, q)
    assert np.max(np.abs(np.sum(Lq * g.dy[:, None, None], axis=0))) <= 1e-11


def test_ly_centre_dirichlet_exact_for_linear_profiles():
    # Couette profile q = y with wall values -1, +1 is an exact discrete null vector.
    g = _grid(stretch=2.5)
    a, b, c, wlo, whi = o.ly_centre(g, o.DIRICHLET)
    q = g.yc[:, None, None] * np.ones((1, 1, 1))
    Lq = o.apply_rows(a, b, c, q, wlo, -1.0, whi, 1.0)
    scale = np.max(np.abs(b))
    assert np.max(np.abs(Lq)) <= 1e-13 * scale


def test_ly_centre_uniform_quadratic():
    g = _grid(stretch=0.0)
    a, b, c, wlo, whi = o.ly_centre(g, o.DIRICHLET)
    # q = 1 - y^2 vanishes on the walls; on a uniform grid the 3-point formula is
    # exact for quadratics in the interior, and the half-cell wall closure gives
    # d2q/dy2 with a known O(1) error only in the wall cells.
    q = (1.0 - g.yc ** 2)[:, None, None]
    Lq = o.apply_rows(a, b, c, q, wlo, 0.0, whi, 0.0)[:, 0, 0]
    assert np.max(np.abs(Lq[1:-1] + 2.0)) <= 1e-10
    # wall cell: [(q1 - q0)/dy - (q0 - 0)/(dy/2)]/dy with q0 = 1 - y0^2
    dy = g.dy[0]
    y0, y1 = g.yc[0], g.yc[1]
    expect = (((1 - y1 ** 2) - (1 - y0 ** 2)) / dy - (1 - y0 ** 2) / (0.5 * dy)) / dy
    assert abs(Lq[0] - expect) <= 1e-10 * abs(expect)


def test_ly_face_symmetric_and_exact_for_quadratics():
    g = _grid(stretch=2.0)
    a, b, c = o.ly_face(g)
    W = np.diag(g.h[1:-1]) @ _dense(a, b, c)
    assert np.max(np.abs(W - W.T)) <= 1e-12 * np.max(np.abs(W))
    # v = 1 - y^2 on the faces (zero on walls): exact second derivative -2 on any grid
    v = (1.0 - g.yf[1:-1] ** 2)[:, None, None]
    Lv = o.apply_rows(a, b, c, v)[:, 0, 0]
    assert np.max(np.abs(Lv + 2.0)) <= 1e-9


def _dense_div_grad(g):
    """Brute-force Neumann Laplacian: divergence(grad(e_k)) for every unit vector."""
    shp = (g.nyc, g.nz, g.nx)
    n = int(np.prod(shp))
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        e = e.reshape(shp)
        M[:, k] = o.divergence(g, o.grad_x(g, e), o.grad_y(g, e), o.grad_z(g, e)).ravel()
    return M


def test_poisson_neumann_vs_dense_div_grad():
    g = o.Grid(4, 6, 4, 2 * math.pi, math.pi, stretch=1.5)
    M = _dense_div_grad(g)
    x_true = seeded.field(5, (g.nyc, g.nz, g.nx))
    rhs = (M @ x_true.ravel()).reshape(x_true.shape)
    x = o.poisson_solve(g, rhs, o.NEUMANN)
    # solution unique up to a constant; the pin sets the bottom plane mean to zero
    x_true = x_true - x_true[0].mean()
    assert np.max(np.abs(x - x_true)) <= 1e-11 * np.max(np.abs(x_true))
    assert abs(x[0].mean()) <= 1e-13


def test_poisson_neumann_residual_of_dense_operator():
    g = o.Grid(8, 9, 4, 2.0, 1.0, stretch=2.0)
    M = _dense_div_grad(g)
    r = seeded.field(6, (g.nyc, g.nz, g.nx))
    r -= np.sum(r * g.dy[:, None, None]) / (np.sum(g.dy) * g.nz * g.nx)  # solvable rhs
    x = o.poisson_solve(g, r, o.NEUMANN)
    res = (M @ x.ravel()).reshape(r.shape) - r
    assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(r))


@pytest.mark.parametrize("bc", [o.DIRICHLET, o.NEUMANN])
def test_poisson_discrete_eigenfunctions_uniform(bc):
    # Uniform y: sin(m pi (j+1/2)/N) (Dirichlet at the walls) and cos(m pi (j+1/2)/N)
    # (Neumann) are exact discrete eigenvectors with eigenvalue -(2 - 2cos(m pi/N))/dy^2.
    nx, nz, N = 8, 16, 12
    g = o.Grid(nx, N + 1, nz, 3.0, 2.0, stretch=0.0)
    j = np.arange(N) + 0.5
    i = np.arange(nx)
    k = np.arange(nz)
    for (m, px, pz) in [(1, 0, 0), (3, 1, 2), (5, 3, 7), (2, 4, 1)]:
        fy = np.sin(m * math.pi * j / N) if bc == o.DIRICHLET else np.cos(m * math.pi * j / N)
        lam_y = -(2 - 2 * math.cos(m * math.pi / N)) / g.dy[0] ** 2
        lam_x = -(2 - 2 * math.cos(2 * math.pi * px / nx)) / g.dx ** 2
        lam_z = -(2 - 2 * math.cos(2 * math.pi * pz / nz)) / g.dz ** 2
        f = (fy[:, None, None] * np.cos(2 * math.pi * px * i / nx)[None, None, :]
             * np.cos(2 * math.pi * pz * k / nz + 0.3)[None, :, None])
        x = o.poisson_solve(g, (lam_x + lam_y + lam_z) * f, bc)
        if bc == o.NEUMANN:
            x = x - x[0].mean() + f[0].mean()
        assert np.max(np.abs(x - f)) <= 1e-11


@pytest.mark.parametrize("bc", [o.DIRICHLET, o.NEUMANN])
def test_poisson_continuous_mms_second_order(bc):
    # phi = Y(y) cos(x) cos(2 z) on [0,2pi) x [-1,1] x [0,pi); Y = sin(pi y) (Dirichlet)
    # or cos(pi y) (Neumann). Observed order of the max error must be ~2 on tanh grids.
    errs = []
    for n in (32, 64):
        g = o.Grid(16, n + 1, 16, 2 * math.pi, math.pi, stretch=1.5)
        x = (np.arange(g.nx) + 0.5) * g.dx
        z = (np.arange(g.nz) + 0.5) * g.dz
        Y = np.sin(math.pi * g.yc) if bc == o.DIRICHLET else np.cos(math.pi * g.yc)
        f = Y[:, None, None] * np.cos(2 * z)[None, :, None] * np.cos(x)[None, None, :]
        # discrete x/z operators act exactly on Fourier modes; only y carries error
        lam_xz = (-(2 - 2 * math.cos(g.dx)) / g.dx ** 2 - (2 - 2 * math.cos(2 * g.dz)) / g.dz ** 2)
        rhs = (lam_xz - math.pi ** 2) * f
        sol = o.poisson_solve(g, rhs, bc)
        if bc == o.NEUMANN:  # all x/z modes are non-constant here, so no gauge freedom
            pass
        errs.append(np.max(np.abs(sol - f)))
    order = math.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.3, (errs, order)


def test_divergence_gradient_adjoint():
    # sum u.grad p dV_u + ... = - sum p div(u) dV_c  (summation by parts, zero wall flux)
    g = o.Grid(8, 11, 4, 2.0, 1.5, stretch=2.0)
    shp = (g.nyc, g.nz, g.nx)
    u = seeded.field(11, shp)
    v = seeded.wall_zero_faces(12, (g.ny, g.nz, g.nx))
    w = seeded.field(13, shp)
    p = seeded.field(14, shp)
    dV = g.dx * g.dz
    lhs = dV * (np.sum(u * o.grad_x(g, p) * g.dy[:, None, None])
                + np.sum(v * o.grad_y(g, p) * g.h[:, None, None])
                + np.sum(w * o.grad_z(g, p) * g.dy[:, None, None]))
    rhs = -dV * np.sum(p * o.divergence(g, u, v, w) * g.dy[:, None, None])
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_modified_wavenumbers_are_second_difference_eigenvalues():
    g = o.Grid(16, 5, 8, 2.0, 3.0)
    kx2, kz2 = o.modified_wavenumbers(g)
    i = np.arange(g.nx)
    for m in range(g.nx // 2 + 1):
        e = np.cos(2 * math.pi * m * i / g.nx + 0.2)
        d2 = (np.roll(e, -1) - 2 * e + np.roll(e, 1)) / g.dx ** 2
        assert np.max(np.abs(d2 + kx2[m] * e)) <= 1e-10 * (1 + kx2[m])
    assert kz2[0] == 0.0 and abs(kz2[1] - kz2[-1]) <= 1e-12 * kz2[1]
