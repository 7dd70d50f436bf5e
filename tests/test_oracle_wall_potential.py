"""Pins of the oracle's potential solve with wall potentials that vary along
the walls (the paper's walls may carry any potential; Eq. (4) with Dirichlet
data): against the uniform-wall solve, a dense direct solve of the
finite-volume system with the wall values on the wall faces, and the closed
form of a single-mode wall potential in a charge-free gap (second order)."""
import math

import numpy as np

from oracle import pnp_oracle as o
from tests import seeded


def test_uniform_maps_reproduce_the_uniform_walls():
    g = o.Grid(8, 13, 4, 2.0, 1.0, stretch=1.8)
    prm = o.Params(Re=10.0, lam=0.1, V=1.7)
    cp = seeded.positive_field(1, (g.nyc, g.nz, g.nx), 0.5, 1.5)
    cm = seeded.positive_field(2, (g.nyc, g.nz, g.nx), 0.5, 1.5)
    ref = o.potential_from_ions(g, prm, cp, cm)
    prm2 = o.Params(Re=10.0, lam=0.1, V=1.7, wall=(np.full((4, 8), -1.7), np.full((4, 8), 1.7)))
    assert np.max(np.abs(o.potential_from_ions(g, prm2, cp, cm) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_wall_maps_against_a_dense_direct_solve():
    # Assemble the finite-volume Laplacian of every cell: periodic second
    # differences in x and z; in y the flux through face j is (Phi_j - Phi_{j-1})
    # / (yc_j - yc_{j-1}), and through a wall face (Phi_wall - Phi_edge) over the
    # half cell; divide by the cell height.  Wall values move to the right side.
    nx, ny, nz = 4, 6, 4
    yf = np.array([-1.0, -0.8, -0.3, 0.25, 0.7, 1.0])
    g = o.Grid(nx, ny, nz, 1.5, 1.1, y_faces=yf)
    prm = o.Params(Re=10.0, lam=0.2, V=0.0,
                   wall=(seeded.field(3, (nz, nx)), seeded.field(4, (nz, nx))))
    cp = seeded.positive_field(5, (g.nyc, nz, nx), 0.5, 1.5)
    cm = seeded.positive_field(6, (g.nyc, nz, nx), 0.5, 1.5)
    Pb, Pt = prm.wall
    yc = 0.5 * (yf[1:] + yf[:-1])
    dy = yf[1:] - yf[:-1]
    n = g.nyc * nz * nx
    idx = lambda j, k, i: (j * nz + k) * nx + i
    A = np.zeros((n, n))
    b = (-(cp - cm) / (2 * prm.lam ** 2)).ravel().copy()
    for j in range(g.nyc):
        for k in range(nz):
            for i in range(nx):
                r = idx(j, k, i)
                for di, h2 in ((1, g.dx ** 2), (-1, g.dx ** 2)):
                    A[r, idx(j, k, (i + di) % nx)] += 1 / h2
                    A[r, r] -= 1 / h2
                for dk, h2 in ((1, g.dz ** 2), (-1, g.dz ** 2)):
                    A[r, idx(j, (k + dk) % nz, i)] += 1 / h2
                    A[r, r] -= 1 / h2
                # lower face
                if j > 0:
                    w = 1 / ((yc[j] - yc[j - 1]) * dy[j])
                    A[r, idx(j - 1, k, i)] += w
                    A[r, r] -= w
                else:
                    w = 1 / ((yc[0] - yf[0]) * dy[0])
                    A[r, r] -= w
                    b[r] -= w * Pb[k, i]
                # upper face
                if j < g.nyc - 1:
                    w = 1 / ((yc[j + 1] - yc[j]) * dy[j])
                    A[r, idx(j + 1, k, i)] += w
                    A[r, r] -= w
                else:
                    w = 1 / ((yf[-1] - yc[-1]) * dy[-1])
                    A[r, r] -= w
                    b[r] -= w * Pt[k, i]
    direct = np.linalg.solve(A, b).reshape(g.nyc, nz, nx)
    got = o.potential_from_ions(g, prm, cp, cm)
    assert np.max(np.abs(got - direct)) <= 1e-11 * np.max(np.abs(direct))


def test_single_mode_wall_potential_converges_to_the_closed_form():
    # no charge, Phi_bottom = cos(k x), Phi_top = 0: Phi = cos(k x) sinh(k (1 - y)) / sinh(2 k)
    errs = []
    for m in (1, 2, 4, 8):
        nx, nyc, nz = 16 * m, 8 * m, 4
        Lx = 2 * math.pi
        g = o.Grid(nx, nyc + 1, nz, Lx, 1.0)
        kx = 2 * math.pi / Lx
        xc = (np.arange(nx) + 0.5) * g.dx
        Pb = np.broadcast_to(np.cos(kx * xc), (nz, nx)).copy()
        prm = o.Params(Re=1.0, lam=1.0, V=0.0, wall=(Pb, np.zeros((nz, nx))))
        c = np.ones((g.nyc, nz, nx))
        got = o.potential_from_ions(g, prm, c, c)
        exact = (np.cos(kx * xc)[None, None, :] * (np.sinh(kx * (1 - g.yc)) / np.sinh(2 * kx))[:, None, None])
        errs.append(np.max(np.abs(got - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    # second order, approached from below on the coarsest grids
    assert errs[-1] < 2e-4 and orders[0] < orders[1] < orders[2] and 1.9 < orders[2] < 2.1, (errs, orders)
