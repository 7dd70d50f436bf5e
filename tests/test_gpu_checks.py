"""Device checks of the running state (pnp_diagnostics / pnp_status): the
advective CFL number of the last step, the potential step between
neighbouring cells, and the net ion flux through the walls implied by the
stored explicit terms.  The failing states are made on the host (a dt above
the stability bound, a double layer too thin for its grid); nothing here can
fault a GPU: the checks only set the status word."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded

pytestmark = pytest.mark.gpu


def _solver(g, prm, precision=0):
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta, prm.Uw)
    return s


def _cfl_rate(g, u, v, w):
    """max over cells of |u_c|/dx + |v_c|/dy + |w_c|/dz with cell-centred velocities."""
    uc = 0.5 * (u + np.roll(u, -1, axis=2))
    vc = 0.5 * (v[:-1] + v[1:])
    wc = 0.5 * (w + np.roll(w, -1, axis=1))
    return float(np.max(np.abs(uc) / g.dx + np.abs(vc) / g.dy[:, None, None] + np.abs(wc) / g.dz))


def _max_dphi(Phi):
    return float(max(np.max(np.abs(np.roll(Phi, -1, axis=2) - Phi)), np.max(np.abs(np.roll(Phi, -1, axis=1) - Phi)),
                     np.max(np.abs(Phi[1:] - Phi[:-1]))))


@pytest.mark.parametrize("precision", [0, 1])
def test_cfl_number_and_its_error_code(precision):
    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(16, 17, 8, 2 * math.pi, math.pi, stretch=1.5)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=1.0)
    s = _solver(g, prm, precision)
    s.init_state(1, 3, 0.05)
    dt = 0.01
    s.step(2, dt)
    d = s.diagnostics()
    want = dt * _cfl_rate(g, s.get("u"), s.get("v"), s.get("w"))
    assert abs(d["cfl"] - want) <= (1e-12 if precision == 0 else 2e-6) * want, (d["cfl"], want)
    assert d["status"] == B.PNP_OK and d["cfl"] < 3 ** 0.5
    s.set_limits(cfl_max=0.5 * d["cfl"])
    assert s.diagnostics()["status"] == B.PNP_ERR_CFL
    assert s.status() == B.PNP_ERR_CFL
    s.set_limits()
    assert s.diagnostics()["status"] == B.PNP_OK
    # a dt just above the RK3 bound for two steps: the fields stay finite, the check fires
    dt_big = 1.9 / _cfl_rate(g, s.get("u"), s.get("v"), s.get("w"))
    s.step(2, dt_big)
    d = s.diagnostics()
    assert d["status"] == B.PNP_ERR_CFL, d
    assert d["cfl"] > 3 ** 0.5
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_potential_step_check_flags_an_unresolved_double_layer(precision):
    from paper_1701_02005_gb300 import binding as B

    # V = 10, Debye length 0.1 on a uniform 8-cell grid: the Gouy-Chapman wall
    # layer drops by more than 2 thermal voltages between the first two cells
    g = o.Grid(8, 9, 4, 2 * math.pi, math.pi, stretch=0.0)
    prm = o.Params(Re=100.0, lam=0.1, Sc=1.0, V=10.0)
    st = o.initial_state(g, prm, o.IC_PB)
    s = _solver(g, prm, precision)
    s.set_state(st)
    d = s.diagnostics()
    want = _max_dphi(st.Phi)
    assert want > 2.0
    assert abs(d["max_dphi"] - want) <= (1e-12 if precision == 0 else 5e-6) * want, (d["max_dphi"], want)
    assert d["status"] == B.PNP_ERR_DPHI
    # a resolved layer passes
    g2 = o.Grid(8, 33, 4, 2 * math.pi, math.pi, stretch=2.0)
    prm2 = o.Params(Re=100.0, lam=0.1, Sc=1.0, V=2.0)
    s2 = _solver(g2, prm2, precision)
    st2 = o.initial_state(g2, prm2, o.IC_PB)
    s2.set_state(st2)
    d2 = s2.diagnostics()
    assert d2["status"] == B.PNP_OK and d2["max_dphi"] < 2.0
    assert abs(d2["max_dphi"] - _max_dphi(st2.Phi)) <= 5e-6 * _max_dphi(st2.Phi)
    s.close()
    s2.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_wall_flux_of_the_explicit_ion_terms_vanishes(precision):
    # the cell sums of H_c telescope to the wall-face fluxes, which the scheme
    # sets to zero (Fig. 1 caption): zero to rounding of the sum of |H_c| dV
    g = o.Grid(32, 21, 16, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0)
    st = o.initial_state(g, prm, o.IC_PB, seed=9, amp=0.1)
    shp = (g.nyc, g.nz, g.nx)
    st.cp = st.cp * seeded.positive_field(10, shp, 0.95, 1.05)
    st.cm = st.cm * seeded.positive_field(11, shp, 0.95, 1.05)
    st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
    s = _solver(g, prm, precision)
    s.set_state(st)
    s.eval_explicit()
    d = s.diagnostics()
    _, _, _, Hcp, Hcm = o.explicit_terms(g, prm, st)
    vol = g.cell_volume()
    scale_p, scale_m = float(np.sum(np.abs(Hcp) * vol)), float(np.sum(np.abs(Hcm) * vol))
    tol = 1e-12 if precision == 0 else 1e-6
    assert abs(d["flux_plus"]) <= tol * scale_p and abs(d["flux_minus"]) <= tol * scale_m, (d, scale_p, scale_m)
    assert d["wall_flux"] == abs(d["flux_plus"]) + abs(d["flux_minus"])
    s.step(3, 0.004)
    d = s.diagnostics()
    assert d["status"] == 0
    assert d["wall_flux"] <= tol * (scale_p + scale_m), d
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_posted_diagnostics_equal_the_synchronous_ones(precision):
    """pnp_diagnostics_post / _read: records posted after consecutive steps and
    read afterwards equal pnp_diagnostics taken at the same moments, in both
    precisions, with wall slip on (the plane-mean wall velocities ride along)."""
    import torch

    g = o.Grid(16, 25, 8, 2 * math.pi, math.pi, stretch=1.8)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5)
    s = _solver(g, prm, precision)
    s.init_state(1, 11, 0.05)
    s.step(2, 0.01)
    sync = s.diagnostics()
    raw = s.diag_buffer()
    s.diagnostics_post(raw)
    s.synchronize()
    assert s.diagnostics_read(raw) == sync
    # two posts in flight, one step apart, then read
    raws = [s.diag_buffer(), s.diag_buffer()]
    ref = []
    for k in range(2):
        s.step(1, 0.01)
        s.diagnostics_post(raws[k])
        ref.append(s.diagnostics())
    for k in range(2):
        assert s.diagnostics_read(raws[k]) == ref[k]
    assert ref[1]["nstep"] == ref[0]["nstep"] + 1
    # slip walls: the plane-mean wall velocities enter the wall shear
    from paper_1701_02005_gb300 import wallmodel as wm

    X = wm.features(s, 4)
    Y = torch.zeros((X.shape[0], 5), dtype=torch.float32, device=X.device)
    Y[:, 0] = 0.5
    wm.set_slip(s, X, Y, 4)
    s.step(1, 0.01)
    d = s.diagnostics()
    s.diagnostics_post(raw)
    s.synchronize()
    assert s.diagnostics_read(raw) == d
    s.close()
