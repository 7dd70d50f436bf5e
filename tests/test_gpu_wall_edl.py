"""Double-layer coupling of the wall model on the GPU against the oracle: the
wall-potential offsets (and the potential and steps under them) and the
ion-flux transfer across the first interior face, in both precisions."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from oracle import wall_oracle as w
from tests import seeded

pytestmark = pytest.mark.gpu

FIELDS = ("u", "v", "w", "p", "cp", "cm", "Phi", "Hu", "Hv", "Hw", "Hcp", "Hcm")


def _rel(a, b, floor=1e-300):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor))


def _setup(precision, seed=4):
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(16, 25, 8, 2 * math.pi, math.pi, stretch=1.8)
    prm = o.Params(Re=200.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=seed, amp=0.05)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    s.set_state(st)
    return g, prm, st, s


def _gpu_state(s, st):
    out = st.copy()
    for n in FIELDS:
        setattr(out, n, np.asarray(s.get(n), dtype=np.float64))
    return out


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("precision", [0, 1])
def test_potential_offsets_match_the_oracle(precision):
    from paper_1701_02005_gb300 import wallmodel as wm

    g, prm, st, s = _setup(precision)
    P, nc, gain = g.nz * g.nx, 4, 0.7
    wm.set_coupling(s, 0, 1.0, potential_gain=gain, flux_gain=0.0)
    B, T = np.zeros((g.nz, g.nx)), np.zeros((g.nz, g.nx))
    # (the mixed context solves the potential with its own pipeline once it steps on its shadows)
    tol_phi = 1e-12 if precision == 0 else 1e-5
    tol = 1e-10 if precision == 0 else 1e-5
    dt = 0.01
    for stage, seed in enumerate((11, 12)):   # offsets accumulate over updates
        # the features leave the present offsets' lift out; the update adds it back
        lift = w.offsets_lift(g, prm, B, T) if stage > 0 else None
        X = w.wall_features(g, prm, st, nc, lift).astype(np.float32)
        Y = seeded.field(seed, (2 * P, 5), 0.3).astype(np.float32)
        B, T = w.edl_offsets(g, X, Y, nc, gain, B, T, max(1.0, abs(prm.V)), lift)
        wm.set_wall_edl(s, _dev(X), _dev(Y), nc)
        prmw = o.Params(Re=prm.Re, lam=prm.lam, Sc=prm.Sc, V=prm.V, beta=prm.beta,
                        wall=(-prm.V + B, prm.V + T))
        st = st.copy()
        st.Phi = o.potential_from_ions(g, prmw, st.cp, st.cm)
        assert _rel(s.get("Phi"), st.Phi) <= tol_phi, (stage, _rel(s.get("Phi"), st.Phi))
        # the features the network would now see: the offsets' lift left out
        Xg = wm.features(s, nc).cpu().numpy()
        Xo = w.wall_features(g, prm, st, nc, w.offsets_lift(g, prm, B, T))
        assert _rel(Xg, Xo) <= (1e-6 if precision == 0 else 2e-5), (stage, _rel(Xg, Xo))
        assert np.max(np.abs(B)) > 0.05   # the offsets are not trivially zero
        s.step(3, dt)
        st = o.step(g, prmw, st, dt, 3)
        for n in ("u", "v", "w", "cp", "cm", "Phi"):
            e = _rel(s.get(n), getattr(st, n), 1.0 if (precision == 1 and n in ("u", "v", "w")) else 1e-300)
            assert e <= tol, (stage, n, e)
        assert s.diagnostics()["status"] == 0
    # gain 0 removes the offsets: the uniform walls and their potential return
    wm.clear_edl(s)
    phi0 = o.potential_from_ions(g, prm, s.get("cp"), s.get("cm"))
    assert _rel(s.get("Phi"), phi0) <= tol_phi
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_flux_transfer_matches_the_oracle(precision):
    from paper_1701_02005_gb300 import wallmodel as wm

    g, prm, st, s = _setup(precision, seed=5)
    dt, gain, P = 0.01, 0.6, g.nz * g.nx
    s.step(2, dt)   # the mixed context now steps on its df shadows
    st_g = _gpu_state(s, st)
    Y = seeded.field(13, (2 * P, 5), 0.05).astype(np.float32)
    wm.set_coupling(s, 0, 1.0, potential_gain=0.0, flux_gain=gain)
    wm.correct_wall_flux(s, _dev(Y), dt)
    cp_o, cm_o = w.wall_flux_fix(g, prm, st_g, Y.astype(np.float64), gain, dt)
    assert _rel(cp_o, st_g.cp) > 1e-4   # the transfer is not trivially small
    for n, ref, old in (("cp", cp_o, st_g.cp), ("cm", cm_o, st_g.cm)):
        got = s.get(n)
        assert _rel(got, ref) <= 1e-13, (n, _rel(got, ref))
        cont = lambda c: np.einsum("jkx,j->kx", c, g.dy)
        assert np.allclose(cont(got), cont(old), rtol=1e-13, atol=0)
    # the next step starts from the transferred ions (in the mixed path: from the
    # shadows the transfer rewrote), with the potential it had
    st_o = st_g.copy()
    st_o.cp, st_o.cm = cp_o, cm_o
    st_o = o.step(g, prm, st_o, dt, 1)
    s.step(1, dt)
    tol = 1e-10 if precision == 0 else 1e-5
    for n in ("cp", "cm", "Phi"):
        e = _rel(s.get(n), getattr(st_o, n))
        assert e <= tol, (n, e)
    s.close()


def test_flux_transfer_needs_disjoint_wall_cells():
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(8, 4, 4, 2 * math.pi, math.pi, stretch=1.5)   # Nyc = 3: the walls' cells overlap
    prm = o.Params(Re=100.0, lam=0.1, Sc=1.0, V=1.0)
    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=0, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    s.set_state(o.initial_state(g, prm, o.IC_PB, seed=1, amp=0.0))
    B.check(B.pnp_set_wallmodel_edl(s.ctx, 0.0, 0.5), "pnp_set_wallmodel_edl")
    Y = _dev(np.zeros((2 * g.nz * g.nx, 5)))
    import ctypes as C

    assert B.pnp_correct_wall_flux(s.ctx, C.c_void_p(Y.data_ptr()), 0.01) == B.PNP_ERR_ARG
    s.close()
