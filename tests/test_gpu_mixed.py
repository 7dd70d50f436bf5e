"""GPU mixed precision (FP32 stencils / FP64 ions, solves and sums) against the
FP64 oracle.

Tolerance: 1e-4 on the plane-averaged streamwise profile <u>(y) (absolute, in
units of the wall speed) and relative 1e-4 on the wall shear stress, the
stated accuracy target of the mixed path.  Ion numbers are FP64 sums of FP64
fields and must stay conserved to 1e-10 relative.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from tests import seeded

pytestmark = pytest.mark.gpu


def _mixed(g, prm):
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=B.PNP_MIXED, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta, prm.Uw)
    return s


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_mixed_explicit_terms_close_to_oracle():
    g = o.Grid(32, 21, 16, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=5, amp=0.1)
    shp = (g.nyc, g.nz, g.nx)
    st.cp = st.cp * seeded.positive_field(6, shp, 0.98, 1.02)
    st.cm = st.cm * seeded.positive_field(7, shp, 0.98, 1.02)
    st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
    s = _mixed(g, prm)
    s.set_state(st)
    s.eval_explicit()
    H = o.explicit_terms(g, prm, st)
    errs = {n: _rel(s.get(n), ref) for n, ref in zip(("Hu", "Hv", "Hw", "Hcp", "Hcm"), H)}
    # FP32 stencils: relative 1e-5 of each field's scale
    assert all(e <= 2e-5 for e in errs.values()), errs
    s.close()


def test_mixed_c1_against_fp64_oracle():
    g = o.Grid(32, 33, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st0 = o.initial_state(g, prm, o.IC_PB, seed=1701, amp=1e-2)
    s = _mixed(g, prm)
    s.set_state(st0)
    nsteps, dt = 100, 0.01
    s.step(nsteps, dt)
    ref = o.step(g, prm, st0, dt, nsteps)
    du = np.max(np.abs(s.mean_profile("u") - o.mean_profile(ref.u)))
    d, dr, d0 = s.diagnostics(), o.diagnostics(g, prm, ref), o.diagnostics(g, prm, st0)
    tau_err = max(abs(d["tau_bot"] - dr["tau_bot"]) / abs(dr["tau_bot"]),
                  abs(d["tau_top"] - dr["tau_top"]) / abs(dr["tau_top"]))
    field_errs = {n: _rel(s.get(n), getattr(ref, n)) for n in ("u", "v", "w", "cp", "cm", "Phi")}
    print("mixed C1: <u> err", du, "tau err", tau_err, "fields", field_errs)
    assert du <= 1e-4 and tau_err <= 1e-4, (du, tau_err)
    assert field_errs["cp"] <= 1e-5 and field_errs["cm"] <= 1e-5 and field_errs["Phi"] <= 1e-5, field_errs
    assert abs(d["n_plus"] - d0["n_plus"]) <= 1e-10 * d0["n_plus"]
    assert abs(d["n_minus"] - d0["n_minus"]) <= 1e-10 * d0["n_minus"]
    assert d["status"] == 0
    s.close()


def test_mixed_double_layer_at_rest_stays_poisson_boltzmann():
    # walls at rest: a discrete Poisson-Boltzmann state (from the FP64 oracle march)
    # must stay stationary in mixed precision — the Debye-layer cancellation is FP64.
    g = o.Grid(4, 33, 4, 1.0, 1.0, stretch=1.5)
    prm = o.Params(Re=1.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5, Uw=0.0)
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    st = o.step(g, prm, st, 8e-3, 600)
    s = _mixed(g, prm)
    s.set_state(st)
    s.step(200, 8e-3)
    ref = o.step(g, prm, st, 8e-3, 200)
    for n in ("cp", "cm", "Phi"):
        assert _rel(s.get(n), getattr(ref, n)) <= 1e-9, n
    assert np.max(np.abs(s.get("u"))) <= 1e-6
    s.close()


def test_mixed_laminar_couette_exact():
    g = o.Grid(16, 17, 8, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=0.0)
    s = _mixed(g, prm)
    s.init_state(0, 1, 0.0)
    s.step(20, 0.01)
    d = s.diagnostics()
    # FP32 storage of u: relative 1e-5 on tau_w, 1e-6 absolute on u
    assert abs(d["tau_bot"] - 1 / 400) <= 1e-5 * (1 / 400)
    assert np.max(np.abs(s.get("u") - g.yc[:, None, None])) <= 1e-6
    s.close()


def test_mixed_stencil_kernels_agree():
    # the TMA row kernel (x2 and x1 rows per block) and the cp.async tile kernels
    # (packed pairs 64 and 32 wide, one cell 32 wide) run the same per-cell
    # arithmetic: identical to FP32 rounding
    import ctypes as C

    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(64, 41, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=15, amp=0.1)
    shp = (g.nyc, g.nz, g.nx)
    st.cp = st.cp * seeded.positive_field(16, shp, 0.98, 1.02)
    st.cm = st.cm * seeded.positive_field(17, shp, 0.98, 1.02)
    st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
    s = _mixed(g, prm)
    out = {}
    for bx in (128, 64, 32, 16):
        B.check(B.pnp_set_launch_config(s.ctx, (C.c_int * 4)(bx, 128, 64, 32)), "pnp_set_launch_config")
        s.set_state(st)
        s.eval_explicit()
        out[bx] = {n: s.get(n) for n in ("Hu", "Hv", "Hw", "Hcp", "Hcm")}
    assert s.status() == 0
    for bx in (64, 32, 16):
        for n in out[128]:
            assert _rel(out[bx][n], out[128][n]) <= 1e-6, (bx, n)
    s.close()


def test_mixed_spectral_solve_variants_agree():
    # the spectral y-solve with its forward values in shared memory (launch code
    # 16) and one thread per spectral point (32, 64): the same df operations in
    # the same order, so the fields agree to the last bit
    import ctypes as C

    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(64, 41, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=25, amp=0.1)
    s = _mixed(g, prm)
    out = {}
    for sp in (16, 32, 64):
        B.check(B.pnp_set_launch_config(s.ctx, (C.c_int * 4)(32, 32, sp, 32)), "pnp_set_launch_config")
        s.set_state(st)
        s.step(3, 0.005)
        out[sp] = {n: s.get(n) for n in ("u", "v", "w", "p", "Phi")}
    assert s.status() == 0
    for sp in (16, 64):
        for n in out[32]:
            assert np.array_equal(out[sp][n], out[32][n]), (sp, n)
    s.close()


def test_mixed_cn_variants_agree():
    # the wall-normal CN solves as one thread per line (launch codes 64, 128, 256;
    # the default) and as shared-memory line tiles (32): the same recurrences on
    # the same operands, so the stepped fields agree to FP32 rounding
    import ctypes as C

    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(64, 41, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=27, amp=0.1)
    s = _mixed(g, prm)
    out = {}
    for cn in (32, 64, 128, 256):
        B.check(B.pnp_set_launch_config(s.ctx, (C.c_int * 4)(64, cn, 32, 32)), "pnp_set_launch_config")
        s.set_state(st)
        s.step(3, 0.005)
        out[cn] = {n: s.get(n) for n in ("u", "v", "w", "cp", "cm", "Phi")}
    assert s.status() == 0
    for cn in (64, 128, 256):
        assert all(np.array_equal(out[cn][n], out[64][n]) for n in out[64]), cn   # same kernel, other block size
        for n in out[32]:
            assert _rel(out[cn][n], out[32][n]) <= 1e-6, (cn, n)
    s.close()


def test_mixed_diagnostics_from_shadows_match_the_definition():
    # after steps the mixed diagnostics come straight from the FP32 fields and
    # the double-float ion state; they must match the definitions evaluated in
    # FP64 on the materialised state (read back through pnp_get_state)
    g = o.Grid(64, 41, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    s = _mixed(g, prm)
    s.set_state(o.initial_state(g, prm, o.IC_PB, seed=21, amp=0.05))
    s.step(6, 0.01)
    for _ in range(2):   # twice: the second call sees the same state
        d = s.diagnostics()
        st = o.State(*(s.get(n) for n in ("u", "v", "w", "p", "cp", "cm", "Phi", "Hu", "Hv", "Hw", "Hcp", "Hcm")))
        ref = o.diagnostics(g, prm, st)
        for k in ("n_plus", "n_minus"):
            assert abs(d[k] - ref[k]) <= 1e-13 * abs(ref[k]), (k, d[k], ref[k])
        assert abs(d["net_charge"] - ref["net_charge"]) <= 1e-13 * abs(ref["n_plus"])
        for k in ("tau_bot", "tau_top", "ke"):
            assert abs(d[k] - ref[k]) <= 1e-12 * abs(ref[k]), (k, d[k], ref[k])
        # the divergence summed in double-float against its FP64 evaluation
        assert abs(d["max_div"] - ref["max_div"]) <= 1e-6 * ref["max_div"] + 1e-15
        assert d["status"] == 0
    s.close()


def test_mixed_fp64_solves_policy_against_the_oracle():
    # the policy that runs every transform and tridiagonal solve of the mixed
    # path in FP64 arithmetic: the same tolerances as the default policy
    from paper_1701_02005_gb300 import binding as B

    g = o.Grid(32, 33, 32, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=400.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st0 = o.initial_state(g, prm, o.IC_PB, seed=1701, amp=1e-2)
    s = _mixed(g, prm)
    s.set_policy(B.PNP_POLICY_FP64_SOLVES)
    s.set_state(st0)
    nsteps, dt = 100, 0.01
    s.step(nsteps, dt)
    ref = o.step(g, prm, st0, dt, nsteps)
    du = np.max(np.abs(s.mean_profile("u") - o.mean_profile(ref.u)))
    d, dr, d0 = s.diagnostics(), o.diagnostics(g, prm, ref), o.diagnostics(g, prm, st0)
    tau_err = max(abs(d["tau_bot"] - dr["tau_bot"]) / abs(dr["tau_bot"]),
                  abs(d["tau_top"] - dr["tau_top"]) / abs(dr["tau_top"]))
    field_errs = {n: _rel(s.get(n), getattr(ref, n)) for n in ("u", "v", "w", "cp", "cm", "Phi")}
    print("mixed (FP64 solves) C1: <u> err", du, "tau err", tau_err, "fields", field_errs)
    assert du <= 1e-4 and tau_err <= 1e-4, (du, tau_err)
    assert field_errs["cp"] <= 1e-5 and field_errs["cm"] <= 1e-5 and field_errs["Phi"] <= 1e-5, field_errs
    assert abs(d["n_plus"] - d0["n_plus"]) <= 1e-10 * d0["n_plus"]
    assert d["status"] == 0
    # switching back to the default policy keeps the state and steps on
    s.set_policy(B.PNP_POLICY_DEFAULT)
    s.step(2, dt)
    assert s.diagnostics()["status"] == 0
    s.close()


def test_fp64_solves_policy_needs_a_mixed_context():
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(8, 9, 4, 1.0, 1.0, precision=B.PNP_FP64)
    assert B.pnp_set_policy(s.ctx, B.PNP_POLICY_FP64_SOLVES) == B.PNP_ERR_UNSUPPORTED
    assert B.pnp_set_policy(s.ctx, 7) == B.PNP_ERR_ARG
    assert B.pnp_set_policy(s.ctx, B.PNP_POLICY_DEFAULT) == B.PNP_OK
    s.close()


@pytest.mark.parametrize("shape", [(64, 97, 32), (16, 257, 8)])
def test_fused_forward_elimination_matches_the_unfused_solve(shape):
    # the stencil's chunk-local forward elimination plus the back substitution's
    # chunk fix-up against right-hand sides stored and eliminated in one sweep:
    # the same solve up to FP32 rounding, on grids whose y-march has many chunks
    from paper_1701_02005_gb300 import binding as B

    nx, ny, nz = shape
    g = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=2.0)
    prm = o.Params(Re=300.0, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    st = o.initial_state(g, prm, o.IC_PB, seed=37, amp=0.1)
    out = {}
    for fused in (1, 0):
        s = _mixed(g, prm)
        B.check(B.pnp_set_fusion(s.ctx, fused), "pnp_set_fusion")
        s.set_state(st)
        s.step(3, 0.004)
        out[fused] = {n: s.get(n) for n in ("u", "v", "w", "cp", "cm", "Phi")}
        assert s.status() == 0
        s.close()
    for n in out[0]:
        scale = max(np.max(np.abs(out[0][n])), 1.0 if n in ("u", "v", "w") else 1e-300)
        assert np.max(np.abs(out[1][n] - out[0][n])) <= 1e-6 * scale, n
    ref = o.step(g, prm, st, 0.004, 3)
    for n in out[1]:
        r = getattr(ref, n)
        scale = max(np.max(np.abs(r)), 1.0 if n in ("u", "v", "w") else 1e-300)
        assert np.max(np.abs(out[1][n] - r)) <= 1e-5 * scale, n


@pytest.mark.parametrize("shape", [(1024, 9, 32), (32, 9, 512), (512, 9, 64), (128, 9, 256)])
def test_mixed_steps_at_every_register_transform_length(shape):
    """Two mixed steps against the oracle on flat grids whose x- and z-extents
    reach every FP32 register-transform length (Nx/2 = 512, 16, 256, 64;
    Nz = 32, 512, 64, 256), fields to 1e-5 of their scale."""
    nx, ny, nz = shape
    g = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=1.5)
    prm = o.Params(Re=300.0, lam=0.1, Sc=1.0, V=2.0, beta=0.5)
    st0 = o.initial_state(g, prm, o.IC_PB, seed=17, amp=0.05)
    s = _mixed(g, prm)
    s.set_state(st0)
    s.step(2, 0.005)
    ref = o.step(g, prm, st0, 0.005, 2)
    for n in ("u", "v", "w", "cp", "cm", "Phi"):
        r = getattr(ref, n)
        scale = max(float(np.max(np.abs(r))), 1.0) if n in ("u", "v", "w") else float(np.max(np.abs(r)))
        e = float(np.max(np.abs(s.get(n) - r))) / scale
        assert e <= 1e-5, (shape, n, e)
    assert s.diagnostics()["status"] == 0
    s.close()
