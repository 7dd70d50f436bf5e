"""Parity at the sizes the benchmark runs: the kernel instantiations and tile
paths of the 256 x 193 x 256 turbulent-Couette workload against the FP64
oracle, element by element on the same seeded state.

* mixed precision at 256 x 65 x 256 (the workload's x/z grid and parameters,
  a shorter y-grid): 256-point register transforms, 64-wide stencil tiles with
  neighbouring tiles in x, the stencil's multi-chunk y-march, three steps;
  under both solve policies (default, and FP64 transforms and solves), under
  every launch shape the autotuner can choose (one code at a time), and under
  the shapes it chooses for the 256 x 193 x 256 benchmark grid; and at the
  full 256 x 193 x 256 in those shapes, the benchmark's own configuration.
  Tolerances: fields 1e-5 of each field's scale (velocities at least the wall
  speed), <u>(y) 1e-4 absolute and the wall shear 1e-4 relative (the stated
  accuracy of the mixed path);
* FP64 at the full 256 x 193 x 256 after five steps: 1e-10 relative in the
  max norm of every field (chaotic growth is negligible over five steps).
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o

pytestmark = pytest.mark.gpu

C2 = dict(Lx=2 * math.pi, Lz=math.pi, stretch=2.5, Re=3000.0, lam=0.01, Sc=1.0, V=2.0, beta=0.5, dt=0.004,
          seed=1702, amp=0.1)
STATE = ("u", "v", "w", "p", "cp", "cm", "Phi", "Hu", "Hv", "Hw", "Hcp", "Hcm")
VEL = ("u", "v", "w")


def _setup(nx, ny, nz, precision):
    from paper_1701_02005_gb300.solver import Solver

    g = o.Grid(nx, ny, nz, C2["Lx"], C2["Lz"], stretch=C2["stretch"])
    prm = o.Params(Re=C2["Re"], lam=C2["lam"], Sc=C2["Sc"], V=C2["V"], beta=C2["beta"])
    s = Solver(nx, ny, nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    s.init_state(1, C2["seed"], C2["amp"])
    st0 = o.State(*(s.get(n) for n in STATE))   # the oracle starts from the GPU's initial state
    return g, prm, s, st0


def _scale(name, ref):
    m = float(np.max(np.abs(ref)))
    return max(m, 1.0) if name in VEL else max(m, 1e-300)


MIXED_STEPS = 3
# launch codes {stencil, CN, spectral y-solve, z-transform}: the built-in shapes, and
# every other candidate the autotuner can pick, one code at a time
DEFAULT_CFG = (64, 128, 64, 32)
CANDIDATES = ((32, 64, 128, 16), (32, 64, 256), (16, 32, 128), (8, 16, 64))
CFGS = [DEFAULT_CFG] + [tuple(v if j == i else DEFAULT_CFG[j] for j in range(4))
                        for i, vals in enumerate(CANDIDATES) for v in vals if v != DEFAULT_CFG[i]]


@pytest.fixture(scope="module")
def mixed_reference():
    """The oracle's three steps at 256 x 65 x 256 from the GPU's initial state
    (computed once for every launch configuration)."""
    from paper_1701_02005_gb300 import binding as B

    g, prm, s, st0 = _setup(256, 65, 256, B.PNP_MIXED)
    s.close()
    return g, prm, o.step(g, prm, st0, C2["dt"], MIXED_STEPS)


def _mixed_run(g, prm, ref, cfg=None, policy=0):
    import ctypes as C

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=B.PNP_MIXED, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta)
    if cfg is not None:
        B.check(B.pnp_set_launch_config(s.ctx, (C.c_int * 4)(*cfg)), "pnp_set_launch_config")
    s.set_policy(policy)
    s.init_state(1, C2["seed"], C2["amp"])
    s.step(MIXED_STEPS, C2["dt"])
    errs = {n: float(np.max(np.abs(s.get(n) - getattr(ref, n)))) / _scale(n, getattr(ref, n))
            for n in ("u", "v", "w", "cp", "cm", "Phi")}
    du = float(np.max(np.abs(s.mean_profile("u") - o.mean_profile(ref.u))))
    d, dr = s.diagnostics(), o.diagnostics(g, prm, ref)
    tau = max(abs(d["tau_bot"] - dr["tau_bot"]) / abs(dr["tau_bot"]),
              abs(d["tau_top"] - dr["tau_top"]) / abs(dr["tau_top"]))
    print(f"mixed {g.nx}x{g.ny}x{g.nz} cfg", cfg, "policy", policy, "vs oracle:", errs, "<u>", du, "tau", tau)
    assert d["status"] == 0
    assert all(e <= 1e-5 for e in errs.values()), (cfg, errs)
    assert du <= 1e-4 and tau <= 1e-4, (cfg, du, tau)
    s.close()


@pytest.mark.parametrize("policy", [0, 1])
def test_mixed_at_the_workload_x_z_grid_matches_the_oracle(mixed_reference, policy):
    g, prm, ref = mixed_reference
    _mixed_run(g, prm, ref, None, policy)


@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: "cfg" + "-".join(map(str, c)))
def test_mixed_under_every_launch_shape_the_autotuner_can_pick(mixed_reference, cfg):
    g, prm, ref = mixed_reference
    _mixed_run(g, prm, ref, cfg)


def test_mixed_under_the_benchmarks_tuned_launch_shapes(mixed_reference):
    """The autotuner on the 256 x 193 x 256 benchmark grid (the result is cached,
    so that a benchmark run on the same machine takes the same shapes), its
    choice applied to the parity grid."""
    import math as m

    from paper_1701_02005_gb300 import autotune
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(256, 193, 256, C2["Lx"], C2["Lz"], stretch=C2["stretch"], precision=B.PNP_MIXED)
    s.set_params(C2["Re"], C2["lam"], C2["Sc"], C2["V"], C2["beta"])
    cfg, _ = autotune.tune(s, C2["dt"])
    s.close()
    assert m.isfinite(sum(cfg))
    g, prm, ref = mixed_reference
    _mixed_run(g, prm, ref, tuple(cfg))


@pytest.fixture(scope="module")
def full_mixed_reference():
    """The oracle's three steps at the full 256 x 193 x 256 from the mixed
    context's initial state."""
    from paper_1701_02005_gb300 import binding as B

    g, prm, s, st0 = _setup(256, 193, 256, B.PNP_MIXED)
    s.close()
    return g, prm, o.step(g, prm, st0, C2["dt"], MIXED_STEPS)


def test_mixed_at_the_full_workload_grid_in_the_benchmarks_launch_shapes(full_mixed_reference):
    """The benchmark's own configuration: 256 x 193 x 256, mixed precision, the
    launch shapes the autotuner picks for that grid (as bench.py does), three
    steps against the oracle at the mixed path's tolerances."""
    import math as m

    from paper_1701_02005_gb300 import autotune
    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(256, 193, 256, C2["Lx"], C2["Lz"], stretch=C2["stretch"], precision=B.PNP_MIXED)
    s.set_params(C2["Re"], C2["lam"], C2["Sc"], C2["V"], C2["beta"])
    cfg, _ = autotune.tune(s, C2["dt"])
    s.close()
    assert m.isfinite(sum(cfg))
    g, prm, ref = full_mixed_reference
    _mixed_run(g, prm, ref, tuple(cfg))


def test_fp64_at_the_full_workload_grid_matches_the_oracle_after_five_steps():
    from paper_1701_02005_gb300 import binding as B

    g, prm, s, st0 = _setup(256, 193, 256, B.PNP_FP64)
    nsteps, dt = 5, C2["dt"]
    s.step(nsteps, dt)
    ref = o.step(g, prm, st0, dt, nsteps)
    errs = {}
    for n in ("u", "v", "w", "p", "cp", "cm", "Phi"):
        r = getattr(ref, n)
        errs[n] = float(np.max(np.abs(s.get(n) - r)) / max(np.max(np.abs(r)), 1e-300))
    print("FP64 256x193x256, 5 steps vs oracle:", errs)
    assert all(e <= 1e-10 for e in errs.values()), errs
    d = s.diagnostics()
    assert d["status"] == 0
    s.close()
