"""Learned wall model on the GPU: data kernels and network against the FP64
oracle, training by the library's own kernels, and the gain over the coarse
solver without the model (drag judged against the fine DNS)."""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from oracle import wall_oracle as w
from tests import seeded

pytestmark = pytest.mark.gpu


def _solver(g, prm, precision=0):
    from paper_1701_02005_gb300.solver import Solver

    s = Solver(g.nx, g.ny, g.nz, g.Lx, g.Lz, precision=precision, y_faces=g.yf)
    s.set_params(prm.Re, prm.lam, prm.Sc, prm.V, prm.beta, prm.Uw)
    return s


def _grids():
    gf = o.Grid(16, 33, 8, 2 * math.pi, math.pi, stretch=2.0)
    gc = o.Grid(8, 9, 4, 2 * math.pi, math.pi, y_faces=gf.yf[::4])
    return gf, gc


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


def test_restriction_features_labels_match_oracle():
    from paper_1701_02005_gb300 import wallmodel as wm

    gf, gc = _grids()
    prm = o.Params(Re=200.0, lam=0.1, V=2.0)
    st = o.initial_state(gf, prm, o.IC_PB, seed=21, amp=0.2)
    shp = (gf.nyc, gf.nz, gf.nx)
    st.cp = st.cp * seeded.positive_field(22, shp, 0.9, 1.1)
    st.Phi = st.Phi + seeded.field(23, shp, 0.02)
    sf, sc = _solver(gf, prm), _solver(gc, prm)
    sf.set_state(st)
    wm.restrict(sf, sc)
    for name, vf in (("u", False), ("v", True), ("w", False), ("cp", False), ("Phi", False)):
        assert _rel(sc.get(name), w.restrict(gf, gc, getattr(st, name), vf)) <= 1e-13, name
    stc = o.State(*(w.restrict(gf, gc, getattr(st, n), n == "v") for n in ("u", "v", "w", "p", "cp", "cm", "Phi")),
                  *(np.zeros(1),) * 5)
    X = wm.features(sc, 8).cpu().numpy()
    Xr = w.wall_features(gc, prm, stc, 8)
    assert np.max(np.abs(X - Xr)) <= 1e-6 * np.max(np.abs(Xr))
    T = wm.labels(sf, sc).cpu().numpy()
    Tr = w.wall_labels(gf, gc, prm, st)
    for q in range(5):
        assert np.max(np.abs(T[:, q] - Tr[:, q])) <= 1e-5 * max(np.max(np.abs(Tr[:, q])), 1e-12), q
    sf.close()
    sc.close()


def _norm(seed):
    r = seeded.rng(seed)
    return [r.normal(size=40).astype(np.float32), r.uniform(0.5, 2, 40).astype(np.float32),
            r.normal(size=5).astype(np.float32), r.uniform(0.5, 2, 5).astype(np.float32)]


def test_mlp_forward_and_gradient_match_oracle():
    import torch

    from paper_1701_02005_gb300.wallmodel import MLP

    net = MLP(256, seed=5)
    norm = _norm(6)
    net.set_normalization(*norm)
    p = net.params()
    r = seeded.rng(7)
    X = r.standard_normal((200, 40)).astype(np.float32)
    T = r.standard_normal((200, 5)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    # the tensor-core GEMMs take weights and activation operands in BF16 and
    # accumulate in FP32: against the oracle's BF16-operand reading the results
    # differ by the FP32 accumulation order and by the rare operand whose BF16
    # rounding flips between the two GELU evaluations (one BF16 ulp, 2^-8)
    Y = net.forward(Xd).cpu().numpy()
    Yr, _ = w.forward(p, X, norm, bf16=True, bf16_act=True)
    Yr = np.clip((Yr - norm[2]) * norm[3], -6, 6) / norm[3] + norm[2]   # inference path clips at 6 sigma
    assert np.max(np.abs(Y - Yr)) <= 2e-3 * np.max(np.abs(Yr)), np.max(np.abs(Y - Yr)) / np.max(np.abs(Yr))
    Yx, _ = w.forward(p, X, norm, bf16=True)
    Yx = np.clip((Yx - norm[2]) * norm[3], -6, 6) / norm[3] + norm[2]
    assert np.max(np.abs(Y - Yx)) <= 3e-2 * np.max(np.abs(Yx))   # and to BF16 accuracy of the FP32-operand net
    g, loss = net.gradient(Xd, Td)
    lr, gr = w.loss_and_grad(p, X, T, norm, bf16=True, bf16_act=True)
    assert abs(loss - lr) <= 2e-3 * lr, (loss, lr)
    sl, _ = w.param_slices()
    for ws, bs, _, _ in sl:
        for s_ in (ws, bs):
            err = np.max(np.abs(g[s_] - gr[s_])) / (np.max(np.abs(gr[s_])) + 1e-12)
            assert err <= 5e-3, err
    assert net.status() == 0
    net.close()


def test_mlp_residual_output_matches_oracle():
    """Output 2 as the raw input column 32 plus the network (pnp_mlp_set_skip):
    the fused inference adds the input after the clip and the output scaling,
    the loss and gradient take the residual target t_2 - x_32; removing the skip
    restores the plain outputs; bad columns are rejected."""
    import torch

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300.wallmodel import MLP

    net = MLP(512, seed=15)
    norm = _norm(16)
    net.set_normalization(*norm)
    p = net.params()
    r = seeded.rng(17)
    X = r.standard_normal((300, 40)).astype(np.float32)
    X[:, 32] += 5.0   # an input column far from the target's mean: the residual target differs
    T = r.standard_normal((300, 5)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    Y0 = net.forward(Xd).cpu().numpy()
    net.set_skip(2, 32)
    Y = net.forward(Xd).cpu().numpy()
    assert np.array_equal(np.delete(Y, 2, 1), np.delete(Y0, 2, 1))
    assert np.allclose(Y[:, 2], Y0[:, 2] + X[:, 32], rtol=0, atol=1e-6 * np.max(np.abs(Y[:, 2])))
    Yr, _ = w.forward(p, X, norm, bf16=True, bf16_act=True)
    Yr = np.clip((Yr - norm[2]) * norm[3], -6, 6) / norm[3] + norm[2]
    Yr[:, 2] += X[:, 32]
    assert np.max(np.abs(Y - Yr)) <= 2e-3 * np.max(np.abs(Yr)), np.max(np.abs(Y - Yr)) / np.max(np.abs(Yr))
    g, loss = net.gradient(Xd, Td)
    lr, gr = w.loss_and_grad(p, X, T, norm, bf16=True, bf16_act=True, skip=(2, 32))
    assert abs(loss - lr) <= 2e-3 * lr, (loss, lr)
    assert abs(lr - w.loss_and_grad(p, X, T, norm, bf16=True, bf16_act=True)[0]) > 1e-2 * lr   # the skip matters
    sl, _ = w.param_slices()
    for ws, bs, _, _ in sl:
        for s_ in (ws, bs):
            err = np.max(np.abs(g[s_] - gr[s_])) / (np.max(np.abs(gr[s_])) + 1e-12)
            assert err <= 5e-3, err
    net.set_skip(-1, 0)
    assert np.array_equal(net.forward(Xd).cpu().numpy(), Y0)
    for bad in ((5, 0), (0, 40), (1, -1)):
        assert B.pnp_mlp_set_skip(net.m, *bad) == B.PNP_ERR_ARG
    assert net.status() == 0
    net.close()


def test_mlp_training_reduces_loss():
    import torch

    from paper_1701_02005_gb300.wallmodel import MLP

    r = seeded.rng(9)
    X = r.standard_normal((4096, 40)).astype(np.float32)
    A = r.standard_normal((40, 5)) / math.sqrt(40)
    T = (np.tanh(X @ A) + 0.1 * (X[:, :5] ** 2)).astype(np.float32)
    net = MLP(4096, seed=10)
    net.set_normalization(np.zeros(40), np.ones(40), np.zeros(5), np.ones(5))
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0 = net.train_step(Xd, Td, 1e-3, want_loss=True)
    for _ in range(400):
        net.train_step(Xd, Td, 1e-3)
    l1 = net.train_step(Xd, Td, 1e-3, want_loss=True)
    assert l1 < 0.1 * l0, (l0, l1)
    net.close()


def _impulsive(s, g, seed, amp=0.02):
    """Walls set in motion at t = 0: the seeded, projected noise of pnp_init_state
    minus the Couette profile (a function of y only, so still divergence free)."""
    s.init_state(1, seed, amp)
    s.set("u", s.get("u") - g.yc[:, None, None])


def wall_model_case(nfine=(32, 65, 32), ry=4, rxz=2, Re=500.0, dt=0.002, nsteps=200, every=2, train_iters=3000,
                    passes=3, mode=2, relax=1.0, seed_train=31, seed_judge=32, edl=(0.3, 0.3), residual=False):
    """Fine DNS data -> trained network -> coarse runs with and without it, judged
    on the friction coefficient against the fine DNS.  Training pairs the coarse
    solver's own near-wall features with the fine run's filtered labels at the
    same time and initial state: data pass 0 from the coarse run without the
    model, later passes (dataset aggregation) from the coarse run coupled to the
    previous pass's network in the coupling judged (`mode`, `relax`, `edl`).
    residual: the network's potential output is the first-cell feature plus its
    own value (a residual output)."""
    import torch

    from paper_1701_02005_gb300 import binding as B
    from paper_1701_02005_gb300 import wallmodel as wm

    nx, ny, nz = nfine
    gf = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=2.0)
    gc = o.Grid(nx // rxz, (ny - 1) // ry + 1, nz // rxz, 2 * math.pi, math.pi, y_faces=gf.yf[::ry])
    prm = o.Params(Re=Re, lam=0.05, Sc=1.0, V=2.0, beta=0.5)
    sf, sc, sm = _solver(gf, prm), _solver(gc, prm), _solver(gc, prm)
    skip = wm.PHI_SKIP if residual else None

    def couple(s):
        B.check(B.pnp_set_wallmodel_coupling(s.ctx, mode, relax), "pnp_set_wallmodel_coupling")
        B.check(B.pnp_set_wallmodel_edl(s.ctx, float(edl[0]), float(edl[1])), "pnp_set_wallmodel_edl")

    Xs, Ts = [], []
    net, norm, losses = None, None, []
    for rnd in range(passes):
        _impulsive(sf, gf, seed_train)
        wm.restrict(sf, sc)
        couple(sc)
        for n in range(nsteps // every):
            Xs.append(wm.features(sc, 8))
            Ts.append(wm.labels(sf, sc))
            sf.step(every, dt)
            if net is None:
                sc.step(every, dt)
            else:
                wm.step_with_model(sc, net, every, dt)
        X = torch.cat(Xs)
        T = wm.residual_targets(torch.cat(Ts), X, skip)   # the normalisation describes these
        if net is None:
            Xh, Th = X.cpu().numpy(), T.cpu().numpy()
            xs, ts = Xh.mean(0), Th.mean(0)
            # spreads floored relative to each column's magnitude: columns that hardly
            # vary in the training data must not be amplified into noise at inference
            xsd = np.maximum(Xh.std(0), 1e-2 * np.maximum(np.abs(xs), 1e-2))
            tsd = np.maximum(Th.std(0), 1e-2 * np.maximum(np.abs(ts), 1e-4))
            norm = (xs, 1.0 / xsd, ts, 1.0 / tsd)
            net = wm.MLP(nsteps // every * passes * 2 * gc.nz * gc.nx, seed=33)
            net.set_normalization(*norm)
            if skip is not None:
                net.set_skip(*skip)
        T = torch.cat(Ts)   # the network takes the labels themselves
        lr0, lr1 = (2e-3, 5e-4) if rnd == 0 else (1e-3, 3e-4)
        l0 = net.train_step(X, T, lr0, want_loss=True)
        for it in range(train_iters):
            net.train_step(X, T, lr0 if it < train_iters // 2 else lr1)
        l1 = net.train_step(X, T, lr1, want_loss=True)
        losses.append((l0, l1))
        wm.set_slip(sc, None, None)
        wm.clear_edl(sc)
    # judge run (another seed): fine truth, coarse alone, the network predicting the
    # wall shear along the uncoupled coarse trajectory (one-way), and the two-way
    # coupled run (network -> wall conditions -> coarse solver)
    _impulsive(sf, gf, seed_judge)
    wm.restrict(sf, sc)
    wm.restrict(sf, sm)
    couple(sm)
    d0 = sm.diagnostics()
    N_0 = (d0["n_plus"], d0["n_minus"])
    cf_f, cf_p, cf_m, cf_c = [], [], [], []
    phi_err = {"plain": [], "coupled": []}   # first-cell potential against the filtered fine one
    chunk = 10
    for n in range(nsteps // chunk):
        sf.step(chunk, dt)
        sc.step(chunk, dt)
        wm.step_with_model(sm, net, chunk, dt)
        cf_f.append(sf.diagnostics()["cf"])
        cf_p.append(sc.diagnostics()["cf"])
        Xp = wm.features(sc, 8)
        Y = net.forward(Xp).cpu().numpy()
        cf_m.append(2.0 * prm.nu * float(Y[:, 0].mean()))     # c_f = 2 tau_w / Uw^2, tau_w = nu <du_rel/dy>
        cf_c.append(sm.diagnostics()["cf"])
        phi_f = wm.labels(sf, sc).cpu().numpy()[:, 2]
        for key, s_ in (("plain", sc), ("coupled", sm)):   # the total first-cell potential
            phi_c = wm.first_cell_potential(s_, prm.V, gc.yc)
            phi_err[key].append(float(np.mean(np.abs(phi_c - phi_f)) / np.mean(np.abs(phi_f))))
    cf_f, cf_p, cf_m, cf_c = map(np.array, (cf_f, cf_p, cf_m, cf_c))
    err = lambda a: float(np.mean(np.abs(a - cf_f) / cf_f))
    status = net.status()
    dm = sm.diagnostics()
    N_c = (dm["n_plus"], dm["n_minus"])
    for s in (sf, sc, sm):
        s.close()
    net.close()
    return dict(loss0=losses[0][0], loss1=losses[0][1], err_plain=err(cf_p), err_model=err(cf_m),
                err_coupled=err(cf_c), cf_fine=cf_f.tolist(), cf_plain=cf_p.tolist(), cf_model=cf_m.tolist(),
                cf_coupled=cf_c.tolist(), rows=int(Xs[0].shape[0] * len(Xs)), status=status, ions_coupled=N_c,
                ions_start=N_0, err_phi_plain=float(np.mean(phi_err["plain"])),
                err_phi_coupled=float(np.mean(phi_err["coupled"])))


@pytest.mark.parametrize("residual", [False, True])
def test_wall_model_gains_over_coarse_solver(residual):
    """The coarse solver coupled to the network (plane-mean predicted wall stress,
    wall-potential offsets and ion-flux transfers at gain 0.3, three passes of
    dataset aggregation) tracks the fine DNS's friction coefficient better than
    the coarse solver alone, its first-cell potential follows the filtered fine
    one, and the flux transfers keep the ion numbers; with the potential output
    absolute or residual (the coarse first-cell potential plus the network)."""
    r = wall_model_case(residual=residual)
    print("wall model:", {k: v for k, v in r.items() if not k.startswith("cf_")})
    print("cf fine ", np.round(r["cf_fine"], 6).tolist())
    print("cf plain", np.round(r["cf_plain"], 6).tolist())
    print("cf model", np.round(r["cf_model"], 6).tolist())
    print("cf coupled", np.round(r["cf_coupled"], 6).tolist())
    assert r["status"] == 0
    assert r["loss1"] < 0.1 * r["loss0"]
    assert r["err_model"] < r["err_plain"], r
    assert r["err_coupled"] < 0.75 * r["err_plain"], r
    assert r["err_phi_coupled"] < 0.1 * r["err_phi_plain"], r
    for n0, n1 in zip(r["ions_start"], r["ions_coupled"]):
        assert abs(n1 - n0) <= 1e-12 * n0, r


def test_fused_inference_matches_the_layer_by_layer_forward():
    """The outputs-only kernel (all layers in one launch, activations kept on chip)
    against the layer-by-layer forward the gradient runs, over several tiles and a
    ragged last tile: the loss of the fused outputs equals the gradient call's loss
    (same BF16 operands, same FP32 accumulation; nothing near the 6-sigma clip)."""
    import torch

    from paper_1701_02005_gb300.wallmodel import MLP

    rows = 5 * 128 + 37
    net = MLP(rows, seed=11)
    norm = _norm(12)
    norm[2], norm[3] = np.zeros(5, np.float32), np.ones(5, np.float32)   # unit-scale targets
    net.set_normalization(*norm)
    r = seeded.rng(13)
    X = r.standard_normal((rows, 40)).astype(np.float32)
    T = r.standard_normal((rows, 5)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    for _ in range(100):   # towards unit-scale outputs, well inside the clip
        net.train_step(Xd, Td, 1e-3)
    Y = net.forward(Xd).cpu().numpy().astype(np.float64)
    yn = (Y - norm[2]) * norm[3]
    assert np.max(np.abs(yn)) < 5.9
    loss_fused = float(np.mean((yn - (T - norm[2]) * norm[3]) ** 2))
    _, loss = net.gradient(Xd, Td)
    assert abs(loss_fused - loss) <= 1e-5 * loss, (loss_fused, loss)
    # the parity of the fused outputs with the oracle, row by row
    Yr, _ = w.forward(net.params(), X, norm, bf16=True, bf16_act=True)
    assert np.max(np.abs(Y - Yr)) <= 2e-3 * np.max(np.abs(Yr))
    assert net.status() == 0
    net.close()
