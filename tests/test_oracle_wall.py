"""Pins of the wall-model oracle (network, restriction, features, labels).

GELU against its closed-form values and a numerical derivative, backprop
against central finite differences, BF16 rounding against exactly
representable cases, restriction conserving volume integrals, and labels of
states whose answers are fixed: laminar Couette needs no slip, a discrete
Boltzmann state carries no ion flux, identical grids give the identity.
"""
import math

import numpy as np
import pytest

from oracle import pnp_oracle as o
from oracle import wall_oracle as w
from tests import seeded


def test_gelu_closed_forms():
    z = np.array([0.0, 1.0, -1.0, 10.0, -10.0])
    g = w.gelu(z)
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) < 1e-15           # Phi(1)
    assert abs(g[2] + 0.15865525393145707) < 1e-15          # -Phi(-1)
    assert abs(g[3] - 10.0) < 1e-15 and abs(g[4]) < 1e-20
    assert w.gelu_d(np.array([0.0]))[0] == 0.5
    zz = np.linspace(-4, 4, 33)
    hh = 1e-6
    fd = (w.gelu(zz + hh) - w.gelu(zz - hh)) / (2 * hh)
    assert np.max(np.abs(fd - w.gelu_d(zz))) < 1e-8


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, math.pi, -2.5, 0.0], dtype=np.float32)
    r = w.bf16_round(vals)
    assert list(r) == [1.0, 1.0, 1.0 + 2 ** -6, 3.140625, -2.5, 0.0]


def _norm(seed):
    r = seeded.rng(seed)
    return (r.normal(size=40), r.uniform(0.5, 2, 40), r.normal(size=5), r.uniform(0.5, 2, 5))


def test_mlp_gradient_matches_finite_differences():
    _, total = w.param_slices()
    assert total == 40 * 128 + 128 + 3 * (128 * 128 + 128) + 128 * 5 + 5
    r = seeded.rng(3)
    p = 0.2 * r.standard_normal(total)
    X = r.standard_normal((12, 40))
    T = r.standard_normal((12, 5))
    norm = _norm(4)
    loss, g = w.loss_and_grad(p, X, T, norm, bf16=False)
    idx = r.choice(total, 40, replace=False)
    idx = np.concatenate([idx, [0, 5119, 5120 + 5, total - 1, total - 6]])
    for i in idx:
        e = np.zeros(total)
        e[i] = 1e-6
        lp, _ = w.loss_and_grad(p + e, X, T, norm, bf16=False)
        lm, _ = w.loss_and_grad(p - e, X, T, norm, bf16=False)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_residual_output_adds_the_input_column():
    """skip = (j, i): with zero parameters every output is its shift, and output j
    the shift plus the raw input x_i; the loss is the mean squared normalised
    difference of the physical outputs and the targets (so the target of the
    network's own value is t_j - x_i), and its gradient matches finite differences."""
    _, total = w.param_slices()
    r = seeded.rng(5)
    X = r.standard_normal((9, 40))
    T = r.standard_normal((9, 5))
    norm = _norm(6)
    y0, _ = w.forward(np.zeros(total), X, norm, bf16=False, skip=(2, 32))
    want = np.tile(norm[2], (9, 1))
    want[:, 2] += X[:, 32]
    assert np.allclose(y0, want, rtol=0, atol=1e-15)
    p = 0.2 * r.standard_normal(total)
    y, _ = w.forward(p, X, norm, bf16=False, skip=(2, 32))
    y_plain, _ = w.forward(p, X, norm, bf16=False)
    assert np.allclose(np.delete(y, 2, 1), np.delete(y_plain, 2, 1), rtol=0, atol=0)
    loss, g = w.loss_and_grad(p, X, T, norm, bf16=False, skip=(2, 32))
    direct = lambda q: float(np.mean(((w.forward(q, X, norm, bf16=False, skip=(2, 32))[0] - T) * norm[3]) ** 2))
    assert abs(loss - direct(p)) <= 1e-12 * loss
    assert abs(loss - w.loss_and_grad(p, X, T, norm, bf16=False)[0]) > 1e-3 * loss   # the skip matters
    for i in np.concatenate([r.choice(total, 12, replace=False), [total - 3]]):   # total - 3: output 2's bias
        e = np.zeros(total)
        e[i] = 1e-6
        fd = (direct(p + e) - direct(p - e)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = w.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-7)


def _grids():
    gf = o.Grid(16, 33, 8, 2 * math.pi, math.pi, stretch=2.0)
    gc = o.Grid(8, 9, 4, 2 * math.pi, math.pi, y_faces=gf.yf[::4])
    return gf, gc


def test_restriction_conserves_volume_integrals():
    gf, gc = _grids()
    q = seeded.field(7, (gf.nyc, gf.nz, gf.nx))
    qc = w.restrict(gf, gc, q)
    assert abs(np.sum(qc * gc.cell_volume()) - np.sum(q * gf.cell_volume())) <= 1e-12 * np.sum(np.abs(q))
    assert np.allclose(w.restrict(gf, gc, np.full_like(q, 2.5)), 2.5, atol=1e-15)


def test_features_of_laminar_couette():
    gf, gc = _grids()
    prm = o.Params(Re=100.0, lam=0.1, V=0.0)
    st = o.initial_state(gc, prm, o.IC_LAMINAR)
    X = w.wall_features(gc, prm, st, 8)
    for d in range(8):
        assert np.allclose(X[:, d], gc.yc[d] + 1.0, atol=1e-14)   # u relative to the wall
    assert np.allclose(X[:, 16:32], 1.0) and np.allclose(X[:, 32:40], 0.0, atol=1e-14)


def test_labels_laminar_shear_and_rest_has_no_flux():
    gf, gc = _grids()
    prm = o.Params(Re=100.0, lam=0.1, V=0.0)
    st = o.initial_state(gf, prm, o.IC_LAMINAR)
    T = w.wall_labels(gf, gc, prm, st)
    # Couette u = y: wall shear rate exactly 1 in the wall frame at both walls, w = 0
    assert np.max(np.abs(T[:, 0] - 1.0)) <= 1e-13 and np.max(np.abs(T[:, 1])) <= 1e-14
    assert np.max(np.abs(T[:, 3:])) <= 1e-14
    # discrete Boltzmann ions at rest: zero total flux through every interior face
    prm2 = o.Params(Re=1.0, lam=0.1, V=1.0, Uw=0.0)
    Phi1 = 0.3 * np.cumsum(seeded.field(8, gf.nyc))
    cols = {}
    for s in (1.0, -1.0):
        c = np.empty(gf.nyc)
        c[0] = 1.2
        for j in range(1, gf.nyc):
            d = Phi1[j] - Phi1[j - 1]
            c[j] = c[j - 1] * (2 - s * d) / (2 + s * d)
        cols[s] = c[:, None, None] * np.ones((1, gf.nz, gf.nx))
    st2 = o.initial_state(gf, prm2, o.IC_LAMINAR)
    st2.cp, st2.cm = cols[1.0], cols[-1.0]
    st2.Phi = Phi1[:, None, None] * np.ones((1, gf.nz, gf.nx))
    T2 = w.wall_labels(gf, gc, prm2, st2)
    assert np.max(np.abs(T2[:, 3:])) <= 1e-12 * np.max(np.abs(cols[1.0]))


def test_labels_identity_on_identical_grids():
    # on identical grids the label shear rate is the first-cell value over h_0
    g = o.Grid(8, 9, 4, 2.0, 1.0, stretch=1.5)
    prm = o.Params(Re=50.0, lam=0.1, V=1.0)
    st = o.initial_state(g, prm, o.IC_PB, seed=2, amp=0.1)
    T = w.wall_labels(g, g, prm, st)
    X = w.wall_features(g, prm, st, 1)
    assert np.allclose(T[:, 0], X[:, 0] / g.h[0], rtol=1e-13)
    assert np.allclose(T[:, 1], X[:, 1] / g.h[0], rtol=1e-13, atol=1e-14)
    assert np.allclose(T[:, 2], X[:, 4], atol=1e-14)   # first-cell phi


# ---------------------------------------------------------------------------
# Top-wall mapping and the sign / species of the ion-flux labels
# ---------------------------------------------------------------------------
def _symmetric_grid(nx, ny, nz, stretch):
    """tanh faces made exactly antisymmetric, so that the mirror image of a
    state lives on the same grid to the last bit."""
    g = o.Grid(nx, ny, nz, 2 * math.pi, math.pi, stretch=stretch)
    yf = 0.5 * (g.yf - g.yf[::-1])
    return o.Grid(nx, ny, nz, 2 * math.pi, math.pi, y_faces=yf)


def _mirror(g, st):
    """Image of a state under the half turn about the z-axis, (x, y) -> (-x, -y),
    with c+ <-> c- and Phi -> -Phi: it maps the top wall (speed +Uw, potential
    +V) onto the bottom one (-Uw, -V), so the image solves the same problem.
    x: centres i -> nx-1-i, x-faces i -> (nx-i) mod nx; y: cells j -> nyc-1-j,
    faces j -> ny-1-j; z unchanged.  u and v change sign, w does not."""
    xc = (g.nx - 1 - np.arange(g.nx))
    xf = (g.nx - np.arange(g.nx)) % g.nx
    img = st.copy()
    img.u = -st.u[::-1][:, :, xf]
    img.v = -st.v[::-1][:, :, xc]
    img.w = st.w[::-1][:, :, xc]
    img.cp = st.cm[::-1][:, :, xc]
    img.cm = st.cp[::-1][:, :, xc]
    img.Phi = -st.Phi[::-1][:, :, xc]
    return img


def _random_wall_state(g, prm, seed):
    shp = (g.nyc, g.nz, g.nx)
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    st.u = seeded.field(seed, shp, 0.3) + g.yc[:, None, None]
    st.v = seeded.wall_zero_faces(seed + 1, (g.ny, g.nz, g.nx), 0.1)
    st.w = seeded.field(seed + 2, shp, 0.2)
    st.cp = seeded.positive_field(seed + 3, shp, 0.5, 2.0)
    st.cm = seeded.positive_field(seed + 4, shp, 0.2, 3.0)
    st.Phi = prm.V * g.yc[:, None, None] + seeded.field(seed + 5, shp, 0.4)
    return st


def test_top_wall_features_are_the_bottom_features_of_the_mirror_image():
    g = _symmetric_grid(8, 17, 4, 1.8)
    prm = o.Params(Re=100.0, lam=0.1, V=1.5)
    st = _random_wall_state(g, prm, 61)
    img = _mirror(g, st)
    nc = 6
    X = w.wall_features(g, prm, st, nc)
    Xi = w.wall_features(g, prm, img, nc)
    P = g.nz * g.nx
    top = X[P:].reshape(g.nz, g.nx, 5 * nc)
    bot_img = Xi[:P].reshape(g.nz, g.nx, 5 * nc)
    xc = g.nx - 1 - np.arange(g.nx)
    xf = (g.nx - np.arange(g.nx)) % g.nx
    # u (x-faces) maps its own way in x; the centred quantities another
    assert np.allclose(top[:, :, :nc], bot_img[:, xf, :nc], rtol=0, atol=1e-14)
    assert np.allclose(top[:, :, nc:], bot_img[:, xc, nc:], rtol=0, atol=1e-14)
    # the mapping is not trivially satisfied: the species and the sign matter
    assert np.max(np.abs(top[:, :, 2 * nc:3 * nc] - top[:, :, 3 * nc:4 * nc])) > 0.1
    assert np.max(np.abs(top[:, :, 4 * nc:])) > 0.1


def test_top_wall_labels_are_the_bottom_labels_of_the_mirror_image():
    gf = _symmetric_grid(8, 33, 8, 1.8)
    gc = o.Grid(8, 9, 4, 2 * math.pi, math.pi, y_faces=gf.yf[::4])   # rx = 1 keeps the x-face map block-aligned
    prm = o.Params(Re=100.0, lam=0.1, V=1.5)
    st = _random_wall_state(gf, prm, 71)
    img = _mirror(gf, st)
    T = w.wall_labels(gf, gc, prm, st)
    Ti = w.wall_labels(gf, gc, prm, img)
    Pc = gc.nz * gc.nx
    top = T[Pc:].reshape(gc.nz, gc.nx, 5)
    bot_img = Ti[:Pc].reshape(gc.nz, gc.nx, 5)
    xc = gc.nx - 1 - np.arange(gc.nx)
    xf = (gc.nx - np.arange(gc.nx)) % gc.nx
    assert np.allclose(top[:, :, 0], bot_img[:, xf, 0], rtol=1e-13, atol=1e-13)
    assert np.allclose(top[:, :, 1:], bot_img[:, xc, 1:], rtol=1e-13, atol=1e-13)
    assert np.max(np.abs(top[:, :, 3] - top[:, :, 4])) > 1e-3


def test_flux_labels_of_linear_profiles_have_closed_forms():
    """Uniform gradients give face fluxes known in closed form: diffusion of
    c = a + b y carries -D b in +y, migration in Phi = E y carries -/+ D c E
    for c+/c-, advection by a uniform v carries v c.  Column 3 is the counter-
    ion (c- at the top wall, held at +V), column 4 the co-ion, both counted
    away from their wall; distinct values per species catch a swap."""
    gf = o.Grid(8, 33, 4, 2 * math.pi, math.pi, stretch=1.6)
    gc = o.Grid(4, 9, 2, 2 * math.pi, math.pi, y_faces=gf.yf[::4])
    shp = (gf.nyc, gf.nz, gf.nx)
    prm = o.Params(Re=50.0, lam=0.1, V=0.0, Sc=2.0, Uw=0.0)
    D = prm.D
    P = gc.nz * gc.nx

    def labels(cp, cm, Phi, v0=0.0):
        st = o.initial_state(gf, prm, o.IC_LAMINAR)
        st.u[...] = 0.0
        st.cp, st.cm, st.Phi = cp, cm, Phi
        st.v = np.zeros((gf.ny, gf.nz, gf.nx))
        st.v[1:-1] = v0
        T = w.wall_labels(gf, gc, prm, st)
        return T[:P], T[P:]

    ones = np.ones(shp)
    y = gf.yc[:, None, None] * ones
    # diffusion: c+ = 1 + 0.3 y, c- = 2 - 0.7 y
    bot, top = labels(1.0 + 0.3 * y, 2.0 - 0.7 * y, 0.0 * ones)
    assert np.allclose(bot[:, 3], -D * 0.3, rtol=1e-12) and np.allclose(bot[:, 4], -D * -0.7, rtol=1e-12)
    assert np.allclose(top[:, 3], +D * -0.7, rtol=1e-12) and np.allclose(top[:, 4], +D * 0.3, rtol=1e-12)
    # migration in a uniform field E = 0.4 with c+ = 1.5, c- = 0.5
    E = 0.4
    bot, top = labels(1.5 * ones, 0.5 * ones, E * y)
    assert np.allclose(bot[:, 3], -D * 1.5 * E, rtol=1e-12) and np.allclose(bot[:, 4], +D * 0.5 * E, rtol=1e-12)
    assert np.allclose(top[:, 3], -D * 0.5 * E, rtol=1e-12) and np.allclose(top[:, 4], +D * 1.5 * E, rtol=1e-12)
    # advection by v = 0.05 with c+ = 1.5, c- = 0.5
    bot, top = labels(1.5 * ones, 0.5 * ones, 0.0 * ones, v0=0.05)
    assert np.allclose(bot[:, 3], 0.05 * 1.5, rtol=1e-12) and np.allclose(bot[:, 4], 0.05 * 0.5, rtol=1e-12)
    assert np.allclose(top[:, 3], -0.05 * 0.5, rtol=1e-12) and np.allclose(top[:, 4], -0.05 * 1.5, rtol=1e-12)


def test_bf16_operand_reading_is_exact_on_representable_values():
    # with weights, inputs and every intermediate GEMM operand exactly
    # representable in BF16 the BF16-operand reading equals the exact network;
    # on random values it differs by the BF16 rounding of the operands only
    _, total = w.param_slices()
    p = np.zeros(total)
    sl, _ = w.param_slices()
    r = seeded.rng(11)
    for ws, bs, fi, fo in sl:   # weights k / 8 (k small), zero biases
        p[ws] = r.integers(-2, 3, size=ws.stop - ws.start) / 8.0
    X = r.integers(-2, 3, size=(6, 40)).astype(np.float64)
    norm = (np.zeros(40), np.ones(40), np.zeros(5), np.ones(5))
    # the first layer's pre-activations are small integers / 8: representable;
    # GELU of them is not, so compare only the first layer's GEMM
    _, (ins_a, zs_a, _) = w.forward(p, X, norm, bf16=True, bf16_act=True)
    _, (ins_b, zs_b, _) = w.forward(p, X, norm, bf16=True, bf16_act=False)
    assert np.array_equal(zs_a[0], zs_b[0])
    # random values: the two readings agree to the BF16 operand rounding
    p2 = 0.1 * r.standard_normal(total)
    X2 = r.standard_normal((20, 40))
    ya, _ = w.forward(p2, X2, norm, bf16=True, bf16_act=True)
    yb, _ = w.forward(p2, X2, norm, bf16=True, bf16_act=False)
    rel = np.max(np.abs(ya - yb)) / np.max(np.abs(yb))
    assert 0 < rel < 3e-2, rel
    la, ga = w.loss_and_grad(p2, X2, X2[:, :5], norm, bf16=True, bf16_act=True)
    lb, gb = w.loss_and_grad(p2, X2, X2[:, :5], norm, bf16=True, bf16_act=False)
    assert abs(la - lb) <= 3e-2 * lb and np.max(np.abs(ga - gb)) <= 5e-2 * np.max(np.abs(gb))
