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
