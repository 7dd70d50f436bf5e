"""Host-side logic of the wall model that needs no GPU: the residual targets
of the network's potential output, and the feature column that output adds
back (PHI_SKIP), checked against the oracle's feature layout."""
import math

import numpy as np
import torch

from oracle import pnp_oracle as o
from oracle import wall_oracle as w
from tests import seeded


def test_residual_targets_subtract_the_skip_column_from_a_copy():
    from paper_1701_02005_gb300 import wallmodel as wm

    r = seeded.rng(3)
    T = torch.from_numpy(r.standard_normal((7, 5)))
    X = torch.from_numpy(r.standard_normal((7, 40)))
    T0 = T.clone()
    assert wm.residual_targets(T, X, None) is T
    R = wm.residual_targets(T, X, wm.PHI_SKIP)
    j, i = wm.PHI_SKIP
    assert torch.equal(T, T0)   # the labels themselves are untouched
    assert torch.equal(R[:, j], T[:, j] - X[:, i])
    others = [c for c in range(5) if c != j]
    assert torch.equal(R[:, others], T[:, others])


def test_the_skip_column_is_the_first_cells_potential_in_the_wall_frame():
    """Feature column PHI_SKIP[1] of a row is its first cell's phi = Phi - V y_c
    (the top wall's sign flipped), the quantity label column PHI_SKIP[0] holds
    for the filtered fine state."""
    from paper_1701_02005_gb300 import wallmodel as wm

    g = o.Grid(8, 9, 4, 2 * math.pi, math.pi, stretch=1.5)
    prm = o.Params(Re=100.0, lam=0.1, Sc=1.0, V=2.0)
    st = o.initial_state(g, prm, o.IC_PB, seed=7, amp=0.05)
    X = w.wall_features(g, prm, st, 8)
    j, i = wm.PHI_SKIP
    assert j == 2
    P = g.nz * g.nx
    bottom = (st.Phi[0] - prm.V * g.yc[0]).ravel()
    top = -(st.Phi[-1] - prm.V * g.yc[-1]).ravel()
    assert np.allclose(X[:P, i], bottom, rtol=0, atol=1e-14)
    assert np.allclose(X[P:, i], top, rtol=0, atol=1e-14)
    assert np.max(np.abs(X[:, i])) > 1e-3   # not a column of zeros
