"""Pins of the oracle's double-layer coupling (wall-potential offsets and the
ion-flux transfer across the first coarse face).

The transfer conserves ions per column, is idle when the prediction equals the
state's own face flux (which the label pins fix), matches closed forms on
linear profiles, treats the top wall as the bottom wall of the mirror image,
and never takes more than half a cell's ions.  The offsets drive the first
cell's potential to the prediction: on a charge-free state they converge to the
closed form -a / y_c0 of the symmetric grid.
"""
import numpy as np

from oracle import pnp_oracle as o
from oracle import wall_oracle as w
from tests import seeded
from tests.test_oracle_wall import _mirror, _random_wall_state, _symmetric_grid


def _col_content(g, c):
    return np.einsum("jkx,j->kx", c, g.dy)


def _Y(g, seed, scale=0.05):
    return seeded.field(seed, (2 * g.nz * g.nx, 5), scale)


def test_flux_transfer_conserves_ions_per_column_and_touches_four_planes():
    g = o.Grid(8, 13, 4, 2.0, 1.0, stretch=1.7)
    prm = o.Params(Re=80.0, lam=0.1, V=1.0)
    st = _random_wall_state(g, prm, 5)
    for gain in (1.0, 0.4):
        cp, cm = w.wall_flux_fix(g, prm, st, _Y(g, 6), gain, 0.01)
        for new, old in ((cp, st.cp), (cm, st.cm)):
            assert np.allclose(_col_content(g, new), _col_content(g, old), rtol=1e-14, atol=0)
            changed = np.nonzero(np.any(new != old, axis=(1, 2)))[0].tolist()
            assert changed == [0, 1, g.nyc - 2, g.nyc - 1]


def test_flux_transfer_is_idle_at_the_states_own_fluxes():
    # on identical grids the flux labels are the state's own first-face fluxes
    g = o.Grid(8, 11, 4, 2.0, 1.0, stretch=1.5)
    prm = o.Params(Re=50.0, lam=0.1, V=1.0)
    st = _random_wall_state(g, prm, 9)
    Y = _Y(g, 10)
    Y[:, 3:] = w.wall_labels(g, g, prm, st)[:, 3:]
    cp, cm = w.wall_flux_fix(g, prm, st, Y, 1.0, 0.02)
    assert np.allclose(cp, st.cp, rtol=0, atol=1e-15)
    assert np.allclose(cm, st.cm, rtol=0, atol=1e-15)


def test_flux_transfer_closed_form_on_linear_profiles():
    """c+ = 1 + 0.3 y, c- = 2 - 0.7 y at rest carry -0.3 D and +0.7 D in +y.
    A prediction of zero flux (column 3 the counter-ion: c+ at the bottom, c- at
    the top) holds back what diffusion carries towards each wall: 0.3 D gain dt
    of c+ moves from the bottom cell 0 up into cell 1, and 0.7 D gain dt of c-
    from the top cell Nyc-1 down into Nyc-2."""
    g = o.Grid(4, 9, 2, 2.0, 1.0, stretch=1.6)
    prm = o.Params(Re=50.0, lam=0.1, V=0.0, Sc=2.0, Uw=0.0)
    D, P, gain, dt = prm.D, 2 * 4, 0.6, 0.05
    st = o.initial_state(g, prm, o.IC_LAMINAR)
    y = g.yc[:, None, None] * np.ones((g.nyc, g.nz, g.nx))
    st.cp, st.cm, st.Phi = 1.0 + 0.3 * y, 2.0 - 0.7 * y, 0.0 * y
    st.v = np.zeros((g.ny, g.nz, g.nx))
    Y = np.zeros((2 * P, 5))
    # co-ion predictions equal to the state's flux: bottom c- carries +0.7 D, top c+ carries +0.3 D away (= -y)
    Y[:P, 4] = 0.7 * D
    Y[P:, 4] = 0.3 * D
    cp, cm = w.wall_flux_fix(g, prm, st, Y, gain, dt)
    n = g.nyc - 1
    assert np.allclose(cp[0] - st.cp[0], -0.3 * D * gain * dt / g.dy[0], rtol=1e-12)
    assert np.allclose(cp[1] - st.cp[1], +0.3 * D * gain * dt / g.dy[1], rtol=1e-12)
    assert np.allclose(cm[n] - st.cm[n], -0.7 * D * gain * dt / g.dy[n], rtol=1e-12)
    assert np.allclose(cm[n - 1] - st.cm[n - 1], +0.7 * D * gain * dt / g.dy[n - 1], rtol=1e-12)
    # the co-ions were predicted exactly: untouched
    assert np.allclose(cm[:2], st.cm[:2], rtol=0, atol=1e-15)
    assert np.allclose(cp[n - 1:], st.cp[n - 1:], rtol=0, atol=1e-15)


def test_flux_transfer_top_wall_is_the_bottom_wall_of_the_mirror_image():
    g = _symmetric_grid(8, 17, 4, 1.8)
    prm = o.Params(Re=100.0, lam=0.1, V=1.5)
    st = _random_wall_state(g, prm, 21)
    img = _mirror(g, st)
    P = g.nz * g.nx
    Y = _Y(g, 22, 0.2)
    xc = g.nx - 1 - np.arange(g.nx)
    # the image's bottom rows are the original top rows (centred x map), and back
    Yi = np.empty_like(Y)
    Yi[:P] = Y[P:].reshape(g.nz, g.nx, 5)[:, xc].reshape(P, 5)
    Yi[P:] = Y[:P].reshape(g.nz, g.nx, 5)[:, xc].reshape(P, 5)
    cp, cm = w.wall_flux_fix(g, prm, st, Y, 0.8, 0.03)
    cpi, cmi = w.wall_flux_fix(g, prm, img, Yi, 0.8, 0.03)
    assert np.allclose(cpi, cm[::-1][:, :, xc], rtol=1e-13, atol=1e-14)
    assert np.allclose(cmi, cp[::-1][:, :, xc], rtol=1e-13, atol=1e-14)
    assert np.max(np.abs(cp - st.cp)) > 1e-3


def test_flux_transfer_gives_at_most_half_a_cell():
    g = o.Grid(4, 9, 2, 2.0, 1.0, stretch=1.4)
    prm = o.Params(Re=50.0, lam=0.1, V=1.0)
    st = _random_wall_state(g, prm, 31)
    P = g.nz * g.nx
    Y = np.zeros((2 * P, 5))
    Y[:, 3] = 1e6    # far more than any cell holds, away from both walls
    cp, cm = w.wall_flux_fix(g, prm, st, Y, 1.0, 0.01)
    assert np.allclose(cp[0], 0.5 * st.cp[0], rtol=1e-14)   # bottom counter-ion c+ leaves cell 0
    n = g.nyc - 1
    assert np.allclose(cm[n], 0.5 * st.cm[n], rtol=1e-14)   # top counter-ion c- leaves cell Nyc-1
    assert np.allclose(_col_content(g, cp), _col_content(g, st.cp), rtol=1e-14)


def test_offsets_idle_at_the_present_potential_clipped_and_finite():
    g = o.Grid(8, 9, 4, 2.0, 1.0, stretch=1.5)
    prm = o.Params(Re=50.0, lam=0.1, V=1.0)
    st = _random_wall_state(g, prm, 41)
    nc = 3
    X = w.wall_features(g, prm, st, nc)
    P = g.nz * g.nx
    B0, T0 = seeded.field(42, (g.nz, g.nx), 0.1), seeded.field(43, (g.nz, g.nx), 0.1)
    Y = _Y(g, 44)
    Y[:, 2] = X[:, 4 * nc]
    B, T = w.edl_offsets(g, X, Y, nc, 0.7, B0, T0, 1.0)
    assert np.array_equal(B, B0) and np.array_equal(T, T0)
    # with a lift the present potential is the feature plus the lift
    lift = seeded.field(45, (g.nyc, g.nz, g.nx), 0.1)
    Y2 = Y.copy()
    Y2[:P, 2] = X[:P, 4 * nc] + lift[0].ravel()
    Y2[P:, 2] = X[P:, 4 * nc] - lift[g.nyc - 1].ravel()
    B, T = w.edl_offsets(g, X, Y2, nc, 0.7, B0, T0, 1.0, lift)
    assert np.allclose(B, B0, rtol=0, atol=1e-15) and np.allclose(T, T0, rtol=0, atol=1e-15)
    Y[:, 2] = X[:, 4 * nc] + 100.0
    Y[0, 2] = np.nan
    B, T = w.edl_offsets(g, X, Y, nc, 1.0, B0, T0, 1.0)
    assert B.ravel()[0] == B0.ravel()[0]
    assert np.all(B.ravel()[1:] == 1.0) and np.all(T == -1.0)   # the top wall's sign flips back
    assert P == B.size


def test_offsets_converge_to_the_closed_form_on_a_charge_free_state():
    """Neutral uniform ions carry no charge, so Phi is the linear blend of the wall
    potentials: the first-cell perturbations are (1 - y0)/2 dB + (1 + y0)/2 dT at
    the bottom and minus the mirror at the top.  Asking both walls (wall frame)
    for a gives dB = -a / y0, dT = a / y0 on the symmetric grid."""
    g = _symmetric_grid(8, 17, 4, 1.8)
    prm0 = o.Params(Re=100.0, lam=0.1, V=1.5)
    st = o.initial_state(g, prm0, o.IC_LAMINAR)
    st.cp = np.ones((g.nyc, g.nz, g.nx))
    st.cm = np.ones((g.nyc, g.nz, g.nx))
    a, nc, P = 0.25, 2, g.nz * g.nx
    B, T = np.zeros((g.nz, g.nx)), np.zeros((g.nz, g.nx))
    for it in range(40):
        prm = o.Params(Re=100.0, lam=0.1, V=1.5, wall=(-prm0.V + B, prm0.V + T))
        st.Phi = o.potential_from_ions(g, prm, st.cp, st.cm)
        lift = w.offsets_lift(g, prm0, B, T)
        X = w.wall_features(g, prm0, st, nc, lift)   # what the network sees: no ions, no charge
        assert np.allclose(X[:, 4 * nc], 0.0, atol=1e-13)
        Y = np.zeros((2 * P, 5))
        Y[:, 2] = a
        B, T = w.edl_offsets(g, X, Y, nc, 1.0, B, T, 4.0, lift)
    y0 = g.yc[0]
    assert np.allclose(B, -a / y0, rtol=1e-12)
    assert np.allclose(T, a / y0, rtol=1e-12)
    # the total first-cell potential reached the prediction
    Xt = w.wall_features(g, prm0, st, nc)
    assert np.allclose(Xt[:, 4 * nc], a, rtol=1e-12)


def test_offsets_lift_is_the_charge_free_potential_of_the_offsets():
    """Uniform offsets give the linear blend (1 - y)/2 dB + (1 + y)/2 dT exactly;
    and the lift is linear in the offsets."""
    g = o.Grid(8, 13, 4, 2.0, 1.0, stretch=1.6)
    prm = o.Params(Re=50.0, lam=0.1, V=1.0)
    L = w.offsets_lift(g, prm, 0.3 * np.ones((g.nz, g.nx)), -0.2 * np.ones((g.nz, g.nx)))
    y = g.yc[:, None, None]
    assert np.allclose(L, 0.5 * (1 - y) * 0.3 + 0.5 * (1 + y) * -0.2 + 0 * L, rtol=0, atol=1e-13)
    B1, T1 = seeded.field(51, (g.nz, g.nx), 0.2), seeded.field(52, (g.nz, g.nx), 0.2)
    B2, T2 = seeded.field(53, (g.nz, g.nx), 0.2), seeded.field(54, (g.nz, g.nx), 0.2)
    assert np.allclose(w.offsets_lift(g, prm, B1 + B2, T1 + T2),
                       w.offsets_lift(g, prm, B1, T1) + w.offsets_lift(g, prm, B2, T2), rtol=0, atol=1e-12)
