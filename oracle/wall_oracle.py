"""FP64 NumPy oracle of the learned wall model's data and network (TEST
INFRASTRUCTURE ONLY; see oracle/__init__.py).

The paper resolves the double layer and has no wall model; this restates the
definitions the CUDA kernels implement, in plain array code: restriction of a
fine state onto a coarse grid made of every ry-th y-face and rx x rz cell
blocks, near-wall feature columns in the wall frame (rotation (x, y) -> (-x,
-y) with c+ <-> c-, Phi -> -Phi maps the top wall onto the bottom), training
labels (filtered fine wall shear rates, first-cell potential perturbation,
ion fluxes through the first coarse face), the double-layer coupling that
imposes the predicted first-cell potential (wall-potential offsets) and ion
fluxes (conservative transfers across the first face), and the
MLP 40 -> 128 x 4 -> 5 with erf-GELU, MSE loss on normalised outputs,
backpropagation and Adam.  Pinned by tests/test_oracle_wall.py.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .pnp_oracle import Grid  # noqa: F401  (grids are the oracle's)

LAYERS = [(40, 128), (128, 128), (128, 128), (128, 128), (128, 5)]


def ratios(gf, gc):
    return gf.nx // gc.nx, gf.nyc // gc.nyc, gf.nz // gc.nz


def restrict(gf, gc, q, vfield=False):
    rx, ry, rz = ratios(gf, gc)
    if vfield:
        qq = q[::ry].reshape(gc.ny, gc.nz, rz, gc.nx, rx)
        return qq.mean(axis=(2, 4))
    qq = q.reshape(gc.nyc, ry, gc.nz, rz, gc.nx, rx)
    w = gf.dy.reshape(gc.nyc, ry)
    num = (qq.sum(axis=(3, 5)) * w[:, :, None, None]).sum(axis=1)
    return num / (w.sum(axis=1) * rx * rz)[:, None, None]


def wall_features(g, prm, st, ncells=8, lift=None):
    """Feature rows; lift (cells, optional): the charge-free potential of wall-model
    offsets, left out of the potential column."""
    P = g.nz * g.nx
    X = np.empty((2 * P, 5 * ncells))
    phi = st.Phi - prm.V * g.yc[:, None, None]
    if lift is not None:
        phi = phi - lift
    for wall in (0, 1):
        for d in range(ncells):
            j = d if wall == 0 else g.nyc - 1 - d
            ur = st.u[j] + prm.Uw if wall == 0 else prm.Uw - st.u[j]
            rows = slice(wall * P, (wall + 1) * P)
            X[rows, 0 * ncells + d] = ur.ravel()
            X[rows, 1 * ncells + d] = st.w[j].ravel()
            X[rows, 2 * ncells + d] = (st.cp[j] if wall == 0 else st.cm[j]).ravel()
            X[rows, 3 * ncells + d] = (st.cm[j] if wall == 0 else st.cp[j]).ravel()
            X[rows, 4 * ncells + d] = (phi[j] if wall == 0 else -phi[j]).ravel()
    return X


def _block_mean(gf, gc, a2d):
    rx, _, rz = ratios(gf, gc)
    return a2d.reshape(gc.nz, rz, gc.nx, rx).mean(axis=(1, 3))


def wall_labels(gf, gc, prm, st):
    rx, ry, rz = ratios(gf, gc)
    Pc = gc.nz * gc.nx
    T = np.empty((2 * Pc, 5))
    D = prm.D
    for wall in (0, 1):
        sl = slice(0, ry) if wall == 0 else slice(gf.nyc - ry, gf.nyc)
        w = gf.dy[sl]
        urel = st.u + prm.Uw if wall == 0 else prm.Uw - st.u
        phi = st.Phi - prm.V * gf.yc[:, None, None]
        phi = phi if wall == 0 else -phi

        def first_cell(q):
            qq = q[sl].reshape(ry, gc.nz, rz, gc.nx, rx).sum(axis=(2, 4))
            return (qq * w[:, None, None]).sum(axis=0) / (w.sum() * rx * rz)

        pa = first_cell(phi)
        j0 = 0 if wall == 0 else gf.nyc - 1
        hw = gf.h[0] if wall == 0 else gf.h[gf.nyc]
        gu = _block_mean(gf, gc, urel[j0] / hw)
        gw = _block_mean(gf, gc, st.w[j0] / hw)
        jf = ry if wall == 0 else gf.nyc - ry
        a, b = jf - 1, jf
        dP = (st.Phi[b] - st.Phi[a]) / gf.h[jf]
        cpf, cmf = 0.5 * (st.cp[a] + st.cp[b]), 0.5 * (st.cm[a] + st.cm[b])
        Fp = st.v[jf] * cpf - D * ((st.cp[b] - st.cp[a]) / gf.h[jf] + cpf * dP)
        Fm = st.v[jf] * cmf - D * ((st.cm[b] - st.cm[a]) / gf.h[jf] - cmf * dP)
        f3, f4 = (Fp, Fm) if wall == 0 else (-Fm, -Fp)
        rows = slice(wall * Pc, (wall + 1) * Pc)
        T[rows, 0] = gu.ravel()
        T[rows, 1] = gw.ravel()
        T[rows, 2] = pa.ravel()
        T[rows, 3] = _block_mean(gf, gc, f3).ravel()
        T[rows, 4] = _block_mean(gf, gc, f4).ravel()
    return T


# ---------------------------------------------------------------------------
# Double-layer coupling: the network's columns 2-4 imposed on a coarse state
# ---------------------------------------------------------------------------
def offsets_lift(g, prm, B, T):
    """The charge-free potential of wall offsets B, T (lab frame) on top of the
    uniform walls: the potential of no ions between walls -V + B, V + T less that
    between -V, V (the solution is linear in the wall data)."""
    from .pnp_oracle import Params, potential_from_ions
    zero = np.zeros((g.nyc, g.nz, g.nx))
    pw = Params(Re=prm.Re, lam=prm.lam, Sc=prm.Sc, V=prm.V, beta=prm.beta, Uw=prm.Uw,
                wall=(-prm.V + np.asarray(B), prm.V + np.asarray(T)))
    p0 = Params(Re=prm.Re, lam=prm.lam, Sc=prm.Sc, V=prm.V, beta=prm.beta, Uw=prm.Uw)
    return potential_from_ions(g, pw, zero, zero) - potential_from_ions(g, p0, zero, zero)


def edl_offsets(g, X, Y, ncells, gain, B, T, lim, lift=None):
    """Wall-potential offsets (lab frame, on top of the uniform walls -V, +V)
    after one update: each wall column's offset moves by gain (phi_pred - phi_1),
    phi_pred column 2 of the prediction (wall frame: the top wall's sign flips
    back) and phi_1 the first cell's present potential perturbation: the feature
    row's value (which leaves the offsets' lift out) plus lift (the offsets'
    charge-free potential, cells; none: zero); clipped to +-lim, a non-finite step
    leaves the offset alone."""
    P = g.nz * g.nx
    lb = np.zeros(P) if lift is None else lift[0].ravel()
    lt = np.zeros(P) if lift is None else -lift[g.nyc - 1].ravel()   # wall frame
    db = gain * (Y[:P, 2].astype(np.float64) - (X[:P, 4 * ncells].astype(np.float64) + lb))
    dt = gain * (Y[P:, 2].astype(np.float64) - (X[P:, 4 * ncells].astype(np.float64) + lt))
    Bn, Tn = np.asarray(B, dtype=np.float64).ravel().copy(), np.asarray(T, dtype=np.float64).ravel().copy()
    okb, okt = np.isfinite(db), np.isfinite(dt)
    Bn[okb] = np.clip(Bn[okb] + db[okb], -lim, lim)
    Tn[okt] = np.clip(Tn[okt] - dt[okt], -lim, lim)
    return Bn.reshape(g.nz, g.nx), Tn.reshape(g.nz, g.nx)


def face_fluxes(g, prm, st, jf):
    """Total ion fluxes (lab frame, +y) through interior y-face jf, the labels'
    discrete form F = v c_f - D (dc/dy + s c_f dPhi/dy), c_f the face mean."""
    a, b = jf - 1, jf
    dP = (st.Phi[b] - st.Phi[a]) / g.h[jf]
    cpf, cmf = 0.5 * (st.cp[a] + st.cp[b]), 0.5 * (st.cm[a] + st.cm[b])
    Fp = st.v[jf] * cpf - prm.D * ((st.cp[b] - st.cp[a]) / g.h[jf] + cpf * dP)
    Fm = st.v[jf] * cmf - prm.D * ((st.cm[b] - st.cm[a]) / g.h[jf] - cmf * dP)
    return Fp, Fm


def wall_flux_fix(g, prm, st, Y, gain, dt):
    """c+, c- after one ion-flux transfer: across the first interior face of each
    wall column (face 1 at the bottom, Nyc-1 at the top) the flux grows by
    gain (F_pred - F) (F_pred columns 3, 4 of the prediction in the wall frame)
    for a time dt, moving ions from one of the two cells sharing the face to the
    other; the cell that gives ions gives at most half of them."""
    if g.nyc < 4:
        raise ValueError("the two walls' transfers need disjoint cells (Nyc >= 4)")
    P = g.nz * g.nx
    cp, cm = st.cp.copy(), st.cm.copy()
    for wall in (0, 1):
        jf = 1 if wall == 0 else g.nyc - 1
        a, b = jf - 1, jf
        Fp, Fm = face_fluxes(g, prm, st, jf)
        y = Y[wall * P:(wall + 1) * P].astype(np.float64).reshape(g.nz, g.nx, 5)
        if wall == 0:
            dFp, dFm = gain * (y[..., 3] - Fp), gain * (y[..., 4] - Fm)
        else:   # wall frame: away from the top wall is -y, and its column 3 is c-
            dFm, dFp = -gain * (y[..., 3] + Fm), -gain * (y[..., 4] + Fp)
        for c, dF in ((cp, dFp), (cm, dFm)):
            dF = np.where(np.isfinite(dF), dF, 0.0)
            cap = np.where(dF > 0, 0.5 * np.maximum(c[a], 0.0) * g.dy[a] / dt,
                           0.5 * np.maximum(c[b], 0.0) * g.dy[b] / dt)
            dF = np.clip(dF, -cap, cap)
            c[a] = c[a] - dF * dt / g.dy[a]
            c[b] = c[b] + dF * dt / g.dy[b]
    return cp, cm


# ---------------------------------------------------------------------------
# MLP
# ---------------------------------------------------------------------------
def param_slices():
    out, off = [], 0
    for fi, fo in LAYERS:
        w = slice(off, off + fi * fo)
        off += fi * fo
        b = slice(off, off + fo)
        off += fo
        out.append((w, b, fi, fo))
    return out, off


def bf16_round(p):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(p, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _weights(p, bf16):
    sl, _ = param_slices()
    Ws, bs = [], []
    for w, b, fi, fo in sl:
        W = np.asarray(p[w], dtype=np.float64).reshape(fo, fi)
        Ws.append(bf16_round(p[w]).reshape(fo, fi) if bf16 else W)
        bs.append(np.asarray(p[b], dtype=np.float64))
    return Ws, bs


def forward(p, X, norm, bf16=True, bf16_act=False, skip=None):
    """Physical outputs and the cache for backpropagation.  bf16: the GEMMs use
    BF16-rounded weights; bf16_act: their activation operands are rounded to
    BF16 as well (tensor-core GEMMs take both operands in BF16 and accumulate
    in FP32); biases, GELU and the accumulation stay FP64 here.  skip = (j, i):
    output j is the network's value plus the raw input column i (a residual
    output: the network learns y_j - x_i)."""
    in_shift, in_scale, out_shift, out_scale = (np.asarray(a, dtype=np.float64) for a in norm)
    Ws, bs = _weights(p, bf16)
    a = (np.asarray(X, dtype=np.float64) - in_shift) * in_scale
    ins, zs = [], []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        x = a if l == 0 else gelu(zs[-1])
        if bf16_act:
            x = bf16_round(x)
        ins.append(x)
        zs.append(x @ W.T + b)
    y = zs[-1] / out_scale + out_shift
    if skip is not None:
        y[:, skip[0]] += np.asarray(X, dtype=np.float64)[:, skip[1]]
    return y, (ins, zs, Ws)


def loss_and_grad(p, X, T, norm, bf16=True, bf16_act=False, skip=None):
    """MSE of normalised outputs and its gradient w.r.t. the parameter vector
    (w.r.t. the weights the forward pass used).  bf16_act: the backward GEMMs
    take the output gradients dz in BF16 as well (the weight gradient pairs
    them with the BF16 layer inputs; the bias gradient sums them).  skip: as in
    forward; the normalisation of output j then applies to y_j - x_i."""
    _, _, out_shift, out_scale = (np.asarray(a, dtype=np.float64) for a in norm)
    _, (ins, zs, Ws) = forward(p, X, norm, bf16, bf16_act, skip)
    y = np.array(T, dtype=np.float64)
    if skip is not None:
        y[:, skip[0]] -= np.asarray(X, dtype=np.float64)[:, skip[1]]
    tn = (y - out_shift) * out_scale
    e = zs[-1] - tn
    n = e.size
    loss = float(np.sum(e * e) / n)
    sl, total = param_slices()
    g = np.zeros(total)
    dz = 2.0 * e / n
    for l in range(len(LAYERS) - 1, -1, -1):
        w, b, fi, fo = sl[l]
        dzo = bf16_round(dz) if bf16_act else dz
        g[w] = (dzo.T @ ins[l]).ravel()
        g[b] = dzo.sum(axis=0)
        if l > 0:
            dz = (dzo @ Ws[l]) * gelu_d(zs[l - 1])
    return loss, g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
