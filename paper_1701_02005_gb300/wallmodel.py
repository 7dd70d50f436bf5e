"""Learned double-layer wall model: the MLP of libpnp (pnp_mlp_* in include/pnp.h)
with torch-owned workspace, and the data calls that couple it to solver contexts."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B

N_IN, N_OUT = 40, 5


def _fp(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


class MLP:
    def __init__(self, max_batch, seed=1705, device=0, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        nb = C.c_size_t()
        B.check(B.pnp_mlp_workspace_bytes(int(max_batch), C.byref(nb)), "pnp_mlp_workspace_bytes")
        self.ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        # the network's stream clears and then owns the workspace: it must come after
        # whatever torch still has queued on that memory (a block freed a moment ago,
        # such as the temporary of a reduction still running, may be handed out here)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.ws.record_stream(self.stream)
        m = C.c_void_p()
        B.check(B.pnp_mlp_create(C.byref(m), int(max_batch), C.c_void_p(self.ws.data_ptr() + off),
                                 C.c_size_t(int(nb.value)), C.c_void_p(self.stream.cuda_stream), C.c_uint64(seed)),
                "pnp_mlp_create")
        self.m = m
        self.max_batch = int(max_batch)
        n = C.c_size_t()
        B.check(B.pnp_mlp_param_count(C.byref(n)), "pnp_mlp_param_count")
        self.nparam = int(n.value)
        self.skip = None

    def params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        B.check(B.pnp_mlp_get_params(self.m, out.ctypes.data_as(C.POINTER(C.c_float)), self.nparam),
                "pnp_mlp_get_params")
        return out

    def set_params(self, p):
        a, ptr = _fp(p)
        B.check(B.pnp_mlp_set_params(self.m, ptr, a.size), "pnp_mlp_set_params")

    def set_normalization(self, in_shift, in_scale, out_shift, out_scale):
        arrs = [_fp(x) for x in (in_shift, in_scale, out_shift, out_scale)]
        B.check(B.pnp_mlp_set_normalization(self.m, *[p for _, p in arrs]), "pnp_mlp_set_normalization")

    def set_skip(self, out_col, in_col):
        """Residual output: output out_col = the network's value + input column in_col
        (out_col < 0: none); the output normalisation of out_col then describes the
        difference, the labels' column minus that input."""
        B.check(B.pnp_mlp_set_skip(self.m, int(out_col), int(in_col)), "pnp_mlp_set_skip")
        self.skip = (int(out_col), int(in_col)) if out_col >= 0 else None

    def _after_torch(self, *tensors):
        """Order the network's stream after the work torch has queued on the tensors
        it reads (its current stream), and keep their memory from being reused by
        torch's allocator until the network's stream has used it."""
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        for t in tensors:
            t.record_stream(self.stream)

    def forward(self, X):
        """X: device float32 tensor [B, 40] -> device tensor [B, 5]."""
        Y = self.torch.empty((X.shape[0], N_OUT), dtype=self.torch.float32, device=self.device)
        self._after_torch(X, Y)
        B.check(B.pnp_mlp_forward(self.m, C.c_void_p(X.data_ptr()), int(X.shape[0]), C.c_void_p(Y.data_ptr())),
                "pnp_mlp_forward")
        self.stream.synchronize()
        return Y

    def gradient(self, X, T):
        g = np.empty(self.nparam, dtype=np.float32)
        loss = C.c_float()
        self._after_torch(X, T)
        B.check(B.pnp_mlp_gradient(self.m, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), int(X.shape[0]),
                                   g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)), "pnp_mlp_gradient")
        return g, float(loss.value)

    def train_step(self, X, T, lr, want_loss=False):
        loss = C.c_float()
        self._after_torch(X, T)
        B.check(B.pnp_mlp_train_step(self.m, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), int(X.shape[0]),
                                     float(lr), C.byref(loss) if want_loss else None), "pnp_mlp_train_step")
        return float(loss.value) if want_loss else None

    def status(self):
        """Device status of the network's kernels (PNP_ERR_TIMEOUT if a tensor-core wait ran out)."""
        return int(B.pnp_mlp_status(self.m))

    def close(self):
        if getattr(self, "m", None):
            self.stream.synchronize()
            B.pnp_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PHI_SKIP = (2, 4 * 8)   # first-cell potential: output 2 on feature column 4 ncells (ncells = 8)


def residual_targets(T, X, skip):
    """The targets the network's own outputs learn under a residual output: column
    skip[0] of T less column skip[1] of X (a copy; T itself when skip is None)."""
    if skip is None:
        return T
    R = T.clone()
    R[:, skip[0]] -= X[:, skip[1]]
    return R


def features(solver, ncells=8):
    """Feature rows [2 Nz Nx, 5 ncells] of a solver's state (device tensor)."""
    torch = solver.torch
    X = torch.empty((2 * solver.nz * solver.nx, 5 * ncells), dtype=torch.float32, device=solver.device)
    torch.cuda.synchronize(solver.device)
    B.check(B.pnp_wall_features(solver.ctx, int(ncells), C.c_void_p(X.data_ptr())), "pnp_wall_features")
    solver.synchronize()
    return X


def labels(fine, coarse):
    torch = fine.torch
    T = torch.empty((2 * coarse.nz * coarse.nx, N_OUT), dtype=torch.float32, device=fine.device)
    torch.cuda.synchronize(fine.device)
    B.check(B.pnp_wall_labels(fine.ctx, coarse.ctx, C.c_void_p(T.data_ptr())), "pnp_wall_labels")
    return T


def first_cell_potential(solver, V, yc):
    """The first cells' potential perturbation Phi - V y_c in the wall frame (the
    top wall's sign flipped), rows [bottom Nz Nx, top Nz Nx] as in the feature
    rows: the total potential, wall-model offsets included (host array)."""
    Phi = solver.get("Phi")
    return np.concatenate([(Phi[0] - V * yc[0]).ravel(), -(Phi[-1] - V * yc[-1]).ravel()])


def restrict(fine, coarse):
    B.check(B.pnp_restrict_state(fine.ctx, coarse.ctx), "pnp_restrict_state")


def set_slip(solver, X, Y, ncells=8):
    solver.torch.cuda.synchronize(solver.device)
    if Y is None:
        B.check(B.pnp_set_wall_slip(solver.ctx, None, 0, None), "pnp_set_wall_slip")
    else:
        B.check(B.pnp_set_wall_slip(solver.ctx, C.c_void_p(X.data_ptr()), int(ncells), C.c_void_p(Y.data_ptr())),
                "pnp_set_wall_slip")


def set_coupling(solver, mode=0, relax=1.0, potential_gain=0.0, flux_gain=0.0):
    """How step_with_model couples the network: wall shear by slip (0), stress (1)
    or plane-mean stress (2), its relaxation, and the double-layer gains."""
    B.check(B.pnp_set_wallmodel_coupling(solver.ctx, int(mode), float(relax)), "pnp_set_wallmodel_coupling")
    B.check(B.pnp_set_wallmodel_edl(solver.ctx, float(potential_gain), float(flux_gain)), "pnp_set_wallmodel_edl")


def clear_edl(solver):
    """Switch the double-layer coupling off and restore the uniform walls."""
    B.check(B.pnp_set_wallmodel_edl(solver.ctx, 0.0, 0.0), "pnp_set_wallmodel_edl")


def set_wall_edl(solver, X, Y, ncells=8):
    solver.torch.cuda.synchronize(solver.device)
    B.check(B.pnp_set_wall_edl(solver.ctx, C.c_void_p(X.data_ptr()), int(ncells), C.c_void_p(Y.data_ptr())),
            "pnp_set_wall_edl")
    solver.synchronize()


def correct_wall_flux(solver, Y, dt):
    solver.torch.cuda.synchronize(solver.device)
    B.check(B.pnp_correct_wall_flux(solver.ctx, C.c_void_p(Y.data_ptr()), float(dt)), "pnp_correct_wall_flux")
    solver.synchronize()


def step_with_model(solver, mlp, nsteps, dt):
    B.check(B.pnp_step_wallmodel(solver.ctx, mlp.m, int(nsteps), float(dt)), "pnp_step_wallmodel")
