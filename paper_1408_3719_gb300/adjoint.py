"""Gradients of the LTS ALE ADER-WENO run through ``torch.autograd``.

``LtsRun.apply(Q0, xy0, solver, n_sweeps, ckpt_every)`` loads the initial
averages ``Q0`` [n_tris, 4] on node positions ``xy0`` [n_nodes, 2] into a
``Solver`` whose mesh is loaded, runs ``n_sweeps`` LTS sweeps on the GPU
(checkpoints every ``ckpt_every`` sweeps) and returns the final averages
[n_tris, 4] and element corners [n_tris, 6].  Its backward is the hand-written
discrete adjoint of the library (``aw_adjoint``): the sweep map for the
schedule the run took, i.e. with the ready sets and integer time steps held
fixed and the stencils of the loaded mesh kept.
"""
from __future__ import annotations

import numpy as np
import torch


def _settle(t):
    """The library reads and writes through its own stream: finish the work
    queued on torch's current stream of t's device first."""
    if t.device.type == "cuda":
        torch.cuda.current_stream(t.device).synchronize()


class LtsRun(torch.autograd.Function):
    """Tensors stay where they are: device tensors are handed to the C ABI
    by pointer (no host round trip), host tensors likewise."""

    @staticmethod
    def forward(ctx, Q0, xy0, solver, n_sweeps, ckpt_every=10):
        dev = Q0.device
        Qd = Q0.detach().to(dtype=torch.float64).contiguous()
        xyd = xy0.detach().to(device=dev, dtype=torch.float64).contiguous()
        _settle(Qd)
        solver.load_state_xy(Qd, xyd)
        solver.adjoint_forward(int(n_sweeps), int(ckpt_every))
        Q = torch.empty((solver.n_tris, 4), dtype=torch.float64, device=dev)
        X = torch.empty((solver.n_tris, 6), dtype=torch.float64, device=dev)
        solver.get_elem_into(Q=Q, X=X)
        ctx.solver = solver
        ctx.dev = dev
        ctx.n_nodes = xy0.shape[0]
        return Q, X

    @staticmethod
    def backward(ctx, gQ, gX):
        s, dev = ctx.solver, ctx.dev
        gq = None if gQ is None else gQ.detach().to(device=dev, dtype=torch.float64).contiguous()
        gx = None if gX is None else gX.detach().to(device=dev, dtype=torch.float64).contiguous()
        for g in (gq, gx):
            if g is not None:
                _settle(g)
        gQ0 = torch.empty((s.n_tris, 4), dtype=torch.float64, device=dev)
        gxy0 = torch.empty((ctx.n_nodes, 2), dtype=torch.float64, device=dev)
        s.adjoint(gq, gx, None, out_Q=gQ0, out_xy=gxy0)
        return gQ0, gxy0, None, None, None


def triangle_areas(X):
    """Signed areas of triangles given as [n, 6] corner coordinates."""
    return 0.5 * ((X[:, 2] - X[:, 0]) * (X[:, 5] - X[:, 1]) - (X[:, 3] - X[:, 1]) * (X[:, 4] - X[:, 0]))


def kinetic_energy(Q, X, mask):
    """sum over the masked elements of |T| (rho u^2 + rho v^2) / (2 rho)."""
    ke = 0.5 * (Q[:, 1] ** 2 + Q[:, 2] ** 2) / Q[:, 0]
    return (triangle_areas(X) * ke * mask).sum()


def disc_mask(X, centre, radius, period=None):
    """1 for the elements whose centroid lies within radius of centre (the
    nearest periodic image when period is given)."""
    c = X.reshape(-1, 3, 2).mean(1) - np.asarray(centre)
    if period is not None:
        p = np.asarray(period)
        c = c - p * np.round(c / p)
    return (np.hypot(c[:, 0], c[:, 1]) < radius).astype(np.float64)
