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


class LtsRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q0, xy0, solver, n_sweeps, ckpt_every=10):
        Qh = Q0.detach().to("cpu", torch.float64).contiguous().numpy()
        xyh = xy0.detach().to("cpu", torch.float64).contiguous().numpy()
        solver.load_state_xy(Qh, xyh)
        solver.adjoint_forward(int(n_sweeps), int(ckpt_every))
        e = solver.get_elem()
        ctx.solver = solver
        ctx.dev = Q0.device
        return (torch.from_numpy(e["Q"]).to(Q0.device), torch.from_numpy(e["X"]).to(Q0.device))

    @staticmethod
    def backward(ctx, gQ, gX):
        s = ctx.solver
        gq = None if gQ is None else gQ.detach().to("cpu", torch.float64).contiguous().numpy()
        gx = None if gX is None else gX.detach().to("cpu", torch.float64).contiguous().numpy()
        gQ0, gxy0 = s.adjoint(gq, gx, None)
        return torch.from_numpy(gQ0).to(ctx.dev), torch.from_numpy(gxy0).to(ctx.dev), None, None, None


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
