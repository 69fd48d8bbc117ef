"""1D reference solutions for the cylindrical explosions of Sec. 3.3.

Radially symmetric flow of the 2D Euler equations reduces to the 1D system
with geometric source terms of eqs. inhomEuler / matrixInhomEuler,

    Q_t + F(Q)_r = S(Q),   Q = (rho, rho u, rho E),
    F = (rho u, rho u^2 + p, u (rho E + p)),   S = -(alpha / r) (rho u, rho u^2, u (rho E + p)),

with alpha = 1 (alpha = 0 gives the planar shock tube).  The paper solves it
on 15,000 points of [0, 1] with a second-order TVD scheme and a Rusanov-type
flux.  This module does the same with the MUSCL-Hancock scheme of Toro's book:
van Leer-limited slopes of the primitive variables, a half-step evolution of
the face values by the primitive quasi-linear form (sources included),
Rusanov-type face fluxes, and the source taken at the evolved cell-centre
state.  Mirror cells at r = 0 (reflective), copies at the outer end
(transmissive).

The module is an analysis tool for the configuration runs; it shares nothing
with the solver library.
"""
from __future__ import annotations

import numpy as np


def _prim(U, g):
    rho = U[0]
    u = U[1] / rho
    p = (g - 1.0) * (U[2] - 0.5 * rho * u * u)
    return rho, u, p


def _flux(rho, u, p, g):
    E = p / (g - 1.0) + 0.5 * rho * u * u
    return np.stack([rho * u, rho * u * u + p, u * (E + p)])


def _vanleer(a, b):
    ab = a * b
    return np.where(ab > 0.0, 2.0 * ab / np.where(ab > 0.0, a + b, 1.0), 0.0)


def solve(inner, outer, r_d=0.5, t_end=0.25, n=15000, length=1.0, alpha=1, gamma=1.4, cfl=0.9,
          max_steps=10_000_000, budget=None):
    """Advance the 1D system from a jump at r = r_d between the primitive
    states ``inner`` (r < r_d) and ``outer`` = (rho, u, p) to ``t_end`` on
    ``n`` equal cells of [0, length].  alpha = 1: cylindrical (explosions,
    Sec. 3.3); alpha = 0: planar (the left end is then a wall).  Returns
    (cell centres, rho, u, p).

    If ``budget`` is a dict it receives the time integrals that close the
    balance laws of the r-weighted form (r^alpha Q)_t + (r^alpha F)_r =
    (0, alpha p, 0): ``outflow`` = int length^alpha F(length) dt (3 values)
    and ``pressure`` = int int alpha p dr dt, both taken at the mid-step
    states the update uses, and ``steps``."""
    g = gamma
    dx = length / n
    r = (np.arange(n) + 0.5) * dx
    ql = np.array(inner, dtype=np.float64)
    qr = np.array(outer, dtype=np.float64)
    inside = r < r_d
    rho = np.where(inside, ql[0], qr[0])
    u = np.where(inside, ql[1], qr[1])
    p = np.where(inside, ql[2], qr[2])
    U = np.stack([rho, rho * u, p / (g - 1.0) + 0.5 * rho * u * u])
    t = 0.0
    rg = np.concatenate([[-0.5 * dx], r, [length + 0.5 * dx]])  # centres with one ghost each side
    inv_r = np.where(rg > 0, alpha / np.abs(rg), 0.0)
    for _ in range(max_steps):
        if t >= t_end:
            break
        rho, u, p = _prim(U, g)
        c = np.sqrt(g * p / rho)
        dt = min(cfl * dx / np.max(np.abs(u) + c), t_end - t)
        # ghost cells: mirror at r = 0, copy at the outer end
        W = np.stack([rho, u, p])
        W = np.concatenate([W[:, :1] * np.array([[1.0], [-1.0], [1.0]]), W, W[:, -1:]], axis=1)
        # limited slopes (ghosts keep zero slope)
        d = np.zeros_like(W)
        d[:, 1:-1] = _vanleer(W[:, 1:-1] - W[:, :-2], W[:, 2:] - W[:, 1:-1])
        rh, uh, ph = W
        drh, duh, dph = d / dx
        # half-step evolution of the primitive variables (quasi-linear form + sources)
        s = 0.5 * dt
        rt = -(uh * drh + rh * duh) - inv_r * rh * uh
        ut = -(uh * duh + dph / rh)
        pt = -(uh * dph + g * ph * duh) - inv_r * g * ph * uh
        Wm = np.stack([rh + s * rt, uh + s * ut, ph + s * pt])  # cell centre at t + dt/2
        WL = Wm + 0.5 * d  # value at the right face of each cell
        WR = Wm - 0.5 * d  # value at the left face of each cell
        # the ghosts' face values: mirror of the first cell's left face (no
        # flux through r = 0), copy of the last cell's right face
        WL[:, 0] = WR[:, 1] * np.array([1.0, -1.0, 1.0])
        WR[:, -1] = WL[:, -2]
        a, b = WL[:, :-1], WR[:, 1:]  # the two sides of every face
        ca = np.sqrt(g * a[2] / a[0])
        cb = np.sqrt(g * b[2] / b[0])
        smax = np.maximum(np.abs(a[1]) + ca, np.abs(b[1]) + cb)
        Ua = np.stack([a[0], a[0] * a[1], a[2] / (g - 1.0) + 0.5 * a[0] * a[1] ** 2])
        Ub = np.stack([b[0], b[0] * b[1], b[2] / (g - 1.0) + 0.5 * b[0] * b[1] ** 2])
        F = 0.5 * (_flux(*a, g) + _flux(*b, g)) - 0.5 * smax * (Ub - Ua)
        # source at the evolved centre state of the real cells
        rm, um, pm = Wm[:, 1:-1]
        Em = pm / (g - 1.0) + 0.5 * rm * um * um
        S = -inv_r[1:-1] * np.stack([rm * um, rm * um * um, um * (Em + pm)])
        U = U - dt / dx * (F[:, 1:] - F[:, :-1]) + dt * S
        t += dt
        if budget is not None:
            budget["outflow"] = budget.get("outflow", 0.0) + dt * length ** alpha * F[:, -1]
            budget["pressure"] = budget.get("pressure", 0.0) + dt * alpha * dx * float(np.sum(pm))
            budget["steps"] = budget.get("steps", 0) + 1
    rho, u, p = _prim(U, g)
    return r, rho, u, p


def sample(r_query, r, field):
    """Linear interpolation of a 1D profile at the radii ``r_query``."""
    return np.interp(r_query, r, field)
