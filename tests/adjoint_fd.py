"""Objective and finite-difference helpers of the adjoint tests.  No torch
import: the oracle's difference quotients run in spawned worker processes that
import only this module, numpy and the oracle."""
import numpy as np

from paper_1408_3719_gb300 import workloads as W

H = 1e-6          # central-difference step
TOL = 1e-6        # relative agreement of <dJ/dx, v> with the difference quotient
ROUND = 1e-15     # relative rounding noise of one evaluation of J


def agree(ad, fd, J0):
    """|ad - fd| within TOL of fd, plus the rounding error of the quotient
    itself (ROUND |J| / H, a few 1e-10 here)"""
    return abs(ad - fd) <= TOL * abs(fd) + ROUND * abs(J0) / H


def _areas(X):
    return 0.5 * ((X[:, 2] - X[:, 0]) * (X[:, 5] - X[:, 1]) - (X[:, 3] - X[:, 1]) * (X[:, 4] - X[:, 0]))


def _mask(mesh):
    """elements whose initial centroid is within 1 of the vortex centre (5, 5)"""
    c = W._corner_coords(mesh).mean(1) - 5.0
    return (np.hypot(c[:, 0], c[:, 1]) < 1.0).astype(np.float64)


def wavy_vortex(nv, gamma=1.4):
    """The isentropic vortex with a smooth periodic entropy wave on the density
    (velocity and pressure kept), so that no characteristic field is flat.
    On the plain isentropic vortex the entropy field is flat to the
    discretisation error: its nonlinear weights then work at sigma ~ epsilon =
    1e-14, where they curve so strongly that a central difference of step 1e-6
    along a random perturbation of the averages leaves the linear regime."""
    mesh, _ = W.vortex(nv)

    def fun(x, y):
        q = W.vortex_state(x, y, gamma, mesh["period"])
        rho = q[..., 0]
        u, v = q[..., 1] / rho, q[..., 2] / rho
        p = (gamma - 1.0) * (q[..., 3] - 0.5 * rho * (u * u + v * v))
        f = 1.0 + 0.1 * np.sin(0.2 * np.pi * x) * np.cos(0.2 * np.pi * y)
        return W.prim_to_cons(f * rho, u, v, p, gamma)

    return mesh, W.cell_average(mesh, fun, W._duffy_rule(8))


def _J(Q, X, mask):
    return float(np.sum(mask * _areas(X) * 0.5 * (Q[:, 1] ** 2 + Q[:, 2] ** 2) / Q[:, 0]))


def _dJ(Q, X, mask):
    A = _areas(X)
    ke = 0.5 * (Q[:, 1] ** 2 + Q[:, 2] ** 2) / Q[:, 0]
    gQ = np.zeros_like(Q)
    gQ[:, 0] = -mask * A * ke / Q[:, 0]
    gQ[:, 1] = mask * A * Q[:, 1] / Q[:, 0]
    gQ[:, 2] = mask * A * Q[:, 2] / Q[:, 0]
    s = mask * ke
    gX = np.zeros_like(X)
    gX[:, 0] = 0.5 * s * (X[:, 3] - X[:, 5])
    gX[:, 1] = 0.5 * s * (X[:, 4] - X[:, 2])
    gX[:, 2] = 0.5 * s * (X[:, 5] - X[:, 1])
    gX[:, 3] = 0.5 * s * (X[:, 0] - X[:, 4])
    gX[:, 4] = 0.5 * s * (X[:, 1] - X[:, 3])
    gX[:, 5] = 0.5 * s * (X[:, 2] - X[:, 0])
    return gQ, gX


def _direction(rng, Q, xy, kind):
    vQ = rng.standard_normal(Q.shape) * np.array([0.1, 0.1, 0.1, 0.3]) if kind in ("Q", "both") else np.zeros_like(Q)
    vxy = rng.standard_normal(xy.shape) * 0.01 if kind in ("xy", "both") else np.zeros_like(xy)
    return vQ, vxy


def _oracle_fd(args):
    """Central difference of the oracle along one direction, in a process of
    its own (spawned: no CUDA state): record the base schedule, replay it."""
    mesh, Q0, order, n_sweeps, vQ, vxy = args
    from oracle.pyoracle import Oracle
    o = Oracle(order_M=order, t_end=1.0)
    o.load_mesh(mesh)
    o.schedule("record", n_sweeps + 2)
    o.load_state_xy(Q0, mesh["xy"])
    for _ in range(n_sweeps):
        o.sweep()
    log = o.get_schedule()
    o.schedule("replay")
    mask = _mask(mesh)
    out = []
    for sgn in (1.0, -1.0):
        o.load_state_xy(Q0 + sgn * H * vQ, mesh["xy"] + sgn * H * vxy)
        for _ in range(n_sweeps):
            o.sweep()
        e = o.get_elem()
        out.append(_J(e["Q"], e["X"], mask))
    return (out[0] - out[1]) / (2 * H), log


def _oracle_tlm(args):
    """The oracle's tangent-linear product J'(x0) v in a process of its own
    (spawned): the dual-number build of the oracle run from the seeded
    tangents (vQ, vxy), the objective's derivative applied to the final
    tangents.  The schedule is the run's own (values equal the plain
    oracle's bit for bit); it is returned for comparison."""
    mesh, Q0, order, n_sweeps, vQ, vxy = args
    from oracle.pyoracle import TangentOracle
    o = TangentOracle(order_M=order, t_end=1.0)
    o.load_mesh(mesh)
    o.schedule("record", n_sweeps + 2)
    o.load_state_xy(Q0, mesh["xy"], vQ, vxy)
    for _ in range(n_sweeps):
        o.sweep()
    val, tan = o.get_elem()
    gQ, gX = _dJ(val["Q"], val["X"], _mask(mesh))
    return float(np.sum(gQ * tan["Q"]) + np.sum(gX * tan["X"])), o.get_schedule()
