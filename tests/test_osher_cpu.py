"""Pins of the oracle's Osher-type ALE flux (eq. osher with the straight path
of eq. path, reading R14), independent of the oracle's own eigenvectors:
* consistency: with equal states it is the exact ALE flux F.n_xy + q n_t;
* for a small jump it is 1/2 (F(q-) + F(q+)) - 1/2 |J| (q+ - q-), with J the
  Jacobian of the ALE flux taken by central differences here and |J| from
  numpy's eigendecomposition;
* on a Sod tube it is less dissipative than the Rusanov-type flux: a smaller
  L1 density error against the exact Riemann solution (the paper's reason for
  using it)."""
import numpy as np
import pytest

from oracle.pyoracle import Oracle
from paper_1408_3719_gb300 import exact
from paper_1408_3719_gb300 import workloads as W

G = 1.4


def ale_flux(q, n):
    rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
    p = (G - 1.0) * (q[3] - 0.5 * rho * (u * u + v * v))
    w = u * n[0] + v * n[1] + n[2]
    vn = u * n[0] + v * n[1]
    return np.array([q[0] * w, q[1] * w + p * n[0], q[2] * w + p * n[1], q[3] * w + p * vn])


def jacobian(q, n, h=1e-6):
    J = np.zeros((4, 4))
    for j in range(4):
        d = np.zeros(4)
        d[j] = h * max(1.0, abs(q[j]))
        J[:, j] = (ale_flux(q + d, n) - ale_flux(q - d, n)) / (2 * d[j])
    return J


def cases():
    rng = np.random.default_rng(11)
    for _ in range(6):
        rho, u, v, p = 0.5 + rng.random(), rng.normal() * 0.5, rng.normal() * 0.5, 0.5 + rng.random()
        q = np.array([rho, rho * u, rho * v, p / (G - 1) + 0.5 * rho * (u * u + v * v)])
        n = np.array([rng.normal(), rng.normal(), 0.3 * rng.normal()])
        yield q, n


def test_osher_is_consistent():
    o = Oracle(order_M=1, flux="osher")
    for q, n in cases():
        F = o.flux(q, q, n)
        assert np.allclose(F, ale_flux(q, n), rtol=1e-13, atol=1e-13)


def test_osher_dissipation_is_the_absolute_jacobian_for_small_jumps():
    o = Oracle(order_M=1, flux="osher")
    rng = np.random.default_rng(12)
    for q, n in cases():
        dq = 1e-5 * rng.normal(size=4) * np.abs(q)
        qp = q + dq
        J = jacobian(q + 0.5 * dq, n)
        lam, V = np.linalg.eig(J)
        absJ = (V @ np.diag(np.abs(lam.real)) @ np.linalg.inv(V)).real
        expect = 0.5 * (ale_flux(q, n) + ale_flux(qp, n)) - 0.5 * absJ @ dq
        F = o.flux(q, qp, n)
        scale = np.abs(absJ @ dq).max()
        assert np.abs(F - expect).max() < 1e-6 * scale, (F, expect)


def test_osher_is_less_dissipative_than_rusanov_on_a_sod_tube():
    mesh, Q = W.sod_tube(60, 6)
    err = {}
    for fl in ("rusanov", "osher"):
        o = Oracle(order_M=1, t_end=0.2, gts=True, flux=fl)
        o.load_mesh(mesh)
        o.load_state(Q)
        o.advance()
        e = o.get_elem()
        X = e["X"]
        A = 0.5 * ((X[:, 2] - X[:, 0]) * (X[:, 5] - X[:, 1]) - (X[:, 3] - X[:, 1]) * (X[:, 4] - X[:, 0]))
        cxf = X.reshape(-1, 3, 2).mean(1)[:, 0]
        exf = exact.sample(cxf, 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1))
        err[fl] = float(np.sum(np.abs(e["Q"][:, 0] - exf[:, 0]) * A) / A.sum())
    assert err["osher"] < err["rusanov"], err
    assert err["osher"] < 0.05
