"""The Kidder compression of Sec. 3.4 (eqs. KidderIC, KidderEx): the closed
form the inputs and the comparisons use is checked against the Euler
equations themselves, and the oracle driven by its exact boundary state
(tag 3) is checked against the closed form's frontier positions and state."""
import math

import numpy as np

from oracle.pyoracle import Oracle
from paper_1408_3719_gb300 import workloads as W

G = 2.0


def _cons(x, y, t):
    return W.prim_to_cons(*W.kidder_prim(x, y, t), G)


def _flux(q):
    rho, mu, mv, E = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    u, v = mu / rho, mv / rho
    p = (G - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    f = np.stack([mu, mu * u + p, mu * v, u * (E + p)], -1)
    g = np.stack([mv, mv * u, mv * v + p, v * (E + p)], -1)
    return f, g


def test_closed_form_solves_the_euler_equations():
    rng = np.random.default_rng(5)
    tau = W.kidder_tau()
    d = 2e-5
    # fourth-order central differences (the solution's third derivatives put
    # second-order ones 1e-6 off at this step)
    D = lambda f: (8.0 * (f(d) - f(-d)) - (f(2 * d) - f(-2 * d))) / (12.0 * d)
    worst = 0.0
    for _ in range(20):
        t = rng.uniform(0.0, 0.85 * tau)
        h = math.sqrt(1.0 - t * t / tau ** 2)
        r = h * rng.uniform(0.9, 1.0)
        th = rng.uniform(0.0, 0.5 * math.pi)
        x, y = r * math.cos(th), r * math.sin(th)
        dq_dt = D(lambda e: _cons(x, y, t + e))
        df_dx = D(lambda e: _flux(_cons(x + e, y, t))[0])
        dg_dy = D(lambda e: _flux(_cons(x, y + e, t))[1])
        res = dq_dt + df_dx + dg_dy
        worst = max(worst, np.abs(res).max() / np.abs(_cons(x, y, t)).max())
    assert worst < 1e-7


def test_focalisation_time_and_final_compression():
    tau = W.kidder_tau()
    # c_i0^2 = 2, c_e0^2 = 4 (gamma = 2, s0 = 1): tau^2 = (1/2)(1 - 0.81)/2
    assert abs(tau * tau - 0.0475) < 1e-15
    _, _, tf = W.kidder(2, 8)
    assert abs(math.sqrt(1.0 - tf * tf / tau ** 2) - 0.5) < 1e-15
    # mass: the exact density times the area of the shell is conserved
    rho0 = lambda r: W.kidder_prim(r, 0.0, 0.0)[0]
    rho1 = lambda r: W.kidder_prim(r, 0.0, tf)[0]
    rr0 = np.linspace(0.9, 1.0, 20001)
    rr1 = 0.5 * rr0
    m0 = np.trapezoid(rho0(rr0) * rr0, rr0)
    m1 = np.trapezoid(rho1(rr1) * rr1, rr1)
    assert abs(m1 / m0 - 1.0) < 1e-12


def test_oracle_compresses_the_shell_to_the_exact_radii():
    mesh, Q, tf = W.kidder(5, 40)
    o = Oracle(order_M=2, gamma=G, t_end=tf, flux="osher")
    o.load_mesh(mesh)
    o.load_state(Q)
    o.advance()
    X, _ = o.get_nodes()
    r0 = np.hypot(*mesh["xy"].T)
    rn = np.hypot(*X.T)
    assert abs(rn[np.abs(r0 - 0.9) < 1e-12].mean() - 0.45) < 2e-4
    assert abs(rn[np.abs(r0 - 1.0) < 1e-12].mean() - 0.5) < 2e-4
    e = o.get_elem()
    c = e["X"].reshape(-1, 3, 2).mean(1)
    rho_ex = W.kidder_prim(c[:, 0], c[:, 1], tf)[0]
    assert np.abs(e["Q"][:, 0] / rho_ex - 1.0).mean() < 2e-3
