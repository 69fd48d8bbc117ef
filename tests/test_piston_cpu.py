"""The moving slip wall and the global-step start-up of the Saltzman problem
(Sec. 3.5) in the oracle, against what the mathematics fixes: the outer
state of a wall moving with the gas carries no mass or energy through the
wall beyond the pressure work, a uniform flow pushed by a wall moving with
it stays uniform, the wall's nodes move exactly with the wall, and the
start-up takes global steps until t_switch and local ones after."""
import numpy as np
import pytest

from oracle.pyoracle import Oracle
from paper_1408_3719_gb300 import workloads as W

G = 5.0 / 3.0


def test_moving_wall_flux_of_a_gas_moving_with_the_wall():
    o = Oracle(order_M=1, gamma=G, wall_velocity=(1.0, 0.0))
    p = 0.3
    q = W.prim_to_cons(1.2, 1.0, 0.0, p, G)
    # a wall edge facing +x that moves with (1, 0): n_t = -(v_wall . n_xy)
    F = o.flux(q, None, np.array([1.0, 0.0, -1.0]), 2)
    assert np.allclose(F, [0.0, p, 0.0, p], rtol=0, atol=1e-15)
    # gas at rest before the piston: the outer state moves at twice the wall's
    # speed with the same density and pressure (its energy holds the new
    # kinetic energy), so the flux is finite and carries no mass
    rest = W.prim_to_cons(1.0, 0.0, 0.0, (G - 1.0) * 1e-4, G)
    Fr = o.flux(rest, None, np.array([-1.0, 0.0, 1.0]), 2)
    assert np.all(np.isfinite(Fr)) and abs(Fr[0]) < 1e-15 and Fr[1] < 0.0
    # a fixed wall hit by the same gas: no mass through it, and the mirrored
    # outer state pushes back harder than the pressure
    F0 = Oracle(order_M=1, gamma=G).flux(q, None, np.array([1.0, 0.0, 0.0]), 0)
    assert abs(F0[0]) < 1e-15 and F0[1] > p + 1.0


def _channel(nx=20, ny=4):
    mesh, _ = W.saltzman(nx, ny)
    P = W._corner_coords(mesh)
    bc = mesh["bc"].copy()
    for i, e in zip(*np.nonzero(bc == W.BC_WALL)):
        a, b = P[i, e], P[i, (e + 1) % 3]
        if abs(a[0] - 1.0) < 1e-12 and abs(b[0] - 1.0) < 1e-12:
            bc[i, e] = W.BC_TRANSMISSIVE
    return dict(mesh, bc=bc)


@pytest.mark.parametrize("M", [1, 2])
def test_uniform_flow_pushed_by_a_wall_moving_with_it(M):
    mesh = _channel()
    q0 = W.prim_to_cons(1.0, 1.0, 0.0, 0.5, G)
    Q = np.tile(q0, (mesh["tri"].shape[0], 1))
    o = Oracle(order_M=M, gamma=G, t_end=0.2, wall_velocity=(1.0, 0.0))
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(30):
        o.sweep()
    e = o.get_elem()
    assert np.abs(e["Q"] - q0).max() < 1e-12
    X, t = o.get_nodes()
    tick = 0.2 / 2 ** 20
    wall = np.abs(mesh["xy"][:, 0]) < 1e-12
    assert np.all(X[wall, 0] == t[wall] * tick)  # the wall's nodes ride with it exactly
    assert np.all(X[wall, 1] == mesh["xy"][wall, 1])
    assert o.diag()["gcl_max"] < 1e-13


def test_start_up_takes_global_steps_until_the_switch():
    mesh, Q = W.saltzman(20, 4)
    cfg = dict(order_M=1, gamma=G, t_end=0.6, wall_velocity=(1.0, 0.0))
    o = Oracle(t_switch=0.01, cfl_start=0.1, **cfg)
    o.load_mesh(mesh)
    o.load_state(Q)
    # the first step is the global minimum of the CFL-0.1 steps: the same as a
    # global-step run with CFL 0.1
    g = Oracle(gts=True, cfl=0.1, **cfg)
    g.load_mesh(mesh)
    g.load_state(Q)
    assert np.array_equal(o.get_elem()["dt"], g.get_elem()["dt"])
    T_sw = int(np.floor(0.01 / (0.6 / 2 ** 20)))
    n_start = 0
    while True:
        e = o.get_elem()
        if e["t"][0] >= T_sw:
            break
        assert np.all(e["t"] == e["t"][0]) and np.all(e["dt"] == e["dt"][0])
        assert e["t"][0] + e["dt"][0] <= T_sw
        assert o.sweep() == mesh["tri"].shape[0]
        n_start += 1
    assert np.all(o.get_elem()["t"] == T_sw) and n_start > 5
    for _ in range(20):
        o.sweep()
    e = o.get_elem()
    assert len(np.unique(e["t"])) > 1  # local steps after the switch


def test_piston_shock_state_is_the_rankine_hugoniot_state():
    s, rho1, p1 = W.piston_shock()
    # the paper's final shock position x_f = 0.8 at t_f = 0.6
    assert abs(0.6 * s - 0.8) < 1e-3
    # mass and momentum balance across the shock in the shock frame
    rho0, p0 = 1.0, (G - 1.0) * 1e-4
    assert abs(rho0 * s - rho1 * (s - 1.0)) < 1e-12
    assert abs((p0 + rho0 * s * s) - (p1 + rho1 * (s - 1.0) ** 2)) < 1e-12
