"""The shock tubes and explosions as the paper sets them up (Sec. 3.2: box
[-0.5, 0.5] x [-0.05, 0.05], periodic in y, transmissive in x, N_E = 8862;
Sec. 3.3: unit disc, h = 1/100 inside r = 0.5 and 1/50 outside, N_E = 43756),
and the oracle on a mesh that is periodic in one direction only."""
import numpy as np
import pytest

from oracle.pyoracle import Oracle
from paper_1408_3719_gb300 import workloads as W


def _areas(P):
    return 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                  - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))


def test_riemann_problem_mesh_matches_the_paper_set_up():
    mesh, Q, t_end = W.riemann_problem("RP2")
    assert mesh["tri"].shape[0] == 8862 and t_end == 0.1
    P = W._corner_coords(mesh)
    assert abs(_areas(P).sum() - 0.1) < 1e-12  # the rectangle, tiled exactly
    assert np.all(mesh["shift"][..., 0] == 0) and mesh["period"][0] == 0.0
    # transmissive edges only at the two x ends, one per row of quads
    tx = np.nonzero(mesh["bc"] == W.BC_TRANSMISSIVE)
    assert len(tx[0]) == 2 * 21
    for i, e in zip(*tx):
        a, b = P[i, e], P[i, (e + 1) % 3]
        assert abs(a[0] - b[0]) < 1e-15 and abs(abs(a[0]) - 0.5) < 1e-15
    left = P[:, :, 0].max(1) < 0  # elements wholly left of x_d = 0
    assert left.sum() > 4000
    assert np.abs(Q[left] - W.prim_to_cons(0.445, 0.698, 0.0, 3.528, 1.4)[None]).max() < 1e-13


def test_explosion_mesh_matches_the_paper_sizes():
    mesh, Q, t_end = W.explosion_problem("EP2")
    n = mesh["tri"].shape[0]
    assert abs(n - 43756) / 43756 < 0.01 and t_end == 0.012
    P = W._corner_coords(mesh)
    A = _areas(P)
    assert abs(A.sum() - np.pi) < 2e-3
    r = np.linalg.norm(P.mean(1), axis=1)
    h_in = np.sqrt(4 * A[r < 0.45] / np.sqrt(3)).mean()
    h_out = np.sqrt(4 * A[r > 0.6] / np.sqrt(3)).mean()
    assert 1.6 < h_out / h_in < 2.4
    assert np.all(mesh["bc"][mesh["bc"] >= 0] == W.BC_TRANSMISSIVE)
    assert Q[:, 3].max() == pytest.approx(1000.0 / 0.4)


def test_stencils_wrap_in_y_and_not_in_x():
    mesh = W.tube_mesh_periodic_y(40, 6)
    o = Oracle(order_M=2)
    o.load_mesh(mesh)
    c = W._corner_coords(mesh).mean(1)
    ly = mesh["period"][1]
    wrapped_y = False
    sw = {}
    for i in range(mesh["tri"].shape[0]):
        mem, s = o.stencils(i)
        sw[i] = set(s.tolist())
        d = c[mem[mem >= 0]] - c[i]
        assert np.abs(d[:, 0]).max() < 0.2  # no member across the transmissive ends
        dy = d[:, 1]
        wrapped_y |= bool(np.any(np.abs(dy) > 0.5 * ly))
    assert wrapped_y  # members of the boundary rows come through the periodic images
    for i, s in sw.items():
        for j in s:
            assert i in sw[j]


@pytest.mark.parametrize("M", [1, 2])
def test_free_stream_through_transmissive_ends_and_periodic_y(M):
    mesh = W.tube_mesh_periodic_y(24, 4)
    q0 = np.array([1.0, 0.3, -0.2, 2.5])
    Q = np.tile(q0, (mesh["tri"].shape[0], 1))
    o = Oracle(order_M=M, t_end=0.5)
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(30):
        o.sweep()
    e = o.get_elem()
    assert np.abs(e["Q"] - q0).max() < 1e-12
    X, _ = o.get_nodes()
    assert np.abs(X - mesh["xy"]).max() > 1e-3  # the mesh moved, through both ends
    assert o.diag()["gcl_max"] < 1e-13


def test_period_components_are_validated():
    mesh = W.tube_mesh_periodic_y(10, 4)
    o = Oracle(order_M=1)
    bad = dict(mesh)
    bad["period"] = np.array([0.0, 0.0])
    with pytest.raises(Exception):
        o.load_mesh(bad)
    bad["period"] = np.array([-1.0, 0.1])
    with pytest.raises(Exception):
        o.load_mesh(bad)


def test_gas_at_rest_beside_transmissive_ends_stays_at_rest():
    """Reading R15: the outer state of a transmissive edge is the boundary
    element's average.  Taking the inner trace value instead makes the flux
    through the edge the bare physical flux of an extrapolated state; an
    incoming characteristic then sees downwind differencing and a gas at rest
    grows from roundoff (about 4 % per step at P1 on this mesh: 1e-15 to 1e-10
    in 300 steps)."""
    mesh = W.tube_mesh_periodic_y(40, 4)
    Q = np.tile(W.prim_to_cons(1.0, 0.0, 0.0, 1.0, 1.4), (mesh["tri"].shape[0], 1))
    o = Oracle(order_M=1, t_end=10.0, gts=True)
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(300):
        o.sweep()
    q = o.get_elem()["Q"]
    assert np.abs(q[:, 1:3]).max() < 1e-13
    assert np.abs(q[:, 0] - 1.0).max() < 1e-13
