"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (the parity contract): one sweep from a shared snapshot matches to
1e-12 relative in the conserved variables and node positions; multi-sweep and
full runs to 1e-9 relative L-infinity; element times, time steps and update
counts are integers and must match exactly.  Predictor degrees of freedom
match to 1e-12 relative as well: the two sides solve the least-squares fits
differently (Householder QR on the CPU; on the GPU the normal equations with
one step of the corrected semi-normal equations, which brings the solution to
the accuracy of an orthogonal factorisation).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.pyoracle import Oracle  # noqa: E402
from paper_1408_3719_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def aw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno
    aleweno.load()
    return aleweno


def rel(a, b):
    """L-infinity difference relative to the largest magnitude of the
    reference state (a variable that is zero up to roundoff everywhere, such
    as the momentum of a state at rest, is measured on the state's scale)."""
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def make_pair(aw, mesh, Q, **cfg):
    g = aw.Solver(**cfg)
    o = Oracle(**cfg)
    for s in (g, o):
        s.load_mesh(mesh)
        s.load_state(Q)
    return g, o


CASES = {
    "tube_p1": (lambda: W.sod_tube(40, 6), dict(order_M=1, t_end=0.2)),
    "tube_p2": (lambda: W.sod_tube(40, 6), dict(order_M=2, t_end=0.2)),
    "vortex_p1": (lambda: W.vortex(10), dict(order_M=1, t_end=1.0)),
    "vortex_p2": (lambda: W.vortex(10), dict(order_M=2, t_end=1.0)),
    "vortex_p3": (lambda: W.vortex(10), dict(order_M=3, t_end=1.0)),
    "disc_p2": (lambda: W.explosion(0.04), dict(order_M=2, t_end=0.25)),
    "disc_p3": (lambda: W.explosion(0.04), dict(order_M=3, t_end=0.25)),
    "vortex_p2_gts": (lambda: W.vortex(10), dict(order_M=2, t_end=1.0, gts=True)),
    "tube_p1_eulerian": (lambda: W.sod_tube(40, 6), dict(order_M=1, t_end=0.2, eulerian=True)),
    "rp1_periodic_y_p2": (lambda: W.riemann_problem("RP1", 40, 6, jitter=0.1)[:2], dict(order_M=2, t_end=0.2)),
    # the Saltzman piston (Sec. 3.5), coarse: a moving slip wall and the
    # global-step start-up with CFL 0.1 until t = 0.01, local steps after
    "saltzman_p1": (lambda: W.saltzman(20, 4), dict(order_M=1, gamma=5.0 / 3.0, t_end=0.6, wall_velocity=(1.0, 0.0),
                                                    t_switch=0.01, cfl_start=0.1)),
    "saltzman_p2": (lambda: W.saltzman(20, 4), dict(order_M=2, gamma=5.0 / 3.0, t_end=0.6, wall_velocity=(1.0, 0.0),
                                                    t_switch=0.01, cfl_start=0.1)),
    # the Kidder compression (Sec. 3.4): exact state on the two arcs
    "kidder_p2": (lambda: W.kidder(5, 40)[:2], dict(order_M=2, gamma=2.0, t_end=0.5 * 3 ** 0.5 * W.kidder_tau())),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_preprocessing_phase(aw, case):
    (mesh, Q), cfg = CASES[case][0](), CASES[case][1]
    g, o = make_pair(aw, mesh, Q, **cfg)
    eg, eo = g.get_elem(), o.get_elem()
    assert np.array_equal(eg["dt"], eo["dt"])
    assert np.array_equal(eg["X"], eo["X"])
    assert rel(eg["qhat"].reshape(-1, 4), eo["qhat"].reshape(-1, 4)) < 1e-12


@pytest.mark.parametrize("case", sorted(CASES))
def test_single_sweep_from_snapshot(aw, case):
    (mesh, Q), cfg = CASES[case][0](), CASES[case][1]
    o = Oracle(**cfg)
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(4):
        o.sweep()
    snap, (nX, nt) = o.get_elem(), o.get_nodes()
    g = aw.Solver(**cfg)
    g.load_mesh(mesh)
    g.set_elem(snap)
    g.set_nodes(nX, nt)
    ng, no = g.sweep(), o.sweep()
    assert ng == no and ng > 0
    eg, eo = g.get_elem(), o.get_elem()
    for k in ("t", "dt", "count"):
        assert np.array_equal(eg[k], eo[k]), k
    assert rel(eg["Q"], eo["Q"]) < 1e-12
    gX, gt = g.get_nodes()
    oX, ot = o.get_nodes()
    assert np.array_equal(gt, ot)
    assert np.abs(gX - oX).max() < 1e-12 * np.abs(oX).max()
    assert np.abs(eg["X"] - eo["X"]).max() < 1e-12 * np.abs(eo["X"]).max()
    qs = np.abs(eo["Q"]).max(axis=0)
    assert np.abs(eg["QM"] - eo["QM"]).max() / qs.max() < 1e-12
    assert np.abs(eg["HM"] - eo["HM"]).max() < 1e-12 * np.abs(eo["X"]).max() ** 2
    assert rel(eg["qhat"].reshape(-1, 4), eo["qhat"].reshape(-1, 4)) < 1e-12


@pytest.mark.parametrize("case", sorted(CASES))
def test_many_sweeps(aw, case):
    (mesh, Q), cfg = CASES[case][0](), CASES[case][1]
    g, o = make_pair(aw, mesh, Q, **cfg)
    for _ in range(40):
        ng, no = g.sweep(), o.sweep()
        assert ng == no
        if no == 0:
            break
    eg, eo = g.get_elem(), o.get_elem()
    assert np.array_equal(eg["count"], eo["count"])
    assert np.array_equal(eg["t"], eo["t"])
    assert rel(eg["Q"], eo["Q"]) < 1e-9
    gX, _ = g.get_nodes()
    oX, _ = o.get_nodes()
    assert np.abs(gX - oX).max() < 1e-9 * np.abs(oX).max()
    assert g.diag()["gcl_max"] < 1e-12


def test_full_run_shock_tube_gts_p1(aw):
    """The 2000-triangle Sod tube, P1, GTS, to t_end = 0.2."""
    mesh, Q = W.sod_tube()
    g, o = make_pair(aw, mesh, Q, order_M=1, t_end=0.2, gts=True)
    sg, ug = g.advance()
    so, uo = o.advance()
    assert (sg, ug) == (so, uo)
    assert ug == sg * mesh["tri"].shape[0]
    eg, eo = g.get_elem(), o.get_elem()
    assert np.all(eg["t"] == 2 ** 20)
    assert rel(eg["Q"], eo["Q"]) < 1e-9
    gX, _ = g.get_nodes()
    oX, _ = o.get_nodes()
    assert np.abs(gX - oX).max() < 1e-9


def test_full_run_vortex_lts_p3(aw):
    mesh, Q = W.vortex(12)
    g, o = make_pair(aw, mesh, Q, order_M=3, t_end=1.0)
    sg, ug = g.advance()
    so, uo = o.advance()
    assert (sg, ug) == (so, uo)
    eg, eo = g.get_elem(), o.get_elem()
    assert np.array_equal(eg["count"], eo["count"])
    assert rel(eg["Q"], eo["Q"]) < 1e-9


def test_finished_run_has_empty_ready_set(aw):
    mesh, Q = W.sod_tube(20, 4)
    g = aw.Solver(order_M=1, t_end=0.01)
    g.load_mesh(mesh)
    g.load_state(Q)
    g.advance()
    assert g.sweep() == 0
    per, tot = g.update_counts()
    assert per.sum() == tot > 0


def test_bad_inputs_raise(aw):
    mesh, Q = W.sod_tube(20, 4)
    g = aw.Solver(order_M=1)
    bad = dict(mesh)
    bad["tri"] = mesh["tri"][:, ::-1].copy()
    with pytest.raises(aw.AwError) as e:
        g.load_mesh(bad)
    assert e.value.code == -2
    g.load_mesh(mesh)
    Qb = Q.copy()
    Qb[3, 3] = 0.0
    with pytest.raises(aw.AwError) as e:
        g.load_state(Qb)
    assert e.value.code == -3
    with pytest.raises(aw.AwError) as e:
        g.sweep()
    assert e.value.code == -7


def test_device_pointers(aw):
    mesh, Q = W.vortex(6)
    g = aw.Solver(order_M=1, t_end=1.0)
    g.load_mesh(mesh)
    g.load_state(torch.tensor(Q, device="cuda"))
    g.sweep()
    out = torch.empty((Q.shape[0], 4), dtype=torch.float64, device="cuda")
    g.get_state(out)
    host = g.get_state()
    assert np.array_equal(out.cpu().numpy(), host)


def test_moving_wall_and_start_up_guards(aw):
    mesh, Q = W.saltzman(20, 4)
    bad = dict(mesh)
    bad["bc"] = mesh["bc"].copy()
    bad["bc"][bad["bc"] == 2] = 4
    g = aw.Solver(order_M=1, gamma=5.0 / 3.0)
    with pytest.raises(aw.AwError) as e:
        g.load_mesh(bad)
    assert e.value.code == -2
    with pytest.raises(aw.AwError):
        aw.Solver(order_M=1, t_switch=0.01, cfl_start=0.0)
    s = aw.Solver(order_M=2, gamma=5.0 / 3.0, t_end=0.6, wall_velocity=(1.0, 0.0))
    s.load_mesh(mesh)
    s.load_state(Q)
    with pytest.raises(aw.AwError) as e:
        s.adjoint_forward(2, 1)
    assert e.value.code == -1
