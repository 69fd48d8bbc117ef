"""Parity of the CUDA path with the oracle under the Osher-type ALE flux
(Eq. 14's path integral through the straight segment in conserved variables,
three Gauss-Legendre points on the path).  Same bar as the Rusanov-type
parity tests: integers exact, one sweep from a shared snapshot to 1e-12
relative, many sweeps and full runs to 1e-9."""
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
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {
    "tube_p1_gts": (lambda: W.sod_tube(40, 6), dict(order_M=1, t_end=0.2, gts=True)),
    "tube_p2": (lambda: W.sod_tube(40, 6), dict(order_M=2, t_end=0.2)),
    "vortex_p2": (lambda: W.vortex(10), dict(order_M=2, t_end=1.0)),
    "vortex_p3": (lambda: W.vortex(10), dict(order_M=3, t_end=1.0)),
    "disc_p2": (lambda: W.explosion(0.04), dict(order_M=2, t_end=0.25)),
    "tube_p1_eulerian": (lambda: W.sod_tube(40, 6), dict(order_M=1, t_end=0.2, eulerian=True)),
    # the paper's set-ups, small: Lax tube periodic in y and transmissive in
    # x (Sec. 3.2), the EP2 explosion with its pressure ratio of 1e5 (Sec. 3.3)
    "rp2_periodic_y_p2": (lambda: W.riemann_problem("RP2", 40, 6, jitter=0.1)[:2], dict(order_M=2, t_end=0.1)),
    "ep2_p2": (lambda: W.explosion(0.04, inner=(1, 0, 0, 1000), outer=(1, 0, 0, 0.01)),
               dict(order_M=2, t_end=0.012)),
    # the Kidder compression at the paper's fourth order (Sec. 3.4)
    "kidder_p3": (lambda: W.kidder(5, 40)[:2], dict(order_M=3, gamma=2.0, t_end=0.5 * 3 ** 0.5 * W.kidder_tau())),
}


def make_pair(aw, mesh, Q, **cfg):
    g = aw.Solver(flux="osher", **cfg)
    o = Oracle(flux="osher", **cfg)
    for s in (g, o):
        s.load_mesh(mesh)
        s.load_state(Q)
    return g, o


@pytest.mark.parametrize("case", sorted(CASES))
def test_single_sweep_from_snapshot(aw, case):
    (mesh, Q), cfg = CASES[case][0](), CASES[case][1]
    o = Oracle(flux="osher", **cfg)
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(4):
        o.sweep()
    snap, (nX, nt) = o.get_elem(), o.get_nodes()
    g = aw.Solver(flux="osher", **cfg)
    g.load_mesh(mesh)
    g.set_elem(snap)
    g.set_nodes(nX, nt)
    ng, no = g.sweep(), o.sweep()
    assert ng == no and ng > 0
    eg, eo = g.get_elem(), o.get_elem()
    for k in ("t", "dt", "count"):
        assert np.array_equal(eg[k], eo[k]), k
    assert rel(eg["Q"], eo["Q"]) < 1e-12
    gX, _ = g.get_nodes()
    oX, _ = o.get_nodes()
    assert np.abs(gX - oX).max() < 1e-12 * np.abs(oX).max()
    qs = np.abs(eo["Q"]).max()
    assert np.abs(eg["QM"] - eo["QM"]).max() / qs < 1e-12
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


def test_full_run_shock_tube_gts_p1(aw):
    """The 2000-triangle Sod tube, P1, GTS, to t_end = 0.2, with the flux
    differing from the Rusanov-type run (the switch reaches the kernel)."""
    mesh, Q = W.sod_tube()
    g, o = make_pair(aw, mesh, Q, order_M=1, t_end=0.2, gts=True)
    sg, ug = g.advance()
    so, uo = o.advance()
    assert (sg, ug) == (so, uo)
    eg, eo = g.get_elem(), o.get_elem()
    assert rel(eg["Q"], eo["Q"]) < 1e-9
    r = aw.Solver(order_M=1, t_end=0.2, gts=True)
    r.load_mesh(mesh)
    r.load_state(Q)
    r.advance()
    assert rel(r.get_elem()["Q"], eg["Q"]) > 1e-6


def test_adjoint_refuses_the_osher_flux(aw):
    mesh, Q = W.vortex(6)
    g = aw.Solver(order_M=2, t_end=1.0, flux="osher")
    g.load_mesh(mesh)
    g.load_state(Q)
    with pytest.raises(aw.AwError) as e:
        g.adjoint_forward(2, 1)
    assert e.value.code == -1


def test_bad_flux_name_raises(aw):
    with pytest.raises((ValueError, KeyError)):
        aw.Solver(order_M=1, flux="roe")


def test_paper_shock_tube_full_size(aw):
    """RP1 as the paper sets it up (8862 triangles, P2, Osher-type flux, LTS):
    60 sweeps against the oracle."""
    mesh, Q, t_end = W.riemann_problem("RP1")
    g, o = make_pair(aw, mesh, Q, order_M=2, t_end=t_end)
    for _ in range(60):
        assert g.sweep() == o.sweep()
    eg, eo = g.get_elem(), o.get_elem()
    for k in ("t", "dt", "count"):
        assert np.array_equal(eg[k], eo[k]), k
    assert rel(eg["Q"], eo["Q"]) < 1e-9
