"""Runs to a sync time before t_end (aw_advance_to, reading R18) through the
C ABI against the oracle's oc_advance_to: the cut of the steps that cross the
sync time (with the predictors re-solved over the shorter steps), the run to
the sync time, and the resumption past it.  Integers exact; predictor dofs and
conserved variables to the tolerances of the other parity tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.pyoracle import Oracle  # noqa: E402
from tests.test_gpu_parity import CASES, make_pair, rel  # noqa: E402


@pytest.fixture(scope="module")
def aw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno
    aleweno.load()
    return aleweno


def _same(g, o, tol):
    eg, eo = g.get_elem(), o.get_elem()
    for k in ("t", "dt", "count"):
        assert np.array_equal(eg[k], eo[k]), k
    assert rel(eg["Q"], eo["Q"]) < tol
    assert rel(eg["qhat"].reshape(-1, 4), eo["qhat"].reshape(-1, 4)) < max(tol, 1e-12)
    gX, gt = g.get_nodes()
    oX, ot = o.get_nodes()
    assert np.array_equal(gt, ot)
    assert np.abs(gX - oX).max() < tol * np.abs(oX).max()
    return eg


@pytest.mark.parametrize("case", ["vortex_p2", "disc_p2", "tube_p1", "vortex_p2_gts", "saltzman_p1", "kidder_p2"])
def test_advance_to_sync_time(aw, case):
    (mesh, Q), cfg = CASES[case][0](), CASES[case][1]
    g, o = make_pair(aw, mesh, Q, **cfg)
    # a sync time at the median first step: the cut acts on the elements
    # with the longer steps (all of them when the steps are global)
    d0 = o.get_elem()["dt"]
    ticks = int(np.median(d0)) - 1
    ts = ticks * o.tick
    assert (d0 > ticks).any()
    for s in (g, o):
        assert s.advance_to(ts, max_sweeps=0) == (0, 0)
    eg = _same(g, o, 1e-12)
    assert eg["dt"].max() <= ticks
    rg, ro = g.advance_to(ts), o.advance_to(ts)
    assert rg == ro and ro[1] > 0
    eg = _same(g, o, 1e-9)
    assert np.all(eg["t"] == ticks) and np.all(eg["dt"] == 0)
    assert g.sweep() == 0  # nothing moves until the sync time does
    rg, ro = g.advance_to(2 * ts, max_sweeps=25), o.advance_to(2 * ts, max_sweeps=25)
    assert rg == ro and ro[1] > 0
    _same(g, o, 1e-9)


def test_advance_to_rejects_bad_sync_times(aw):
    (mesh, Q), cfg = CASES["vortex_p1"][0](), CASES["vortex_p1"][1]
    g = aw.Solver(**cfg)
    g.load_mesh(mesh)
    g.load_state(Q)
    with pytest.raises(aw.AwError) as ex:
        g.advance_to(0.3)  # not a whole number of ticks
    assert ex.value.code == -1
    g.advance_to(0.25)
    with pytest.raises(aw.AwError) as ex:
        g.advance_to(0.125)  # behind the elements
    assert ex.value.code == -1
    assert g.advance_to(1.0)[1] > 0
    assert np.all(g.get_elem()["t"] == 2 ** 20)
