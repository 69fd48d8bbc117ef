"""CPU checks behind the adjoint (no GPU):
* every element-level reverse of the CUDA library (reconstruction with the
  characteristic WENO weights, predictor with its Picard iterations, swept-edge
  Rusanov flux, node solver) agrees with fourth-order central differences of
  its own forward, run on the host;
* the oracle's frozen schedule: replaying a recorded run reproduces it bit
  for bit, loading the mesh's own node positions equals a plain load, and with
  the schedule replayed the run is a smooth function of the data (difference
  quotients at two steps agree), which is what central differences of the
  oracle need."""
import numpy as np
import pytest

from oracle.pyoracle import Oracle
from paper_1408_3719_gb300 import aleweno, build
from paper_1408_3719_gb300 import workloads as W
from tests.adjoint_fd import _J, _mask


@pytest.mark.parametrize("order", [1, 2, 3])
def test_element_reverses_match_central_differences(order):
    build.build()
    for seed in (1, 2, 3):
        r = aleweno.adjoint_selftest(order, seed)
        for part, err in r.items():
            assert err < 1e-5, (order, seed, part, err)


def _run(o, Q, xy, n):
    o.load_state_xy(Q, xy)
    for _ in range(n):
        o.sweep()
    return o.get_elem()


def test_replayed_schedule_reproduces_the_recorded_run():
    mesh, Q = W.vortex(8)
    o = Oracle(order_M=2, t_end=1.0)
    o.load_mesh(mesh)
    o.schedule("record", 14)
    e1 = _run(o, Q, mesh["xy"], 12)
    log = o.get_schedule()
    assert log[:, 0].min() > 0 and e1["count"].sum() > 12
    o.schedule("replay")
    e2 = _run(o, Q, mesh["xy"], 12)
    for k in ("Q", "QM", "X", "t", "dt", "count", "qhat"):
        assert np.array_equal(e1[k], e2[k]), k
    # loading the mesh's own node positions is the plain load
    o.schedule("free")
    o.load_state(Q)
    a = o.get_elem()
    o.load_state_xy(Q, mesh["xy"])
    b = o.get_elem()
    assert np.array_equal(a["qhat"], b["qhat"]) and np.array_equal(a["dt"], b["dt"])


def test_replay_beyond_the_log_is_an_error():
    mesh, Q = W.vortex(6)
    o = Oracle(order_M=1, t_end=1.0)
    o.load_mesh(mesh)
    o.schedule("record", 1)  # room for the initial step only
    o.load_state(Q)
    with pytest.raises(Exception):
        for _ in range(5):
            o.sweep()


def test_frozen_schedule_makes_the_run_smooth_in_the_data():
    mesh, Q = W.vortex(16)
    mask = _mask(mesh)
    o = Oracle(order_M=2, t_end=1.0)
    o.load_mesh(mesh)
    n = 20
    o.schedule("record", n + 2)
    _run(o, Q, mesh["xy"], n)
    o.schedule("replay")
    rng = np.random.default_rng(5)
    for kind in ("Q", "xy"):
        vQ = 0.1 * rng.standard_normal(Q.shape) * (kind == "Q")
        vxy = 0.01 * rng.standard_normal(mesh["xy"].shape) * (kind == "xy")

        def fd(h):
            ep = _run(o, Q + h * vQ, mesh["xy"] + h * vxy, n)
            em = _run(o, Q - h * vQ, mesh["xy"] - h * vxy, n)
            return (_J(ep["Q"], ep["X"], mask) - _J(em["Q"], em["X"], mask)) / (2 * h)

        d1, d2 = fd(1e-6), fd(1e-7)
        assert abs(d1 - d2) < 3e-6 * abs(d2), (kind, d1, d2)
