"""Runs to an intermediate time (reading R18) on the oracle.

A run stopped at a sync time t_s is the run whose final time is t_s: every
step is clipped at it (as the last steps are clipped at t_f, reading R1), and
the elements stop there.  With the same tick length (t_end / 2^K = t_s /
2^(K - k)) the two runs must agree bit for bit:
* from the start, with steps that cross t_s cut back and their predictors
  re-solved over the shorter steps;
* when continued from t_s, with the run started afresh from the state at t_s
  (every element at t_s, no memory variables left: the elements that reached
  t_s first have all their nodes at t_s, so no later surface touches them),
  up to the rounding of absolute tick counts.
"""
import numpy as np
import pytest

from oracle.pyoracle import Oracle, OracleError
from paper_1408_3719_gb300 import workloads as W

KEYS = ("Q", "QM", "HM", "X", "t", "dt", "count", "qhat")


def _pair(mesh, Q, M, t_end, K, t_s, k, **cfg):
    a = Oracle(order_M=M, t_end=t_end, time_quantum_log2=K, **cfg)
    b = Oracle(order_M=M, t_end=t_s, time_quantum_log2=K - k, **cfg)
    for o in (a, b):
        o.load_mesh(mesh)
        o.load_state(Q)
    assert a.tick == b.tick
    return a, b


@pytest.mark.parametrize("M,gts", [(1, False), (2, False), (3, False), (2, True)])
def test_stop_at_sync_time_is_the_run_that_ends_there(M, gts):
    mesh, Q = W.vortex(8)
    a, b = _pair(mesh, Q, M, 1.0, 20, 0.25, 2, gts=gts)
    sa, ua = a.advance_to(0.25)
    sb, ub = b.advance()
    assert (sa, ua) == (sb, ub) and ua > 0
    ea, eb = a.get_elem(), b.get_elem()
    for key in KEYS:
        assert np.array_equal(ea[key], eb[key]), key
    assert np.all(ea["t"] == 2 ** 18) and np.all(ea["dt"] == 0)
    xa, ta = a.get_nodes()
    xb, tb = b.get_nodes()
    assert np.array_equal(xa, xb) and np.array_equal(ta, tb)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_steps_crossing_the_sync_time_are_cut_back(M):
    """t_s = 2^-9: every initial step crosses it, so every predictor is
    re-solved over the shorter step from its own tau = 0 dofs; the run that
    ends at t_s computes those steps clipped in the first place."""
    mesh, Q = W.vortex(8)
    a, b = _pair(mesh, Q, M, 1.0, 20, 2.0 ** -9, 9)
    d0 = a.get_elem()["dt"]
    assert np.all(d0 > 2 ** 11)
    a.advance_to(2.0 ** -9, max_sweeps=0)  # the cut alone
    ea, eb = a.get_elem(), b.get_elem()
    for key in KEYS:
        assert np.array_equal(ea[key], eb[key]), key
    assert np.all(ea["dt"] == 2 ** 11)
    assert a.advance_to(2.0 ** -9) == b.advance()
    ea, eb = a.get_elem(), b.get_elem()
    for key in KEYS:
        assert np.array_equal(ea[key], eb[key]), key


@pytest.mark.parametrize("M", [1, 2])
def test_continuing_from_the_sync_time_is_a_fresh_start_there(M):
    mesh, Q = W.vortex(8)
    a = Oracle(order_M=M, t_end=1.0)
    a.load_mesh(mesh)
    a.load_state(Q)
    _, u1 = a.advance_to(0.5)
    e1 = a.get_elem()
    x1, t1 = a.get_nodes()
    assert np.all(e1["QM"] == 0) and np.all(e1["HM"] == 0) and np.all(t1 == 2 ** 19)
    _, u2 = a.advance_to(1.0)
    c = Oracle(order_M=M, t_end=0.5, time_quantum_log2=19)
    c.load_mesh(mesh)
    c.load_state_xy(e1["Q"], x1)
    _, uc = c.advance()
    assert uc == u2
    ea, ec = a.get_elem(), c.get_elem()
    for key in ("Q", "X", "qhat"):
        # equal up to rounding: the surfaces interpolate absolute tick
        # counts (2^19 more on the continued run) at their Gauss points
        assert np.abs(ea[key] - ec[key]).max() <= 1e-12 * np.abs(ec[key]).max(), key
    assert np.array_equal(ea["t"], ec["t"] + 2 ** 19)
    assert np.array_equal(ea["count"], ec["count"] + e1["count"])
    assert u1 + u2 == int(ea["count"].sum())


def test_sync_time_arguments():
    mesh, Q = W.vortex(6)
    a = Oracle(order_M=1, t_end=1.0)
    a.load_mesh(mesh)
    a.load_state(Q)
    with pytest.raises(OracleError):
        a.advance_to(0.3)  # not a whole number of ticks
    a.advance_to(0.25)
    with pytest.raises(OracleError):
        a.advance_to(0.125)  # behind the elements
    assert a.advance_to(0.25) == (0, 0)
    assert a.advance_to(1.0)[1] > 0
    assert np.all(a.get_elem()["t"] == 2 ** 20)
