"""The oracle's two C++ builds over the same source (oracle/oc_scalar.hpp).

* Tangent-linear (dual numbers): its values equal the plain build's bit for
  bit, and its directional derivative of the adjoint's objective agrees with
  central differences of the plain oracle (schedule recorded and replayed) to
  the differences' own accuracy; along a direction that changes nothing the
  tangent stays exactly zero.
* Operation counting: values equal bit for bit; every phase of a sweep that
  does floating-point work is counted, and the reconstruction and predictor
  counts per update grow with the order.
"""
import numpy as np
import pytest

from oracle.pyoracle import Oracle, TangentOracle, flop_counts, flop_reset
from paper_1408_3719_gb300 import workloads as W
from tests.adjoint_fd import _direction, _oracle_fd, _oracle_tlm, wavy_vortex


@pytest.mark.parametrize("M", [1, 2, 3])
def test_builds_take_the_plain_values(M):
    mesh, Q = W.vortex(8)
    a = Oracle(order_M=M, t_end=1.0)
    b = TangentOracle(order_M=M, t_end=1.0)
    c = Oracle(order_M=M, t_end=1.0, kind="count")
    for o in (a, b, c):
        o.load_mesh(mesh)
        o.load_state(Q)
        for _ in range(6):
            o.sweep()
    ea, (vb, tb), ec = a.get_elem(), b.get_elem(), c.get_elem()
    for k in ea:
        assert np.array_equal(ea[k], vb[k]) and np.array_equal(ea[k], ec[k]), k
    assert np.all(tb["Q"] == 0) and np.all(tb["qhat"] == 0)  # no seeded tangent


@pytest.mark.parametrize("M,kind", [(1, "both"), (2, "Q"), (2, "xy"), (3, "both")])
def test_tangent_linear_matches_central_differences(M, kind):
    mesh, Q = wavy_vortex(16)
    vQ, vxy = _direction(np.random.default_rng(31 + M), Q, mesh["xy"], kind)
    tlm, log_t = _oracle_tlm((mesh, Q, M, 8, vQ, vxy))
    fd, log_f = _oracle_fd((mesh, Q, M, 8, vQ, vxy))
    assert np.array_equal(log_t, log_f)
    assert abs(tlm - fd) <= 1e-7 * abs(fd), (tlm, fd)


def test_operation_counts_by_phase():
    mesh, Q = W.vortex(8)
    per = {}
    for M in (1, 2, 3):
        o = Oracle(order_M=M, t_end=1.0, kind="count")
        o.load_mesh(mesh)
        o.load_state(Q)
        o.sweep()
        flop_reset(o)
        n = o.sweep()
        f = flop_counts(o)
        assert n > 0 and all(f[k] > 0 for k in ("nodes", "flux", "update", "recon", "dt", "predictor")), f
        per[M] = (f["recon"] / n, f["predictor"] / n)
    assert per[1][0] < per[2][0] < per[3][0] and per[1][1] < per[2][1] < per[3][1]
