"""Failure detection on the oracle with host-made snapshots (see
tests/failure_snapshots.py): the update criterion that no element satisfies
is DEADLOCK, an update that leaves a negative density is NONPHYSICAL with the
element named, and the context refuses further sweeps afterwards."""
import pytest

from oracle.pyoracle import Oracle, OracleError
from tests import failure_snapshots as F


@pytest.mark.parametrize("case", sorted(F.cases()))
def test_deadlock_is_reported(case):
    (mesh, Q), cfg = F.cases()[case][0](), F.cases()[case][1]
    o = Oracle(**cfg)
    o.load_mesh(mesh)
    o.load_state(Q)
    st, nodes = F.deadlock_snapshot(o)
    o.set_elem(st)
    o.set_nodes(*nodes)
    with pytest.raises(OracleError) as ex:
        o.sweep()
    assert ex.value.code == -4


@pytest.mark.parametrize("case", sorted(F.cases()))
def test_nonphysical_update_is_reported(case):
    (mesh, Q), cfg = F.cases()[case][0](), F.cases()[case][1]
    st, nodes, i = F.nonphysical_snapshot(lambda: Oracle(**cfg), mesh, Q)
    o = Oracle(**cfg)
    o.load_mesh(mesh)
    o.set_elem(st)
    o.set_nodes(*nodes)
    with pytest.raises(OracleError) as ex:
        o.sweep()
    assert ex.value.code == -3
    assert f"element {i} " in str(ex.value)
    with pytest.raises(OracleError) as ex:
        o.sweep()
    assert ex.value.code == -7  # no valid state after the failed sweep
