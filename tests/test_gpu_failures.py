"""Failure detection through the C ABI with host-made snapshots (no GPU fault
is involved; see tests/failure_snapshots.py): DEADLOCK when no element
satisfies the update criterion, NONPHYSICAL naming the element whose update
leaves rho < 0, as the oracle reports them; the context then refuses further
sweeps (STATE) until a state is loaded again."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.pyoracle import Oracle, OracleError  # noqa: E402
from tests import failure_snapshots as F  # noqa: E402


@pytest.fixture(scope="module")
def aw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno
    aleweno.load()
    return aleweno


@pytest.mark.parametrize("case", sorted(F.cases()))
def test_deadlock_matches_the_oracle(aw, case):
    (mesh, Q), cfg = F.cases()[case][0](), F.cases()[case][1]
    o = Oracle(**cfg)
    o.load_mesh(mesh)
    o.load_state(Q)
    st, nodes = F.deadlock_snapshot(o)
    g = aw.Solver(**cfg)
    g.load_mesh(mesh)
    for s in (g, o):
        s.set_elem(st)
        s.set_nodes(*nodes)
    with pytest.raises(OracleError) as eo:
        o.sweep()
    with pytest.raises(aw.AwError) as eg:
        g.sweep()
    assert eo.value.code == eg.value.code == -4
    with pytest.raises(aw.AwError) as eg:
        g.sweep()
    assert eg.value.code == -7
    g.load_state(Q)  # a new state clears the failure
    assert g.sweep() > 0


@pytest.mark.parametrize("case", sorted(F.cases()))
def test_nonphysical_update_matches_the_oracle(aw, case):
    (mesh, Q), cfg = F.cases()[case][0](), F.cases()[case][1]
    st, nodes, i = F.nonphysical_snapshot(lambda: Oracle(**cfg), mesh, Q)
    o = Oracle(**cfg)
    g = aw.Solver(**cfg)
    for s in (g, o):
        s.load_mesh(mesh)
        s.set_elem(st)
        s.set_nodes(*nodes)
    with pytest.raises(OracleError) as eo:
        o.sweep()
    with pytest.raises(aw.AwError) as eg:
        g.sweep()
    assert eo.value.code == eg.value.code == -3
    assert f"element {i} " in str(eo.value) and f"element {i} " in str(eg.value)
    with pytest.raises(aw.AwError) as eg:
        g.sweep()
    assert eg.value.code == -7
