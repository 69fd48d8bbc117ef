"""Host-made snapshots that drive a sweep into a failure, for the oracle and
the CUDA library alike (no GPU fault is involved: the failing state is loaded
through the state-setting entry points and the sweep reports it).

* deadlock: the elements split into two sets; set A at t = 0 with steps
  ending at tick 10, set B at t = 20.  An A element has a B member in its
  total stencil that is beyond its new time (the first half of eq.
  WENOupdate fails), a B element has an A member whose step ends before its
  own (the second half fails): no element can be updated although all are
  unfinished.
* non-physical update: a valid snapshot in which one element that the next
  sweep updates carries a memory variable Q^M that removes ten times its
  mass, so the FV update (eq. PDEfinal) leaves rho < 0 there.
"""
import numpy as np

from paper_1408_3719_gb300 import workloads as W


def deadlock_snapshot(oracle, seed=5):
    """(elem, nodes) for a loaded oracle: every element's total stencil holds
    members of both sets (checked)."""
    e = oracle.get_elem()
    ne = e["Q"].shape[0]
    rng = np.random.default_rng(seed)
    inB = rng.uniform(size=ne) < 0.5
    for i in range(ne):
        _, sw = oracle.stencils(i)
        others = sw[sw != i]
        assert inB[others].any() and (~inB[others]).any(), i
    st = dict(e)
    st["t"] = np.where(inB, 20, 0).astype(np.int64)
    st["dt"] = np.where(inB, 3, 10).astype(np.int64)
    X, t = oracle.get_nodes()
    return st, (X, np.zeros_like(t))


def nonphysical_snapshot(make_oracle, mesh, Q, warm=3):
    """A snapshot after `warm` sweeps in which one element that the next sweep
    updates (the lowest index) carries Q^M = -10 |T| Q; returns (elem, nodes,
    element index)."""
    o = make_oracle()
    o.load_mesh(mesh)
    o.load_state(Q)
    for _ in range(warm):
        o.sweep()
    st, nodes = o.get_elem(), o.get_nodes()
    probe = make_oracle()
    probe.load_mesh(mesh)
    probe.set_elem(st)
    probe.set_nodes(*nodes)
    probe.sweep()
    upd = np.nonzero(probe.get_elem()["count"] > st["count"])[0]
    i = int(upd[0])
    X = st["X"][i]
    area = 0.5 * ((X[2] - X[0]) * (X[5] - X[1]) - (X[3] - X[1]) * (X[4] - X[0]))
    st = {k: v.copy() for k, v in st.items()}
    st["QM"][i] = -10.0 * area * st["Q"][i]
    return st, nodes, i


def cases():
    return {"vortex_p2": (lambda: W.vortex(8), dict(order_M=2, t_end=1.0)),
            "tube_p1": (lambda: W.sod_tube(30, 4), dict(order_M=1, t_end=0.2))}
