"""Oracle runs that the GPU parity tests hand to spawned worker processes, so
that several serial oracle runs proceed side by side on the host's cores
while the GPU tests go on (spawned, never forked: a process forked after the
first CUDA call can hang).  Imports neither torch nor the CUDA library."""
from __future__ import annotations

import multiprocessing
import os
from concurrent.futures import ProcessPoolExecutor

_POOL = None


def pool() -> ProcessPoolExecutor:
    global _POOL
    if _POOL is None:
        import atexit
        _POOL = ProcessPoolExecutor(max_workers=max(1, min(12, (os.cpu_count() or 2) - 1)),
                                    mp_context=multiprocessing.get_context("spawn"))
        atexit.register(_POOL.shutdown, wait=False, cancel_futures=True)
    return _POOL


def _result(o):
    e = o.get_elem()
    X, t = o.get_nodes()
    return dict(Q=e["Q"], t=e["t"], count=e["count"], X=e["X"], nX=X, nt=t)


def vortex_to_final_time(n: int, M: int, eps: float = 0.0):
    """The isentropic vortex on the n x n torus, LTS, to t_end = 1; with eps
    > 0 every initial average is multiplied by 1 +- eps (seeded signs)."""
    import numpy as np
    from oracle.pyoracle import Oracle
    from paper_1408_3719_gb300 import workloads as W
    mesh, Q = W.vortex(n)
    if eps > 0:
        Q = Q * (1.0 + eps * np.random.default_rng(5).choice([-1.0, 1.0], Q.shape))
    o = Oracle(order_M=M, t_end=1.0)
    o.load_mesh(mesh)
    o.load_state(Q)
    sweeps, updates = o.advance()
    return dict(_result(o), sweeps=sweeps, updates=updates)


def explosion_window(h_centre: float, M: int, snap: dict, nX, nt, n_sweeps: int):
    """n_sweeps sweeps of the graded-disc explosion from a snapshot."""
    from oracle.pyoracle import Oracle
    from paper_1408_3719_gb300 import workloads as W
    mesh, _ = W.explosion(h_centre)
    o = Oracle(order_M=M, t_end=0.25)
    o.load_mesh(mesh)
    o.set_elem(snap)
    o.set_nodes(nX, nt)
    per_sweep = [o.sweep() for _ in range(n_sweeps)]
    return dict(_result(o), per_sweep=per_sweep)


def batch_instance(k: int, n_sweeps: int, M: int = 2):
    """Instance k of the benchmark's batch, alone, for n_sweeps sweeps."""
    from oracle.pyoracle import Oracle
    from paper_1408_3719_gb300 import workloads as W
    d = W.batched_instances()[k]
    o = Oracle(order_M=M, t_end=d["t_end"])
    o.load_mesh(d["mesh"])
    o.load_state(d["q"])
    for _ in range(n_sweeps):
        o.sweep()
    return _result(o)
