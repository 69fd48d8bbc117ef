"""The GPU adjoint against the oracle's tangent-linear product.

The oracle's dual-number build (oracle/oc_scalar.hpp: the oracle's own
arithmetic on (value, tangent) pairs) gives J'(x0) v exactly up to rounding
for a seeded direction v; the adjoint gives <dJ/dx0, v> from one reverse pass.
Both differentiate the same discrete map (the run's schedule and the loaded
mesh's stencils held fixed), so they must agree to 1e-10 relative with no
allowance for a difference quotient's truncation or cancellation: on the
512-triangle vortex with an entropy wave (P1-P3, 50 sweeps) and on the
49,928-triangle adjoint workload (P2, 50 sweeps, checkpoints every 10)."""
import multiprocessing as mp

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_3719_gb300 import workloads as W  # noqa: E402

from tests.adjoint_fd import _direction, _oracle_tlm, wavy_vortex  # noqa: E402
from tests.test_gpu_adjoint import GpuCase, _need_gpu  # noqa: E402

TOL = 1e-10


def _against_tlm(mesh, Q0, order, n_sweeps, n_dirs, workers, seed):
    aleweno = _need_gpu()
    run = GpuCase(aleweno, mesh, Q0, order, n_sweeps, 10)
    rng = np.random.default_rng(seed)
    dirs = [_direction(rng, Q0, run.xy0, ("Q", "xy", "both")[k % 3]) for k in range(n_dirs)]
    with mp.get_context("spawn").Pool(min(workers, n_dirs)) as pool:
        res = pool.map(_oracle_tlm, [(mesh, Q0, order, n_sweeps, vQ, vxy) for vQ, vxy in dirs])
    worst = 0.0
    for (vQ, vxy), (tlm, log) in zip(dirs, res):
        assert np.array_equal(log, run.log)  # both sides took the same schedule
        ad = float(np.sum(run.gQ0 * vQ) + np.sum(run.gxy0 * vxy))
        worst = max(worst, abs(ad - tlm) / abs(tlm))
        assert abs(ad - tlm) <= TOL * abs(tlm), (ad, tlm)
    return worst


@pytest.mark.parametrize("order", [1, 2, 3])
def test_adjoint_matches_oracle_tangent_linear_small(order):
    _against_tlm(*wavy_vortex(16), order, 50, 6, 6, 77 + order)


def test_adjoint_matches_oracle_tangent_linear_full_size():
    """The adjoint workload: P2, 50 sweeps, 49,928 triangles, 3 directions."""
    _against_tlm(*W.vortex(158), 2, 50, 3, 3, 4242)
