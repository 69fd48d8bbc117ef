"""Batched instances (one sweep advances many independent meshes): each
instance of the batch must evolve exactly as the oracle evolves it alone —
same ready sets (so the batch's update count per sweep is the sum of the
instances'), same update counts, conserved variables to 1e-9 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.pyoracle import Oracle  # noqa: E402
from paper_1408_3719_gb300 import workloads as W  # noqa: E402


def test_batched_instances_match_the_oracle_one_by_one():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno

    inst = W.batched_instances(4, lo=400, hi=1600, seed=W.SEED_BASE + 40)
    t_ends = [d["t_end"] for d in inst]
    t_ends[1] = 0.004  # finishes while the others keep running
    g = aleweno.Solver(order_M=2, t_end=max(t_ends))
    g.load_batch([d["mesh"] for d in inst], t_ends)
    g.load_state(np.concatenate([d["q"] for d in inst]))
    oracles = []
    for d, te in zip(inst, t_ends):
        o = Oracle(order_M=2, t_end=te)
        o.load_mesh(d["mesh"])
        o.load_state(d["q"])
        oracles.append(o)
    for _ in range(40):
        n_g = g.sweep()
        n_o = sum(o.sweep() for o in oracles)
        assert n_g == n_o
    eg = g.get_elem()
    off = g.tri_offsets
    for k, o in enumerate(oracles):
        eo = o.get_elem()
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(eg["count"][sl], eo["count"])
        assert np.array_equal(eg["t"][sl], eo["t"])
        err = np.abs(eg["Q"][sl] - eo["Q"]).max() / np.abs(eo["Q"]).max()
        assert err < 1e-9, (k, err)
    assert np.all(eg["t"][off[1]:off[2]] == 2 ** 20)  # the short instance reached its end
    t_host = np.empty(g.n_tris)
    g.get_state(t=t_host)
    assert np.allclose(t_host[off[1]:off[2]], t_ends[1])


def test_fullsize_batch_sampled_instances_against_the_oracle():
    """The benchmark's batch (256 instances, 2k-60k triangles, P2) in its
    launch configuration (autotuned tiles, the captured sweep graph): after
    a number of batch sweeps, the three smallest instances match the oracle
    run alone on each, element by element."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno

    inst = W.batched_instances()
    sizes = np.array([d["mesh"]["tri"].shape[0] for d in inst])
    t_ends = [d["t_end"] for d in inst]
    g = aleweno.Solver(order_M=2, t_end=max(t_ends))
    g.load_batch([d["mesh"] for d in inst], t_ends)
    g.load_state(np.concatenate([d["q"] for d in inst]))
    tiles, _ = g.autotune(20)
    assert g.get_tiles() == tiles
    n_sweeps = 30
    g.enqueue(n_sweeps)
    g.sync()
    eg = g.get_elem()
    off = g.tri_offsets
    for k in np.argsort(sizes, kind="stable")[:3]:
        o = Oracle(order_M=2, t_end=t_ends[k])
        o.load_mesh(inst[k]["mesh"])
        o.load_state(inst[k]["q"])
        for _ in range(n_sweeps):
            o.sweep()
        eo = o.get_elem()
        sl = slice(off[k], off[k + 1])
        assert np.array_equal(eg["count"][sl], eo["count"]), k
        assert np.array_equal(eg["t"][sl], eo["t"]), k
        assert eo["count"].sum() > 0
        err = np.abs(eg["Q"][sl] - eo["Q"]).max() / np.abs(eo["Q"]).max()
        assert err < 1e-9, (k, err)
