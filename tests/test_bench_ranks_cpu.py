"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the
whole-job rate uses the slowest rank's time and the sum of the replicas'
element updates."""
import os
import socket

import numpy as np

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    ups = [1000, 3000][rank]
    out[rank] = bench.aggregate(ms, ups, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (20.0, 4000.0)


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(3.0, 7) == (3.0, 7.0)


def test_batched_instances_are_sharded_once_and_balanced():
    import bench
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(2000), np.log(60000), 256))]
    for world in (1, 2, 3, 8):
        parts = bench.shard_instances(sizes, world)
        assert sorted(k for p in parts for k in p) == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than one instance
        assert max(loads) <= sum(sizes) / world + max(sizes)
        assert parts == bench.shard_instances(sizes, world)  # deterministic
