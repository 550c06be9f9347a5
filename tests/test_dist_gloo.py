"""The multi-rank path of bench.py on CPU: two gloo ranks, no GPU.

Every rank solves its own parameters (weak scaling, no data-path collective);
the only exchange is the max-reduction of the step time.  The test checks the
sharding (distinct draws of the same distribution), the max-over-ranks timing
and the whole-job throughput every rank would report.
"""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = np.random.default_rng(0).uniform(0.0, 1.0, (64, 4))
    mine = bench.rank_params(base, rank)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, dist)
    value = bench.job_throughput(world, mine.shape[0], slowest)
    gathered = [torch.zeros(64 * 4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(mine.reshape(-1).copy()))
    out[rank] = (slowest, value, [g.numpy().copy() for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        slowest, value, gathered = out[r]
        assert slowest == 15.0                     # max over ranks
        assert value == pytest.approx(2 * 64 / 15e-3)
        p0, p1 = (g.reshape(64, 4) for g in gathered)
        assert not np.allclose(p0, p1)             # every rank has its own parameters
        assert p1.min() >= p0.min() - 1e-12 and p1.max() <= p0.max() + 1e-12
