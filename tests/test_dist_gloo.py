"""The multi-rank path of bench.py on CPU: two gloo ranks, no GPU.

The job's parameters form one global batch that the ranks partition into
contiguous blocks (weak scaling: each block has the workload's size); every
rank solves its block with no data-path collective, and the only exchanges are
the max-reduction of the step time and, for checking, the gather of the
outputs.  The test runs the solve on each rank's block with the oracle (the
CUDA path needs a GPU), reassembles the blocks with the bench's gather and
requires the result to be bit-identical to one unsplit solve of the whole
batch; it also checks the max-over-ranks timing and the whole-job throughput
every rank reports.

The Gaussian-kernel rows split over points: each rank forms the partial rows
K_sigma(X_J, X_g) S_g of its block of points (plus lambda S_J on rank 0) with
the oracle's kernel entries, and the library's all-reduce of the rows
(solver.allreduce_rows) must give every rank the full rows M(sigma, lambda).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from oracle import problem, selection
    from workloads import get_config
    from workloads import snapshots as wsnap
    prob = get_config("reaction_diffusion_1d", n=200, r=8, s=16, m=12)
    S = wsnap.basis(prob)
    J, _ = selection.cpqr_rows(np.asarray(problem.full_matrix(prob, prob.sel_param) @ S), prob.s)
    return prob, S, J


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from oracle import online
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, S, J = _problem()
    mine = bench.rank_params(prob.test_params, rank, world)
    Y, _ = online.solve_many(prob, S, J, mine)
    X = torch.from_numpy(np.ascontiguousarray(Y @ S.T))
    whole = bench.gather_rows(X, dist, world).numpy()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, dist)
    value = bench.job_throughput(world, mine.shape[0], slowest)
    out[rank] = (slowest, value, mine.copy(), whole)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_solve_and_reassemble():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from oracle import online
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    prob, S, J = _problem()
    glob = bench.global_batch(prob.test_params, world)
    Yg, _ = online.solve_many(prob, S, J, glob)
    Xg = Yg @ S.T
    blocks = []
    for r in range(world):
        slowest, value, mine, whole = out[r]
        assert slowest == 15.0                              # max over ranks
        assert value == pytest.approx(world * prob.test_params.shape[0] / 15e-3)
        assert mine.shape == prob.test_params.shape         # weak scaling: the workload's size per rank
        np.testing.assert_array_equal(whole, Xg)            # reassembled = one unsplit solve, bit for bit
        blocks.append(mine)
    np.testing.assert_array_equal(blocks[0], prob.test_params)  # rank 0 keeps the workload's draw
    np.testing.assert_array_equal(np.concatenate(blocks), glob)  # the blocks partition the batch


def test_rank_slices_partition_any_batch():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for m in (1, 7, 64, 4097):
        for world in (1, 2, 3, 8):
            idx = np.concatenate([np.arange(m)[bench.rank_slice(m, r, world)] for r in range(world)])
            np.testing.assert_array_equal(idx, np.arange(m))


def _kernel_problem():
    from oracle import krr, selection
    from workloads import get_config
    from workloads import snapshots as wsnap
    prob = get_config("kernel_ridge", N=300, r=9, s=18, m=5)
    S = wsnap.basis(prob)
    V = krr.full_matrix(prob.X, prob.sel_param) @ S
    J, _ = selection.cpqr_rows(V, prob.s)
    return prob, S, np.asarray(J)


def _kernel_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import krr
    from paper_2510_04825_gb300.solver import allreduce_rows, point_shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, S, J = _kernel_problem()
    sh = point_shard(prob.n, rank, world)
    XJ, Xg, Sg = prob.X[J], prob.X[sh], S[sh]
    s = len(J)
    parts = []
    for sigma, lam in prob.test_params:
        Kg = krr.kernel_rows(np.vstack([XJ, Xg]), np.arange(s), sigma)[:, s:]  # K(X_J, X_g)
        Mg = Kg @ Sg + (lam * S[J] if rank == 0 else 0.0)
        parts.append(Mg)
    M = torch.from_numpy(np.ascontiguousarray(np.stack(parts)))
    allreduce_rows(M, dist)
    out[rank] = (sh.start, sh.stop, M.numpy().copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_kernel_rows_over_point_shards():
    from oracle import krr
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_kernel_worker, args=(world, port, out), nprocs=world, join=True)
    prob, S, J = _kernel_problem()
    Mo = np.stack([krr.subsampled_matrix(prob.X, S, J, p) for p in prob.test_params])
    bounds = sorted((out[r][0], out[r][1]) for r in range(world))
    assert bounds[0][0] == 0 and bounds[-1][1] == prob.n
    assert all(bounds[i][1] == bounds[i + 1][0] for i in range(world - 1))  # the shards tile the points
    for r in range(world):
        M = out[r][2]
        assert np.abs(M - Mo).max() <= 1e-13 * np.abs(Mo).max()  # every rank holds the full rows


def test_point_shards_partition_the_points():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2510_04825_gb300.solver import point_shard
    for n in (1, 7, 2500, 200_000):
        for world in (1, 2, 3, 8):
            idx = np.concatenate([np.arange(n)[point_shard(n, g, world)] for g in range(world)])
            np.testing.assert_array_equal(idx, np.arange(n))
