"""The multi-GPU path (replicas) on CPU: two gloo ranks.

Every rank solves its own replica -- the same workload with problem index =
rank, so independent random streams -- and the benchmark reports the work of
all ranks over the slowest rank's time.  Here two processes check the
reductions the benchmark uses and that replicas of a small problem, run by
the oracle, are independent (different walks) and estimate the same thing.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_2305_04403_gb300 import inputs as I
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    assert bench._over_ranks(dist, 1.0 + rank, "max", "cpu") == float(world)
    assert bench._over_ranks(dist, 10.0 * (rank + 1), "sum", "cpu") == 10.0 * world * (world + 1) / 2
    # this rank's replica: problem index = rank
    v, f = I.icosphere(2)
    q = I.ball_queries(4, 0.6, 1)
    res = O.dl_walks(v, f, q, 400, 3, seed=0, problem=rank, poly=I.POLY_CONFIG1)
    pw = torch.from_numpy(res["per_walk"])
    got = [torch.zeros_like(pw) for _ in range(world)]
    dist.all_gather(got, pw)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        np.save(os.path.join(out_dir, "replicas.npy"), torch.stack(got).numpy())


def test_two_gloo_ranks_reduce_and_replicate(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    rep = np.load(tmp_path / "replicas.npy")          # (ranks, Q, N)
    assert rep.shape[0] == 2
    assert not np.array_equal(rep[0], rep[1])         # independent streams
    m, s = rep.mean(2), rep.std(2, ddof=1) / np.sqrt(rep.shape[2])
    assert np.all(np.abs(m[0] - m[1]) <= 5 * np.sqrt(s[0] ** 2 + s[1] ** 2))
