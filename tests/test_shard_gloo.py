"""Multi-rank split of independent problems, on CPU with the gloo backend
(world size 2): every problem is solved exactly once and the gathered results
equal a single-rank run.  The per-problem solver here is the oracle (CPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2107_11810_gb300 import shard


def test_partition_covers_each_problem_once_and_balances():
    sizes = [1000, 3, 77, 999, 5000, 12, 12, 800]
    parts = shard.partition(sizes, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)
    assert shard.partition(sizes, 3) == parts                       # deterministic
    assert shard.partition([], 2) == [[], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    import oracle
    from paper_2107_11810_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = inputs.pose3dof_batch(num=7, n_lo=10, n_hi=400, seed=61)

    def solve_one(p):
        r = oracle.solve(p.family, p.eps, p.bounds, p.params)
        return (r["depth"], tuple(int(x) for x in r["best_leaf"]))

    res = shard.solve_sharded(solve_one, probs, rank, world)
    if rank == 0:
        np.save(out_path, np.array([[d, *leaf] for d, leaf in res]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_single_rank(tmp_path):
    import oracle
    from paper_2107_11810_gb300 import inputs
    oracle.build()
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    probs = inputs.pose3dof_batch(num=7, n_lo=10, n_hi=400, seed=61)
    for row, p in zip(got, probs):
        r = oracle.solve(p.family, p.eps, p.bounds, p.params)
        assert row[0] == r["depth"]
        assert tuple(row[1:]) == tuple(int(x) for x in r["best_leaf"])
