"""Multi-rank path of bench.py on CPU: two gloo ranks, one process each.

Cells are independent, so the multi-GPU path shards the seeded batch by cell range with
no data-path collective and takes the max of the per-rank step times.  Here each rank
evaluates its shard with the oracle (CPU stands in for the rank's GPU); rank 0 gathers
the shards and checks them against a single-process evaluation of the whole batch, and
checks the max-over-ranks reduction.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

N, L, M, CELLS_PER_RANK, SEED = 8, 4.0, 8, 3, 20165


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, root: str, out_path: str):
    import sys

    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_1608_08009_gb300 import workloads as W

    g = O.make_grid(N, L, M=M)
    mine = bench.shard_cells(rank, CELLS_PER_RANK)
    f = W.two_maxwellians(CELLS_PER_RANK * world, N, L, SEED, cells=mine)
    Q = torch.from_numpy(O.collide(f, g))
    parts = [torch.empty_like(Q) for _ in range(world)]
    dist.all_gather(parts, Q)
    t_max = bench.max_over_ranks(10.0 + rank)
    if rank == 0:
        torch.save({"Q": torch.cat(parts), "t_max": t_max}, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_cells_without_exchange(tmp_path):
    world = 2
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "gathered.pt")
    mp.start_processes(_worker, args=(world, _free_port(), root, out), nprocs=world, join=True,
                       start_method="spawn")
    res = torch.load(out)
    import oracle as O
    from paper_1608_08009_gb300 import workloads as W

    full = O.collide(W.two_maxwellians(CELLS_PER_RANK * world, N, L, SEED), O.make_grid(N, L, M=M))
    # same cells, same arithmetic; batch-size-dependent BLAS blocking may change the last bit
    assert np.max(np.abs(res["Q"].numpy() - full)) <= 1e-13 * np.abs(full).max()
    assert res["t_max"] == 11.0


def test_shard_ranges_partition_the_batch():
    import bench

    ranges = [bench.shard_cells(r, 5) for r in range(4)]
    cells = [c for rg in ranges for c in rg]
    assert cells == list(range(20))
