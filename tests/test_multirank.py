"""Multi-rank paths of bench.py on CPU: two gloo ranks, one process each.

Cells are independent, so the multi-GPU path of the collision shards the seeded batch by
cell range with no data-path collective and takes the max of the per-rank step times.
Here each rank evaluates its shard with the oracle (CPU stands in for the rank's GPU);
rank 0 gathers the shards and checks them against a single-process evaluation of the
whole batch, and checks the max-over-ranks reduction.

The Fast Kinetic Scheme couples neighbouring cells through the transport stage: the 1D
domain is split into x-slabs whose edge cells are exchanged after every step (Sec. 4.2,
fig. mpi-decomp; bench.fks_ghosts).  Each rank steps its slab with the oracle's FKS and
the exchanged ghost cells; the gathered slabs equal the whole domain.
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


def _fks_worker(rank: int, world: int, port: int, root: str, out_path: str):
    import sys

    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from oracle import fks as K

    g = O.make_grid(8, 4.0, M=8)
    f0, left, right, dx = K.sod(g, FKS_CELLS, length=2.0)
    per = FKS_CELLS // world
    f = torch.from_numpy(f0[rank * per:(rank + 1) * per].copy())
    lo_bc, hi_bc = torch.from_numpy(left[None].copy()), torch.from_numpy(right[None].copy())
    t = 0.0
    for _ in range(FKS_STEPS):
        lo, hi = bench.fks_ghosts(f, lo_bc, hi_bc)
        f = torch.from_numpy(K.step(f.numpy(), g, t, FKS_DT, dx, FKS_TAU, lo.numpy()[0], hi.numpy()[0]))
        t += FKS_DT
    parts = [torch.empty_like(f) for _ in range(world)]
    dist.all_gather(parts, f)
    if rank == 0:
        torch.save({"f": torch.cat(parts)}, out_path)
    dist.barrier()
    dist.destroy_process_group()


FKS_CELLS, FKS_STEPS, FKS_DT, FKS_TAU = 8, 5, 0.02, 2.0


def test_two_gloo_ranks_fks_slabs_with_ghost_exchange(tmp_path):
    world = 2
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "fks.pt")
    mp.start_processes(_fks_worker, args=(world, _free_port(), root, out), nprocs=world, join=True,
                       start_method="spawn")
    import oracle as O
    from oracle import fks as K

    g = O.make_grid(8, 4.0, M=8)
    f0, left, right, dx = K.sod(g, FKS_CELLS, length=2.0)
    full = K.run(f0, g, FKS_DT, FKS_STEPS, dx, FKS_TAU, left, right)
    got = torch.load(out)["f"].numpy()
    # same arithmetic per cell; batch-size-dependent BLAS blocking may change the last bit
    assert np.max(np.abs(got - full)) <= 1e-13 * np.abs(full).max()
    # the columns did cross the slab boundary during the run
    assert any(K.shift(g.v[k], FKS_STEPS * FKS_DT, dx) != 0 for k in range(8))


def test_shard_ranges_partition_the_batch():
    import bench

    ranges = [bench.shard_cells(r, 5) for r in range(4)]
    cells = [c for rg in ranges for c in rg]
    assert cells == list(range(20))
