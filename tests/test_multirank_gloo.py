"""The multi-GPU path of bench.py on CPU: two gloo ranks (no GPU, no NCCL).

Sources shard across ranks with no exchange on the data path (each rank
solves its own 8 sources); only the per-step time is reduced (MAX over ranks)
and the traversed-edge counts summed, as bench.py does under torchrun.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen as gg


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.rmat(gg.BASE_SEED + 900, 12, 16 << 12)
    ws, r, _ = bench.dist_env()
    srcs = bench.rank_sources(g, r)
    # every rank learns every other rank's sources (test only: the bench itself exchanges none)
    allsrc = [torch.zeros(8, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allsrc, torch.from_numpy(srcs.astype(np.int64)))
    # the bench's reductions: slowest rank's step time, total traversed edges
    ms = torch.tensor([10.0 + rank], dtype=torch.float64)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    edges = torch.tensor([1000.0 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(edges, op=dist.ReduceOp.SUM)
    out[rank] = (ws, r, [a.tolist() for a in allsrc], float(ms.item()), float(edges.item()))
    dist.destroy_process_group()


def test_two_ranks_shard_sources_and_reduce_timing():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    res = [out[r] for r in range(world)]
    for rank, (ws, r, allsrc, ms, edges) in enumerate(res):
        assert (ws, r) == (world, rank)
        assert ms == 11.0 and edges == 3000.0
    s0, s1 = res[0][2]
    assert len(set(s0)) == 8 and len(set(s1)) == 8
    assert s0 != s1  # ranks solve different sources (weak scaling)
    assert res[0][2] == res[1][2]  # both ranks derived the same assignment independently
    # rank 0's sources are reproducible from the seed alone
    g = gg.rmat(gg.BASE_SEED + 900, 12, 16 << 12)
    import bench
    assert bench.rank_sources(g, 0).tolist() == s0
