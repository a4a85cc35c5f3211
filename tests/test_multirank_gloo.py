"""The multi-GPU paths on CPU: two gloo ranks (no GPU, no NCCL).

Sources shard across ranks with no exchange on the data path (each rank
solves its own 8 sources); only the per-step time is reduced (MAX over ranks)
and the traversed-edge counts summed, as bench.py does under torchrun.  The
batched form shards its (graph, source) problems with the library's planner
(sssp_shard_problems, host only), and the differentiable form shards its
sources and sums dL/dw over the ranks with one all-reduce.
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


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch

    import oracle
    import paper_2103_12012_gb300 as sssp

    dist.init_process_group("gloo", rank=rank, world_size=world)
    # batched form: the full 512-graph recipe, 16 sources per graph
    graphs, sources = gg.workload_batch512()
    keep_g, keep_s = sssp.shard_batch(graphs, sources, rank, world)
    mine = [(g, int(s)) for g, ss in zip(keep_g, keep_s) for s in ss.tolist()]
    load = sum(int(graphs[g].E_raw) + int(graphs[g].V) for g, _ in mine)
    # differentiable form: float32 R-MAT, 8 sources dealt out over the ranks; each rank's
    # dL/dw (the oracle's tree gradient over its own sources) summed by one all-reduce
    gf = gg.rmat(gg.BASE_SEED + 901, 9, 8 << 9, wf32=(0.5, 2.0, 1e-4))
    ref = oracle.csr_of(gf)
    srcs = gg.pick_sources(gg.BASE_SEED + 901, gf, 8)
    gup = gg.normal_f32(11, (len(srcs), ref.V))
    idx = sssp.shard_sources(len(srcs), rank, world)
    d = np.stack([oracle.dijkstra(ref, int(srcs[i]))[0] for i in idx])
    p = np.stack([oracle.dijkstra(ref, int(srcs[i]))[1] for i in idx])
    grad = torch.from_numpy(oracle.tree_grad(ref, d, p, gup[idx]))
    sssp.allreduce_sum(grad)
    out[rank] = (mine, load, idx.tolist(), grad.numpy())
    dist.destroy_process_group()


def test_two_ranks_shard_the_batch_and_sum_the_gradient():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    res = [out[r] for r in range(world)]
    graphs, sources = gg.workload_batch512()
    every = [(g, int(s)) for g, ss in enumerate(sources) for s in np.asarray(ss).tolist()]
    got = res[0][0] + res[1][0]
    # disjoint and complete: every (graph, source) problem solved by exactly one rank
    assert sorted(got) == sorted(every) and len(got) == 512 * 16
    assert not set(res[0][0]) & set(res[1][0])
    # balanced by estimated edges: the ranks differ by at most the largest single problem
    biggest = max(int(g.E_raw) + int(g.V) for g in graphs)
    assert abs(res[0][1] - res[1][1]) <= biggest
    assert abs(res[0][1] - res[1][1]) / (res[0][1] + res[1][1]) < 0.01
    # gradient: sources split without overlap, and the all-reduced sum equals the whole
    assert sorted(res[0][2] + res[1][2]) == list(range(8)) and not set(res[0][2]) & set(res[1][2])
    import oracle
    gf = gg.rmat(gg.BASE_SEED + 901, 9, 8 << 9, wf32=(0.5, 2.0, 1e-4))
    ref = oracle.csr_of(gf)
    srcs = gg.pick_sources(gg.BASE_SEED + 901, gf, 8)
    gup = gg.normal_f32(11, (len(srcs), ref.V))
    d = np.stack([oracle.dijkstra(ref, int(s))[0] for s in srcs])
    p = np.stack([oracle.dijkstra(ref, int(s))[1] for s in srcs])
    whole = oracle.tree_grad(ref, d, p, gup)
    for r in range(world):
        assert np.allclose(res[r][3], whole, rtol=1e-12, atol=1e-12)
    assert np.abs(whole).sum() > 0


def test_planner_assignments():
    """sssp_shard_problems: longest first to the least loaded rank (ties: lowest index, lowest
    rank); the largest load stays within the mean plus the largest cost; bad arguments refused."""
    import paper_2103_12012_gb300 as sssp
    rank_of, load = sssp.shard_problems([5, 5, 4, 3, 3, 2, 2, 2], 3)
    assert rank_of.tolist() == [0, 1, 2, 2, 0, 1, 1, 2] and load.tolist() == [8, 9, 9]
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        c = rng.integers(1, 10 ** 6, 1000)
        r, ld = sssp.shard_problems(c, world)
        assert r.max() < world and ld.sum() == c.sum()
        assert np.array_equal(np.bincount(r, weights=c, minlength=world).astype(np.uint64), ld)
        assert ld.max() <= c.sum() / world + c.max()
    assert sssp.shard_sources(8, 1, 3).tolist() == [1, 4, 7]
    with pytest.raises(sssp.SsspError):
        sssp.shard_problems([1, 2], 0)


def _reduce_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = {"graph_replay_ms": 40.0 + rank, "per_graph_launches_ms": 400.0, "per_problem_launches_ms": 4000.0 + rank,
         "problems": 4096 + rank, "edges_total": 10 ** 6}
    d = {"forward_ms": 1.0, "backward_ms": 0.5 + rank, "forward_backward_ms": 1.6, "sources_this_rank": 16}
    bad = {"error": "boom"} if rank == 1 else dict(d)
    out[rank] = (bench._reduce_sharded("batched", b, world, "cpu"), bench._reduce_sharded("differentiable", d, world, "cpu"),
                 bench._reduce_sharded("differentiable", bad, world, "cpu"))
    dist.destroy_process_group()


def test_two_ranks_reduce_the_sharded_extras():
    """bench.py's reduction of the sharded extras: times by MAX, counts by SUM, rates recomputed
    from the reduced values; a rank whose extra failed makes every rank report an error (the
    collectives still match)."""
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_reduce_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        b, d, bad = out[r]
        assert b["graph_replay_ms"] == 41.0 and b["problems"] == 8193 and b["per_problem_launches_ms"] == 4001.0
        assert b["solves_per_s"] == round(8193 / 41.0 * 1e3, 1) and b["ranks"] == 2
        assert d["backward_ms"] == 1.5 and d["sources_this_rank"] == 32
        assert "error" in bad
