"""Full-size workloads on the CUDA path, in the launch configuration the benchmark uses.

For every workload the GPU CSR equals the oracle's, every source of the R-MAT,
grid and differentiable workloads (and a sample of the 8,192 batch problems)
is compared with the oracle's Dijkstra element by element, in the schedule
the benchmark's autotuner picks, and every source and every batch problem is
checked against properties that hold at any size: d(s)=0,
d[v] <= d[u] + w(u,v) on every edge, every predecessor edge is tight, and the
predecessor is the smallest-id tight in-neighbour.  Float32 distances must be
bit-exact as well (both sides round each d(u)+w once).
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sssp():
    import paper_2103_12012_gb300 as m
    m.lib()
    return m


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def check_csr_equal(g, ref):
    assert g.E == ref.E
    assert np.array_equal(u32(g.row_ptr), ref.row_ptr)
    assert np.array_equal(u32(g.col), ref.col)
    assert np.array_equal(u32(g.w), ref.w.view(np.uint32))


def check_invariants(g, dist, pred, sources):
    """Properties of a shortest-path result that hold at any size (checked with torch on the device)."""
    V = g.V
    rp = g.row_ptr.long()
    tail = torch.repeat_interleave(torch.arange(V, device="cuda"), rp[1:] - rp[:-1])
    head = g.col.long()
    f32 = g.wtype == 1
    INF = torch.tensor(float("inf") if f32 else 0xFFFFFFFF, device="cuda", dtype=torch.float64)
    w = g.w.double() if f32 else (g.w.long() & 0xFFFFFFFF).double()
    for i, s in enumerate(sources):
        d = dist[i].double() if f32 else (dist[i].long() & 0xFFFFFFFF).double()
        p = pred[i].long() & 0xFFFFFFFF
        assert d[s] == 0 and p[s] == 0xFFFFFFFF
        du, dv = d[tail], d[head]
        fin = du != INF
        # candidate in the arithmetic of the weights: float32 sum rounded once, or exact integers
        cand = (dist[i][tail].float() + g.w.float()).double() if f32 else du + w
        assert bool((dv[fin] <= cand[fin]).all()), "an edge is not relaxed"
        tight = fin & (cand == dv) & (head != s)
        # canonical predecessor: smallest tight in-neighbour
        best = torch.full((V,), 0xFFFFFFFF, dtype=torch.long, device="cuda")
        best.scatter_reduce_(0, head[tight], tail[tight], reduce="amin")
        reached = (d != INF)
        reached[s] = False
        assert torch.equal(p[reached], best[reached])
        assert bool((p[~reached & (torch.arange(V, device="cuda") != s)] == 0xFFFFFFFF).all())


def oracle_runs(ref, sources):
    """The oracle's Dijkstra for every source, in threads (the C oracle runs without the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(len(sources), 8)) as ex:
        return list(ex.map(lambda s: oracle.dijkstra(ref, int(s))[:2], list(sources)))


def check_oracle_sources(ref, dist, pred, sources, which=None, runs=None):
    which = range(len(sources)) if which is None else which
    runs = runs or oracle_runs(ref, [sources[i] for i in which])
    for (d, p), i in zip(runs, which):
        assert np.array_equal(u32(dist[i]), d.view(np.uint32)), f"source #{i}"
        assert np.array_equal(u32(pred[i]), p), f"source #{i}"
    return runs


def bench_options(sssp, g, srcs, monkeypatch, tmp_path):
    """The schedule the benchmark times: the autotuner's choice for this graph and these sources
    (a fresh cache, as on a fresh machine)."""
    monkeypatch.setenv("SSSP_TUNE_CACHE", str(tmp_path / "tune.json"))
    opts, ms = sssp.autotune(g, srcs, trials=2)
    assert ms is not None
    return opts


def test_rmat22_eight_sources(sssp, monkeypatch, tmp_path):
    """All 8 sources element by element against the oracle, on the graph as built and on the
    locality layout the benchmark solves on, in the benchmark's autotuned schedule."""
    g0, srcs, P = gg.workload_rmat22()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    check_csr_equal(g, ref)
    del g0
    dist, pred, st, stats = sssp.solve(g, srcs)
    assert st == sssp.SSSP_OK
    runs = check_oracle_sources(ref, dist, pred, srcs)
    check_invariants(g, dist, pred, srcs.tolist())
    # the benchmark solves on the locality layout: the renaming equals the oracle's, and the
    # solve on it returns the same distances and canonical predecessors, in the caller's ids
    h = sssp.layout(g)
    ids, slots, rh = oracle.layout(ref, P)
    assert np.array_equal(u32(h.ids), ids) and np.array_equal(u32(h.slots), slots)
    check_csr_equal(h, rh)
    assert np.array_equal(u32(h.eid), rh.eid)
    del rh
    opts = bench_options(sssp, h, srcs, monkeypatch, tmp_path)
    dist2, pred2, st, _ = sssp.solve(h, srcs, opts)
    assert st == sssp.SSSP_OK
    check_oracle_sources(ref, dist2, pred2, srcs, runs=runs)


def test_grid4096_corner(sssp, monkeypatch, tmp_path):
    """The grid in the benchmark's autotuned schedule (and in a fixed wide-bucket one)."""
    g0, srcs, P = gg.workload_grid4096()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    check_csr_equal(g, ref)
    del g0
    opts = bench_options(sssp, g, srcs, monkeypatch, tmp_path)
    runs = None
    for o in (opts, sssp.options(delta=2048, tile=4096)):
        dist, pred, st, stats = sssp.solve(g, srcs, o)
        assert st == sssp.SSSP_OK
        runs = check_oracle_sources(ref, dist, pred, srcs, runs=runs)
    check_invariants(g, dist, pred, srcs.tolist())


def test_er16k_prune_and_solve(sssp):
    g0, srcs, P = gg.workload_er16k()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    check_csr_equal(g, ref)
    for mode in (0, 1):
        keep, wit = sssp.prune(g, mode)
        rk, rw = oracle.trishla(ref, P, mode)
        assert np.array_equal(keep.cpu().numpy(), rk) and np.array_equal(u32(wit), rw)
    gp = sssp.compact(g, keep)
    for graph in (g, gp):
        dist, pred, st, _ = sssp.solve(graph, srcs)
        assert st == sssp.SSSP_OK
        check_oracle_sources(ref, dist, pred, srcs, [0])
        check_invariants(graph, dist, pred, srcs.tolist())


def test_rmat22_trishla_witnesses_and_sampled_completeness(sssp):
    """Trishla (Algorithm 1, local mode) on the full R-MAT scale-22 graph with 148 partitions.
    Every pruned edge (u, v_j) names a witness v_i in u's partition for which (u, v_i) and
    (v_i, v_j) are edges and w(u, v_j) > w(u, v_i) + w(v_i, v_j); every kept edge names none.
    On a seeded sample of edges the least witness found by brute force from that definition
    (or none) equals the GPU's keep flag and witness."""
    g0, _, P = gg.workload_rmat22()
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    del g0
    keep, wit = sssp.prune(g, 0)
    V, E, NONE = g.V, g.E, 0xFFFFFFFF
    B = -(-V // P)
    rp = g.row_ptr.long()
    deg = rp[1:] - rp[:-1]
    tail = torch.repeat_interleave(torch.arange(V, device="cuda"), deg)
    head = g.col.long()
    w = g.w.long() & 0xFFFFFFFF
    keys = tail * V + head
    assert bool((keys[1:] > keys[:-1]).all())  # canonical CSR: rows sorted, no parallel edges
    wt = wit.long() & 0xFFFFFFFF
    pruned = keep == 0
    assert bool((wt[~pruned] == NONE).all())

    def edge_index(a, b):  # index of edge (a, b), or -1
        k = a * V + b
        i = torch.searchsorted(keys, k).clamp(max=E - 1)
        return torch.where(keys[i] == k, i, torch.full_like(i, -1))

    e = torch.nonzero(pruned).squeeze(1)
    assert e.numel() > 0
    u, vj, vi = tail[e], head[e], wt[e]
    assert bool((vi < V).all()) and bool((vi // B == u // B).all())
    e1, e2 = edge_index(u, vi), edge_index(vi, vj)
    assert bool((e1 >= 0).all()) and bool((e2 >= 0).all())
    assert bool((w[e] > w[e1] + w[e2]).all())
    del e, u, vj, vi, e1, e2

    rng = np.random.default_rng(2103)
    se = torch.from_numpy(rng.choice(E, 20000, replace=False).astype(np.int64)).cuda()
    su, sv = tail[se], head[se]
    lens = deg[su]
    pair = torch.repeat_interleave(torch.arange(se.numel(), device="cuda"), lens)
    start = torch.cumsum(lens, 0) - lens
    ce = rp[su][pair] + torch.arange(pair.numel(), device="cuda") - start[pair]  # edge (u, v_i)
    ci = head[ce]
    e2 = edge_index(ci, sv[pair])
    ok = (ci // B == su[pair] // B) & (e2 >= 0)
    ok &= w[se][pair] > w[ce] + torch.where(e2 >= 0, w[e2.clamp(min=0)], torch.zeros_like(e2))
    least = torch.full((se.numel(),), NONE, dtype=torch.long, device="cuda")
    least.scatter_reduce_(0, pair[ok], ci[ok], reduce="amin")
    assert torch.equal(least, wt[se])
    assert torch.equal(least != NONE, pruned[se])
    assert int(pruned[se].sum()) > 0


def test_rmat18_f32_forward_backward(sssp, monkeypatch, tmp_path):
    """The differentiable workload as the benchmark runs it: 16 partitions, autotuned schedule."""
    g0, srcs, gup = gg.workload_rmat18_f32()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=16)
    check_csr_equal(g, ref)
    opts = bench_options(sssp, g, srcs, monkeypatch, tmp_path)
    dist, pred, st, _ = sssp.solve(g, srcs, opts)
    assert st == sssp.SSSP_OK
    rd = np.empty((len(srcs), g.V), np.float32)
    rp = np.empty((len(srcs), g.V), np.uint32)
    for i, (d, p) in enumerate(oracle_runs(ref, srcs)):
        rd[i], rp[i] = d, p
    assert np.array_equal(u32(dist), rd.view(np.uint32))
    assert np.array_equal(u32(pred), rp)
    check_invariants(g, dist, pred, srcs.tolist())
    grad = sssp.backward(g, pred, torch.from_numpy(gup).cuda()).cpu().numpy().astype(np.float64)
    rg = oracle.tree_grad(ref, rd, rp, gup)
    # float64 accumulation on both sides; the float32 output rounding bounds the difference
    assert np.allclose(grad, rg, rtol=1e-6, atol=1e-6 * np.abs(rg).max())
    assert (grad[rg == 0] == 0).all()


def test_batch512_sampled_and_certified(sssp):
    """The full batch in the schedule the benchmark times (the batch tuner's choice: block size,
    tile and bucket width), replayed from its CUDA graph."""
    graphs0, sources = gg.workload_batch512()
    graphs = [oracle.csr_of(g) for g in graphs0]
    del graphs0
    b = sssp.Batch(graphs, sources)
    b.autotune()
    b.make_plan()
    b.replay()
    st, stats = b.status()
    assert st == sssp.SSSP_OK
    assert b.n_problems == sum(len(s) for s in sources) == 512 * 16
    rng = np.random.default_rng(7)
    for i in rng.choice(b.n_problems, 96, replace=False):
        gi, s = int(b.prob_graph[i]), int(b.prob_source[i])
        d, p, _ = oracle.dijkstra(graphs[gi], s)
        bd, bp = b.result(i)
        assert np.array_equal(u32(bd), d) and np.array_equal(u32(bp), p), (i, gi, s)
    # every one of the 8,192 problems: the full certificate (d(s) = 0, every edge relaxed, the
    # predecessor the smallest tight in-neighbour, unreached vertices unlabelled), per graph on
    # the device over its 16 problems at once
    first = {}
    for i in range(b.n_problems):
        first.setdefault(int(b.prob_graph[i]), []).append(i)
    for gi, probs in first.items():
        G = graphs[gi]
        gd = sssp.upload_csr(G.V, G.row_ptr, G.col, G.w)
        dist = torch.stack([b.result(i)[0] for i in probs])
        pred = torch.stack([b.result(i)[1] for i in probs])
        check_invariants(gd, dist, pred, [int(b.prob_source[i]) for i in probs])
