"""Parity of the CUDA path (through the C ABI) with the CPU oracle on seeded inputs.

Sizes span several tiles and partition blocks with ragged tails.  Integer
results (CSR, keep masks, witnesses, uint32 distances, predecessors) must be
bit-exact; float32 distances must be bit-exact as well (both sides round every
d(u)+w once to float32 and reach the same fixpoint), which is tighter than
the 1e-6 relative bound the float32 workload allows.  Gradients: float64
accumulation on both sides, compared at rtol 1e-5 (float32 output rounding).
"""
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


def raw_graph(seed, V, E, f32=False, wlo=1, whi=255, loops=True):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, V, E).astype(np.uint32)
    dst = rng.integers(0, V, E).astype(np.uint32)
    if not loops:
        dst = np.where(src == dst, (dst + 1) % V, dst).astype(np.uint32)
    w = rng.uniform(0.5, 2.0, E).astype(np.float32) if f32 else rng.integers(wlo, whi + 1, E).astype(np.uint32)
    return src, dst, w


def check_solve(sssp, g_dev, ref, sources, opts=None):
    dist, pred, st, stats = sssp.solve(g_dev, np.asarray(sources, np.uint32), opts)
    assert st == sssp.SSSP_OK
    for i, s in enumerate(sources):
        d, p, _ = oracle.dijkstra(ref, int(s))
        assert np.array_equal(u32(dist[i]), d.view(np.uint32)), f"dist mismatch, source {s}"
        assert np.array_equal(u32(pred[i]), p), f"pred mismatch, source {s}"
    return stats


# --------------------------------------------------------------------- K1 / K2

@pytest.mark.parametrize("seed,V,E,f32", [(0, 1000, 20000, False), (1, 5000, 3000, False), (2, 777, 50000, True),
                                          (3, 1, 5, False), (4, 64, 0, False), (5, 100000, 400000, False)])
def test_csr_build_parity(sssp, seed, V, E, f32):
    src, dst, w = raw_graph(seed, V, E, f32=f32, whi=9)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w)
    assert g.E == ref.E
    assert np.array_equal(u32(g.row_ptr), ref.row_ptr)
    if ref.E:
        assert np.array_equal(u32(g.col), ref.col)
        assert np.array_equal(u32(g.w), ref.w.view(np.uint32))
        assert np.array_equal(u32(g.eid), ref.eid)


def test_csr_build_rejects_bad_ids_and_weights(sssp):
    with pytest.raises(sssp.SsspError):
        sssp.build_csr(10, np.array([0, 10], np.uint32), np.array([1, 2], np.uint32), np.array([1, 1], np.uint32))
    with pytest.raises(sssp.SsspError):
        sssp.build_csr(10, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), np.array([1, 0], np.uint32))


@pytest.mark.parametrize("V,P", [(16384, 4), (1000, 7), (4194, 148), (10, 10)])
def test_partition_parity(sssp, V, P):
    src, dst, w = raw_graph(11, V, 8 * V)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    b, inter = sssp.partition(g)
    rb, ri = oracle.partition(V, P, ref)
    assert np.array_equal(u32(b), rb)
    assert np.array_equal(inter.cpu().numpy().astype(np.uint64), ri)


# ------------------------------------------------------------- locality layout

@pytest.mark.parametrize("seed,V,E,P,f32", [(30, 1000, 20000, 7, False), (31, 5000, 40000, 148, False),
                                            (32, 777, 9000, 1, True), (33, 64, 0, 4, False),
                                            (34, 100000, 800000, 148, False), (35, 10, 40, 10, False)])
def test_layout_parity(sssp, seed, V, E, P, f32):
    src, dst, w = raw_graph(seed, V, E, f32=f32)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    h = sssp.layout(g)
    ids, slots, rh = oracle.layout(ref, P)
    assert np.array_equal(u32(h.ids), ids) and np.array_equal(u32(h.slots), slots)
    assert h.E == rh.E and np.array_equal(u32(h.row_ptr), rh.row_ptr)
    if rh.E:
        assert np.array_equal(u32(h.col), rh.col)
        assert np.array_equal(u32(h.w), rh.w.view(np.uint32))
        assert np.array_equal(u32(h.eid), rh.eid)


def test_layout_rmat_skewed_and_partition_counts_unchanged(sssp):
    g0 = gg.rmat(gg.BASE_SEED + 77, 14, 16 << 14)
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=37)
    h = sssp.layout(g)
    ids, slots, _ = oracle.layout(ref, 37)
    assert np.array_equal(u32(h.ids), ids)
    # renaming inside partitions keeps every partition's inter-edge count (Sec. III.D's threshold input)
    b0, i0 = sssp.partition(g)
    b1, i1 = sssp.partition(h)
    assert torch.equal(b0, b1) and torch.equal(i0, i1)


@pytest.mark.parametrize("seed,V,E,P,f32,split", [(40, 20000, 300000, 148, False, 1), (41, 20000, 300000, 37, False, 2),
                                                  (42, 5000, 60000, 5, True, 1), (43, 3000, 2000, 3, False, 1)])
def test_solve_on_layout_graph(sssp, seed, V, E, P, f32, split):
    src, dst, w = raw_graph(seed, V, E, f32=f32, whi=9)  # narrow weights: many equal-distance ties
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    h = sssp.layout(g)
    check_solve(sssp, h, ref, [0, 1, V - 1, 12345 % V], sssp.options(split=split))


def test_solve_on_layout_rmat(sssp):
    g0 = gg.rmat(gg.BASE_SEED + 78, 15, 16 << 15)
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=148)
    h = sssp.layout(g)
    srcs = gg.pick_sources(gg.BASE_SEED + 78, g0, 4)
    check_solve(sssp, h, ref, srcs.tolist())
    with pytest.raises(sssp.SsspError):
        sssp.backward(h, torch.zeros((1, g0.V), dtype=torch.int32, device="cuda"),
                      torch.zeros((1, g0.V), device="cuda"))


# ------------------------------------------------------------------------ K3

@pytest.mark.parametrize("mode", [0, 1])
def test_prune_parity_er16k(sssp, mode):
    g0, _, P = gg.workload_er16k()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    keep, wit = sssp.prune(g, mode)
    rk, rw = oracle.trishla(ref, P, mode)
    assert np.array_equal(keep.cpu().numpy(), rk)
    assert np.array_equal(u32(wit), rw)


@pytest.mark.parametrize("seed,V,E,P,mode,f32", [(20, 300, 6000, 3, 0, False), (21, 300, 6000, 3, 1, False),
                                                 (22, 2000, 30000, 5, 1, True), (23, 50, 2000, 1, 0, True)])
def test_prune_parity_dense_and_f32(sssp, seed, V, E, P, mode, f32):
    src, dst, w = raw_graph(seed, V, E, f32=f32, whi=30)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    keep, wit = sssp.prune(g, mode)
    rk, rw = oracle.trishla(ref, P, mode)
    assert (rk == 0).any()
    assert np.array_equal(keep.cpu().numpy(), rk)
    assert np.array_equal(u32(wit), rw)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("f32", [False, True])
def test_solve_prune_equals_solve_and_prune(sssp, mode, f32):
    """sssp_solve_prune: idle blocks of the solve run Trishla chunks (the rest right after the
    solve); the keep mask and least witnesses equal the oracle's Algorithm 1 and the distances
    and predecessors equal its Dijkstra.  Many partitions and few sources leave blocks idle."""
    V = 6000
    src, dst, w = raw_graph(90 + mode, V, 90000, f32=f32)
    ref = oracle.csr(V, src, dst, w)
    P = 40
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    srcs = [0, 5999]
    dist, pred, keep, wit, st, _ = sssp.solve_prune(g, np.array(srcs, np.uint32), mode, sssp.options(split=2))
    assert st == sssp.SSSP_OK
    rk, rw = oracle.trishla(ref, P, mode)
    assert np.array_equal(keep.cpu().numpy(), rk) and np.array_equal(u32(wit), rw)
    assert (rk == 0).sum() > 0
    for i, s_ in enumerate(srcs):
        d, p, _ = oracle.dijkstra(ref, s_)
        assert np.array_equal(u32(dist[i]), d.view(np.uint32)) and np.array_equal(u32(pred[i]), p)
    # without a witness array: the same keep mask and result
    d2, p2, k2, w2, st, _ = sssp.solve_prune(g, np.array(srcs, np.uint32), mode, witness=False)
    assert st == sssp.SSSP_OK and w2 is None
    assert np.array_equal(k2.cpu().numpy(), rk) and torch.equal(d2, dist) and torch.equal(p2, pred)


def test_solve_prune_er16k_and_grid(sssp):
    """The paper's configuration (ER 16K, 4 partitions, local Trishla) and a grid, where
    Trishla finds nothing to prune (no triangles) but most blocks are idle."""
    g0, srcs, P = gg.workload_er16k()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    dist, pred, keep, wit, st, _ = sssp.solve_prune(g, srcs, 0)
    assert st == sssp.SSSP_OK
    rk, rw = oracle.trishla(ref, P, 0)
    assert np.array_equal(keep.cpu().numpy(), rk) and np.array_equal(u32(wit), rw)
    d, p, _ = oracle.dijkstra(ref, int(srcs[0]))
    assert np.array_equal(u32(dist[0]), d) and np.array_equal(u32(pred[0]), p)
    gr = gg.grid(gg.BASE_SEED + 95, 256, 256, 1, 1000)
    rg = oracle.csr_of(gr)
    G = sssp.build_csr(gr.V, gr.src, gr.dst, gr.w, partitions=64)
    dist, pred, keep, wit, st, _ = sssp.solve_prune(G, np.array([0], np.uint32), 1)
    assert st == sssp.SSSP_OK and bool((keep == 1).all()) and bool((wit == -1).all())
    d, p, _ = oracle.dijkstra(rg, 0)
    assert np.array_equal(u32(dist[0]), d) and np.array_equal(u32(pred[0]), p)


def test_compact_and_solve_on_pruned_graph(sssp):
    g0, srcs, P = gg.workload_er16k()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    keep, _ = sssp.prune(g, 0)
    gp = sssp.compact(g, keep)
    rk, _ = oracle.trishla(ref, P, 0)
    rp = oracle.compact(ref, rk)
    assert gp.E == rp.E
    assert np.array_equal(u32(gp.row_ptr), rp.row_ptr)
    assert np.array_equal(u32(gp.col), rp.col)
    assert np.array_equal(u32(gp.w), rp.w)
    # pruned edges are never tight, so distances and canonical predecessors are unchanged (Sec. III.B)
    check_solve(sssp, gp, ref, [0, 1, 9999])


# ------------------------------------------------------------------- K0/K4

def test_solve_er16k_p4(sssp):
    g0, srcs, P = gg.workload_er16k()
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    stats = check_solve(sssp, g, ref, srcs.tolist())
    assert stats["edges_scanned"] >= ref.E * 0.5  # most of the graph is reachable and scanned


@pytest.mark.parametrize("P", [1, 2, 4, 7, 148])
@pytest.mark.parametrize("split", [1, 3])
@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("policy", [0, 1, 2, 3])
def test_solve_partition_counts(sssp, P, split, f32, policy):
    """Every frontier policy (relative, fixed, near-far, all) on every partition count and split,
    uint32 and float32 weights: the same distances and predecessors as the oracle."""
    V = 5000
    src, dst, w = raw_graph(30 + P, V, 40000, f32=f32)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    delta = 0.1 if f32 else 16
    check_solve(sssp, g, ref, [0, 4999, 2500, 0], sssp.options(split=split, policy=policy, delta=delta))


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("policy", [0, 1, 2, 3])
def test_hubs_wait_for_a_narrower_bucket(sssp, f32, policy):
    """hub_count on a layout graph (the first hub_count stored vertices of each partition take a
    quarter-width bucket, the next 3 * hub_count a half-width one): exact for every policy, for 1
    hub, some, and more than a partition holds; on a graph in the caller's ids the option is
    ignored."""
    g0 = gg.rmat(gg.BASE_SEED + 630, 14, 16 << 14, wf32=(0.5, 2.0, 1e-4) if f32 else None)
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=16)
    h = sssp.layout(g)
    srcs = gg.pick_sources(gg.BASE_SEED + 630, g0, 4).tolist()
    delta = 0.5 if f32 else 24
    for hubs in (1, 64, 100000):
        check_solve(sssp, h, ref, srcs, sssp.options(policy=policy, delta=delta, hub_count=hubs, split=2))
    check_solve(sssp, g, ref, srcs, sssp.options(policy=policy, delta=delta, hub_count=64))


@pytest.mark.parametrize("prune", [False, True])
@pytest.mark.parametrize("msg", [0, 8])
@pytest.mark.parametrize("hubs", [0, 48])
def test_every_solve_kernel_variant(sssp, prune, msg, hubs):
    """Each compiled variant of the persistent solve (prune on idle time x held messages x hub
    widths) on a layout graph, against the oracle; with prune, the keep mask against Algorithm 1."""
    g0 = gg.rmat(gg.BASE_SEED + 640, 13, 16 << 13)
    ref = oracle.csr_of(g0)
    P = 24
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    h = sssp.layout(g)
    srcs = gg.pick_sources(gg.BASE_SEED + 640, g0, 3)
    o = sssp.options(delta=16, msg_buffer=msg, hub_count=hubs)
    if prune:
        dist, pred, keep, wit, st, _ = sssp.solve_prune(h, srcs, 0, o)
        rk, _ = oracle.trishla(oracle.csr(h.V, np.repeat(np.arange(h.V, dtype=np.uint32),
                                                          np.diff(u32(h.row_ptr).astype(np.int64))),
                                          u32(h.col[:h.E]), u32(h.w[:h.E])), P, 0)
        assert np.array_equal(keep.cpu().numpy(), rk)
    else:
        dist, pred, st, _ = sssp.solve(h, srcs, o)
    assert st == sssp.SSSP_OK
    for i, s_ in enumerate(srcs):
        d, p, _ = oracle.dijkstra(ref, int(s_))
        assert np.array_equal(u32(dist[i]), d) and np.array_equal(u32(pred[i]), p)


@pytest.mark.parametrize("msg", [1, 8, 32])
@pytest.mark.parametrize("P,split", [(7, 1), (148, 1), (37, 3)])
@pytest.mark.parametrize("f32", [False, True])
def test_message_buffering_gives_the_same_result(sssp, msg, P, split, f32):
    """Messages held per warp and pushed out at msg of them and at the end of each sub-round:
    the oracle's distances and predecessors for every buffer size, partitioning and weight type."""
    V = 20000
    src, dst, w = raw_graph(50 + P, V, 200000, f32=f32)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    stats = check_solve(sssp, g, ref, [0, 19999, 777], sssp.options(split=split, msg_buffer=msg,
                                                                     delta=0.25 if f32 else 16))
    assert stats["remote_activations"] > 0


def test_message_buffering_with_layout_policies_and_warm_start(sssp):
    g0 = gg.rmat(gg.BASE_SEED + 620, 14, 16 << 14)
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=64)
    srcs = gg.pick_sources(gg.BASE_SEED + 620, g0, 4)
    for pol in range(4):
        check_solve(sssp, sssp.layout(g), ref, srcs.tolist(), sssp.options(policy=pol, msg_buffer=16, delta=6))
    src, dst, w = raw_graph(621, 8000, 64000, loops=False)
    s2, d2, w2, tails = _lowered(622, src, dst, w, 8000)
    g1 = sssp.build_csr(8000, src, dst, w, partitions=16)
    g2 = sssp.build_csr(8000, s2, d2, w2, partitions=16)
    o = sssp.options(msg_buffer=4)
    d, p, st, _ = sssp.solve(g1, np.array([5, 77], np.uint32), o)
    d, p, st, _ = sssp.update(g2, d, p, tails, o)
    assert st == sssp.SSSP_OK
    ref2 = oracle.csr(8000, s2, d2, w2)
    for i, s_ in enumerate((5, 77)):
        rd, rp, _ = oracle.dijkstra(ref2, s_)
        assert np.array_equal(u32(d[i]), rd) and np.array_equal(u32(p[i]), rp)


@pytest.mark.parametrize("policy", [0, 1, 2, 3])
def test_policies_on_layout_grid_and_warm_start(sssp, policy):
    """The policies on a layout graph (skewed R-MAT), on a grid whose distances have a closed form
    (constant weights: c * (r + col) from the corner), and in a warm start."""
    g0 = gg.rmat(gg.BASE_SEED + 610, 13, 16 << 13)
    ref = oracle.csr_of(g0)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=37)
    srcs = gg.pick_sources(gg.BASE_SEED + 610, g0, 4)
    check_solve(sssp, sssp.layout(g), ref, srcs.tolist(), sssp.options(policy=policy, delta=8, split=2))
    side, c = 300, 7
    gr = gg.grid(gg.BASE_SEED + 611, side, side, c, c)
    G = sssp.build_csr(gr.V, gr.src, gr.dst, gr.w, partitions=12)
    dist, pred, st, _ = sssp.solve(G, np.array([0], np.uint32), sssp.options(policy=policy, delta=3 * c))
    assert st == sssp.SSSP_OK
    r, q = np.divmod(np.arange(side * side), side)
    assert np.array_equal(u32(dist[0]), (c * (r + q)).astype(np.uint32))
    src, dst, w = raw_graph(612, 8000, 64000, loops=False)
    s2, d2, w2, tails = _lowered(613, src, dst, w, 8000)
    g1 = sssp.build_csr(8000, src, dst, w, partitions=16)
    g2 = sssp.build_csr(8000, s2, d2, w2, partitions=16)
    o = sssp.options(policy=policy, delta=12)
    d, p, st, _ = sssp.solve(g1, np.array([5, 77], np.uint32), o)
    d, p, st, _ = sssp.update(g2, d, p, tails, o)
    assert st == sssp.SSSP_OK
    ref2 = oracle.csr(8000, s2, d2, w2)
    for i, s_ in enumerate((5, 77)):
        rd, rp, _ = oracle.dijkstra(ref2, s_)
        assert np.array_equal(u32(d[i]), rd) and np.array_equal(u32(p[i]), rp)


@pytest.mark.parametrize("opts", [dict(threads=128, tile=32, delta=1), dict(threads=256, tile=64, delta=10),
                                  dict(threads=512, tile=4096, delta=1e9), dict(threads=512, tile=100, delta=50,
                                                                                 blocks_per_sm=1)])
def test_solve_schedule_does_not_change_result(sssp, opts):
    V = 20000
    src, dst, w = raw_graph(40, V, 160000)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=16)
    check_solve(sssp, g, ref, [3, 19999, 12345], sssp.options(**opts))


def _lowered(seed, src, dst, w, V, frac=0.02, add=0.01, f32=False):
    """The edge list after some weights fell and some edges were added; returns it and the
    tails of the changed edges."""
    rng = np.random.default_rng(seed)
    E = len(src)
    pick = rng.random(E) < frac
    w2 = w.copy()
    if f32:
        w2[pick] = (w2[pick] * rng.uniform(0.3, 1.0, int(pick.sum()))).astype(np.float32)
    else:
        w2[pick] = np.maximum(1, w2[pick] // rng.integers(1, 4, int(pick.sum()))).astype(np.uint32)
    na = int(add * E)
    s_add = rng.integers(0, V, na).astype(np.uint32)
    d_add = rng.integers(0, V, na).astype(np.uint32)
    w_add = (rng.uniform(0.5, 2.0, na).astype(np.float32) if f32 else rng.integers(1, 256, na).astype(np.uint32))
    tails = np.concatenate([src[pick], s_add]).astype(np.uint32)
    return (np.concatenate([src, s_add]), np.concatenate([dst, d_add]), np.concatenate([w2, w_add]), tails)


@pytest.mark.parametrize("seed,V,E,P,f32,lay", [(70, 20000, 200000, 148, False, False), (71, 20000, 200000, 37, False, True),
                                                (72, 5000, 40000, 5, True, False), (73, 3000, 9000, 3, False, False)])
def test_update_warm_start_equals_fresh_solve(sssp, seed, V, E, P, f32, lay):
    src, dst, w = raw_graph(seed, V, E, f32=f32, whi=60)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    if lay:
        g = sssp.layout(g)
    sources = np.array([0, 11, V - 1], np.uint32)
    dist, pred, st, _ = sssp.solve(g, sources)
    assert st == sssp.SSSP_OK
    src2, dst2, w2, tails = _lowered(seed + 1, src, dst, w, V, f32=f32)
    ref2 = oracle.csr(V, src2, dst2, w2)
    g2 = sssp.build_csr(V, src2, dst2, w2, partitions=P)
    if lay:
        g2 = sssp.layout(g2)
    dist, pred, st, stats = sssp.update(g2, dist, pred, tails)
    assert st == sssp.SSSP_OK
    for i, s in enumerate(sources):
        d, p, _ = oracle.dijkstra(ref2, int(s))
        assert np.array_equal(u32(dist[i]), d.view(np.uint32)), f"dist mismatch, source {s}"
        assert np.array_equal(u32(pred[i]), p), f"pred mismatch, source {s}"
    # far less work than a fresh solve on the changed graph
    _, _, _, fresh = sssp.solve(g2, sources)
    assert stats["edges_scanned"] < fresh["edges_scanned"]


def test_update_with_nothing_changed_and_unreached_tails(sssp):
    V = 4000
    src, dst, w = raw_graph(74, V, 6000)
    g = sssp.build_csr(V, src, dst, w, partitions=4)
    sources = np.array([5], np.uint32)
    dist, pred, _, _ = sssp.solve(g, sources)
    d0, p0 = dist.clone(), pred.clone()
    sssp.update(g, dist, pred, np.zeros(0, np.uint32))
    assert torch.equal(dist, d0) and torch.equal(pred, p0)
    unreached = np.flatnonzero(u32(d0[0]) == 0xFFFFFFFF).astype(np.uint32)[:50]
    assert len(unreached) > 0
    dist, pred, st, stats = sssp.update(g, dist, pred, np.concatenate([unreached, unreached]))
    assert st == sssp.SSSP_OK and torch.equal(dist, d0) and torch.equal(pred, p0)
    assert stats["edges_scanned"] == 0
    with pytest.raises(sssp.SsspError):
        sssp.update(g, dist, pred, np.array([V + 3], np.uint32))


def test_solve_f32_bit_exact(sssp):
    g0 = gg.rmat(gg.BASE_SEED + 50, 14, 8 << 14, wf32=(0.5, 2.0, 1e-4))
    ref = oracle.csr_of(g0)
    g = sssp.upload_csr(ref.V, ref.row_ptr, ref.col, ref.w, partitions=12)
    srcs = gg.pick_sources(gg.BASE_SEED + 50, g0, 5)
    check_solve(sssp, g, ref, srcs.tolist(), sssp.options(delta=0.25))


def test_solve_grid_closed_form_and_unreachable(sssp):
    # constant-weight grid: d = c*(r+q) from corner 0; plus a second component never reached
    R, C, c = 60, 70, 7
    g0 = gg.grid(1, R, C, c, c)
    src = np.concatenate([g0.src, np.array([R * C, R * C + 1], np.uint32)])
    dst = np.concatenate([g0.dst, np.array([R * C + 1, R * C + 2], np.uint32)])
    w = np.concatenate([g0.w, np.array([1, 1], np.uint32)])
    V = R * C + 3
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=9)
    dist, pred, st, _ = sssp.solve(g, np.array([0], np.uint32))
    d = u32(dist[0])
    r, q = np.divmod(np.arange(R * C), C)
    assert np.array_equal(d[:R * C], (c * (r + q)).astype(np.uint32))
    assert (d[R * C:] == 0xFFFFFFFF).all() and (u32(pred[0])[R * C:] == 0xFFFFFFFF).all()
    check_solve(sssp, g, ref, [0, R * C])


def test_solve_tiny_and_isolated(sssp):
    g = sssp.build_csr(1, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    dist, pred, st, _ = sssp.solve(g, np.array([0], np.uint32))
    assert u32(dist).tolist() == [[0]] and u32(pred).tolist() == [[0xFFFFFFFF]]
    src = np.array([0, 1], np.uint32)
    dst = np.array([1, 2], np.uint32)
    ref = oracle.csr(40, src, dst, np.array([5, 6], np.uint32))
    g = sssp.build_csr(40, src, dst, np.array([5, 6], np.uint32), partitions=40)
    check_solve(sssp, g, ref, [0, 39, 2])


def _subround_graph(f32):
    """A path 0..9 (one edge per vertex: sub-rounds of one edge, whose entries alternate
    between the halves of the selection arrays), a hub at 9 (1000 edges: a general
    sub-round that follows a small one whose entries sit in the upper half), a fan of 200
    at 5 whose heads each have two edges (a small sub-round of more than 32 vertices, with
    heads lowered twice in one sub-round), and random heavier edges that relax nothing."""
    rng = np.random.default_rng(77)
    src, dst, w = [], [], []
    def add(a, b, x):
        src.append(a); dst.append(b); w.append(x)
    for i in range(9):
        add(i, i + 1, 1)
    for j in range(1000):
        add(9, 100 + j, 1 + j % 3)
        add(100 + j, 2000 + j, 2)
    for i in range(200):
        add(5, 4000 + i, 7)
        add(4000 + i, 5000 + i % 150, 1 + i % 5)
        add(4000 + i, 5000 + (7 * i) % 150, 2)
    for _ in range(3000):
        add(int(rng.integers(0, 6000)), int(rng.integers(0, 6000)), int(rng.integers(200, 255)))
    src, dst = np.array(src, np.uint32), np.array(dst, np.uint32)
    w = np.array(w, np.float32) if f32 else np.array(w, np.uint32)
    return src, dst, w


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("P", [1, 4])
@pytest.mark.parametrize("opts", [dict(delta=1e6), dict(delta=1e6, tile=256), dict()])
def test_solve_small_and_general_subround_mix(sssp, f32, P, opts):
    src, dst, w = _subround_graph(f32)
    V = 6000
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    check_solve(sssp, g, ref, [0, 9, 5, 4000], sssp.options(**opts))


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("P,opts", [(12, dict(tile=32, delta=1e6)), (40, dict(tile=64, split=4, delta=300)),
                                    (148, dict(tile=1024, split=2, delta=3000)),
                                    (12, dict(tile=32, msg_buffer=8, delta=1e6)),
                                    (7, dict(tile=32, threads=128, delta=50))])
def test_grid_wavefront_messages_of_small_subrounds(sssp, f32, P, opts):
    """A random-weight grid from a corner, the middle and the far corner: the wavefront runs
    sub-rounds of a few vertices on the small path, whose messages into the next unit (and,
    with tiles of 32 or 64, into this unit once its local queue is full) are sent by the next
    sub-round or before the round settles; also on the locality layout with hubs."""
    side = 120
    g0 = gg.grid(gg.BASE_SEED + 620, side, side, 1, 1000)
    w = (g0.w.astype(np.float32) * np.float32(0.01)) if f32 else g0.w
    o = dict(opts)
    if f32 and o["delta"] < 1e6:
        o["delta"] *= 0.01
    ref = oracle.csr(g0.V, g0.src, g0.dst, w)
    g = sssp.build_csr(g0.V, g0.src, g0.dst, w, partitions=P)
    srcs = [0, side * (side // 2) + side // 2, side * side - 1]
    check_solve(sssp, g, ref, srcs, sssp.options(**o))
    check_solve(sssp, sssp.layout(g), ref, srcs, sssp.options(hub_count=16, **o))


def test_solve_overflow_status(sssp):
    w = np.array([0xFFFFFFFE, 2, 1], np.uint32)
    src, dst = np.array([0, 1, 0], np.uint32), np.array([1, 2, 3], np.uint32)
    ref = oracle.csr(4, src, dst, w)
    g = sssp.build_csr(4, src, dst, w)
    dist, pred, st, _ = sssp.solve(g, np.array([0], np.uint32), check=False)
    assert st == sssp.SSSP_EOVERFLOW
    d, p, rst = oracle.dijkstra(ref, 0)
    assert rst == oracle.OVERFLOW
    assert np.array_equal(u32(dist[0]), d) and np.array_equal(u32(pred[0]), p)


def test_solve_bad_source_is_reported(sssp):
    src, dst, w = raw_graph(5, 100, 500)
    g = sssp.build_csr(100, src, dst, w)
    dist, pred, st, _ = sssp.solve(g, np.array([3, 100], np.uint32), check=False)
    assert st == sssp.SSSP_EINVAL
    assert (u32(dist[1]) == 0xFFFFFFFF).all()


def test_solve_wait_limit_returns_timeout_and_device_stays_usable(sssp):
    """The termination count is held one above its true value (a count that nothing will
    release), so every block's idle wait must run out: status SSSP_ETIMEOUT, kernel returns."""
    V = 3000
    src, dst, w = raw_graph(6, V, 20000)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=4)
    o = sssp.options(timeout_ns=50_000_000, flags=sssp.FLAG_TEST_HOLD_PENDING)
    _, _, st, _ = sssp.solve(g, np.array([0], np.uint32), o, check=False)
    assert st == sssp.SSSP_ETIMEOUT
    check_solve(sssp, g, ref, [0])


def test_autotune_picks_a_valid_schedule_and_caches_it(sssp, tmp_path, monkeypatch):
    monkeypatch.setenv("SSSP_TUNE_CACHE", str(tmp_path / "tune.json"))
    V = 30000
    src, dst, w = raw_graph(77, V, 240000)
    ref = oracle.csr(V, src, dst, w)
    g = sssp.build_csr(V, src, dst, w, partitions=24)
    srcs = np.array([1, 2, 29999], np.uint32)
    opts, ms = sssp.autotune(g, srcs)
    assert ms is not None and ms > 0 and opts.delta >= 1 and opts.tile in (1024, 2048, 4096)
    assert opts.split in (1, 2, 4) and opts.policy in (0, 1, 2, 3)
    check_solve(sssp, g, ref, srcs.tolist(), opts)
    again, ms2 = sssp.autotune(g, srcs)
    assert ms2 is None and (again.delta, again.tile, again.split, again.policy) == (opts.delta, opts.tile, opts.split,
                                                                                    opts.policy)


# ------------------------------------------------------------------------ K5

def test_batched_parity_and_graph_replay(sssp):
    graphs, sources = [], []
    for k in range(24):
        t, n = gg.batch_params(gg.BASE_SEED + 77, k, 6.0, 12.0)
        ms = gg.member_seed(gg.BASE_SEED + 77, k)
        if t == 0:
            g0 = gg.erdos_renyi(ms, n, 8 * n, 1, 255)
        else:
            import math
            g0 = gg.rmat(ms, max(1, math.ceil(math.log2(n))), 8 * n, n=n)
        graphs.append(oracle.csr_of(g0))
        sources.append(gg.pick_sources(ms, g0, 4))
    b = sssp.Batch(graphs, sources, sssp.options(tile=256))
    b.solve()
    st, stats = b.status()
    assert st == sssp.SSSP_OK

    def check():
        for i in range(b.n_problems):
            gi, s = int(b.prob_graph[i]), int(b.prob_source[i])
            d, p, _ = oracle.dijkstra(graphs[gi], s)
            bd, bp = b.result(i)
            assert np.array_equal(u32(bd), d) and np.array_equal(u32(bp), p), (i, gi, s)

    check()
    b.dist.fill_(0)
    b.pred.fill_(0)
    b.make_plan()
    for _ in range(2):
        b.replay()
    st, _ = b.status()
    assert st == sssp.SSSP_OK
    check()


@pytest.mark.parametrize("f32,delta,tile", [(False, 1, 32), (False, 1000, 4096), (True, 0.01, 64), (True, 0.5, 1024),
                                             (True, 50.0, 256)])
def test_batched_buckets_extreme_widths_and_f32(sssp, f32, delta, tile):
    # narrow buckets keep the coarse window and the overflow busy (splits, flushes, stale
    # entries); one huge bucket degenerates to label correcting; float32 distances bucket by
    # a rounded quotient
    graphs, sources = [], []
    for k in range(10):
        n = 300 + 250 * k
        ms = gg.member_seed(gg.BASE_SEED + 91, k)
        if f32:
            g0 = gg.rmat(ms, max(1, int(np.ceil(np.log2(n)))), 8 * n, n=n, wf32=(0.5, 2.0, 1e-4))
        elif k % 2:
            g0 = gg.erdos_renyi(ms, n, 8 * n, 1, 255)
        else:
            g0 = gg.rmat(ms, max(1, int(np.ceil(np.log2(n)))), 8 * n, n=n)
        graphs.append(oracle.csr_of(g0))
        sources.append(gg.pick_sources(ms, g0, 3))
    b = sssp.Batch(graphs, sources, sssp.options(delta=delta, tile=tile))
    b.solve()
    st, _ = b.status()
    assert st == sssp.SSSP_OK
    for i in range(b.n_problems):
        gi, s = int(b.prob_graph[i]), int(b.prob_source[i])
        d, p, _ = oracle.dijkstra(graphs[gi], s)
        bd, bp = b.result(i)
        assert np.array_equal(u32(bd), d.view(np.uint32)) and np.array_equal(u32(bp), p), (i, gi, s)


def test_batched_equals_single_solves(sssp):
    g0, srcs, _ = gg.workload_er16k()
    ref = oracle.csr_of(g0)
    srcs = np.array([0, 5, 77, 16383], np.uint32)
    b = sssp.Batch([ref], [srcs])
    b.solve()
    g = sssp.upload_csr(ref.V, ref.row_ptr, ref.col, ref.w, partitions=4)
    dist, pred, _, _ = sssp.solve(g, srcs)
    for i in range(4):
        bd, bp = b.result(i)
        assert torch.equal(bd, dist[i]) and torch.equal(bp, pred[i])


@pytest.mark.parametrize("threads,tile", [(128, 1024), (128, 64), (256, 256), (256, 4096), (512, 512), (384, 32),
                                          (1024, 2048), (1024, 64), (1024, 4096), (768, 1024), (992, 100)])
def test_batched_block_sizes(sssp, threads, tile):
    """The batched kernel with every block size and tile: blocks smaller or larger than the tile
    and than half of it (the small sub-round path keeps its entries in tile halves)."""
    graphs = [oracle.csr_of(gg.rmat(gg.BASE_SEED + 700 + k, 11 + k % 3, 8 << (11 + k % 3))) for k in range(4)]
    graphs.append(oracle.csr_of(gg.erdos_renyi(gg.BASE_SEED + 710, 3000, 24000, 1, 255)))
    srcs = [np.array([0, 1, g.V - 1], np.uint32) for g in graphs]
    b = sssp.Batch(graphs, srcs, sssp.options(threads=threads, tile=tile, delta=8))
    b.solve()
    st, _ = b.status()
    assert st == sssp.SSSP_OK
    for i in range(b.n_problems):
        gi, s_ = int(b.prob_graph[i]), int(b.prob_source[i])
        d, p, _ = oracle.dijkstra(graphs[gi], s_)
        bd, bp = b.result(i)
        assert np.array_equal(u32(bd), d) and np.array_equal(u32(bp), p), (threads, tile, i)


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("opts", [dict(delta=1e6), dict(delta=1e6, tile=256), dict(delta=1),
                                  dict(delta=1e6, threads=1024, tile=2048)])
def test_batched_small_and_general_subround_mix(sssp, f32, opts):
    src, dst, w = _subround_graph(f32)
    ref = oracle.csr(6000, src, dst, w)
    srcs = np.array([0, 9, 5, 4000], np.uint32)
    b = sssp.Batch([ref, ref], [srcs, srcs[::-1].copy()], sssp.options(**opts))
    b.solve()
    st, _ = b.status()
    assert st == sssp.SSSP_OK
    for i, s in enumerate(list(srcs) + list(srcs[::-1])):
        d, p, _ = oracle.dijkstra(ref, int(s))
        bd, bp = b.result(i)
        assert np.array_equal(u32(bd), d.view(np.uint32)) and np.array_equal(u32(bp), p), f"problem {i}"


# ------------------------------------------------------------------------ K6

@pytest.mark.parametrize("scale,S", [(10, 3), (14, 8)])
def test_backward_parity(sssp, scale, S):
    g0 = gg.rmat(gg.BASE_SEED + 60 + scale, scale, 8 << scale, wf32=(0.5, 2.0, 1e-4))
    ref = oracle.csr_of(g0)
    g = sssp.upload_csr(ref.V, ref.row_ptr, ref.col, ref.w, partitions=8)
    srcs = gg.pick_sources(gg.BASE_SEED + 60, g0, S)
    dist, pred, st, _ = sssp.solve(g, srcs)
    gup = torch.from_numpy(gg.normal_f32(scale, (S, ref.V))).cuda()
    grad = sssp.backward(g, pred, gup).cpu().numpy().astype(np.float64)
    rd = np.stack([oracle.dijkstra(ref, int(s))[0] for s in srcs])
    rp = np.stack([oracle.dijkstra(ref, int(s))[1] for s in srcs])
    assert np.array_equal(u32(pred), rp)
    rg = oracle.tree_grad(ref, rd, rp, gup.cpu().numpy())
    assert np.allclose(grad, rg, rtol=1e-5, atol=1e-6 * np.abs(rg).max())
    assert (grad[rg == 0] == 0).all()


def test_autograd_function(sssp):
    g0 = gg.rmat(gg.BASE_SEED + 61, 9, 8 << 9, wf32=(0.5, 2.0, 1e-4))
    ref = oracle.csr_of(g0)
    g = sssp.upload_csr(ref.V, ref.row_ptr, ref.col, ref.w, partitions=2)
    srcs_np = gg.pick_sources(gg.BASE_SEED + 61, g0, 2)
    srcs = torch.from_numpy(srcs_np.view(np.int32)).cuda()
    w = g.w.clone().requires_grad_(True)
    F = sssp.sssp_function()
    dist = F.apply(w, g, srcs)
    gup = torch.from_numpy(gg.normal_f32(3, tuple(dist.shape))).cuda()
    finite = torch.isfinite(dist)
    (torch.where(finite, dist, torch.zeros_like(dist)) * gup).sum().backward()
    rd = np.stack([oracle.dijkstra(ref, int(s))[0] for s in srcs_np])
    rp = np.stack([oracle.dijkstra(ref, int(s))[1] for s in srcs_np])
    rg = oracle.tree_grad(ref, rd, rp, gup.cpu().numpy())
    assert np.allclose(w.grad.cpu().numpy(), rg, rtol=1e-5, atol=1e-6 * np.abs(rg).max())


@pytest.mark.parametrize("seed", range(64))
def test_random_schedules_match_the_oracle(sssp, seed):
    """A seeded sweep of schedules (block size, tile, split, width, policy, hubs, message
    buffering, layout, weight type) on random graphs of random size and partitioning: every
    combination gives the oracle's distances and predecessors."""
    rng = np.random.default_rng(9000 + seed)
    V = int(rng.integers(40, 4000))
    E = int(rng.integers(V, 10 * V))
    f32 = bool(rng.integers(0, 2))
    src, dst, w = raw_graph(9100 + seed, V, E, f32=f32)
    ref = oracle.csr(V, src, dst, w)
    P = int(rng.integers(1, min(148, V) + 1))
    g = sssp.build_csr(V, src, dst, w, partitions=P)
    lay = bool(rng.integers(0, 2))
    if lay:
        g = sssp.layout(g)
    delta = float(rng.choice([0.0, 1.0, 3.0, 17.0, 1e6]))
    if f32 and delta:
        delta *= 0.01
    o = sssp.options(threads=int(rng.choice([128, 256, 384, 512])), tile=int(rng.choice([32, 100, 512, 1024, 4096])),
                     split=int(rng.integers(1, 4)), delta=delta, policy=int(rng.integers(0, 4)),
                     msg_buffer=int(rng.choice([0, 0, 1, 8, 32])), hub_count=int(rng.choice([0, 4, 64])) if lay else 0)
    sources = sorted(set(int(x) for x in rng.integers(0, V, 3)))
    check_solve(sssp, g, ref, sources, o)
    # the same graph in a batch, in a random batched schedule
    bo = sssp.options(threads=int(rng.choice([128, 512, 1024])), tile=int(rng.choice([64, 1024, 2048])),
                      delta=delta)
    b = sssp.Batch([ref], [np.array(sources, np.uint32)], bo)
    b.solve()
    st, _ = b.status()
    assert st == sssp.SSSP_OK
    for i, s in enumerate(sources):
        d, p, _ = oracle.dijkstra(ref, s)
        bd, bp = b.result(i)
        assert np.array_equal(u32(bd), d.view(np.uint32)) and np.array_equal(u32(bp), p), (seed, i)
