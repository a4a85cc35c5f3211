"""Pins for the CPU oracle (no GPU).

Each test ties one oracle function to something other than itself: values
worked out by hand (tests/golden), brute force on tiny inputs, library
routines (scipy.sparse.csgraph), closed forms, and central finite
differences.  A dropped term, a wrong index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import pins

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")
NONE = oracle.NONE


def _edges(case, dtype=np.uint32):
    e = np.array(case["edges"], dtype=np.int64).reshape(-1, 3)
    return (e[:, 0].astype(np.uint32), e[:, 1].astype(np.uint32), e[:, 2].astype(dtype))


def _rand_graph(seed, V, E, wlo=1, whi=20, f32=False):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, V, E).astype(np.uint32)
    dst = rng.integers(0, V, E).astype(np.uint32)
    if f32:
        w = rng.uniform(0.5, 2.0, E).astype(np.float32)
    else:
        w = rng.integers(wlo, whi + 1, E).astype(np.uint32)
    return src, dst, w


# ------------------------------------------------------------------ golden

def test_golden_sssp_cases():
    cases = json.load(open(GOLD))["sssp"]
    for c in cases:
        src, dst, w = _edges(c)
        g = oracle.csr(c["V"], src, dst, w)
        d, p, st = oracle.dijkstra(g, c["source"])
        assert st == oracle.OK
        assert d.tolist() == c["dist"], c["name"]
        assert p.tolist() == c["pred"], c["name"]


def _check_trishla_case(V, P, mode, edges, keep_exp, wit_exp):
    src, dst, w = edges
    g = oracle.csr(V, src, dst, w)
    keep, wit = oracle.trishla(g, P, mode)
    for u in range(V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            key = f"{u},{g.col[e]}"
            assert keep[e] == keep_exp[key], key
            assert wit[e] == wit_exp.get(key, NONE), key


def test_golden_trishla_cases():
    for c in json.load(open(GOLD))["trishla"]:
        edges = _edges(c)
        if "cases" in c:
            for sub in c["cases"]:
                _check_trishla_case(c["V"], c["P"], sub["mode"], edges, sub["keep"], sub["witness"])
        else:
            _check_trishla_case(c["V"], c["P"], c["mode"], edges, c["keep"], c["witness"])


# --------------------------------------------------------------------- CSR

@pytest.mark.parametrize("seed", range(6))
def test_csr_matches_dictionary_construction(seed):
    V = 50
    src, dst, w = _rand_graph(seed, V, 400, 1, 6)  # many duplicates and weight ties
    g = oracle.csr(V, src, dst, w)
    best = pins.canonical_edges(V, src, dst, w)
    keys = sorted(best)
    assert g.E == len(keys)
    got = []
    for u in range(V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            got.append(((u, int(g.col[e])), (int(g.w[e]), int(g.eid[e]))))
    assert got == [(k, best[k]) for k in keys]


def test_csr_f32_and_rejects_bad_endpoint():
    src, dst, w = _rand_graph(7, 30, 200, f32=True)
    g = oracle.csr(30, src, dst, w)
    best = pins.canonical_edges(30, src, dst, w)
    assert g.w.dtype == np.float32 and g.E == len(best)
    for u in range(30):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            assert g.w[e] == np.float32(best[(u, int(g.col[e]))][0])
    with pytest.raises(ValueError):
        oracle.csr(3, np.array([0, 3], np.uint32), np.array([1, 1], np.uint32), np.array([1, 1], np.uint32))


# --------------------------------------------------------------- partition

@pytest.mark.parametrize("seed,mask", [(s, m) for s in range(3) for m in ("random", "trishla", "none", "all")])
def test_compact_matches_dictionary_construction(seed, mask):
    """oracle.compact against a pure-Python construction: the canonical edge dictionary (pins)
    in sorted (tail, head) order, filtered by the keep mask, with row offsets counted per tail.
    The masks: random, the dense-algebra Trishla keep mask (pins.trishla_dense, local mode),
    nothing kept, everything kept."""
    V, P = 40, 3
    src, dst, w = _rand_graph(100 + seed, V, 300, 1, 9)
    g = oracle.csr(V, src, dst, w)
    best = pins.canonical_edges(V, src, dst, w)
    keys = sorted(best)
    if mask == "random":
        keep = np.random.default_rng(seed).integers(0, 2, len(keys)).astype(np.uint8)
    elif mask == "trishla":
        dense = pins.trishla_dense(V, best, P, 0)
        keep = np.array([dense[k][0] for k in keys], np.uint8)
        assert 0 < keep.sum() < len(keys)
    else:
        keep = np.full(len(keys), 0 if mask == "none" else 1, np.uint8)
    h = oracle.compact(g, keep)
    kept = [k for k, f in zip(keys, keep.tolist()) if f]
    row_ptr = [sum(1 for (a, _) in kept if a < u) for u in range(V + 1)]
    assert h.V == V and h.E == len(kept)
    assert h.row_ptr.tolist() == row_ptr
    assert h.col.tolist() == [b for (_, b) in kept]
    assert h.w.tolist() == [best[k][0] for k in kept]
    assert h.eid.tolist() == [best[k][1] for k in kept]


def test_partition_closed_forms():
    b, _ = oracle.partition(16384, 4)
    assert b.tolist() == [0, 4096, 8192, 12288, 16384]
    b, _ = oracle.partition(4194304, 148)
    assert b[1] == 28340 and b[-1] == 4194304 and b[-1] - b[-2] == 28324
    b, _ = oracle.partition(10, 4)  # B = 3: 3,3,3,1
    assert b.tolist() == [0, 3, 6, 9, 10]
    b, _ = oracle.partition(5, 8)  # B = 1; empty tail partitions
    assert b.tolist() == [0, 1, 2, 3, 4, 5, 5, 5, 5]


def test_partition_inter_edges_brute_force():
    V, P = 97, 5
    src, dst, w = _rand_graph(3, V, 800)
    g = oracle.csr(V, src, dst, w)
    _, inter = oracle.partition(V, P, g)
    B = -(-V // P)
    cnt = np.zeros(P, np.int64)
    for (a, b_) in pins.canonical_edges(V, src, dst, w):
        if a // B != b_ // B:
            cnt[a // B] += 1
    assert inter.tolist() == cnt.tolist()


# ---------------------------------------------------------------- Dijkstra

@pytest.mark.parametrize("seed,V,E", [(0, 12, 30), (1, 25, 60), (2, 40, 400), (3, 40, 45), (4, 2, 1), (5, 33, 0)])
def test_dijkstra_u32_vs_floyd_warshall(seed, V, E):
    src, dst, w = _rand_graph(seed, V, E, 1, 9)
    g = oracle.csr(V, src, dst, w)
    best = pins.canonical_edges(V, src, dst, w)
    D, INF = pins.floyd_warshall_int(pins.dense_int(V, best))
    for s in range(0, V, max(1, V // 7)):
        d, p, st = oracle.dijkstra(g, s)
        assert st == oracle.OK
        exp = np.where(D[s] >= INF, 0xFFFFFFFF, D[s]).astype(np.uint32)
        assert np.array_equal(d, exp)
        ep = pins.min_tight_pred(V, best, D[s], s, lambda x: x < INF, lambda a, b: a + b)
        assert np.array_equal(p, ep)


def test_dijkstra_u32_vs_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    V = 3000
    src, dst, w = _rand_graph(11, V, 15000, 1, 255)
    g = oracle.csr(V, src, dst, w)
    A = sp.csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr.astype(np.int64)), shape=(V, V))
    for s in (0, 17, 2999):
        ref = csg.dijkstra(A, directed=True, indices=s)
        d, _, _ = oracle.dijkstra(g, s)
        exp = np.where(np.isinf(ref), 0xFFFFFFFF, ref).astype(np.uint32)
        assert np.array_equal(d, exp)


@pytest.mark.parametrize("seed", range(5))
def test_dijkstra_f32_bit_exact_vs_float32_bellman_ford(seed):
    V = 30
    src, dst, w = _rand_graph(seed, V, 120, f32=True)
    g = oracle.csr(V, src, dst, w)
    best = pins.canonical_edges(V, src, dst, w)
    for s in (0, 5, 29):
        d, p, _ = oracle.dijkstra(g, s)
        ref = pins.bellman_ford_f32(V, best, s)
        assert np.array_equal(d.view(np.uint32), ref.view(np.uint32))
        ep = pins.min_tight_pred(V, best, ref, s, np.isfinite,
                                 lambda a, b: np.float32(np.float32(a) + np.float32(b)))
        assert np.array_equal(p, ep)


def test_dijkstra_closed_form_grid_constant_weight():
    R, C, c = 7, 11, 5
    g0 = gg.grid(1, R, C, c, c)
    g = oracle.csr(g0.V, g0.src, g0.dst, g0.w)
    d, p, _ = oracle.dijkstra(g, 0)
    r, q = np.divmod(np.arange(R * C), C)
    assert np.array_equal(d, (c * (r + q)).astype(np.uint32))
    # canonical pred: the tight neighbours are (r-1,q) and (r,q-1); the smaller id is (r-1,q)
    exp = np.where(r > 0, (r - 1) * C + q, r * C + q - 1)
    exp[0] = NONE
    assert np.array_equal(p, exp.astype(np.uint32))


def test_dijkstra_unit_weights_are_bfs_levels():
    V = 500
    src, dst, _ = _rand_graph(21, V, 1500)
    w = np.ones_like(src)
    g = oracle.csr(V, src, dst, w)
    best = pins.canonical_edges(V, src, dst, w)
    d, _, _ = oracle.dijkstra(g, 3)
    lvl = np.array(pins.bfs_levels(V, best, 3))
    assert np.array_equal(d, np.where(lvl < 0, 0xFFFFFFFF, lvl).astype(np.uint32))


def test_dijkstra_path_prefix_sums_and_overflow():
    V = 9
    w = np.arange(1, V, dtype=np.uint32) * 3
    src = np.arange(V - 1, dtype=np.uint32)
    dst = src + 1
    g = oracle.csr(V, src, dst, w)
    d, p, st = oracle.dijkstra(g, 0)
    assert d.tolist() == [0] + np.cumsum(w).tolist() and st == oracle.OK
    assert p.tolist() == [NONE] + list(range(V - 1))
    # 0 ->1 fits, 0->1->2 = 2^32 does not: reported unreachable with an overflow status
    w = np.array([0xFFFFFFFE, 2, 1], np.uint32)
    g = oracle.csr(4, np.array([0, 1, 0], np.uint32), np.array([1, 2, 3], np.uint32), w)
    d, p, st = oracle.dijkstra(g, 0)
    assert st == oracle.OVERFLOW
    assert d.tolist() == [0, 0xFFFFFFFE, 0xFFFFFFFF, 1]
    assert p.tolist() == [NONE, 0, NONE, 0]


def test_tight_ties_counts():
    g = oracle.csr(4, np.array([0, 0, 2, 1], np.uint32), np.array([2, 1, 3, 3], np.uint32),
                   np.array([1, 1, 2, 2], np.uint32))
    d, _, _ = oracle.dijkstra(g, 0)
    assert oracle.tight_ties(g, 0, d) == 1


# ----------------------------------------------------------------- Trishla

@pytest.mark.parametrize("seed,mode,P,f32", [(0, 0, 1, False), (1, 1, 3, False), (2, 0, 3, False),
                                             (3, 1, 1, True), (4, 0, 2, True), (5, 1, 4, False)])
def test_trishla_vs_dense_formulation(seed, mode, P, f32):
    V = 24
    src, dst, w = _rand_graph(seed, V, 160, 1, 12, f32=f32)
    g = oracle.csr(V, src, dst, w)
    best = pins.canonical_edges(V, src, dst, w)
    ref = pins.trishla_dense(V, best, P, mode, f32=f32)
    keep, wit = oracle.trishla(g, P, mode)
    for u in range(V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            assert (int(keep[e]), int(wit[e])) == ref[(u, int(g.col[e]))]
    assert (keep == 0).any()


@pytest.mark.parametrize("seed", range(4))
def test_trishla_removal_preserves_all_distances(seed):
    """Sec. III.B's correctness argument: a deleted edge's head stays reachable at lower cost,
    so deleting every pruned edge at once changes no shortest distance from any source."""
    csg = pytest.importorskip("scipy.sparse.csgraph")
    sp = pytest.importorskip("scipy.sparse")
    V = 60
    src, dst, w = _rand_graph(100 + seed, V, 600, 1, 30)
    g = oracle.csr(V, src, dst, w)
    keep, wit = oracle.trishla(g, 1, 1)
    assert (keep == 0).sum() > 0

    def apsp(mask):
        rows = np.repeat(np.arange(V), np.diff(g.row_ptr.astype(np.int64)))
        A = sp.csr_matrix((g.w[mask].astype(np.float64), (rows[mask], g.col[mask])), shape=(V, V))
        return csg.shortest_path(A, directed=True)

    full = apsp(np.ones(g.E, bool))
    pruned = apsp(keep.astype(bool))
    assert np.array_equal(full, pruned)
    # every pruned edge is dominated through its recorded witness
    rows = np.repeat(np.arange(V), np.diff(g.row_ptr.astype(np.int64)))
    for e in np.nonzero(keep == 0)[0]:
        u, vj, vi = rows[e], g.col[e], wit[e]
        lo, hi = g.row_ptr[vi], g.row_ptr[vi + 1]
        k = lo + np.searchsorted(g.col[lo:hi], vj)
        e1 = g.row_ptr[u] + np.searchsorted(g.col[g.row_ptr[u]:g.row_ptr[u + 1]], vi)
        assert g.col[k] == vj and g.w[e] > g.w[e1] + g.w[k]


def test_trishla_row_range():
    src, dst, w = _rand_graph(9, 40, 300)
    g = oracle.csr(40, src, dst, w)
    k_all, w_all = oracle.trishla(g, 2, 0)
    k_part, w_part = oracle.trishla(g, 2, 0, 10, 25)
    sl = slice(int(g.row_ptr[10]), int(g.row_ptr[25]))
    assert np.array_equal(k_all[sl], k_part[sl]) and np.array_equal(w_all[sl], w_part[sl])
    assert (k_part[:g.row_ptr[10]] == 1).all()


# ----------------------------------------------------------- tree gradient

def test_tree_grad_path_closed_form():
    """On a path 0->1->...->n, dL/dw(k,k+1) = sum_{j>k} g_j."""
    n = 10
    src = np.arange(n, dtype=np.uint32)
    g = oracle.csr(n + 1, src, src + 1, np.linspace(0.5, 1.5, n).astype(np.float32))
    d, p, _ = oracle.dijkstra(g, 0)
    gup = np.linspace(-1, 2, n + 1).astype(np.float32)
    grad = oracle.tree_grad(g, d[None], p[None], gup[None])
    exp = np.array([gup[k + 1:].astype(np.float64).sum() for k in range(n)])
    assert np.allclose(grad, exp, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_tree_grad_vs_central_finite_differences(seed):
    """Float64 central differences of L = sum_s sum_v g[s,v] d_s(v) (distances by scipy) on graphs with
    unique shortest paths; edges whose tree changes under +-h are skipped."""
    csg = pytest.importorskip("scipy.sparse.csgraph")
    sp = pytest.importorskip("scipy.sparse")
    V, S, h = 120, 3, 1e-3
    src, dst, w = _rand_graph(40 + seed, V, 700, f32=True)
    g = oracle.csr(V, src, dst, w)
    srcs = [0, 7, 50]
    dist = np.empty((S, V), np.float32)
    pred = np.empty((S, V), np.uint32)
    for i, s in enumerate(srcs):
        dist[i], pred[i], _ = oracle.dijkstra(g, s)
    gup = np.random.default_rng(seed).standard_normal((S, V)).astype(np.float32)
    grad = oracle.tree_grad(g, dist, pred, gup)
    rows = np.repeat(np.arange(V), np.diff(g.row_ptr.astype(np.int64)))
    base_w = g.w.astype(np.float64)

    def solve(wv):
        A = sp.csr_matrix((wv, g.col, g.row_ptr.astype(np.int64)), shape=(V, V))
        D, Pr = csg.dijkstra(A, directed=True, indices=srcs, return_predecessors=True)
        return D, Pr

    D0, P0 = solve(base_w)
    fin = np.isfinite(D0)
    checked = 0
    for e in np.random.default_rng(seed).choice(g.E, 150, replace=False):
        wp, wm = base_w.copy(), base_w.copy()
        wp[e] += h
        wm[e] -= h
        Dp, Pp = solve(wp)
        Dm, Pm = solve(wm)
        if not (np.array_equal(Pp, P0) and np.array_equal(Pm, P0)):
            continue
        fd = ((np.where(fin, Dp, 0) - np.where(fin, Dm, 0)) * gup.astype(np.float64)).sum() / (2 * h)
        assert abs(fd - grad[e]) <= 1e-6 * max(1.0, abs(fd)), (e, fd, grad[e])
        checked += 1
    assert checked > 100
    # tree edges only: an edge that is nobody's predecessor edge has zero gradient
    tree = np.zeros(g.E, bool)
    for i in range(S):
        for v in range(V):
            if pred[i, v] != NONE:
                u = pred[i, v]
                tree[g.row_ptr[u] + np.searchsorted(g.col[g.row_ptr[u]:g.row_ptr[u + 1]], v)] = True
    assert (grad[~tree] == 0).all()
    assert rows.shape[0] == g.E


# ---------------------------------------------------------- locality layout

def test_layout_hand_worked_order():
    # V = 6, P = 2 (B = 3); total degrees (in + out): 0:2 1:2 2:3 3:2 4:2 5:3
    src = np.array([0, 0, 1, 3, 5, 5, 2], np.uint32)
    dst = np.array([1, 2, 2, 4, 3, 4, 5], np.uint32)
    w = np.array([4, 1, 2, 7, 1, 9, 3], np.uint32)
    g = oracle.csr(6, src, dst, w)
    ids, slots, h = oracle.layout(g, 2)
    assert ids.tolist() == [2, 0, 1, 5, 3, 4]  # each block: degree 3 first, then the degree-2 ids ascending
    assert slots.tolist() == [1, 2, 0, 4, 5, 3]
    # edge 0 -> 2 (w 1) becomes 1 -> 0; edge 2 -> 5 (w 3) becomes 0 -> 3
    row = lambda u: list(zip(h.col[h.row_ptr[u]:h.row_ptr[u + 1]].tolist(), h.w[h.row_ptr[u]:h.row_ptr[u + 1]].tolist()))
    assert row(1) == [(0, 1), (2, 4)] and row(0) == [(3, 3)]


@pytest.mark.parametrize("seed,V,E,P", [(0, 50, 300, 4), (1, 97, 500, 5), (2, 64, 64, 64), (3, 33, 0, 3), (4, 200, 3000, 7)])
def test_layout_order_properties_brute_force(seed, V, E, P):
    src, dst, w = _rand_graph(seed, V, E)
    g = oracle.csr(V, src, dst, w)
    ids, slots, h = oracle.layout(g, P)
    B = -(-V // P)
    deg = [0] * V
    for u in range(V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            deg[u] += 1
            deg[int(g.col[e])] += 1
    assert sorted(ids.tolist()) == list(range(V))
    for n in range(V):
        assert slots[ids[n]] == n
        assert ids[n] // B == n // B  # same partition
        if n + 1 < V and (n + 1) // B == n // B:
            a, b = int(ids[n]), int(ids[n + 1])
            assert deg[a] > deg[b] or (deg[a] == deg[b] and a < b)
    # the renamed graph holds exactly the renamed edges, each mapped back by eid
    want = sorted((int(slots[u]), int(slots[g.col[e]]), int(g.w[e]))
                  for u in range(V) for e in range(g.row_ptr[u], g.row_ptr[u + 1]))
    got = []
    for n in range(V):
        for k in range(h.row_ptr[n], h.row_ptr[n + 1]):
            got.append((n, int(h.col[k]), int(h.w[k])))
            e = int(h.eid[k])
            assert slots[np.searchsorted(g.row_ptr, e, side="right") - 1] == n and slots[g.col[e]] == h.col[k]
    assert sorted(got) == want


def test_layout_keeps_distances():
    V, P = 120, 6
    src, dst, w = _rand_graph(9, V, 900)
    g = oracle.csr(V, src, dst, w)
    ids, slots, h = oracle.layout(g, P)
    for s in (0, 17, 119):
        d0, _, _ = oracle.dijkstra(g, s)
        d1, _, _ = oracle.dijkstra(h, int(slots[s]))
        assert np.array_equal(d1[slots], d0)
