"""The seeded input generators: shapes, counts, ranges and determinism (no GPU)."""
import numpy as np

import graphgen as gg


def test_er_distinct_no_loops_and_weights():
    g, s, P = gg.workload_er16k()
    assert (g.V, g.E_raw, P, s.tolist()) == (16384, 131072, 4, [0])
    key = g.src.astype(np.uint64) << np.uint64(32) | g.dst
    assert np.unique(key).size == g.E_raw and not (g.src == g.dst).any()
    assert g.w.min() >= 1 and g.w.max() <= 255 and g.w.dtype == np.uint32
    # weights are uniform: every value appears with roughly equal frequency
    h = np.bincount(g.w, minlength=256)[1:]
    assert h.min() > 0.8 * h.mean() and h.max() < 1.2 * h.mean()


def test_rmat_quadrant_probabilities_without_permutation():
    scale, m = 12, 200000
    g = gg.rmat(5, scale, m, permute=False)
    top_s = g.src >> (scale - 1)
    top_d = g.dst >> (scale - 1)
    # first level: P(src bit=0, dst bit=0) = a = .57, P(src bit = 1) = c + d = .24
    assert abs(np.mean((top_s == 0) & (top_d == 0)) - 0.57) < 0.01
    assert abs(np.mean(top_s == 1) - 0.24) < 0.01


def test_rmat_permutation_and_rejection():
    g = gg.rmat(6, 10, 8000, n=700, permute=True)
    assert g.src.max() < 700 and g.dst.max() < 700
    p = gg.permutation(3, 1000)
    assert np.array_equal(np.sort(p), np.arange(1000, dtype=np.uint32))


def test_grid_edge_count_and_symmetry():
    R, C = 6, 9
    g = gg.grid(2, R, C, 1, 1000)
    assert g.E_raw == 2 * (R * (C - 1) + (R - 1) * C)
    d = {(a, b): x for a, b, x in zip(g.src.tolist(), g.dst.tolist(), g.w.tolist())}
    assert all(d[(b, a)] == x for (a, b), x in d.items())
    assert all(abs(a - b) in (1, C) for a, b in d)
    # full-size grid count: 2*(4096*4095*2) = 67,092,480
    assert 2 * (4096 * 4095 + 4095 * 4096) == 67092480


def test_sources_have_out_edges_and_are_distinct():
    g = gg.rmat(8, 12, 20000)
    s = gg.pick_sources(8, g, 16)
    assert len(set(s.tolist())) == 16
    has_out = np.zeros(g.V, bool)
    has_out[g.src[g.src != g.dst]] = True
    assert has_out[s].all()


def test_f32_weights_and_normals():
    w = gg.weights_f32(1, 100000, 0.5, 2.0, 1e-4)
    assert w.dtype == np.float32 and w.min() >= 0.5 and w.max() < 2.0001
    z = gg.normal_f32(2, (4, 50000))
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02


def test_determinism():
    a = gg.rmat(77, 10, 5000)
    b = gg.rmat(77, 10, 5000)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.w, b.w)
    t, n = gg.batch_params(gg.BASE_SEED + 4, 0)
    assert t in (0, 1) and 1024 <= n <= 131072
