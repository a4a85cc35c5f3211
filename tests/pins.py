"""Independent brute-force statements used to pin the oracle.

Nothing here calls the oracle or the CUDA library: each helper recomputes a
quantity by a different procedure (dense matrices, dictionaries, pure-Python
fixpoints, library routines) so that a mistake in the oracle shows up as a
disagreement.
"""
from __future__ import annotations

from collections import deque

import numpy as np

NONE = 0xFFFFFFFF


def canonical_edges(V, src, dst, w):
    """dict (s,d) -> (w, first index) keeping the minimum weight, earliest index on ties; loops dropped."""
    best = {}
    for i, (s, d, x) in enumerate(zip(src.tolist(), dst.tolist(), w.tolist())):
        if s == d:
            continue
        k = (s, d)
        if k not in best or x < best[k][0]:
            best[k] = (x, i)
    return best


def dense_int(V, best):
    """V x V int64 matrix of edge weights, -1 where absent."""
    M = np.full((V, V), -1, np.int64)
    for (s, d), (x, _) in best.items():
        M[s, d] = x
    return M


def floyd_warshall_int(M):
    """All-pairs shortest distances over int weights; INF as a large sentinel."""
    V = M.shape[0]
    INF = np.iinfo(np.int64).max // 4
    D = np.where(M >= 0, M, INF).astype(np.int64)
    np.fill_diagonal(D, 0)
    for k in range(V):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D, INF


def bellman_ford_f32(V, best, s):
    """Fixpoint of d(v) = min(d(v), fl32(d(u)+w)) by repeated sweeps (float32 arithmetic)."""
    d = np.full(V, np.float32(np.inf), np.float32)
    d[s] = np.float32(0)
    edges = [(a, b, np.float32(x)) for (a, b), (x, _) in best.items()]
    changed = True
    while changed:
        changed = False
        for a, b, x in edges:
            if np.isinf(d[a]):
                continue
            c = np.float32(d[a] + x)
            if c < d[b]:
                d[b] = c
                changed = True
    return d


def bfs_levels(V, best, s):
    adj = [[] for _ in range(V)]
    for (a, b) in best:
        adj[a].append(b)
    lvl = [-1] * V
    lvl[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for v in adj[u]:
            if lvl[v] < 0:
                lvl[v] = lvl[u] + 1
                q.append(v)
    return lvl


def min_tight_pred(V, best, dist, s, finite, add):
    """Smallest u with a tight edge (u,v) for every reached v != s, by brute force over the edge dict."""
    pred = [NONE] * V
    for (a, b), (x, _) in best.items():
        if b == s or not finite(dist[a]) or not finite(dist[b]):
            continue
        if add(dist[a], x) == dist[b] and a < pred[b]:
            pred[b] = a
    return np.array(pred, np.uint32)


def trishla_dense(V, best, P, mode, f32=False):
    """Algorithm 1 by dense boolean algebra: prune[u,j] = OR_i A[u,i] & A[i,j] & (W[u,j] > W[u,i]+W[i,j])
    (with i restricted to u's block in local mode).  Returns dict (u,j) -> (keep, witness)."""
    A = np.zeros((V, V), bool)
    W = np.zeros((V, V), np.float32 if f32 else np.int64)
    for (a, b), (x, _) in best.items():
        A[a, b] = True
        W[a, b] = x
    B = -(-V // P)
    owner = np.arange(V) // B
    out = {}
    for (u, j) in best:
        cand = A[u, :] & A[:, j]
        cand[j] = False
        if mode == 0:
            cand &= owner == owner[u]
        if f32:
            sums = (W[u, :] + W[:, j]).astype(np.float32)
        else:
            sums = W[u, :] + W[:, j]
        dom = cand & (W[u, j] > sums)
        idx = np.nonzero(dom)[0]
        out[(u, j)] = (0, int(idx[0])) if idx.size else (1, NONE)
    return out
