"""CPU oracle for the SP_Async hot path (arXiv 2103.12012).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, one function per definition,
each citing the passage of the paper it states); this module only compiles
it with gcc and marshals numpy arrays.  Pins that tie the oracle to facts
other than itself are in ``tests/test_oracle_pins.py``.

Status of each function's parity pin:
  csr, partition, dijkstra (u32 and f32), trishla, tree_grad -- pinned
  (brute force, library routines, closed forms, finite differences).
  layout -- pinned (a hand-worked order; brute-force order properties;
  distances invariant under the renaming).
  compact -- pinned (a pure-Python construction from the canonical edge
  dictionary, filtered by random, Trishla, empty and full keep masks).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None

NONE = 0xFFFFFFFF
INF_U32 = 0xFFFFFFFF
OK, EINVAL, OVERFLOW = 0, 1, 5


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u32, u64, i = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.orc_csr.argtypes = [u32, u64, P, P, P, i, P, P, P, P]
        lib.orc_csr.restype = ctypes.c_int64
        lib.orc_partition.argtypes = [u32, u32, P, P, P, P]
        lib.orc_partition.restype = i
        lib.orc_dijkstra.argtypes = [u32, P, P, P, i, u32, P, P]
        lib.orc_dijkstra.restype = i
        lib.orc_tight_ties.argtypes = [u32, P, P, P, i, u32, P]
        lib.orc_tight_ties.restype = u64
        lib.orc_trishla.argtypes = [u32, P, P, P, i, u32, i, u32, u32, P, P]
        lib.orc_trishla.restype = i
        lib.orc_tree_grad.argtypes = [u32, P, P, u32, P, P, P, P]
        lib.orc_tree_grad.restype = i
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _wbits(w: np.ndarray):
    w = np.ascontiguousarray(w)
    if w.dtype == np.float32:
        return w.view(np.uint32), 1
    return w.astype(np.uint32, copy=False), 0


class CSR:
    """Canonical CSR: rows sorted by head, no self-loops, parallel edges collapsed."""

    def __init__(self, V, row_ptr, col, w, eid):
        self.V, self.row_ptr, self.col, self.w, self.eid = V, row_ptr, col, w, eid

    @property
    def E(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def wtype(self) -> int:
        return 1 if self.w.dtype == np.float32 else 0

    def wbits(self):
        return _wbits(self.w)[0]


def csr(V: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray) -> CSR:
    src = np.ascontiguousarray(src, np.uint32)
    dst = np.ascontiguousarray(dst, np.uint32)
    wb, wt = _wbits(w)
    E_raw = src.shape[0]
    row_ptr = np.zeros(V + 1, np.uint32)
    col = np.empty(max(E_raw, 1), np.uint32)
    wo = np.empty(max(E_raw, 1), np.uint32)
    eid = np.empty(max(E_raw, 1), np.uint32)
    E = _load().orc_csr(V, E_raw, _p(src), _p(dst), _p(wb), wt, _p(row_ptr), _p(col), _p(wo), _p(eid))
    if E < 0:
        raise ValueError("endpoint out of range")
    wo = wo[:E].copy()
    return CSR(V, row_ptr, col[:E].copy(), wo.view(np.float32) if wt else wo, eid[:E].copy())


def csr_of(graph) -> CSR:
    return csr(graph.V, graph.src, graph.dst, graph.w)


def partition(V: int, P: int, g: CSR | None = None):
    """Returns (bounds[P+1] uint32, inter[P] uint64)."""
    bounds = np.zeros(P + 1, np.uint32)
    inter = np.zeros(P, np.uint64)
    rc = _load().orc_partition(V, P, _p(g.row_ptr) if g else None, _p(g.col) if g else None,
                               _p(bounds), _p(inter))
    if rc != OK:
        raise ValueError("bad partition arguments")
    return bounds, inter


def dijkstra(g: CSR, s: int):
    """Returns (dist, pred, status). dist is uint32 (u32 weights) or float32."""
    dist = np.empty(g.V, np.uint32)
    pred = np.empty(g.V, np.uint32)
    wb, wt = _wbits(g.w)
    st = _load().orc_dijkstra(g.V, _p(g.row_ptr), _p(g.col), _p(wb), wt, int(s), _p(dist), _p(pred))
    if st == EINVAL:
        raise ValueError("bad source")
    return (dist.view(np.float32) if wt else dist), pred, st


def tight_ties(g: CSR, s: int, dist: np.ndarray) -> int:
    wb, wt = _wbits(g.w)
    db = np.ascontiguousarray(dist).view(np.uint32)
    return int(_load().orc_tight_ties(g.V, _p(g.row_ptr), _p(g.col), _p(wb), wt, int(s), _p(db)))


def trishla(g: CSR, P: int, mode: int = 0, u_lo: int = 0, u_hi: int | None = None):
    """Algorithm 1. mode 0 = local (v_i in u's partition), 1 = global.
    Returns (keep uint8[E], witness uint32[E]); rows outside [u_lo,u_hi) are left as keep=1, witness=NONE."""
    u_hi = g.V if u_hi is None else u_hi
    keep = np.ones(max(g.E, 1), np.uint8)
    witness = np.full(max(g.E, 1), NONE, np.uint32)
    wb, wt = _wbits(g.w)
    rc = _load().orc_trishla(g.V, _p(g.row_ptr), _p(g.col), _p(wb), wt, P, mode, u_lo, u_hi, _p(keep),
                             _p(witness))
    if rc != OK:
        raise ValueError("bad trishla arguments")
    return keep[:g.E], witness[:g.E]


def tree_grad(g: CSR, dist: np.ndarray, pred: np.ndarray, gup: np.ndarray) -> np.ndarray:
    """float64 dL/dw per CSR edge for L = sum g * dist, summed over sources."""
    dist = np.ascontiguousarray(dist, np.float32)
    pred = np.ascontiguousarray(pred, np.uint32)
    gup = np.ascontiguousarray(gup, np.float32)
    S = dist.shape[0]
    grad = np.zeros(max(g.E, 1), np.float64)
    rc = _load().orc_tree_grad(g.V, _p(g.row_ptr), _p(g.col), S, _p(dist), _p(pred), _p(gup), _p(grad))
    if rc != OK:
        raise ValueError("predecessor edge missing from graph")
    return grad[:g.E]


def compact(g: CSR, keep: np.ndarray) -> CSR:
    """The graph with the edges of keep == 0 removed (eid still maps to the raw input)."""
    keep = keep.astype(bool)
    deg = np.diff(g.row_ptr.astype(np.int64))
    rows = np.repeat(np.arange(g.V), deg)
    kept_deg = np.bincount(rows[keep], minlength=g.V)
    row_ptr = np.zeros(g.V + 1, np.uint32)
    row_ptr[1:] = np.cumsum(kept_deg)
    return CSR(g.V, row_ptr, g.col[keep].copy(), g.w[keep].copy(), g.eid[keep].copy())


def layout(g: CSR, P: int):
    """The locality layout (a renaming of vertices; the paper has no such step): inside each
    1D block partition of Sec. III.A (B = ceil(V/P)), vertices ordered by total degree
    (in + out) descending, ties by id ascending.  Returns (ids, slots, h): ids[n] = old id of
    new vertex n, slots = its inverse, h = the renamed graph as a canonical CSR whose eid maps
    each edge to its index in g."""
    V = g.V
    deg = np.diff(g.row_ptr.astype(np.int64)) + np.bincount(g.col.astype(np.int64), minlength=V)
    v = np.arange(V, dtype=np.int64)
    part = v // (-(-V // P))
    ids = np.lexsort((v, -deg, part)).astype(np.uint32)  # primary: partition, then degree desc, then id
    slots = np.empty(V, np.uint32)
    slots[ids] = np.arange(V, dtype=np.uint32)
    tails = np.repeat(np.arange(V, dtype=np.uint32), np.diff(g.row_ptr.astype(np.int64)))
    h = csr(V, slots[tails], slots[g.col], g.w)
    return ids, slots, h

