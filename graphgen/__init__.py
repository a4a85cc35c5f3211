"""Seeded synthetic inputs for the SSSP library, its tests and its benchmark.

This module only draws graphs, sources and upstream gradients; it contains
none of the shortest-path, pruning or gradient arithmetic, so both the CUDA
path and the CPU oracle may take their inputs from it.

The generators are written in C (``graphgen.c``, counter-based SplitMix64 so
results do not depend on the thread count or the CPU architecture) and loaded
through ctypes.  ``build()`` compiles them with gcc.

The paper's own graphs (Graph1-4 of its experiment section, made with ParMat)
are not available here; the recipes below stand in for them with the five
workload shapes the library is measured on (see ``WORKLOADS``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lib = None

BASE_SEED = 0x53535350  # base seed of the workload recipes; workload k uses BASE_SEED + k

WTYPE_U32 = 0
WTYPE_F32 = 1


def build(force: bool = False) -> str:
    """Compile graphgen.c into an in-tree shared object (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u64, u32, dbl, i = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
        lib.gg_weights_u32.argtypes = [u64, u64, u32, u32, P]
        lib.gg_weights_f32.argtypes = [u64, u64, dbl, dbl, dbl, P]
        lib.gg_normal_f32.argtypes = [u64, u64, P]
        lib.gg_permutation.argtypes = [u64, u32, P]
        lib.gg_rmat.argtypes = [u64, u32, u32, u64, dbl, dbl, dbl, i, P, P]
        lib.gg_er.argtypes = [u64, u32, u64, P, P]
        lib.gg_er.restype = i
        lib.gg_grid.argtypes = [u64, u32, u32, u32, u32, P, P, P]
        lib.gg_grid.restype = u64
        lib.gg_pick_sources.argtypes = [u64, u32, u64, P, P, u32, P]
        lib.gg_pick_sources.restype = u32
        lib.gg_batch_params.argtypes = [u64, u32, dbl, dbl, P, P]
        lib.gg_member_seed.argtypes = [u64, u32]
        lib.gg_member_seed.restype = u64
        lib.gg_rand_u64.argtypes = [u64, u64, u64]
        lib.gg_rand_u64.restype = u64
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """A raw directed edge list (COO) with weights; duplicates and self-loops allowed."""
    V: int
    src: np.ndarray  # uint32 [E_raw]
    dst: np.ndarray  # uint32 [E_raw]
    w: np.ndarray  # uint32 or float32 [E_raw]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def E_raw(self) -> int:
        return int(self.src.shape[0])

    @property
    def wtype(self) -> int:
        return WTYPE_F32 if self.w.dtype == np.float32 else WTYPE_U32


def rand_u64(seed: int, stream: int, ctr: int) -> int:
    return int(_load().gg_rand_u64(seed, stream, ctr))


def weights_u32(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    w = np.empty(n, np.uint32)
    _load().gg_weights_u32(seed, n, lo, hi, _p(w))
    return w


def weights_f32(seed: int, n: int, lo: float, hi: float, jitter: float) -> np.ndarray:
    w = np.empty(n, np.float32)
    _load().gg_weights_f32(seed, n, lo, hi, jitter, _p(w))
    return w


def normal_f32(seed: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    out = np.empty(n, np.float32)
    _load().gg_normal_f32(seed, n, _p(out))
    return out.reshape(shape)


def permutation(seed: int, n: int) -> np.ndarray:
    p = np.empty(n, np.uint32)
    _load().gg_permutation(seed, n, _p(p))
    return p


def rmat(seed: int, scale: int, nedges: int, a=0.57, b=0.19, c=0.19, n: int | None = None,
         permute: bool = True, wlo: int = 1, whi: int = 255, wf32: tuple | None = None) -> Graph:
    """R-MAT edge list of 2^scale vertices (or n < 2^scale with endpoint rejection)."""
    n = (1 << scale) if n is None else n
    src = np.empty(nedges, np.uint32)
    dst = np.empty(nedges, np.uint32)
    _load().gg_rmat(seed, scale, n, nedges, a, b, c, 1 if permute else 0, _p(src), _p(dst))
    w = weights_f32(seed, nedges, *wf32) if wf32 else weights_u32(seed, nedges, wlo, whi)
    return Graph(n, src, dst, w, name=f"rmat-s{scale}", meta=dict(a=a, b=b, c=c, permute=permute))


def erdos_renyi(seed: int, n: int, M: int, wlo: int = 1, whi: int = 255) -> Graph:
    """G(n, M): M distinct non-loop directed pairs, uniform integer weights."""
    src = np.empty(M, np.uint32)
    dst = np.empty(M, np.uint32)
    rc = _load().gg_er(seed, n, M, _p(src), _p(dst))
    if rc != 0:
        raise ValueError("M too large for n")
    return Graph(n, src, dst, weights_u32(seed, M, wlo, whi), name=f"er-{n}-{M}")


def grid(seed: int, rows: int, cols: int, wlo: int = 1, whi: int = 1000) -> Graph:
    """rows x cols 4-neighbour grid, both directions, symmetric weights U{wlo..whi}."""
    E = 2 * (rows * (cols - 1) + (rows - 1) * cols)
    src = np.empty(E, np.uint32)
    dst = np.empty(E, np.uint32)
    w = np.empty(E, np.uint32)
    got = _load().gg_grid(seed, rows, cols, wlo, whi, _p(src), _p(dst), _p(w))
    assert got == E
    return Graph(rows * cols, src, dst, w, name=f"grid-{rows}x{cols}", meta=dict(rows=rows, cols=cols))


def pick_sources(seed: int, g: Graph, count: int) -> np.ndarray:
    """`count` distinct vertices with a non-loop out-edge, seeded uniform."""
    out = np.empty(max(count, 1), np.uint32)
    got = _load().gg_pick_sources(seed, g.V, g.E_raw, _p(g.src), _p(g.dst), count, _p(out))
    return out[:got].copy()


def batch_params(seed: int, g: int, lo_exp=10.0, hi_exp=17.0):
    t = np.zeros(1, np.uint32)
    n = np.zeros(1, np.uint32)
    _load().gg_batch_params(seed, g, lo_exp, hi_exp, _p(t), _p(n))
    return int(t[0]), int(n[0])


def member_seed(seed: int, g: int) -> int:
    return int(_load().gg_member_seed(seed, g))


# ------------------------------------------------------------------ recipes

def workload_er16k(seed: int = BASE_SEED + 1):
    """ER directed graph, 16,384 vertices, 131,072 distinct edges, w ~ U{1..255};
    source 0; 4 vertex-id block partitions."""
    g = erdos_renyi(seed, 16384, 131072, 1, 255)
    return g, np.array([0], np.uint32), 4


def workload_rmat22(seed: int = BASE_SEED + 2, scale: int = 22, edge_factor: int = 16, n_sources: int = 8,
                    partitions: int = 148):
    """R-MAT scale 22, edge factor 16 (67,108,864 raw edges), a/b/c/d = .57/.19/.19/.05,
    seeded vertex permutation, w ~ U{1..255}; 8 sources; 148 partitions."""
    g = rmat(seed, scale, edge_factor << scale, permute=True, wlo=1, whi=255)
    return g, pick_sources(seed, g, n_sources), partitions


def workload_grid4096(seed: int = BASE_SEED + 3, side: int = 4096, partitions: int = 148):
    """4096 x 4096 road-like grid, 4-neighbour, both directions, symmetric w ~ U{1..1000};
    source at corner 0."""
    g = grid(seed, side, side, 1, 1000)
    return g, np.array([0], np.uint32), partitions


def workload_batch512(seed: int = BASE_SEED + 4, n_graphs: int = 512, n_sources: int = 16,
                      lo_exp: float = 10.0, hi_exp: float = 17.0):
    """512 independent graphs: fair coin between ER out-degree 8 (M = 8n) and R-MAT
    edge factor 8 (scale ceil(log2 n), endpoints >= n rejected); n = round(2^U(10,17));
    w ~ U{1..255}; 16 sources each."""
    graphs, sources = [], []
    for gi in range(n_graphs):
        t, n = batch_params(seed, gi, lo_exp, hi_exp)
        ms = member_seed(seed, gi)
        if t == 0:
            g = erdos_renyi(ms, n, 8 * n, 1, 255)
        else:
            scale = max(1, math.ceil(math.log2(n)))
            g = rmat(ms, scale, 8 * n, n=n, permute=True, wlo=1, whi=255)
        graphs.append(g)
        sources.append(pick_sources(ms, g, n_sources))
    return graphs, sources


def workload_rmat18_f32(seed: int = BASE_SEED + 5, scale: int = 18, edge_factor: int = 8, n_sources: int = 32):
    """R-MAT scale 18 (262,144 vertices), edge factor 8, fp32 w ~ U[0.5,2.0) + 1e-4 U[0,1);
    32 sources; upstream dL/d dist ~ N(0,1) fp32 of shape [32, V]."""
    g = rmat(seed, scale, edge_factor << scale, permute=True, wf32=(0.5, 2.0, 1e-4))
    srcs = pick_sources(seed, g, n_sources)
    gout = normal_f32(seed, (len(srcs), g.V))
    return g, srcs, gout


WORKLOADS = {
    "er16k": workload_er16k,
    "rmat22": workload_rmat22,
    "grid4096": workload_grid4096,
    "batch512": workload_batch512,
    "rmat18_f32": workload_rmat18_f32,
}
