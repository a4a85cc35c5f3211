"""Python binding of libsssp, a GB300 (sm_103a) implementation of the hot path of
SP_Async (arXiv 2103.12012): CSR build, 1D block partition, Trishla prune,
asynchronous partitioned SSSP, batched SSSP and the tree backward.

This module only marshals arguments: torch tensors provide device memory and
the stream, every step runs in the CUDA kernels of ``_lib/libsssp.so`` behind
the C ABI of ``include/sssp.h``.  There is no CPU fallback: if the library is
missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsssp.so")
_lib = None

SSSP_OK, SSSP_EINVAL, SSSP_ENOMEM, SSSP_ECUDA, SSSP_ETIMEOUT, SSSP_EOVERFLOW, SSSP_EINTERNAL, SSSP_EUNSUPPORTED = \
    range(8)
W_U32, W_F32 = 0, 1
POLICY_RELATIVE, POLICY_FIXED, POLICY_NEAR_FAR, POLICY_ALL = range(4)
POLICY_NAMES = ("relative", "fixed", "near_far", "all")
FLAG_TEST_HOLD_PENDING = 0x1
NONE = 0xFFFFFFFF

P = ctypes.c_void_p
u32, u64, i32, sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t


class SsspGraph(ctypes.Structure):
    _fields_ = [("V", u32), ("E", u32), ("row_ptr", P), ("col", P), ("w", P), ("wtype", i32),
                ("partitions", u32), ("ids", P), ("slots", P)]


class SsspOptions(ctypes.Structure):
    _fields_ = [("threads", u32), ("blocks_per_sm", u32), ("tile", u32), ("split", u32),
                ("delta", ctypes.c_double), ("timeout_ns", u64), ("flags", u32), ("policy", u32),
                ("msg_buffer", u32), ("hub_count", u32), ("ev_relax_begin", P), ("ev_relax_end", P)]


class SsspStats(ctypes.Structure):
    _fields_ = [("edges_scanned", u64), ("atomics", u64), ("improved", u64), ("activations", u64),
                ("rounds", u64), ("vertices", u64), ("remote_activations", u64), ("idle_us", u64),
                ("prune_chunks", u64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class SsspBatchGraph(ctypes.Structure):
    _fields_ = [("row_off", u64), ("edge_off", u64), ("V", u32), ("E", u32)]


class SsspBatch(ctypes.Structure):
    _fields_ = [("n_graphs", u32), ("n_problems", u32), ("graphs", P), ("prob_graph", P), ("prob_source", P),
                ("row_ptr", P), ("col", P), ("w", P), ("wtype", i32), ("dist", P), ("pred", P)]


# name -> (restype, argtypes); the names are exactly the header's entry points
_SIGS = {
    "sssp_status_string": (ctypes.c_char_p, [i32]),
    "sssp_version": (ctypes.c_char_p, []),
    "sssp_build_csr_workspace_size": (sz, [u32, u64]),
    "sssp_build_csr": (i32, [u32, u64, P, P, P, i32, P, P, P, P, P, P, sz, P]),
    "sssp_layout_workspace_size": (sz, [P]),
    "sssp_layout": (i32, [P, P, P, P, P, P, P, P, sz, P]),
    "sssp_partition": (i32, [P, P, P, P]),
    "sssp_prune": (i32, [P, i32, P, P, P]),
    "sssp_compact_workspace_size": (sz, [u32, u32]),
    "sssp_compact": (i32, [P, P, P, P, P, P, P, P, sz, P]),
    "sssp_solve_workspace_size": (sz, [P, u32, P]),
    "sssp_solve": (i32, [P, P, u32, P, P, P, P, sz, P]),
    "sssp_workspace_status": (i32, [P, P, P]),
    "sssp_update": (i32, [P, u32, P, P, P, u32, P, P, sz, P]),
    "sssp_autotune": (i32, [P, P, u32, P, P, P, sz, P, u32, P, P, P]),
    "sssp_solve_noalloc": (i32, [P, P, u32, P, P, P, P, P]),
    "sssp_batch_workspace_size": (sz, [P, P]),
    "sssp_solve_batched": (i32, [P, P, P, sz, P]),
    "sssp_batch_plan_create": (i32, [P, P, P, sz, P, P]),
    "sssp_batch_plan_launch": (i32, [P, P]),
    "sssp_batch_plan_destroy": (None, [P]),
    "sssp_backward_workspace_size": (sz, [u32, u32, u32]),
    "sssp_backward": (i32, [P, u32, P, P, P, P, sz, P]),
    "sssp_shard_problems": (i32, [u32, P, u32, P, P]),
    "sssp_solve_prune": (i32, [P, P, u32, P, P, i32, P, P, P, P, sz, P]),
}


class SsspError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def lib():
    """The loaded libsssp (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsssp is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().sssp_status_string(int(s)).decode()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsssp needs a CUDA GPU")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(st, where):
    if st != SSSP_OK:
        raise SsspError(st, where)


def _ws(nbytes):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def options(threads=0, blocks_per_sm=0, tile=0, split=0, delta=0.0, timeout_ns=0, flags=0,
            policy=POLICY_RELATIVE, msg_buffer=0, hub_count=0) -> SsspOptions:
    return SsspOptions(threads, blocks_per_sm, tile, split, float(delta), int(timeout_ns), flags, int(policy),
                       int(msg_buffer), int(hub_count), None, None)


@dataclass
class DeviceGraph:
    """A canonical CSR in device memory (torch int32 tensors holding uint32 values)."""
    V: int
    E: int
    row_ptr: object
    col: object
    w: object  # int32 (uint32 bits) or float32
    wtype: int
    partitions: int = 1
    eid: object = None  # kept edge -> index in the input edge list (for a layout graph: in the graph it came from)
    ids: object = None  # layout graph: stored vertex -> caller's id
    slots: object = None  # layout graph: caller's id -> stored vertex

    def c(self) -> SsspGraph:
        return SsspGraph(self.V, self.E, self.row_ptr.data_ptr(), self.col.data_ptr() if self.E else None,
                         self.w.data_ptr() if self.E else None, self.wtype, self.partitions,
                         _ptr(self.ids), _ptr(self.slots))

    def with_partitions(self, P):
        if self.ids is not None:
            raise ValueError("a layout graph keeps the partitions it was made for")
        return DeviceGraph(self.V, self.E, self.row_ptr, self.col, self.w, self.wtype, P, self.eid)


def _as_dev_u32(x):
    torch = _torch()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x).view(np.int32))
    return x.to("cuda", non_blocking=False).contiguous()


def _w_dev(w):
    torch = _torch()
    if isinstance(w, np.ndarray):
        if w.dtype == np.float32:
            return torch.from_numpy(np.ascontiguousarray(w)).cuda(), W_F32
        return torch.from_numpy(np.ascontiguousarray(w.astype(np.uint32)).view(np.int32)).cuda(), W_U32
    return w.contiguous(), (W_F32 if w.dtype == torch.float32 else W_U32)


def build_csr(V, src, dst, w, partitions=1, stream=None) -> DeviceGraph:
    """K1: raw edge list -> canonical CSR (self-loops dropped, parallel edges collapsed to min weight)."""
    torch = _torch()
    src_d, dst_d = _as_dev_u32(src), _as_dev_u32(dst)
    w_d, wt = _w_dev(w)
    n = int(src_d.numel())
    row_ptr = torch.empty(V + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    w_out = torch.empty(max(n, 1), dtype=w_d.dtype, device="cuda")
    eid = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    E_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = lib()
    nb = L.sssp_build_csr_workspace_size(V, n)
    ws = _ws(nb)
    st = _stream(stream)
    _check(L.sssp_build_csr(V, n, _ptr(src_d), _ptr(dst_d), _ptr(w_d), wt, _ptr(row_ptr), _ptr(col), _ptr(w_out),
                            _ptr(eid), _ptr(E_out), _ptr(ws), nb, st), "sssp_build_csr")
    _check(L.sssp_workspace_status(_ptr(ws), st, None), "sssp_build_csr (device)")
    E = int(E_out.item())
    return DeviceGraph(V, E, row_ptr, col[:max(E, 1)], w_out[:max(E, 1)], wt, partitions, eid[:max(E, 1)])


def upload_csr(V, row_ptr, col, w, partitions=1, eid=None) -> DeviceGraph:
    """A CSR already in canonical form (e.g. from the oracle) copied to the device."""
    w_d, wt = _w_dev(np.asarray(w))
    E = int(np.asarray(row_ptr)[-1])
    return DeviceGraph(V, E, _as_dev_u32(np.asarray(row_ptr, np.uint32)), _as_dev_u32(np.asarray(col, np.uint32)),
                       w_d, wt, partitions, None if eid is None else _as_dev_u32(np.asarray(eid, np.uint32)))


def layout(g: DeviceGraph, stream=None) -> DeviceGraph:
    """sssp_layout: g with its vertices renumbered inside each block partition by degree (a
    memory layout for the solve; solves on the result take and return the caller's ids)."""
    torch = _torch()
    row_ptr = torch.empty(g.V + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(g.E, 1), dtype=torch.int32, device="cuda")
    w = torch.empty(max(g.E, 1), dtype=g.w.dtype, device="cuda")
    emap = torch.empty(max(g.E, 1), dtype=torch.int32, device="cuda")
    ids = torch.empty(g.V, dtype=torch.int32, device="cuda")
    slots = torch.empty(g.V, dtype=torch.int32, device="cuda")
    L = lib()
    gc = g.c()
    nb = L.sssp_layout_workspace_size(ctypes.byref(gc))
    if nb == 0:
        raise SsspError(SSSP_EINVAL, "sssp_layout_workspace_size")
    ws = _ws(nb)
    st = _stream(stream)
    _check(L.sssp_layout(ctypes.byref(gc), _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(emap), _ptr(ids), _ptr(slots),
                         _ptr(ws), nb, st), "sssp_layout")
    _check(L.sssp_workspace_status(_ptr(ws), st, None), "sssp_layout (device)")
    return DeviceGraph(g.V, g.E, row_ptr, col[:max(g.E, 1)], w[:max(g.E, 1)], g.wtype, g.partitions,
                       emap[:max(g.E, 1)], ids, slots)


def partition(g: DeviceGraph, stream=None):
    """K2: (bounds [P+1], inter-edges per partition [P]) as torch tensors."""
    torch = _torch()
    bounds = torch.empty(g.partitions + 1, dtype=torch.int32, device="cuda")
    inter = torch.empty(g.partitions, dtype=torch.int64, device="cuda")
    gc = g.c()
    _check(lib().sssp_partition(ctypes.byref(gc), _ptr(bounds), _ptr(inter), _stream(stream)), "sssp_partition")
    return bounds, inter


def prune(g: DeviceGraph, mode=0, witness=True, stream=None):
    """K3 Trishla: (keep uint8 [E], witness int32 [E] or None)."""
    torch = _torch()
    keep = torch.empty(max(g.E, 1), dtype=torch.uint8, device="cuda")
    wit = torch.empty(max(g.E, 1), dtype=torch.int32, device="cuda") if witness else None
    gc = g.c()
    _check(lib().sssp_prune(ctypes.byref(gc), int(mode), _ptr(keep), _ptr(wit), _stream(stream)), "sssp_prune")
    return keep[:g.E], (wit[:g.E] if wit is not None else None)


def compact(g: DeviceGraph, keep, stream=None) -> DeviceGraph:
    """The graph without the pruned edges; .eid maps kept edges to g's edge indices."""
    torch = _torch()
    row_ptr = torch.empty(g.V + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(g.E, 1), dtype=torch.int32, device="cuda")
    w = torch.empty(max(g.E, 1), dtype=g.w.dtype, device="cuda")
    emap = torch.empty(max(g.E, 1), dtype=torch.int32, device="cuda")
    E_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = lib()
    nb = L.sssp_compact_workspace_size(g.V, g.E)
    ws = _ws(nb)
    gc = g.c()
    st = _stream(stream)
    _check(L.sssp_compact(ctypes.byref(gc), _ptr(keep), _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(emap), _ptr(E_out),
                          _ptr(ws), nb, st), "sssp_compact")
    E = int(E_out.item())
    return DeviceGraph(g.V, E, row_ptr, col[:max(E, 1)], w[:max(E, 1)], g.wtype, g.partitions, emap[:max(E, 1)])


class Solver:
    """Reusable sssp_solve call: holds the workspace for (graph, S, options)."""

    def __init__(self, g: DeviceGraph, S: int, opts: SsspOptions | None = None):
        torch = _torch()
        self.g, self.S = g, int(S)
        self.opts = opts or options()
        self.gc = g.c()
        L = lib()
        self.ws_bytes = L.sssp_solve_workspace_size(ctypes.byref(self.gc), self.S, ctypes.byref(self.opts))
        if self.ws_bytes == 0:
            raise SsspError(SSSP_EINVAL, "sssp_solve_workspace_size")
        self.ws = _ws(self.ws_bytes)
        dt = torch.float32 if g.wtype == W_F32 else torch.int32
        self.dist = torch.empty((self.S, g.V), dtype=dt, device="cuda")
        self.pred = torch.empty((self.S, g.V), dtype=torch.int32, device="cuda")

    def launch(self, sources, dist=None, pred=None, stream=None):
        """Asynchronous: enqueue the solve; returns the (dist, pred) tensors it writes."""
        dist = self.dist if dist is None else dist
        pred = self.pred if pred is None else pred
        st = lib().sssp_solve(ctypes.byref(self.gc), _ptr(sources), self.S, _ptr(dist), _ptr(pred),
                              ctypes.byref(self.opts), _ptr(self.ws), self.ws_bytes, _stream(stream))
        _check(st, "sssp_solve")
        return dist, pred

    def launch_prune(self, sources, mode, keep, witness=None, dist=None, pred=None, stream=None):
        """sssp_solve_prune, asynchronous: the solve of launch(), with Trishla (mode 0 local, 1 global)
        run on the solve's idle time into keep (uint8 [E]) and witness (int32 [E] or None)."""
        dist = self.dist if dist is None else dist
        pred = self.pred if pred is None else pred
        st = lib().sssp_solve_prune(ctypes.byref(self.gc), _ptr(sources), self.S, _ptr(dist), _ptr(pred), int(mode),
                                    _ptr(keep), _ptr(witness), ctypes.byref(self.opts), _ptr(self.ws), self.ws_bytes,
                                    _stream(stream))
        _check(st, "sssp_solve_prune")
        return dist, pred

    def update(self, dist, pred, tails, stream=None):
        """sssp_update (warm start), asynchronous: dist/pred hold a result for this solver's S
        sources on the graph before some weights fell or edges were added; they are updated in
        place to the result on this solver's graph.  tails: device int32 tensor of the changed
        edges' tails (caller's ids)."""
        n = 0 if tails is None else int(tails.numel())
        st = lib().sssp_update(ctypes.byref(self.gc), self.S, _ptr(dist), _ptr(pred), _ptr(tails) if n else None, n,
                               ctypes.byref(self.opts), _ptr(self.ws), self.ws_bytes, _stream(stream))
        _check(st, "sssp_update")
        return dist, pred

    def status(self, stream=None):
        stats = SsspStats()
        st = lib().sssp_workspace_status(_ptr(self.ws), _stream(stream), ctypes.byref(stats))
        return st, stats.as_dict()

    def __call__(self, sources, check=True, stream=None):
        torch = _torch()
        if isinstance(sources, np.ndarray) or isinstance(sources, (list, tuple)):
            sources = _as_dev_u32(np.asarray(sources, np.uint32))
        dist, pred = self.launch(sources, stream=stream)
        st, stats = self.status(stream)
        if check and st not in (SSSP_OK,):
            raise SsspError(st, "sssp_solve (device)")
        self.last_status, self.last_stats = st, stats
        return dist, pred


def _tune_cache_path():
    return os.environ.get("SSSP_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sssp_gb300",
                                                           "tune.json"))


def _graph_class(g: DeviceGraph, S: int) -> str:
    """Cache key: sizes, weight type, partitions, sources and the weight scale (mean of a sample)."""
    wm = float(g.w[:min(g.E, 65536)].float().mean().item()) if g.E and g.wtype == W_F32 else (
        float((g.w[:min(g.E, 65536)].long() & 0xFFFFFFFF).double().mean().item()) if g.E else 0.0)
    return f"V{g.V}:E{g.E}:w{g.wtype}:P{g.partitions}:S{S}:m{wm:.3g}" + (":layout" if g.ids is not None else "")


def autotune(g: DeviceGraph, sources, base: SsspOptions | None = None, trials: int = 1, cache: bool = True):
    """Options for sssp_solve on graphs of this class: from the JSON cache (SSSP_TUNE_CACHE), else
    measured by sssp_autotune and stored.  Returns (options, ms or None if cached)."""
    import json
    S = len(sources) if not hasattr(sources, "numel") else int(sources.numel())
    key = _graph_class(g, S)
    path = _tune_cache_path()
    db = {}
    if cache and os.path.exists(path):
        try:
            with open(path) as f:
                db = json.load(f)
        except ValueError:
            db = {}
    if key in db and "hub_count" in db[key]:
        o = db[key]
        return options(threads=o["threads"], tile=o["tile"], split=o["split"], delta=o["delta"],
                       policy=o["policy"], hub_count=o["hub_count"]), None
    solver = Solver(g, S, options(split=4))  # workspace large enough for every split candidate
    if isinstance(sources, np.ndarray) or isinstance(sources, (list, tuple)):
        sources = _as_dev_u32(np.asarray(sources, np.uint32))
    best = SsspOptions()
    ms = ctypes.c_float()
    b = base or options()
    _check(lib().sssp_autotune(ctypes.byref(solver.gc), _ptr(sources), S, _ptr(solver.dist), _ptr(solver.pred),
                               _ptr(solver.ws), solver.ws_bytes, ctypes.byref(b), trials, ctypes.byref(best),
                               ctypes.byref(ms), _stream()), "sssp_autotune")
    rec = dict(threads=int(best.threads), tile=int(best.tile), split=int(best.split), delta=float(best.delta),
               policy=int(best.policy), hub_count=int(best.hub_count), ms=round(float(ms.value), 4))
    if cache:
        db[key] = rec
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return options(threads=rec["threads"], tile=rec["tile"], split=rec["split"], delta=rec["delta"],
                   policy=rec["policy"], hub_count=rec["hub_count"]), rec["ms"]


def solve(g: DeviceGraph, sources, opts: SsspOptions | None = None, check=True):
    """sssp_solve for the given sources; returns (dist [S,V], pred [S,V]) torch tensors."""
    s = Solver(g, len(sources) if not hasattr(sources, "numel") else sources.numel(), opts)
    d, p = s(sources, check=check)
    return d.clone(), p.clone(), s.last_status, s.last_stats


def solve_prune(g: DeviceGraph, sources, mode=0, opts: SsspOptions | None = None, witness=True, check=True):
    """sssp_solve_prune: (dist, pred, keep, witness or None, status, stats) -- the solve, with
    Trishla on g run by the solve's idle blocks (and finished right after it)."""
    torch = _torch()
    S = len(sources) if not hasattr(sources, "numel") else int(sources.numel())
    s = Solver(g, S, opts)
    if isinstance(sources, np.ndarray) or isinstance(sources, (list, tuple)):
        sources = _as_dev_u32(np.asarray(sources, np.uint32))
    keep = torch.empty(max(g.E, 1), dtype=torch.uint8, device="cuda")
    wit = torch.empty(max(g.E, 1), dtype=torch.int32, device="cuda") if witness else None
    s.launch_prune(sources, mode, keep, wit)
    st, stats = s.status()
    if check and st != SSSP_OK:
        raise SsspError(st, "sssp_solve_prune (device)")
    return s.dist.clone(), s.pred.clone(), keep[:g.E], (wit[:g.E] if wit is not None else None), st, stats


def update(g: DeviceGraph, dist, pred, tails, opts: SsspOptions | None = None, check=True):
    """Warm start: dist/pred ([S, V] tensors from a solve before some weights fell or edges were
    added) updated in place to the result on g; tails = the changed edges' tails.  Returns
    (dist, pred, status, stats)."""
    s = Solver(g, int(dist.shape[0]), opts)
    if isinstance(tails, np.ndarray) or isinstance(tails, (list, tuple)):
        tails = _as_dev_u32(np.asarray(tails, np.uint32))
    s.update(dist, pred, tails)
    st, stats = s.status()
    if check and st != SSSP_OK:
        raise SsspError(st, "sssp_update (device)")
    return dist, pred, st, stats


class Batch:
    """A batch of independent (graph, source) problems over several graphs, solved in one launch."""

    def __init__(self, graphs, sources, opts: SsspOptions | None = None):
        """graphs: DeviceGraph objects (from build_csr) or canonical CSRs with numpy V, row_ptr, col, w;
        sources: list of source arrays, one per graph."""
        torch = _torch()
        self.opts = opts or options()
        if any(getattr(g, "ids", None) is not None for g in graphs):
            raise ValueError("batched solves take graphs in the caller's ids, not layout graphs")
        Vs = [int(g.V) for g in graphs]
        self.row_off = np.concatenate([[0], np.cumsum([v + 1 for v in Vs])[:-1]]).astype(np.uint64)
        if isinstance(graphs[0], DeviceGraph):
            # device CSRs (e.g. from build_csr): concatenate on the device
            Es = [int(g.E) for g in graphs]
            self.row_ptr = torch.cat([g.row_ptr for g in graphs])
            self.col = torch.cat([g.col[:g.E] for g in graphs])
            self.w = torch.cat([g.w[:g.E] for g in graphs])
            wt = self.wtype = graphs[0].wtype
        else:
            Es = [int(g.row_ptr[-1]) for g in graphs]
            rp = np.concatenate([np.asarray(g.row_ptr, np.uint32) for g in graphs])
            col = np.concatenate([np.asarray(g.col, np.uint32) for g in graphs])
            wt = W_F32 if graphs[0].w.dtype == np.float32 else W_U32
            w = np.concatenate([np.asarray(g.w) for g in graphs])
            self.row_ptr = _as_dev_u32(rp)
            self.col = _as_dev_u32(col)
            self.w, self.wtype = _w_dev(w)
        self.edge_off = np.concatenate([[0], np.cumsum(Es)[:-1]]).astype(np.uint64)
        self.Es = Es
        self.gdesc = (SsspBatchGraph * len(graphs))(*[SsspBatchGraph(int(a), int(b), v, e) for a, b, v, e in
                                                      zip(self.row_off, self.edge_off, Vs, Es)])
        pg, ps = [], []
        for gi, s in enumerate(sources):
            for x in np.asarray(s).tolist():
                pg.append(gi)
                ps.append(int(x))
        self.prob_graph = np.asarray(pg, np.uint32)
        self.prob_source = np.asarray(ps, np.uint32)
        self.out_off = np.concatenate([[0], np.cumsum([Vs[g] for g in pg])[:-1]]).astype(np.int64)
        self.Vs = Vs
        total = int(sum(Vs[g] for g in pg))
        dt = torch.float32 if wt == W_F32 else torch.int32
        self.dist = torch.empty(total, dtype=dt, device="cuda")
        self.pred = torch.empty(total, dtype=torch.int32, device="cuda")
        self.c = SsspBatch(len(graphs), len(pg), ctypes.cast(self.gdesc, P), self.prob_graph.ctypes.data,
                           self.prob_source.ctypes.data, self.row_ptr.data_ptr(), self.col.data_ptr(),
                           self.w.data_ptr(), self.wtype, self.dist.data_ptr(), self.pred.data_ptr())
        L = lib()
        self.ws_bytes = L.sssp_batch_workspace_size(ctypes.byref(self.c), ctypes.byref(self.opts))
        if self.ws_bytes == 0:
            raise SsspError(SSSP_EINVAL, "sssp_batch_workspace_size")
        self.ws = _ws(self.ws_bytes)
        self.plan = None

    @property
    def n_problems(self):
        return int(self.prob_graph.shape[0])

    def solve(self, stream=None):
        _check(lib().sssp_solve_batched(ctypes.byref(self.c), ctypes.byref(self.opts), _ptr(self.ws), self.ws_bytes,
                                        _stream(stream)), "sssp_solve_batched")

    def autotune(self, deltas=(2, 4, 8, 16, 32, 64), tiles=(256, 512, 1024, 2048), threads=(512, 1024),
                 stream=None):
        """Choose the batched kernel's bucket width, tile and block size by timing sssp_solve_batched on
        this batch (coordinate search: delta; then tile and block size together; then delta again at
        3/4, 5/4 and 3/2 of the best).  Sets self.opts and returns (options, ms)."""
        torch = _torch()

        def run(o):
            self.opts = o
            self.solve(stream)
            st, _ = self.status(stream)
            if st != SSSP_OK:
                return float("inf")
            s = torch.cuda.current_stream() if stream is None else stream
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            self.solve(stream)
            b.record(s)
            st, _ = self.status(stream)
            return a.elapsed_time(b) if st == SSSP_OK else float("inf")

        base = self.opts
        best, best_ms = base, run(base)

        def consider(o):
            nonlocal best, best_ms
            ms = run(o)
            if ms < best_ms:
                best, best_ms = o, ms

        for d in deltas:
            consider(options(threads=base.threads, tile=base.tile, delta=d))
        d0 = best.delta
        for th in threads:
            for t in tiles:
                consider(options(threads=th, tile=t, delta=d0))
        b0 = best
        for f in (0.75, 1.25, 1.5):
            d = b0.delta * f if self.wtype == W_F32 else max(1, round(b0.delta * f))
            consider(options(threads=b0.threads, tile=b0.tile, delta=d))
        self.opts = best
        if self.plan is not None:
            lib().sssp_batch_plan_destroy(self.plan)
            self.plan = None
        return best, best_ms

    def make_plan(self, stream=None):
        if self.plan is not None:
            lib().sssp_batch_plan_destroy(self.plan)
            self.plan = None
        h = ctypes.c_void_p()
        _check(lib().sssp_batch_plan_create(ctypes.byref(self.c), ctypes.byref(self.opts), _ptr(self.ws),
                                            self.ws_bytes, _stream(stream), ctypes.byref(h)), "sssp_batch_plan_create")
        self.plan = h

    def replay(self, stream=None):
        _check(lib().sssp_batch_plan_launch(self.plan, _stream(stream)), "sssp_batch_plan_launch")

    def status(self, stream=None):
        stats = SsspStats()
        st = lib().sssp_workspace_status(_ptr(self.ws), _stream(stream), ctypes.byref(stats))
        return st, stats.as_dict()

    def result(self, i):
        """(dist, pred) views of problem i."""
        o, v = int(self.out_off[i]), self.Vs[int(self.prob_graph[i])]
        return self.dist[o:o + v], self.pred[o:o + v]

    def __del__(self):
        if getattr(self, "plan", None) is not None and _lib is not None:
            _lib.sssp_batch_plan_destroy(self.plan)
            self.plan = None


def shard_problems(costs, world: int):
    """sssp_shard_problems (host only): (rank of each problem, total cost of each rank) for
    independent problems with the given estimated costs, split over `world` ranks."""
    costs = np.ascontiguousarray(np.asarray(costs, np.uint64))
    rank_of = np.empty(max(costs.size, 1), np.uint32)
    load = np.empty(max(int(world), 1), np.uint64)
    _check(lib().sssp_shard_problems(costs.size, costs.ctypes.data, int(world), rank_of.ctypes.data,
                                     load.ctypes.data), "sssp_shard_problems")
    return rank_of[:costs.size], load[:int(world)]


def shard_batch(graphs, sources, rank: int, world: int):
    """The (graph, source) problems of a batch that `rank` of `world` solves, split by estimated
    cost (the edges of the problem's graph, plus its vertices).  graphs: objects with V and E
    (or E_raw, or a canonical row_ptr); sources: one array per graph.  Returns (graph indices, sources
    per kept graph), ready for Batch; every rank computes the same split, with no exchange."""
    sizes = []
    for g in graphs:
        if hasattr(g, "E"):
            E = int(g.E)
        elif hasattr(g, "E_raw"):  # an edge list not yet made canonical: its raw edges
            E = int(g.E_raw)
        else:
            E = int(np.asarray(g.row_ptr)[-1])
        sizes.append(E + int(g.V))
    costs, owner = [], []
    for gi, s in enumerate(sources):
        for _ in np.asarray(s).tolist():
            costs.append(sizes[gi])
            owner.append(gi)
    rank_of, _ = shard_problems(costs, world)
    keep_g, keep_s = [], []
    k = 0
    for gi, s in enumerate(sources):
        s = np.asarray(s)
        mine = s[rank_of[k:k + s.size] == rank]
        k += s.size
        if mine.size:
            keep_g.append(gi)
            keep_s.append(mine.astype(np.uint32))
    return keep_g, keep_s


def shard_sources(n_sources: int, rank: int, world: int):
    """Indices of the sources of one multi-source solve that `rank` of `world` solves (equal
    costs: the planner deals them out in turn)."""
    rank_of, _ = shard_problems(np.ones(n_sources, np.uint64), world)
    return np.nonzero(rank_of == rank)[0]


def allreduce_sum(t):
    """Sum a tensor over the ranks of the default torch.distributed group (in place; no-op with
    one rank): the single exchange of the sharded differentiable form, dL/dw summed over the
    ranks' sources."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def backward(g: DeviceGraph, pred, grad_dist, stream=None):
    """K6: dL/dw (float32, CSR edge order) for L = sum grad_dist * dist."""
    torch = _torch()
    S = int(pred.shape[0])
    grad_w = torch.empty(max(g.E, 1), dtype=torch.float32, device="cuda")
    L = lib()
    nb = L.sssp_backward_workspace_size(g.V, g.E, S)
    ws = _ws(nb)
    gc = g.c()
    st = _stream(stream)
    _check(L.sssp_backward(ctypes.byref(gc), S, _ptr(pred.contiguous()), _ptr(grad_dist.contiguous()), _ptr(grad_w),
                           _ptr(ws), nb, st), "sssp_backward")
    _check(L.sssp_workspace_status(_ptr(ws), st, None), "sssp_backward (device)")
    return grad_w[:g.E]


def _autograd():
    torch = _torch()

    class SSSPFunction(torch.autograd.Function):
        """dist = SSSP(w) for fixed topology g and sources; differentiable in the float32 weights w."""

        @staticmethod
        def forward(ctx, w, g: DeviceGraph, sources, opts=None):
            gw = DeviceGraph(g.V, g.E, g.row_ptr, g.col, w.detach().contiguous(), W_F32, g.partitions, g.eid)
            solver = Solver(gw, int(sources.numel()), opts)
            dist, pred = solver(sources)
            ctx.g = gw
            ctx.save_for_backward(pred)
            return dist.clone()

        @staticmethod
        def backward(ctx, grad_dist):
            (pred,) = ctx.saved_tensors
            return backward(ctx.g, pred, grad_dist.float()), None, None, None

    return SSSPFunction


def sssp_function():
    """torch.autograd.Function class for differentiable SSSP (created lazily so importing needs no GPU)."""
    return _autograd()
