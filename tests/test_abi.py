"""The C ABI library loads without a GPU, exports every entry point that
include/*.h declares, and rejects bad arguments on the host (no GPU work)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2103_12012_gb300 as sssp
from paper_2103_12012_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return sssp.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sssp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert {"sssp_prune", "sssp_solve", "sssp_solve_batched", "sssp_backward"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(sssp._SIGS) == names, "binding and header disagree"


def test_status_strings(L):
    assert sssp.status_string(sssp.SSSP_OK) == "ok"
    assert sssp.status_string(sssp.SSSP_ETIMEOUT) == "device wait timed out"
    assert L.sssp_version().decode().startswith("libsssp")


def _graph(V=10, E=0, P=1, wtype=0):
    return sssp.SsspGraph(V, E, 16, 16 if E else None, 16 if E else None, wtype, P)


def test_host_argument_checks_without_gpu(L):
    g = _graph()
    opt = sssp.options()
    # NULL graph, zero sources, bad partition counts, bad weight type: rejected before any launch
    assert L.sssp_solve(None, 16, 1, 16, None, None, 16, 1 << 20, None) == sssp.SSSP_EINVAL
    assert L.sssp_solve(ctypes.byref(g), 16, 0, 16, None, None, 16, 1 << 20, None) == sssp.SSSP_EINVAL
    for bad in (_graph(P=0), _graph(P=11), _graph(wtype=7), _graph(V=0)):
        assert L.sssp_solve(ctypes.byref(bad), 16, 1, 16, None, None, 16, 1 << 20, None) == sssp.SSSP_EINVAL
        assert L.sssp_solve_workspace_size(ctypes.byref(bad), 1, None) == 0
    # bad options
    for o in (sssp.options(threads=100), sssp.options(threads=2048), sssp.options(tile=8), sssp.options(delta=-1),
              sssp.options(policy=4), sssp.options(msg_buffer=33)):
        assert L.sssp_solve_workspace_size(ctypes.byref(g), 1, ctypes.byref(o)) == 0
    # the solve kernel runs at most 512 threads per block
    o = sssp.options(threads=1024)
    assert L.sssp_solve(ctypes.byref(g), 16, 1, 16, None, ctypes.byref(o), 256, 1 << 30, None) == sssp.SSSP_EINVAL
    # too-small workspace
    need = L.sssp_solve_workspace_size(ctypes.byref(g), 2, ctypes.byref(opt))
    assert need > 0
    assert L.sssp_solve(ctypes.byref(g), 16, 2, 16, None, ctypes.byref(opt), 256, need - 1, None) == sssp.SSSP_ENOMEM
    assert L.sssp_prune(ctypes.byref(g), 3, 16, None, None) == sssp.SSSP_EINVAL
    assert L.sssp_build_csr(0, 0, None, None, None, 0, None, None, None, None, None, None, 0, None) == sssp.SSSP_EINVAL
    assert L.sssp_backward(ctypes.byref(g), 0, 16, 16, 16, 16, 1 << 20, None) == sssp.SSSP_EINVAL


def test_workspace_sizes_scale(L):
    g = sssp.SsspGraph(4194304, 67108864, 16, 16, 16, 0, 148)
    one = L.sssp_solve_workspace_size(ctypes.byref(g), 1, None)
    eight = L.sssp_solve_workspace_size(ctypes.byref(g), 8, None)
    # packed words dominate: 8 bytes per vertex per source
    assert 8 * 4194304 <= one < 8 * 4194304 * 1.1
    assert abs(eight - 8 * one) < 8 * 4096
    assert L.sssp_build_csr_workspace_size(1000, 5000) > 5000 * 36
    assert L.sssp_backward_workspace_size(1000, 5000, 3) >= 3 * 1000 * 17 + 5000 * 8


def test_batch_tables_checked_on_host(L):
    graphs = (sssp.SsspBatchGraph * 1)(sssp.SsspBatchGraph(0, 0, 10, 0))
    import numpy as np
    pg = np.array([0, 0], np.uint32)
    ps = np.array([3, 11], np.uint32)  # 11 >= V: invalid
    b = sssp.SsspBatch(1, 2, ctypes.cast(graphs, ctypes.c_void_p), pg.ctypes.data, ps.ctypes.data, 16, 16, 16, 0,
                       16, None)
    assert L.sssp_batch_workspace_size(ctypes.byref(b), None) == 0
    ps[1] = 9
    assert L.sssp_batch_workspace_size(ctypes.byref(b), None) > 0


def test_layout_host_checks_without_gpu(L):
    g = _graph(V=1000, E=5000, P=4)
    need = L.sssp_layout_workspace_size(ctypes.byref(g))
    assert need > 5000 * 8 + 1000 * 24  # renumbered edge list + sort keys and values
    assert L.sssp_layout_workspace_size(None) == 0
    lay = _graph(V=1000, E=5000, P=4)
    lay.ids, lay.slots = 16, 16
    assert L.sssp_layout_workspace_size(ctypes.byref(lay)) == 0  # already a layout graph
    half = _graph(V=1000, E=5000, P=4)
    half.ids = 16  # ids without slots: not a graph
    assert L.sssp_solve_workspace_size(ctypes.byref(half), 1, None) == 0
    assert L.sssp_solve(ctypes.byref(half), 16, 1, 16, None, None, 16, 1 << 20, None) == sssp.SSSP_EINVAL
    # missing outputs, misaligned or short workspace
    assert L.sssp_layout(ctypes.byref(g), None, 16, 16, None, 16, 16, 16, need, None) == sssp.SSSP_EINVAL
    assert L.sssp_layout(ctypes.byref(g), 16, 16, 16, None, None, 16, 16, need, None) == sssp.SSSP_EINVAL
    assert L.sssp_layout(ctypes.byref(g), 16, 16, 16, None, 16, 16, 17, need, None) == sssp.SSSP_EINVAL
    assert L.sssp_layout(ctypes.byref(g), 16, 16, 16, None, 16, 16, 16, need - 1, None) == sssp.SSSP_ENOMEM
    assert L.sssp_layout(ctypes.byref(lay), 16, 16, 16, None, 16, 16, 16, need, None) == sssp.SSSP_EINVAL
    # the tree backward indexes edges of the graph it is given: a layout graph is refused
    assert L.sssp_backward(ctypes.byref(lay), 1, 16, 16, 16, 16, 1 << 30, None) == sssp.SSSP_EINVAL


def test_update_host_checks_without_gpu(L):
    g = _graph(V=1000, E=5000, P=4)
    # pred is required (the previous predecessors seed the canonical ones); tails unless n_tails = 0
    assert L.sssp_update(ctypes.byref(g), 1, 16, None, 16, 1, None, 16, 1 << 30, None) == sssp.SSSP_EINVAL
    assert L.sssp_update(ctypes.byref(g), 1, 16, 16, None, 3, None, 16, 1 << 30, None) == sssp.SSSP_EINVAL
    assert L.sssp_update(ctypes.byref(g), 0, 16, 16, 16, 1, None, 16, 1 << 30, None) == sssp.SSSP_EINVAL
    assert L.sssp_update(None, 1, 16, 16, 16, 1, None, 16, 1 << 30, None) == sssp.SSSP_EINVAL
    need = L.sssp_solve_workspace_size(ctypes.byref(g), 2, None)
    assert L.sssp_update(ctypes.byref(g), 2, 16, 16, 16, 1, None, 16, need - 1, None) == sssp.SSSP_ENOMEM



def test_missing_library_raises(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every call fails loudly."""
    monkeypatch.setattr(sssp, "_lib", None)
    monkeypatch.setattr(sssp, "LIB_PATH", str(tmp_path / "libsssp.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sssp.lib()


def test_no_gpu_means_no_solve():
    """On a machine without a GPU the binding raises instead of computing anywhere else."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    src = np.array([0, 1], np.uint32)
    dst = np.array([1, 2], np.uint32)
    w = np.array([3, 4], np.uint32)
    with pytest.raises(RuntimeError, match="CUDA GPU"):
        sssp.build_csr(3, src, dst, w)
    with pytest.raises(RuntimeError, match="CUDA GPU"):
        sssp.Batch([], [])


def test_options_layout_matches_the_header():
    """sssp_options as the header declares it: 4 uint32, a double, a uint64, flags, policy, msg_buffer,
    hub_count, two pointers."""
    O = sssp.SsspOptions
    assert [f[0] for f in O._fields_] == ["threads", "blocks_per_sm", "tile", "split", "delta", "timeout_ns",
                                          "flags", "policy", "msg_buffer", "hub_count", "ev_relax_begin",
                                          "ev_relax_end"]
    assert O.delta.offset == 16 and O.timeout_ns.offset == 24 and O.policy.offset == 36
    assert O.msg_buffer.offset == 40 and O.ev_relax_begin.offset == 48 and ctypes.sizeof(O) == 64
    assert sssp.POLICY_NAMES == ("relative", "fixed", "near_far", "all")
