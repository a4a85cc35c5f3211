"""sssp_solve_noalloc against sssp_solve, through the C ABI.

sssp_solve_noalloc serves callers that cannot allocate device memory (for
example a plugin inside a host application that owns every device allocation
and hands it only input and output buffers): it takes its scratch from a fixed
array the library reserves on each GPU.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sssp():
    import paper_2103_12012_gb300 as m
    m.lib()
    return m


def _noalloc(sssp, g, sources_d, dist, pred, status, opts=None):
    gc = g.c()
    opts = opts or sssp.options()
    st = sssp.lib().sssp_solve_noalloc(ctypes.byref(gc), ctypes.c_void_p(sources_d.data_ptr()), sources_d.numel(),
                                       ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(pred.data_ptr()),
                                       ctypes.byref(opts), None if status is None else ctypes.c_void_p(status.data_ptr()),
                                       sssp._stream())
    return st


def test_noalloc_matches_solve_on_two_calls_in_a_row(sssp):
    g0, _, P = gg.workload_er16k()
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    calls = [np.array([0, 123, 4567, 16383], np.uint32), np.array([9, 10000], np.uint32)]
    for srcs in calls:
        sources_d = torch.from_numpy(srcs.view(np.int32)).cuda()
        ref_dist, ref_pred, st, _ = sssp.solve(g, srcs)
        assert st == sssp.SSSP_OK
        dist = torch.full_like(ref_dist, 7)
        pred = torch.full_like(ref_pred, 7)
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        assert _noalloc(sssp, g, sources_d, dist, pred, status) == sssp.SSSP_OK
        torch.cuda.synchronize()
        assert int(status.item()) == sssp.SSSP_OK
        # integer distances and predecessors: exact equality is the tolerance
        assert torch.equal(dist, ref_dist)
        assert torch.equal(pred, ref_pred)


def test_noalloc_rejects_problems_beyond_its_fixed_scratch(sssp):
    limit = 8 << 20
    V = 1 << 22  # 8 bytes per vertex per source alone exceed the fixed array
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    gc = sssp.SsspGraph(V, 0, dummy.data_ptr(), None, None, 0, 1)
    need = sssp.lib().sssp_solve_workspace_size(ctypes.byref(gc), 1, None)
    assert need > limit
    st = sssp.lib().sssp_solve_noalloc(ctypes.byref(gc), ctypes.c_void_p(dummy.data_ptr()), 1,
                                       ctypes.c_void_p(dummy.data_ptr()), None, None, None, sssp._stream())
    assert st == sssp.SSSP_ENOMEM


def test_noalloc_reports_a_device_error_then_solves_again(sssp):
    """The device-side status reaches status_out: a solve whose termination count is held one
    above its true value must time out (SSSP_ETIMEOUT, after a 50 ms idle limit), and the next
    call on the same fixed array, once without and once with a status word, is exact again."""
    g0, _, P = gg.workload_er16k()
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    srcs = np.array([0, 4567], np.uint32)
    sources_d = torch.from_numpy(srcs.view(np.int32)).cuda()
    ref_dist, ref_pred, st, _ = sssp.solve(g, srcs)
    assert st == sssp.SSSP_OK
    dist = torch.empty_like(ref_dist)
    pred = torch.empty_like(ref_pred)
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    held = sssp.options(timeout_ns=50_000_000, flags=sssp.FLAG_TEST_HOLD_PENDING)
    assert _noalloc(sssp, g, sources_d, dist, pred, status, held) == sssp.SSSP_OK  # launched
    torch.cuda.synchronize()
    assert int(status.item()) == sssp.SSSP_ETIMEOUT
    dist.fill_(7)
    assert _noalloc(sssp, g, sources_d, dist, pred, None) == sssp.SSSP_OK  # no status word
    torch.cuda.synchronize()
    assert torch.equal(dist, ref_dist) and torch.equal(pred, ref_pred)
    dist.fill_(7)
    assert _noalloc(sssp, g, sources_d, dist, pred, status) == sssp.SSSP_OK
    torch.cuda.synchronize()
    assert int(status.item()) == sssp.SSSP_OK
    assert torch.equal(dist, ref_dist) and torch.equal(pred, ref_pred)
