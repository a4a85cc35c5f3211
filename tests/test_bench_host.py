"""Host-side logic of bench.py (no GPU): the kernel-code hash that keys the committed DRAM
capture, the traffic scaling, the peak lookup and the clock-sample parsing that decides
whether a timed run is kept."""
import json

import bench


def test_code_hash_ignores_comments_and_blank_lines(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n    return x + 1;  // one\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("/* a block\n comment */\nint f(int x) {\n\n    return x + 1;  // another note\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.code_sha256(str(a)) == bench.code_sha256(str(b))
    assert bench.code_sha256(str(a)) != bench.code_sha256(str(c))


def test_dram_traffic_scales_by_edges_and_lapses_when_the_code_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"source": "k.cu", "code_sha256": bench.code_sha256(str(src)), "capture": "test capture",
           "dram_bytes_per_scanned_edge": 19.5}
    (tmp_path / "profiles" / "k_solve_dram_traffic.txt").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t, note = bench.dram_traffic(1000)
    assert t == 19500 and note.startswith("test capture")
    src.write_text("// a comment only\n__global__ void k() {}\n")
    assert bench.dram_traffic(1000)[0] == 19500
    src.write_text("__global__ void k() { int a = 0; }\n")
    assert bench.dram_traffic(1000) == (None, "kernel changed since the capture")
    (tmp_path / "profiles" / "k_solve_dram_traffic.txt").unlink()
    assert bench.dram_traffic(1000) == (None, "no capture")


def test_peaks_measured_file_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6794.1, "bf16_tflops": 1900}))
    assert bench.peaks() == (6794.1, "measured")


def test_parse_clocks_median_and_reasons():
    rows = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.parse_clocks(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clocks("0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active")
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.parse_clocks("")["samples"] == 0


def test_cpu_baseline_single_all_cores_and_trishla():
    """The bench's CPU baseline on a small R-MAT: the single-threaded oracle, the all-cores run
    (one source per spawned process, over the saved CSR) and the oracle Trishla timing."""
    import os

    import graphgen as gg
    g0 = gg.rmat(gg.BASE_SEED + 2, 12, 16 << 12, permute=True, wlo=1, whi=255)
    srcs = gg.pick_sources(gg.BASE_SEED + 2, g0, 4)
    out = bench.cpu_baseline(g0, srcs[:1], all_srcs=srcs)
    assert out["kind"] == "oracle" and out["cores"] == 1 and out["value"] > 0
    ac = out["all_cores"]
    assert ac["cores"] == min(4, os.cpu_count() or 1) and ac["value"] > 0 and ac["unit"] == out["unit"]
    tr = out["trishla_er16k"]
    assert tr["edges"] == 131072 and tr["pruned"] > 0 and tr["s"] > 0


def test_tree_path_sums_and_depth_against_brute_force():
    """The grid latency model's hop and crossing counts: per-vertex sums along predecessor paths
    by pointer doubling, against walking each path."""
    import numpy as np
    import torch
    NONE = 0xFFFFFFFF
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 300):
        for _ in range(4):
            order = rng.permutation(n)
            pred = np.full(n, NONE, np.uint32)
            for k in range(1, n):
                if rng.random() < 0.9:
                    pred[order[k]] = order[rng.integers(0, k)]
            w = rng.integers(0, 2, n)
            got = bench.tree_path_sums(torch.from_numpy(pred.view(np.int32)[None]), torch.from_numpy(w)[None])[0]
            hops = bench.tree_path_sums(torch.from_numpy(pred.view(np.int32)[None]))[0]
            for v in range(n):
                s = h = 0
                x = v
                while pred[x] != NONE:
                    s += int(w[x])
                    h += 1
                    x = pred[x]
                assert int(got[v]) == s and int(hops[v]) == h
            assert int(bench.tree_depth(torch.from_numpy(pred.view(np.int32)[None]))[0]) == int(hops.max())
    chain = np.concatenate([np.array([NONE], np.uint32), np.arange(99999, dtype=np.uint32)])
    assert int(bench.tree_depth(torch.from_numpy(chain.view(np.int32)[None]))[0]) == 99999


def test_batched_traffic_lookup(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"source": "k.cu", "code_sha256": bench.code_sha256(str(src)), "dram_bytes_per_scanned_edge": 121.5}
    (tmp_path / "profiles" / "k_batched_dram_traffic.txt").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.batched_traffic(1000) == 121500
    src.write_text("__global__ void k() { int changed = 1; }\n")
    assert bench.batched_traffic(1000) is None


def test_sharded_extras_pass_through_on_one_rank():
    d = {"graph_replay_ms": 47.2, "problems": 8192}
    assert bench._reduce_sharded("batched", d, 1, None) is d
