"""Benchmark of the SP_Async hot path on GB300.

One step = one pass of the per-run phases (the paper's "SSSP + termination",
repeated per source) over one batch: init -> persistent asynchronous
relaxation -> unpack, for the 8 sources of the R-MAT scale-22 workload
(4,194,304 vertices, 67,108,864 raw edges, 148 partitions), graph resident in
HBM.  The one-time phases (CSR build, partition, Trishla prune) are timed once
and reported under "phases".

value  = GTEPS: edges (after dedupe) whose tail is reached, summed over the
         step's sources, / device time per step (CUDA events, max over ranks).
e2e    = the same metric through the C ABI with host buffers: pinned host CSR
         and sources copied in, dist/pred copied out, inside the timed region.
roofline: the persistent relaxation kernel (launch timed alone with events
         recorded by the library on the launching stream); algorithmic bytes
         per source = 8 per reached edge (col + weight) + 16 per reached vertex
         (row_ptr pair + final packed word).
--impl reference: the CPU oracle (binary-heap Dijkstra) on the same workload,
         one source per step, on the host cores.

Multi-GPU (torchrun): every rank solves its own 8 sources (weak scaling, no
collective on the data path); value sums all ranks' edges over the slowest
rank's time.  The batched extra splits its (graph, source) problems over the
ranks with the library's planner (no exchange) and the differentiable extra
splits its sources and sums dL/dw with one all-reduce; the grid and
warm-start extras run on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

METRIC = "GTEPS (SSSP, R-MAT scale 22 ef16, 8 sources per step)"
UNIT = "GTEPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, differentiable and grid workloads")
    ap.add_argument("--extras", default="", help="comma-separated subset of the extras to run (default: all)")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--delta", type=float, default=0.0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--policy", type=int, default=0, help="frontier policy (0 relative, 1 fixed, 2 near-far, 3 all)")
    ap.add_argument("--hubs", type=int, default=0, help="hub_count (layout graphs)")
    ap.add_argument("--no-tune", action="store_true", help="library defaults instead of the autotuned schedule")
    ap.add_argument("--profile-case", choices=["batched", "batched-full", "backward", "prune", "grid", "all"],
                    help="run a small case of one kernel three times and exit (for ncu captures)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_sources(g, rank, count=8):
    """The 8 sources of a rank: rank 0 takes the workload's own sources; other ranks draw their own."""
    seed = gg.BASE_SEED + 2 + 1000 * rank
    return gg.pick_sources(seed, g, count)


def code_sha256(path):
    """sha256 of a CUDA source with its comments and blank lines removed: what the capture of a
    kernel depends on (a comment edit keeps the capture valid, a code edit does not)."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()


def dram_traffic(edges_scanned):
    """DRAM bytes per launch of the relaxation kernel from the committed ncu capture, scaled to this
    launch by edges scanned; None if the kernel code changed since that capture."""
    try:
        rec = json.loads(open(os.path.join(ROOT, "profiles", "k_solve_dram_traffic.txt")).read())
        sha = code_sha256(os.path.join(ROOT, rec["source"]))
    except (OSError, ValueError, KeyError):
        return None, "no capture"
    if sha != rec["code_sha256"]:
        return None, "kernel changed since the capture"
    return int(rec["dram_bytes_per_scanned_edge"] * edges_scanned), rec["capture"] + ", scaled by edges scanned"


def batched_traffic(edges_scanned):
    """DRAM bytes of one k_batched launch from the committed one-pass capture of the full batch,
    scaled by edges scanned; None if there is no capture or the kernel code changed since."""
    try:
        rec = json.loads(open(os.path.join(ROOT, "profiles", "k_batched_dram_traffic.txt")).read())
        if code_sha256(os.path.join(ROOT, rec["source"])) != rec["code_sha256"]:
            return None
    except (OSError, ValueError, KeyError):
        return None
    return int(rec["dram_bytes_per_scanned_edge"] * edges_scanned)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        return parse_clocks(out)


def parse_clocks(out):
    """nvidia-smi rows (the Clocks query, csv, no header, no units) -> median SM clock under load,
    the highest max clock seen, and every throttle reason that was active in any sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(scale):
    if scale == 22:
        g, srcs, P = gg.workload_rmat22()
    else:  # smaller case of the same recipe (profiling captures)
        g, srcs, P = gg.workload_rmat22(scale=scale)
    return g, P


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2103_12012_gb300 as sssp

    ws, rank, local = dist_env()
    if ws > 1:
        import datetime
        dist.init_process_group("nccl", device_id=torch.device("cuda", local),
                                timeout=datetime.timedelta(seconds=600))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    g0, P = make_workload(a.scale)
    srcs = rank_sources(g0, rank)
    S = len(srcs)

    # one-time phases (Sec. IV.B): CSR build, partition
    t0 = time.perf_counter()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    src_d = torch.from_numpy(g0.src.view(np.int32)).to(dev)
    dst_d = torch.from_numpy(g0.dst.view(np.int32)).to(dev)
    w_d = torch.from_numpy(g0.w.view(np.int32)).to(dev)
    torch.cuda.synchronize()
    g = sssp.build_csr(g0.V, src_d, dst_d, w_d, partitions=P)  # first call: allocation and module loading
    del g
    torch.cuda.synchronize()
    e0.record()
    g = sssp.build_csr(g0.V, src_d, dst_d, w_d, partitions=P)
    e1.record()
    torch.cuda.synchronize()
    csr_ms = e0.elapsed_time(e1)
    e0.record()
    bounds, inter = sssp.partition(g)
    e1.record()
    torch.cuda.synchronize()
    part_ms = e0.elapsed_time(e1)
    del src_d, dst_d, w_d
    inter_total = int(inter.sum().item())
    # Trishla (Algorithm 1, local mode) on the full graph: a one-time phase, reported apart
    e0.record()
    keep, _ = sssp.prune(g, 0, witness=False)
    e1.record()
    torch.cuda.synchronize()
    prune_ms = e0.elapsed_time(e1)
    pruned = int((keep == 0).sum().item())
    del keep
    # locality layout: vertices renumbered inside their partitions by degree (one-time); the
    # solves below run on it and take / return the caller's ids
    e0.record()
    h = sssp.layout(g)
    e1.record()
    torch.cuda.synchronize()
    layout_ms = e0.elapsed_time(e1)

    sources_d = torch.from_numpy(srcs.view(np.int32)).to(dev)
    tuned_ms = None
    if a.no_tune or a.threads or a.tile or a.delta or a.split:
        opts = sssp.options(threads=a.threads, tile=a.tile, delta=a.delta, split=a.split, policy=a.policy,
                            hub_count=a.hubs)
    else:
        t0 = time.perf_counter()
        opts, tuned_ms = sssp.autotune(h, sources_d, trials=2)
        tune_s = time.perf_counter() - t0
    solver = sssp.Solver(h, S, opts)

    # warm-up (also the step whose output defines the traversed-edge count)
    for _ in range(max(a.warmup, 1)):
        solver.launch(sources_d)
    st, stats = solver.status()
    if st != sssp.SSSP_OK:
        raise RuntimeError(f"solve failed: {sssp.status_string(st)}")
    deg = (g.row_ptr[1:].to(torch.int64) - g.row_ptr[:-1].to(torch.int64))
    reached = solver.dist.view(torch.int32) != -1
    E_r = int((reached.to(torch.int64) * deg[None, :]).sum().item())
    V_r = int(reached.sum().item())
    alg_bytes = 8 * E_r + 16 * V_r

    # timed region: K steps, events around the whole step and around each relaxation kernel launch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    for b_, e_ in evs:  # create the underlying CUDA events before handing their handles to the library
        b_.record()
        e_.record()
    clocks = Clocks(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]  # step boundaries
    t_start, t_end = marks[0], marks[-1]
    t_start.record()
    for k in range(a.steps):
        solver.opts.ev_relax_begin = evs[k][0].cuda_event
        solver.opts.ev_relax_end = evs[k][1].cuda_event
        solver.launch(sources_d)
        marks[k + 1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    solver.opts.ev_relax_begin = None
    solver.opts.ev_relax_end = None
    if ws > 1:
        dist.barrier()
    st, stats = solver.status()
    if st != sssp.SSSP_OK:
        raise RuntimeError(f"solve failed: {sssp.status_string(st)}")
    total_ms = t_start.elapsed_time(t_end)
    relax_ms = [b.elapsed_time(e) for b, e in evs]
    step_ms = [marks[k].elapsed_time(marks[k + 1]) for k in range(a.steps)]
    ms_step = total_ms / a.steps
    ms_step_median = statistics.median(step_ms)
    if ws > 1:
        t = torch.tensor([ms_step, ms_step_median], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step, ms_step_median = float(t[0].item()), float(t[1].item())
        e = torch.tensor([E_r], device=dev, dtype=torch.float64)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        E_all = float(e.item())
    else:
        E_all = float(E_r)
    gteps = E_all / (ms_step * 1e-3) / 1e9

    peak, peak_kind = peaks()
    relax_avg = statistics.mean(relax_ms)
    achieved = alg_bytes / (relax_avg * 1e-3) / 1e9
    traffic, traffic_note = dram_traffic(stats["edges_scanned"])

    # each frontier policy at its best bucket width (rank 0; outside the timed region)
    policies = messages = None
    if rank == 0 and not a.no_extras:
        policies = policy_table(sssp, h, sources_d, opts, E_r)
        messages = message_table(sssp, h, sources_d, opts, E_r)

    # end to end through the C ABI with host buffers
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(sssp, h, srcs, opts, dev, E_r, max(3, min(a.steps, 10)))

    # CPU baseline: the oracle on this host's cores (rank 0, N=1 only)
    cpu = None
    if not a.no_cpu_baseline and ws == 1 and rank == 0:
        cpu = cpu_baseline(g0, srcs[:1], all_srcs=srcs)

    line = {
        "metric": METRIC, "value": round(gteps, 4), "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_step, 4), "ms_per_step_median": round(ms_step_median, 4),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded R-MAT, weights U{1..255})",
        "config": {"workload": f"rmat-s{a.scale}-ef16 directed, a/b/c=.57/.19/.19, permuted ids, "
                               f"{g0.V} vertices, {g0.E_raw} raw edges ({g.E} after dedupe), "
                               f"{S} sources per GPU, {P} partitions",
                   "partitions": P, "sources_per_gpu": S, "l2": "inputs larger than L2 (CSR and state > 0.5 GB)",
                   "layout": "vertices renumbered inside their partitions by degree (sssp_layout, one-time); "
                             "sources and outputs in the generator's ids",
                   "options": {"threads": opts.threads or 512, "tile": opts.tile or 1024,
                               "delta": opts.delta or 4, "split": opts.split or 1,
                               "policy": sssp.POLICY_NAMES[opts.policy], "hub_count": opts.hub_count,
                               "autotuned": not (a.no_tune or a.threads or a.tile or a.delta or a.split)}},
        "roofline": {"bound": "hbm", "kernel": "k_solve (persistent relaxation)", "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "traffic_note": traffic_note, "alg_bytes_per_launch": alg_bytes,
                     "kernel_ms": round(relax_avg, 4), "kernel_ms_median": round(statistics.median(relax_ms), 4)},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": 4 * a.steps,
        "phases": {"csr_build_ms": round(csr_ms, 3), "partition_ms": round(part_ms, 3),
                   "layout_ms": round(layout_ms, 3),
                   "prune_local_ms": round(prune_ms, 3), "pruned_edges": pruned, "edges": g.E,
                   "toka_threshold_interedges": inter_total, "toka_threshold_msgs": inter_total * P},
        "work": {"reached_edges": E_r, "reached_vertices": V_r, "stats_last_step": stats,
                 "work_inflation": round(stats["edges_scanned"] / max(E_r, 1), 4),
                 "policies": policies, "message_buffering": messages},
    }
    if not a.no_extras:
        ex = extras(sssp, dev, rank, ws, tuple(x for x in a.extras.split(",") if x))
        if rank == 0:
            line["extras"] = ex
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def policy_table(sssp, g, src_d, base, E_ref, reps=3):
    """Each frontier policy at its best bucket width (a sweep over 1/64 .. 4 x the mean weight,
    refined at 3/4 and 3/2 of the best, as the autotuner's) with the given tile and split: ms
    per solve (CUDA events, median of `reps`) and the work inflation (edges scanned / E_ref).
    A candidate whose first run takes over 3x the best so far is not repeated."""
    import torch
    w = g.w[:min(g.E, 65536)]
    mean = float(w.float().mean()) if g.wtype == sssp.W_F32 else float((w.long() & 0xFFFFFFFF).double().mean())
    factors = (1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2, 1, 2, 4)
    S = int(src_d.numel())
    out = {}
    best_all = None
    def width(x):
        return x if g.wtype == sssp.W_F32 else max(1.0, float(int(x)))

    for pol, name in enumerate(sssp.POLICY_NAMES):
        best = None
        coarse = [width(mean * f) for f in factors] if pol != sssp.POLICY_ALL else [1.0]
        for refine in (False, True):
            if refine:  # 3/4 and 3/2 of the best width
                if pol == sssp.POLICY_ALL or best is None:
                    break
                cands = [x for x in (width(best["delta"] * 0.75), width(best["delta"] * 1.5)) if x != best["delta"]]
            else:
                cands = coarse
            for d in cands:
                solver = sssp.Solver(g, S, sssp.options(threads=base.threads, tile=base.tile, split=base.split,
                                                        delta=d, policy=pol, hub_count=base.hub_count))
                a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record()
                solver.launch(src_d)
                b0.record()
                st, stats = solver.status()
                if st != sssp.SSSP_OK:
                    continue
                first = a0.elapsed_time(b0)
                if best_all is not None and first > 3 * best_all:  # far off the pace: one untimed run is enough
                    if best is None or first < best["ms"]:
                        best = {"delta": d, "ms": round(first, 3), "work_inflation": round(stats["edges_scanned"] / E_ref, 3),
                                "rounds": stats["rounds"], "single_run": True}
                    continue
                times = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    solver.launch(src_d)
                    b.record()
                    torch.cuda.synchronize()
                    times.append(a.elapsed_time(b))
                ms = statistics.median(times)
                if best is None or ms < best["ms"]:
                    best = {"delta": d, "ms": round(ms, 3), "work_inflation": round(stats["edges_scanned"] / E_ref, 3),
                            "rounds": stats["rounds"]}
                best_all = ms if best_all is None else min(best_all, ms)
                del solver
        out[name] = best
    return out


def message_table(sssp, g, src_d, base, E_ref, sizes=(0, 1, 8, 32), reps=3):
    """Message buffering (msg_buffer: 0 = direct, k = a warp pushes its held messages out at k and
    at the end of each sub-round) at the given schedule: ms per solve (CUDA events, median of
    `reps`), work inflation (edges scanned / E_ref) and rounds."""
    import torch
    S = int(src_d.numel())
    out = {}
    for k in sizes:
        o = sssp.options(threads=base.threads, tile=base.tile, split=base.split, delta=base.delta,
                         policy=base.policy, msg_buffer=k, hub_count=base.hub_count)
        solver = sssp.Solver(g, S, o)
        solver.launch(src_d)
        st, stats = solver.status()
        if st != sssp.SSSP_OK:
            out[str(k)] = {"error": sssp.status_string(st)}
            continue
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            solver.launch(src_d)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        out[str(k)] = {"ms": round(statistics.median(times), 3),
                       "work_inflation": round(stats["edges_scanned"] / E_ref, 3), "rounds": stats["rounds"],
                       "remote_activations": stats["remote_activations"]}
        del solver
    return out


def run_e2e(sssp, g, srcs, opts, dev, E_r, steps):
    """H2D (pinned CSR [+ layout ids] + sources) -> sssp_solve -> D2H (dist, pred), every step.

    Two slots (device buffers, solver, stream) alternate between steps, so one step's copies
    run on the copy engines while the other step's solve runs; every step still copies all of
    its inputs in and all of its results out inside the timed region.  The same steps run
    one after another on one stream give the serial figure reported beside it."""
    import torch
    host = [g.row_ptr, g.col, g.w] + ([g.ids, g.slots] if g.ids is not None else [])
    host = [t.cpu().pin_memory() for t in host]
    src_h = torch.from_numpy(srcs.view(np.int32)).pin_memory()
    S = len(srcs)

    def make_slot():
        devs = [torch.empty_like(t, device=dev) for t in host]
        gd = sssp.DeviceGraph(g.V, g.E, devs[0], devs[1], devs[2], g.wtype, g.partitions, None,
                              *(devs[3:5] if len(devs) == 5 else (None, None)))
        return dict(devs=devs, src=torch.empty_like(src_h, device=dev), solver=sssp.Solver(gd, S, opts),
                    dist_h=torch.empty((S, g.V), dtype=torch.int32).pin_memory(),
                    pred_h=torch.empty((S, g.V), dtype=torch.int32).pin_memory(), stream=torch.cuda.Stream(dev))

    slots = [make_slot(), make_slot()]
    h2d = sum(t.numel() * 4 for t in host) + src_h.numel() * 4
    d2h = 2 * S * g.V * 4

    def step(sl, stream):
        with torch.cuda.stream(stream):
            for d_, h_ in zip(sl["devs"], host):
                d_.copy_(h_, non_blocking=True)
            sl["src"].copy_(src_h, non_blocking=True)
            sl["solver"].launch(sl["src"], stream=stream)
            sl["dist_h"].copy_(sl["solver"].dist, non_blocking=True)
            sl["pred_h"].copy_(sl["solver"].pred, non_blocking=True)

    def timed(n, pipelined):
        main = torch.cuda.current_stream(dev)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(main)
        for sl in slots:
            sl["stream"].wait_stream(main)
        for k in range(n):
            sl = slots[k % 2] if pipelined else slots[0]
            step(sl, sl["stream"])
        for sl in slots:
            main.wait_stream(sl["stream"])
        t1.record(main)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / n

    timed(2, True)  # warm-up of both slots
    ms_serial = timed(steps, False)
    ms = timed(steps, True)
    for sl in slots:
        st, _ = sl["solver"].status()
        assert st == sssp.SSSP_OK
    assert torch.equal(slots[0]["dist_h"], slots[1]["dist_h"])
    return {"value": round(E_r / (ms * 1e-3) / 1e9, 4), "unit": UNIT, "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": steps,
            "overlap": "two slots on two streams: a step's copies overlap the other step's solve",
            "serial": {"value": round(E_r / (ms_serial * 1e-3) / 1e9, 4), "ms_per_step": round(ms_serial, 4)}}


def _oracle_worker(args):
    """One oracle Dijkstra in a spawned process, over the CSR arrays saved by cpu_baseline (mapped,
    not copied).  Returns (wall-clock start, end, edges with a reached tail)."""
    import oracle
    d, V, s, start_at = args
    rp, col, w = (np.load(os.path.join(d, n + ".npy"), mmap_mode="r") for n in ("row_ptr", "col", "w"))
    ref = oracle.CSR(V, rp, col, w, None)
    time.sleep(max(0.0, start_at - time.time()))  # all workers start together
    t0 = time.time()
    dist, _, _ = oracle.dijkstra(ref, s)
    t1 = time.time()
    deg = np.diff(np.asarray(rp, np.int64))
    return t0, t1, int(deg[dist != 0xFFFFFFFF].sum())


def cpu_baseline(g0, srcs, all_srcs=None, er16k=True):
    """The oracle as it stands: its own CSR from the raw edges (untimed), then binary-heap Dijkstra,
    single-threaded on `srcs`.  Also, as extra keys: the same oracle on all of `all_srcs` at once,
    one source per spawned process (all cores), and the naive Trishla prune of the 16K-vertex ER
    workload (local mode, 4 partitions), single-threaded."""
    import multiprocessing as mp
    import tempfile
    from concurrent.futures import ProcessPoolExecutor
    import oracle
    ref = oracle.csr_of(g0)
    deg = np.diff(ref.row_ptr.astype(np.int64))
    t_total, e_total = 0.0, 0
    for s in srcs:
        t0 = time.perf_counter()
        d, _, _ = oracle.dijkstra(ref, int(s))
        t_total += time.perf_counter() - t0
        e_total += int(deg[d != 0xFFFFFFFF].sum())
    out = {"value": round(e_total / t_total / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{len(srcs)} of 8 sources, full graph, single-threaded binary-heap Dijkstra "
                     f"({t_total:.2f} s)", "host_cores_available": os.cpu_count()}
    if all_srcs is not None and len(all_srcs) > 1:
        n = min(len(all_srcs), os.cpu_count() or 1)
        with tempfile.TemporaryDirectory() as td:
            for name in ("row_ptr", "col", "w"):
                np.save(os.path.join(td, name + ".npy"), getattr(ref, name)[:max(ref.E, 1)] if name != "row_ptr"
                        else ref.row_ptr)
            # spawned (never forked after CUDA started); a worker that dies raises here
            with ProcessPoolExecutor(n, mp_context=mp.get_context("spawn")) as pool:
                start_at = time.time() + 5.0
                res = list(pool.map(_oracle_worker, [(td, ref.V, int(s), start_at) for s in all_srcs]))
        wall = max(r[1] for r in res) - min(r[0] for r in res)
        out["all_cores"] = {"value": round(sum(r[2] for r in res) / wall / 1e9, 6), "unit": UNIT, "cores": n,
                            "sample": f"all {len(all_srcs)} sources, one per process, {wall:.2f} s wall"}
    if er16k:
        e0, _, P1 = gg.workload_er16k()
        r1 = oracle.csr_of(e0)
        t0 = time.perf_counter()
        keep, _ = oracle.trishla(r1, P1, 0)
        out["trishla_er16k"] = {"s": round(time.perf_counter() - t0, 4), "cores": 1, "edges": r1.E,
                                "pruned": int((keep[:r1.E] == 0).sum())}
        out.update(cpu_other_configs())
    return out


def cpu_other_configs():
    """The oracle on bounded samples of the batched and differentiable workloads, single-threaded:
    the first source of every 8th graph of the 512-graph batch (64 problems), and 8 of the 32
    float32 R-MAT scale-18 sources with the tree gradient of their results."""
    import oracle
    out = {}
    graphs, sources = gg.workload_batch512()
    t_total, solves = 0.0, 0
    for gi in range(0, len(graphs), 8):
        ref = oracle.csr_of(graphs[gi])
        t0 = time.perf_counter()
        oracle.dijkstra(ref, int(sources[gi][0]))
        t_total += time.perf_counter() - t0
        solves += 1
    out["batch512_sample"] = {"solves_per_s": round(solves / t_total, 1), "cores": 1, "kind": "oracle",
                              "sample": f"{solves} problems (first source of every 8th graph), {t_total:.2f} s"}
    g0, srcs, gup = gg.workload_rmat18_f32()
    ref = oracle.csr_of(g0)
    t0 = time.perf_counter()
    runs = [oracle.dijkstra(ref, int(s)) for s in srcs[:8]]
    t1 = time.perf_counter()
    oracle.tree_grad(ref, np.stack([r[0] for r in runs]), np.stack([r[1] for r in runs]), gup[:8])
    t2 = time.perf_counter()
    out["rmat18_f32_sample"] = {"forward_ms_per_source": round((t1 - t0) * 1e3 / 8, 2),
                                "backward_ms_per_source": round((t2 - t1) * 1e3 / 8, 2), "cores": 1,
                                "kind": "oracle", "sample": "8 of the 32 sources: Dijkstra, then the tree gradient"}
    return out


def run_reference(a):
    """The CPU oracle on this workload, one source per step (rank 0 only)."""
    import oracle
    ws, rank, local = dist_env()
    if rank != 0:
        return
    g0, P = make_workload(a.scale)
    srcs = rank_sources(g0, 0)
    ref = oracle.csr_of(g0)
    deg = np.diff(ref.row_ptr.astype(np.int64))
    for k in range(a.warmup):
        oracle.dijkstra(ref, int(srcs[k % len(srcs)]))
    t_total, e_total = 0.0, 0
    for k in range(a.steps):
        s = int(srcs[k % len(srcs)])
        t0 = time.perf_counter()
        d, _, _ = oracle.dijkstra(ref, s)
        t_total += time.perf_counter() - t0
        e_total += int(deg[d != 0xFFFFFFFF].sum())
    v = e_total / t_total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(1e3 * t_total / a.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded R-MAT, weights U{1..255})",
        "config": {"workload": f"rmat-s{a.scale}-ef16 directed, {g0.V} vertices, {g0.E_raw} raw edges, "
                               f"1 source per step (of 8), {P} partitions", "partitions": P},
        "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one source's full single-threaded binary-heap Dijkstra per step",
                         "host_cores_available": os.cpu_count()},
        "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _evt():
    import torch
    return torch.cuda.Event(enable_timing=True)


def _time_ms(fn, reps):
    import torch
    a, b = _evt(), _evt()
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extras_batched(sssp, dev, rank=0, world=1):
    """512 graphs x 16 sources: one CUDA-graph replay of the batched kernel vs per-problem sssp_solve
    launches (one source each) and per-graph launches (16 sources each), same options.  With
    several ranks each solves the (graph, source) problems the library's planner gives it
    (split by estimated edges, no exchange); the times are reduced by the caller (MAX)."""
    import torch
    graphs0, sources = gg.workload_batch512()
    if world > 1:
        keep_g, sources = sssp.shard_batch(graphs0, sources, rank, world)
        graphs0 = [graphs0[i] for i in keep_g]
    # the per-solve baseline gets a partition count that spreads one graph over many blocks
    graphs = [sssp.build_csr(g.V, g.src, g.dst, g.w, partitions=max(1, min(148, g.V // 512))) for g in graphs0]
    del graphs0
    n_prob = sum(len(s) for s in sources)
    edges = sum(g.E for g in graphs)
    b = sssp.Batch(graphs, sources)
    tuned, _ = b.autotune()
    b.make_plan()
    b.replay()
    st, stats = b.status()
    assert st == sssp.SSSP_OK, sssp.status_string(st)
    ms_plan = _time_ms(b.replay, 3)
    # algorithmic bytes of the replay: per problem 8 per reached edge + 16 per reached vertex
    E_r = V_r = 0
    by_graph = {}
    for i in range(b.n_problems):
        by_graph.setdefault(int(b.prob_graph[i]), []).append(i)
    for gi, probs in by_graph.items():
        gd = graphs[gi]
        deg = (gd.row_ptr[1:].long() - gd.row_ptr[:-1].long())
        reached = torch.stack([b.result(i)[0] for i in probs]) != -1
        E_r += int((reached.long() * deg[None, :]).sum())
        V_r += int(reached.sum())
    alg = 8 * E_r + 16 * V_r
    peak, peak_kind = peaks()
    achieved = alg / (ms_plan * 1e-3) / 1e9
    # per-graph launches (16 sources in one sssp_solve each)
    solvers = [(sssp.Solver(g, len(s)), torch.from_numpy(s.view(np.int32)).to(dev)) for g, s in zip(graphs, sources)]
    ms_graph = _time_ms(lambda: [sv.launch(src) for sv, src in solvers], 1)
    # per-problem launches (one source per sssp_solve)
    one = [(sssp.Solver(g, 1), torch.from_numpy(s.view(np.int32)).to(dev)) for g, s in zip(graphs, sources)]

    def per_problem():
        for sv, src in one:
            for i in range(src.numel()):
                sv.launch(src[i:i + 1])
    ms_prob = _time_ms(per_problem, 1)
    return {"workload": "512 graphs (ER deg 8 / R-MAT ef 8, n = 2^U(10,17)), 16 sources each",
            "problems": n_prob, "edges_total": int(edges),
            "options": {"delta": tuned.delta, "tile": tuned.tile or 1024, "threads": tuned.threads or 512,
                        "autotuned": True},
            "graph_replay_ms": round(ms_plan, 3), "solves_per_s": round(n_prob / ms_plan * 1e3, 1),
            "reached_edges": E_r, "reached_vertices": V_r, "edges_scanned": stats["edges_scanned"],
            "work_inflation": round(stats["edges_scanned"] / max(E_r, 1), 3),
            "roofline": {"bound": "hbm", "kernel": "k_batched", "achieved": round(achieved, 1), "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "alg_bytes_per_launch": alg, "traffic": batched_traffic(stats["edges_scanned"])},
            "per_graph_launches_ms": round(ms_graph, 3), "per_problem_launches_ms": round(ms_prob, 3),
            "speedup_vs_per_problem": round(ms_prob / ms_plan, 3),
            "speedup_vs_per_graph": round(ms_graph / ms_plan, 3)}


def extras_differentiable(sssp, dev, rank=0, world=1):
    """R-MAT scale 18, fp32 weights, 32 sources: forward solve, backward, forward+backward.  With
    several ranks each takes its share of the sources (the planner deals them out) and dL/dw is
    summed over the ranks by one all-reduce, inside the backward's timing."""
    import torch
    g0, srcs, gup = gg.workload_rmat18_f32()
    if world > 1:
        idx = sssp.shard_sources(len(srcs), rank, world)
        srcs, gup = srcs[idx], gup[idx]
    # 16 partitions: 512 units for the 32 sources keep the persistent blocks busy
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=16)
    src_d = torch.from_numpy(srcs.view(np.int32)).to(dev)
    opts, _ = sssp.autotune(g, src_d, trials=2)
    solver = sssp.Solver(g, len(srcs), opts)
    gup_d = torch.from_numpy(gup).to(dev)
    solver.launch(src_d)
    st, _ = solver.status()
    assert st == sssp.SSSP_OK

    def bwd():
        return sssp.allreduce_sum(sssp.backward(g, solver.pred, gup_d))
    ms_fwd = _time_ms(lambda: solver.launch(src_d), 5)
    ms_bwd = _time_ms(bwd, 5)
    ms_both = _time_ms(lambda: (solver.launch(src_d), bwd()), 5)
    return {"workload": "rmat-s18-ef8 fp32 weights, 32 sources, 16 partitions",
            "sources_this_rank": int(len(srcs)),
            "options": {"delta": opts.delta, "tile": opts.tile, "split": opts.split, "autotuned": True},
            "forward_ms": round(ms_fwd, 3),
            "backward_ms": round(ms_bwd, 3), "forward_backward_ms": round(ms_both, 3),
            "fwd_bwd_over_fwd": round(ms_both / ms_fwd, 3)}


def tree_path_sums(pred, weight=None):
    """For every vertex, the sum of `weight` (default 1) over the tree edges on its path to the
    root, one row of predecessors at a time (pointer doubling on the device); weight[v] belongs
    to the edge (pred[v], v)."""
    import torch
    p = pred.long() & 0xFFFFFFFF
    none = p == 0xFFFFFFFF
    anc = torch.where(none, torch.arange(p.shape[-1], device=p.device).expand_as(p), p)
    dep = (~none).long() if weight is None else weight.long() * (~none).long()
    for _ in range(int(p.shape[-1]).bit_length()):
        dep = dep + torch.gather(dep, -1, anc) * (anc != torch.gather(anc, -1, anc)).long()
        anc = torch.gather(anc, -1, anc)
    return dep


def tree_depth(pred):
    """Edges on the longest tree path (the hops of the deepest shortest path) of each row."""
    return tree_path_sums(pred).max(dim=-1).values


def chain_ms_per_hop(sssp, dev, n=1 << 16, partitions=1, cross=False, reps=3):
    """ms per hop of a pure chain of n vertices (unit weights): every hop waits for the one before
    it.  cross=False: the chain runs through consecutive ids (inside one unit when partitions=1,
    a sub-round per hop); cross=True: consecutive chain vertices lie in different partitions, so
    every hop is a message to another unit."""
    import torch
    if cross:
        n -= n % partitions  # whole blocks: B = n / partitions, every node id below n
    i = np.arange(n, dtype=np.int64)
    if cross:
        B = n // partitions
        node = ((i % partitions) * B + i // partitions).astype(np.uint32)
    else:
        node = i.astype(np.uint32)
    g = sssp.build_csr(n, node[:-1], node[1:], np.ones(n - 1, np.uint32), partitions=partitions)
    solver = sssp.Solver(g, 1, sssp.options(delta=1e9))
    src = torch.full((1,), int(node[0]), dtype=torch.int32, device=dev)
    solver.launch(src)
    st, _ = solver.status()
    assert st == sssp.SSSP_OK
    return statistics.median(_time_ms(lambda: solver.launch(src), 1) for _ in range(reps)) / (n - 1)


def extras_grid(sssp, dev):
    """4096 x 4096 grid, corner source: the high-diameter case (autotuned schedule).  Latency model:
    the deepest shortest path has `depth` hops, each of which waits for the one before it, and
    `crossing` of them lead into another unit; pure chains give the time of a hop inside a unit
    (a sub-round) and across units (a message, its doorbell and the owner's round), so
    (depth - crossing) x t_in + crossing x t_cross is the floor of the grid's solve here."""
    import torch
    g0, srcs, P = gg.workload_grid4096()
    g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
    del g0
    src_d = torch.from_numpy(srcs.view(np.int32)).to(dev)
    opts, _ = sssp.autotune(g, src_d, trials=2)
    solver = sssp.Solver(g, 1, opts)
    solver.launch(src_d)
    st, stats = solver.status()
    assert st == sssp.SSSP_OK
    ms = _time_ms(lambda: solver.launch(src_d), 3)
    # the deepest path's hops, and how many of them cross from one unit to another
    V = g.V
    B = -(-V // g.partitions)
    split = opts.split or 1
    Bq = -(-B // split)
    v = torch.arange(V, device=dev)
    unit = (v // B) * split + (v % B) // Bq
    p = solver.pred[0].long() & 0xFFFFFFFF
    crosses = (p != 0xFFFFFFFF) & (unit[p.clamp(max=V - 1)] != unit)
    hops = tree_path_sums(solver.pred)[0]
    deep = int(torch.argmax(hops))
    depth = int(hops[deep])
    n_cross = int(tree_path_sums(solver.pred, crosses[None, :])[0][deep])
    hop_in = chain_ms_per_hop(sssp, dev, partitions=1)
    hop_cross = chain_ms_per_hop(sssp, dev, partitions=148, cross=True)
    floor = (depth - n_cross) * hop_in + n_cross * hop_cross
    model = {"depth_hops": depth, "crossing_hops": n_cross, "ms_per_hop": round(ms / depth, 6),
             "chain_ms_per_hop_in_unit": round(hop_in, 6), "chain_ms_per_hop_across_units": round(hop_cross, 6),
             "floor_ms": round(floor, 3), "measured_over_floor": round(ms / floor, 2)}
    return {"workload": "grid 4096x4096, corner source", "delta": opts.delta, "tile": opts.tile,
            "latency_model": model,
            "split": opts.split, "policy": sssp.POLICY_NAMES[opts.policy], "ms": round(ms, 3),
            "gteps": round(g.E / (ms * 1e-3) / 1e9, 4), "rounds": stats["rounds"],
            "work_inflation": round(stats["edges_scanned"] / g.E, 3),
            "policies": policy_table(sssp, g, src_d, opts, g.E),
            "message_buffering": message_table(sssp, g, src_d, opts, g.E)}


def extras_warm(sssp, dev):
    """R-MAT scale 22, 8 sources, locality layout: 0.1% of the weights halved; sssp_update from the
    previous result against a fresh solve of the changed graph (results must be equal)."""
    import torch
    g0, srcs, P = gg.workload_rmat22()
    g = sssp.layout(sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P))
    del g0
    src_d = torch.from_numpy(srcs.view(np.int32)).to(dev)
    opts, _ = sssp.autotune(g, src_d, trials=2)
    rng = np.random.default_rng(gg.BASE_SEED + 40)
    idx = torch.from_numpy(np.sort(rng.choice(g.E, g.E // 1000, replace=False)).astype(np.int64)).to(dev)
    w2 = g.w.clone()
    w2[idx] = torch.clamp(w2[idx] // 2, min=1)
    tails = g.ids.long()[torch.searchsorted(g.row_ptr.long(), idx, right=True) - 1].int()  # caller's ids
    g2 = sssp.DeviceGraph(g.V, g.E, g.row_ptr, g.col, w2, g.wtype, g.partitions, g.eid, g.ids, g.slots)
    s1, s2 = sssp.Solver(g, len(srcs), opts), sssp.Solver(g2, len(srcs), opts)
    s1.launch(src_d)
    d0, p0 = s1.dist.clone(), s1.pred.clone()
    s2.launch(src_d)
    st, fresh = s2.status()
    assert st == sssp.SSSP_OK
    fresh_ms = _time_ms(lambda: s2.launch(src_d), 3)
    d, p = d0.clone(), p0.clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(4):
        d.copy_(d0)
        p.copy_(p0)
        e0.record()
        s2.update(d, p, tails)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    st, warm = s2.status()
    assert st == sssp.SSSP_OK
    equal = bool(torch.equal(d, s2.dist) and torch.equal(p, s2.pred))
    upd_ms = statistics.median(times[1:])
    return {"workload": "rmat-s22-ef16, 8 sources, layout; 0.1% of the weights halved", "changed_edges": int(idx.numel()),
            "fresh_solve_ms": round(fresh_ms, 3), "update_ms": round(upd_ms, 3),
            "speedup": round(fresh_ms / upd_ms, 2), "update_edges_scanned": warm["edges_scanned"],
            "fresh_edges_scanned": fresh["edges_scanned"], "equal_to_fresh": equal}


_SHARDED_KEYS = {"batched": ["graph_replay_ms", "per_graph_launches_ms", "per_problem_launches_ms", "problems",
                               "edges_total"],
                 "differentiable": ["forward_ms", "backward_ms", "forward_backward_ms", "sources_this_rank"]}


def _reduce_sharded(name, d, world, dev):
    """Across ranks: times (keys ending in _ms) by MAX, problem counts by SUM; rates recomputed.
    Every rank reduces the same keys (NaN where its extra failed), so the collectives match."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return d
    keys = _SHARDED_KEYS[name]
    t = torch.tensor([float(d.get(k, float("nan"))) for k in keys], dtype=torch.float64, device=dev)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    out = dict(d)
    if any(np.isnan(sm.tolist())) or "error" in d:  # a NaN from any rank survives the SUM
        out["error"] = out.get("error", "an extra failed on another rank")
        return out
    for i, k in enumerate(keys):
        out[k] = round(float(mx[i] if k.endswith("_ms") else sm[i]), 3)
    if "graph_replay_ms" in out:
        out["solves_per_s"] = round(out["problems"] / out["graph_replay_ms"] * 1e3, 1)
        out["speedup_vs_per_problem"] = round(out["per_problem_launches_ms"] / out["graph_replay_ms"], 3)
        out["speedup_vs_per_graph"] = round(out["per_graph_launches_ms"] / out["graph_replay_ms"], 3)
    if "forward_ms" in out:
        out["fwd_bwd_over_fwd"] = round(out["forward_backward_ms"] / out["forward_ms"], 3)
    out["ranks"] = world
    out["sharding"] = "problems split by estimated edges (sssp_shard_problems), no exchange" if \
        "graph_replay_ms" in out else "sources dealt out over the ranks; dL/dw summed by one all-reduce"
    return out


def extras_prune_overlap(sssp, dev):
    """Trishla on the solve's idle time (sssp_solve_prune) against a solve followed by a separate
    prune (sssp_solve + sssp_prune), local mode, on the 16K ER workload, R-MAT scale 22 (8
    sources, locality layout) and the 4096 x 4096 grid (no triangles: nothing to prune, but the
    blocks are idle most of the solve).  Same options for both; CUDA events, median of 3."""
    import torch

    def med(fn, reps=3):
        return statistics.median(_time_ms(fn, 1) for _ in range(reps))

    out = {}
    cases = (("er16k", lambda: gg.workload_er16k(), False), ("rmat22", lambda: gg.workload_rmat22(), True),
             ("grid4096", lambda: gg.workload_grid4096(), False))
    for name, make, lay in cases:
        g0, srcs, P = make()
        g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=P)
        del g0
        if lay:
            g = sssp.layout(g)
        src_d = torch.from_numpy(np.asarray(srcs, np.uint32).view(np.int32)).to(dev)
        opts, _ = sssp.autotune(g, src_d, trials=2)
        solver = sssp.Solver(g, len(srcs), opts)
        keep = torch.empty(max(g.E, 1), dtype=torch.uint8, device=dev)
        solver.launch_prune(src_d, 0, keep)
        st, _ = solver.status()
        assert st == sssp.SSSP_OK
        k_sep, _ = sssp.prune(g, 0, witness=False)
        assert torch.equal(k_sep, keep[:g.E])
        t_solve = med(lambda: solver.launch(src_d))
        t_prune = med(lambda: sssp.prune(g, 0, witness=False))
        t_both = med(lambda: solver.launch_prune(src_d, 0, keep))
        out[name] = {"solve_ms": round(t_solve, 3), "prune_ms": round(t_prune, 3),
                     "solve_then_prune_ms": round(t_solve + t_prune, 3), "solve_prune_ms": round(t_both, 3),
                     "hidden_ms": round(t_solve + t_prune - t_both, 3), "pruned_edges": int((k_sep == 0).sum()),
                     "edges": g.E}
        del solver, keep, k_sep, g
        torch.cuda.empty_cache()
    return out


def extras(sssp, dev, rank=0, world=1, only=()):
    """The other workloads.  batched and differentiable run on every rank, sharded, and are reduced
    over the ranks; grid and warm_start (one graph, one solve) run on rank 0 only."""
    import torch.distributed as dist
    out = {}
    for name, fn, sharded in (("batched", extras_batched, True), ("differentiable", extras_differentiable, True),
                              ("grid", extras_grid, False), ("warm_start", extras_warm, False),
                              ("prune_overlap", extras_prune_overlap, False)):
        if (not sharded and rank != 0) or (only and name not in only):
            continue
        t0 = time.perf_counter()
        try:
            out[name] = fn(sssp, dev, rank, world) if sharded else fn(sssp, dev)
        except Exception as e:  # an extra must not hide the headline line
            out[name] = {"error": repr(e)[:300]}
        if sharded:
            out[name] = _reduce_sharded(name, out[name], world, dev)
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    if world > 1:
        dist.barrier()
    return out


def profile_case(which):
    """Small cases of the other kernels for ncu: batched (64 graphs x 16 sources), backward (R-MAT scale 18
    fp32, 32 sources), Trishla prune (R-MAT scale 16, local mode), and the solve on a 2048 x 2048 grid
    from a corner (the high-diameter case, with the full grid's tuned schedule)."""
    import torch

    import paper_2103_12012_gb300 as sssp
    if which == "all":
        # every kernel of the library once (CSR build, partition, layout, Trishla, compact, solve with
        # its init and unpack, warm start, solve with prune on idle time, batched, backward) on
        # R-MAT scale 21 (CSR 0.5 GB, larger than L2), 8 sources
        g0 = gg.rmat(gg.BASE_SEED + 21, 21, 16 << 21)
        srcs = gg.pick_sources(gg.BASE_SEED + 21, g0, 8)
        g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=148)
        del g0
        sssp.partition(g)
        h = sssp.layout(g)
        keep, _ = sssp.prune(g, 0)
        gp = sssp.compact(g, keep)
        src_d = torch.from_numpy(srcs.view(np.int32)).cuda()
        opts = sssp.options(delta=5)
        s1 = sssp.Solver(h, len(srcs), opts)
        s1.launch(src_d)
        d0, p0 = s1.dist.clone(), s1.pred.clone()
        w2 = h.w.clone()
        w2[::1000] = torch.clamp(w2[::1000] // 2, min=1)
        h2 = sssp.DeviceGraph(h.V, h.E, h.row_ptr, h.col, w2, h.wtype, h.partitions, h.eid, h.ids, h.slots)
        tails = h.ids.long()[torch.searchsorted(h.row_ptr.long(), torch.arange(0, h.E, 1000, device="cuda"),
                                                right=True) - 1].int()
        s2 = sssp.Solver(h2, len(srcs), opts)
        s2.update(d0, p0, tails)
        s3 = sssp.Solver(gp, len(srcs), opts)
        kp = torch.empty(max(gp.E, 1), dtype=torch.uint8, device="cuda")
        s3.launch_prune(src_d, 0, kp)
        for s_ in (s1, s2, s3):
            st, _ = s_.status()
            assert st == sssp.SSSP_OK, st
        graphs0, sources = gg.workload_batch512(n_graphs=64)
        b = sssp.Batch([sssp.build_csr(x.V, x.src, x.dst, x.w) for x in graphs0], sources, sssp.options(delta=8))
        b.solve()
        st, _ = b.status()
        assert st == sssp.SSSP_OK, st
        gf0, fsrcs, gup = gg.workload_rmat18_f32()
        gf = sssp.build_csr(gf0.V, gf0.src, gf0.dst, gf0.w, partitions=16)
        _, fpred, st, _ = sssp.solve(gf, fsrcs)
        gr = sssp.backward(gf, fpred, torch.from_numpy(gup).cuda())
        torch.cuda.synchronize()
        print("all", g.E, h.E, gp.E, float(gr.abs().sum()))
    elif which == "batched-full":
        # the full 512-graph, 16-source batch at the schedule the bench's tuner picks (1024-thread
        # blocks, tile 2048, delta 16)
        graphs0, sources = gg.workload_batch512()
        graphs = [sssp.build_csr(x.V, x.src, x.dst, x.w) for x in graphs0]
        del graphs0
        b = sssp.Batch(graphs, sources, sssp.options(threads=1024, tile=2048, delta=16))
        for _ in range(2):
            b.solve()
        st, stats = b.status()
        assert st == sssp.SSSP_OK, st
        print("batched-full", b.n_problems, stats)
    elif which == "batched":
        graphs0, sources = gg.workload_batch512(n_graphs=64)
        graphs = [sssp.build_csr(g.V, g.src, g.dst, g.w) for g in graphs0]
        b = sssp.Batch(graphs, sources)
        for _ in range(3):
            b.solve()
        st, stats = b.status()
        assert st == sssp.SSSP_OK, st
        print("batched", b.n_problems, stats)
    elif which == "backward":
        g0, srcs, gup = gg.workload_rmat18_f32()
        g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=8)
        _, pred, st, _ = sssp.solve(g, srcs)
        gd = torch.from_numpy(gup).cuda()
        for _ in range(3):
            gr = sssp.backward(g, pred, gd)
        torch.cuda.synchronize()
        print("backward", float(gr.abs().sum()))
    elif which == "grid":
        g0 = gg.grid(gg.BASE_SEED + 3, 2048, 2048, 1, 1000)
        g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=148)
        solver = sssp.Solver(g, 1, sssp.options(delta=2982, tile=2048, split=4))
        src = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(3):
            solver.launch(src)
        st, stats = solver.status()
        assert st == sssp.SSSP_OK, st
        print("grid", g.E, stats)
    else:
        g0 = gg.rmat(gg.BASE_SEED + 16, 16, 16 << 16)
        g = sssp.build_csr(g0.V, g0.src, g0.dst, g0.w, partitions=16)
        for _ in range(3):
            keep, _ = sssp.prune(g, 0)
        torch.cuda.synchronize()
        print("prune", int((keep == 0).sum()), "of", g.E)


if __name__ == "__main__":
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
