"""Benchmark of the algebraic-distance sparsification hot path on one GB300.

Workload (a "step"): R-MAT scale 20 (1,048,576 vertices, edge factor 16,
a/b/c/d = 0.57/0.19/0.19/0.05, symmetrised, no self loops or duplicates, unit
weights), R = 32 Philox test vectors, k = 20 JOR sweeps at omega = 0.5 with a
rescale after every sweep, the per-edge distance, then Alg. 2 sparsification
to 30% of the edges per node in local and in global mode.  Inputs are
resident in device memory when the timed region starts.

Metric: edge-vector updates per second = nnz * R * k / step time (nnz counts
both CSR directions).  Also reported: the end-to-end figure through the C ABI
with host buffers (graph upload and result download inside the timed region),
the HBM roofline fraction of the dominant kernel (one JOR sweep), the same step
with BF16 and FP16 storage of the test vectors (FP32 accumulation) and their
accuracy against the FP32 path, and the FP64 oracle timed on the host cores on
a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--storage fp32|bf16|fp16|q16]
    python bench.py --impl reference      # the FP64 CPU oracle, same metric
    python bench.py --scale 18 ...        # a smaller graph for profiler captures
    python bench.py --workload ws512|ba2m|rmat22   # batched, multilevel, reverse-mode paths
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "JOR+distance edge-vector updates/s (nnz*R*k/s) & % HBM roofline vs FP32 plain"
UNIT = "edge-vector updates/s"
R, K_SWEEPS, OMEGA, SEED, FRACTION = 32, 20, 0.5, 0x1601055270000000, 0.30
SCALE, EDGE_FACTOR, GRAPH_SEED = 20, 16, 2


def workload():
    return (f"R-MAT scale {SCALE} (2^{SCALE} vertices, edge factor {EDGE_FACTOR}, a=0.57 b=0.19 c=0.19 d=0.05, "
            f"symmetrised, dedup, unit weights), R={R}, k={K_SWEEPS}, omega={OMEGA}, per-sweep rescale, "
            f"L2 distance, per-node sparsification to {int(FRACTION * 100)}% local and global")


def sweep_source_digest() -> str:
    h = hashlib.sha256()
    for f in ("sweep_kernels.cuh", "ad_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1601_05527_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sweep_traffic(storage):
    """DRAM bytes per sweep launch from the committed ncu summary, if the
    sweep kernel source is unchanged since it was captured."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(storage)
    if not e or e.get("sweep_cu_sha256_16") != sweep_source_digest():
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 7:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                except ValueError:
                    pass
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_graph():
    from paper_1601_05527_gb300 import graphgen
    return graphgen.rmat(SCALE, EDGE_FACTOR, seed=GRAPH_SEED)


def algorithmic_bytes_per_sweep(g, storage):
    """Compulsory traffic of one sweep (gathers assumed served on chip): column
    indices, row pointers, inverse degrees, and one read + one write of every
    active row of the R-wide vector block."""
    s = 4 if storage == "fp32" else 2
    n_active = int((g.degrees() > 0).sum())
    return g.nnz * 4 + (g.n + 1) * 4 + g.n * 4 + 2 * n_active * R * s, n_active


def cpu_baseline(g):
    """The FP64 oracle as it stands on a bounded sample of the workload (the full
    graph, R = 32, k sweeps), on one host core and with its row loops on all host
    cores (OpenMP over rows, the per-row arithmetic unchanged), seconds per phase."""
    import oracle
    cores = os.cpu_count() or 1
    out = {}
    for label, threads, k in (("one_core", 1, 1), ("all_cores", cores, 4)):
        oracle.set_threads(threads)
        t0 = time.perf_counter()
        oracle.algebraic_distance(g.row_ptr, g.col, None, R=R, k=k, omega=OMEGA, seed=SEED)
        dt = time.perf_counter() - t0
        out[label] = {"value": g.nnz * R * k / dt, "threads": oracle.max_threads(), "k": k, "seconds": dt,
                      "phase_seconds": oracle.last_phase_seconds()}
    oracle.set_threads(cores)
    best = out["all_cores"]
    return {"value": best["value"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
            "sample": f"same R-MAT scale-{SCALE} graph, R={R}, FP64; one core: k=1 sweep "
                      f"({out['one_core']['seconds']:.1f} s); all cores: k=4 sweeps ({best['seconds']:.1f} s), "
                      "each + init and distance",
            "runs": out}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    g = make_graph()
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    k = 1
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.algebraic_distance(g.row_ptr, g.col, None, R=R, k=k, omega=OMEGA, seed=SEED)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = args.steps * g.nnz * R * k / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(), "sample": f"each step: FP64 oracle, R={R}, k={k} sweep on the full graph",
                       "n": g.n, "m": g.m, "nnz": g.nnz},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"R={R}, k={k} sweep (+ init and distance) on the full graph per step, "
                                       "row loops on all host cores"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1601_05527_gb300 import build, _lib as L
    build.build()
    L.load()
    L.use_torch_allocator()
    g = make_graph()
    dev = torch.device("cuda", local)
    # a stream of our own: the library can record a repeated call as a CUDA graph on it
    # (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    h = L.ad_graph_create(g.n, rp_d, col_d, None, 0, stream)
    keep_d = torch.empty(g.m, dtype=torch.uint8, device=dev)
    keep2_d = torch.empty(g.m, dtype=torch.uint8, device=dev)
    storage = args.storage
    # launch shape of the sweep chosen by the library's autotuner (setup, not timed)
    lpr, cpl, per_sm = L.ad_graph_autotune(h, R, storage)
    shape = {"lanes_per_row": lpr, "chunks_per_lane": cpl, "ctas_per_sm": per_sm or "max", "chosen_by": "ad_graph_autotune"}

    def step(handle, keep):
        L.ad_algebraic_distance(handle, R, K_SWEEPS, OMEGA, SEED, 0, storage, 0, None)
        (kl, kg), _ = L.ad_sparsify_local_global(handle, FRACTION, keep, keep2_d)
        return kl, kg

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    from paper_1601_05527_gb300 import replicas

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, dev)

    for _ in range(args.warmup):
        step(h, keep_d)
    clocks = Clocks()
    clocks.start()
    barrier()
    launches0 = L.ad_kernel_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")     # lets a profiler pick out the timed launches
    ev0.record(stream)
    kept = None
    for _ in range(args.steps):
        kept = step(h, keep_d)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = L.ad_kernel_launch_count() - launches0
    clk = clocks.stop()
    units = g.nnz * R * K_SWEEPS
    ms_local = ev0.elapsed_time(ev1)
    value = replicas.whole_job_rate(args.steps * units, ms_local / 1e3, dev)   # all ranks' units / slowest rank
    ms = max_over_ranks(ms_local)

    # the same step with 16-bit storage of the test vectors (FP32 accumulation), and its
    # accuracy against the FP32 path (itself within 1e-5 of the FP64 oracle)
    variants = {}
    if args.variants:
        rho32 = torch.empty(g.m, dtype=torch.float32, device=dev)
        L.ad_algebraic_distance(h, R, K_SWEEPS, OMEGA, SEED, 0, storage, 0, rho32)
        L.ad_sparsify(h, FRACTION, "local", "per_node", keep_d)
        keep32 = keep_d.clone()
        for st in ("bf16", "fp16"):
            if st == storage:
                continue

            def vstep(handle, keep, st=st):
                L.ad_algebraic_distance(handle, R, K_SWEEPS, OMEGA, SEED, 0, st, 0, None)
                L.ad_sparsify_local_global(handle, FRACTION, keep, keep2_d)
            for _ in range(args.warmup):
                vstep(h, keep_d)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                vstep(h, keep_d)
            e1.record(stream)
            barrier()
            vms = max_over_ranks(e0.elapsed_time(e1))
            rv = torch.empty(g.m, dtype=torch.float32, device=dev)
            L.ad_algebraic_distance(h, R, K_SWEEPS, OMEGA, SEED, 0, st, 0, rv)
            L.ad_sparsify(h, FRACTION, "local", "per_node", keep_d)
            d = (rv.double() - rho32.double())
            inter = int((keep_d.bool() & keep32.bool()).sum())
            union = int((keep_d.bool() | keep32.bool()).sum())
            variants[st] = {"value": ws * args.steps * g.nnz * R * K_SWEEPS / (vms / 1e3), "unit": UNIT,
                            "ms_per_step": vms / args.steps,
                            "rho_rms_rel_err_vs_fp32": float(d.pow(2).mean().sqrt() / rho32.double().pow(2).mean().sqrt()),
                            "rho_max_err_over_rms_vs_fp32": float(d.abs().max() / rho32.double().pow(2).mean().sqrt()),
                            "jaccard_local_30pct_vs_fp32": inter / max(union, 1)}
        del rho32, keep32

    # SparsifyB (Alg. 3) on the same distances, timed on its own (not part of the step)
    binned = None
    if args.variants:
        L.ad_algebraic_distance(h, R, K_SWEEPS, OMEGA, SEED, 0, storage, 0, None)
        for _ in range(2):
            L.ad_sparsify_binned(h, None, FRACTION, SEED, keep_d)
        barrier()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nb = 3
        torch.cuda.nvtx.range_push("binned")
        b0.record(stream)
        for _ in range(nb):
            kb, eb = L.ad_sparsify_binned(h, None, FRACTION, SEED, keep_d)
        b1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        binned = {"ms": b0.elapsed_time(b1) / nb, "kept": kb, "e": eb,
                  "what": f"SparsifyB to {int(FRACTION * 100)}% per node on the step's distances (bins, round robin, "
                          "fit of e), timed on its own"}

    # phase split and the dominant kernel's launch time (events on the handle's stream)
    L.ad_graph_set_profiling(h, True)
    for ph in ("init", "sweep", "distance", "select"):
        L.ad_graph_phase_time(h, ph, reset=True)
    prof_steps = 2
    for _ in range(prof_steps):
        step(h, keep_d)
    phase = {ph: L.ad_graph_phase_time(h, ph) for ph in ("init", "sweep", "distance", "select")}
    L.ad_graph_set_profiling(h, False)
    sweep_ms = phase["sweep"][0] / max(phase["sweep"][1], 1)
    b_sweep, n_active = algorithmic_bytes_per_sweep(g, storage)
    peak, peak_kind = measured_peaks()
    achieved = b_sweep / (sweep_ms / 1e3) / 1e9
    jd_ms = (phase["init"][0] + phase["sweep"][0] + phase["distance"][0]) / prof_steps

    # end to end through the C ABI with host buffers (pinned), upload and download timed
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    keep_h = torch.empty(g.m, dtype=torch.uint8).pin_memory()
    keep2_h = torch.empty(g.m, dtype=torch.uint8).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        he = L.ad_graph_create(g.n, rp_h, col_h, None, 0, stream)
        L.ad_algebraic_distance(he, R, K_SWEEPS, OMEGA, SEED, 0, storage, 0, None)
        L.ad_sparsify_local_global(he, FRACTION, keep_h, keep2_h)
        L.ad_graph_destroy(he)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = ws * e2e_steps * units / e2e_s
    h2d = rp_h.numel() * 8 + col_h.numel() * 4
    d2h = 2 * g.m

    L.ad_graph_destroy(h)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if storage == "fp32" else f"{storage} storage, f32 accumulate",
                "data": "synthetic",
                "config": {"workload": workload(), "n": g.n, "n_active": n_active, "m": g.m, "nnz": g.nnz,
                           "R": R, "k": K_SWEEPS, "storage": storage, "graph_digest": g.digest(),
                           "parallelism": "replicas" if ws > 1 else "single GPU", "sweep_shape": shape,
                           "l2": "no flush: per-sweep traffic (column indices 126 MB + vector block) exceeds the 129 MB L2"},
                "phases_ms_per_step": {"init": phase["init"][0] / prof_steps, "sweeps": phase["sweep"][0] / prof_steps,
                                       "distance": phase["distance"][0] / prof_steps,
                                       "select_local_and_global": phase["select"][0] / prof_steps},
                "jor_distance_only": {"value": units / (jd_ms / 1e3), "unit": UNIT, "ms": jd_ms},
                "sparsify_kept": {"local": kept[0] if kept else None, "global": kept[1] if kept else None},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": e2e_steps},
                "roofline": {"kernel": "k_sweep (one JOR sweep + fused rescale min/max)", "bound": "hbm",
                             "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "peak_kind": peak_kind, "algorithmic_bytes_per_launch": b_sweep,
                             "avg_launch_ms": sweep_ms, "traffic": sweep_traffic(storage),
                             # not roofline terms: every CSR entry gathers one R-wide neighbour row, which
                             # the L1/L2 serve; this is the rate the sweep sustains on those gathers
                             "gathered_bytes_per_launch": g.nnz * R * (4 if storage == "fp32" else 2),
                             "gather_rate_gbs": g.nnz * R * (4 if storage == "fp32" else 2) / (sweep_ms / 1e3) / 1e9},
                "gpu_launches": int(launches),
                "storage_variants": variants or None,
                "sparsify_binned": binned,
                "clocks": clk}
        if ws == 1 and args.workloads:
            line["workloads"] = {}
            for name, fn in WORKLOADS.items():
                kw = {} if name in ("grid64", "rmat22") else {"storage": "bf16" if name == "ws512" else "fp32"}
                line["workloads"][name] = fn(L, dev, stream, min(args.steps, 3), max(args.warmup, 3), **kw)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _timed(stream, fn, steps, warmup, mark=True):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if mark:
        torch.cuda.nvtx.range_push("timed_steps")     # lets a profiler pick out the timed launches
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    if mark:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _sweep_ms(L, h, fn, runs=2):
    """Average event time of one JOR sweep launch of handle h over `runs` calls of fn."""
    L.ad_graph_set_profiling(h, True)
    L.ad_graph_phase_time(h, "sweep", reset=True)
    for _ in range(runs):
        fn()
    ms, cnt = L.ad_graph_phase_time(h, "sweep", reset=True)
    L.ad_graph_set_profiling(h, False)
    return ms / max(cnt, 1)


def _roofline(b_sweep, sweep_ms, what):
    peak, kind = measured_peaks()
    ach = b_sweep / (sweep_ms / 1e3) / 1e9
    return {"kernel": what, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": kind, "algorithmic_bytes_per_launch": b_sweep, "avg_launch_ms": sweep_ms}


def sweep_bytes(n, nnz, n_active, R_, s, weighted):
    """Algorithmic bytes of one sweep (gathers assumed on chip): column indices,
    row pointers, inverse degrees, weights if any, one read + one write of
    every active row of the R-wide block."""
    return nnz * 4 + (n + 1) * 4 + n * 4 + (nnz * 4 if weighted else 0) + 2 * n_active * R_ * s


def workload_grid64(L, dev, stream, steps, warmup):
    """2-D 64x64 grid, unit weights, R = 8, k = 20, 50% by global whole-graph ranking:
    a latency-bound case, reported in microseconds per call."""
    import torch
    from paper_1601_05527_gb300 import graphgen
    g = graphgen.grid2d(64, 64)
    h = L.ad_graph_create(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev), None, 0, stream)
    keep = torch.empty(g.m, dtype=torch.uint8, device=dev)

    def ad():
        L.ad_algebraic_distance(h, 8, 20, OMEGA, SEED, 0, "fp32", 0, None)

    def step():
        ad()
        L.ad_sparsify(h, 0.5, "global", "whole_graph", keep)
    reps = max(20, steps * 10)
    ms_ad = _timed(stream, ad, reps, max(warmup, 3), mark=False)
    ms = _timed(stream, step, reps, max(warmup, 3), mark=False)
    L.ad_graph_destroy(h)
    units = g.nnz * 8 * 20
    return {"workload": "2-D grid 64x64 (4,096 vertices, 8,064 edges), unit weights, R=8, k=20, omega=0.5, "
                        "50% by global whole-graph ranking",
            "distance_us": 1e3 * ms_ad, "step_us": 1e3 * ms, "value": units / (ms / 1e3), "unit": UNIT,
            "note": "latency-bound: microseconds per call, repeated calls replay a recorded CUDA graph"}


def workload_ws512(L, dev, stream, steps, warmup, storage="bf16", graphs_in_batch=512):
    """512 Watts-Strogatz graphs in one batched handle, R = 16, k = 15, 16-bit storage,
    per-graph 25% global per-node sparsification; against the plain FP32 form with
    one handle per graph.  graphs_in_batch < 512 takes the first graphs of the same
    batch (a smaller case of the same kernels, e.g. for a profiler)."""
    import torch
    from paper_1601_05527_gb300 import graphgen
    st = storage if storage != "fp32" else "bf16"
    graphs = graphgen.ws_batch(512, seed=5)[:graphs_in_batch]
    voff, big = graphgen.concat(graphs)
    h = L.ad_graph_create_batched(voff, big.n, torch.from_numpy(big.row_ptr).to(dev),
                                  torch.from_numpy(big.col).to(dev), None, 0, stream)
    keep = torch.empty(big.m, dtype=torch.uint8, device=dev)

    def ad():
        L.ad_algebraic_distance(h, 16, 15, OMEGA, SEED, 0, st, 0, None)

    def step():
        ad()
        L.ad_sparsify(h, 0.25, "global", "per_node", keep)
    ms = _timed(stream, step, steps, warmup)
    sw = _sweep_ms(L, h, ad)
    L.ad_graph_destroy(h)
    hs = [L.ad_graph_create(gg.n, torch.from_numpy(gg.row_ptr).to(dev), torch.from_numpy(gg.col).to(dev), None,
                            0, stream) for gg in graphs]
    keeps = [torch.empty(gg.m, dtype=torch.uint8, device=dev) for gg in graphs]

    def plain():
        for hh, kk in zip(hs, keeps):
            L.ad_algebraic_distance(hh, 16, 15, OMEGA, SEED, 0, "fp32", 0, None)
            L.ad_sparsify(hh, 0.25, "global", "per_node", kk)
    ms_plain = _timed(stream, plain, 1, 1, mark=False)
    for hh in hs:
        L.ad_graph_destroy(hh)
    units = big.nnz * 16 * 15
    return {"workload": f"{len(graphs)} Watts-Strogatz graphs, n ~ U{{1000..200000}}, ring degree 10, p=0.1, R=16, "
                        "k=15, per-graph 25% global per-node sparsification, one batched handle",
            "n": big.n, "m": big.m, "nnz": big.nnz, "storage": st, "value": units / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms,
            "roofline": _roofline(sweep_bytes(big.n, big.nnz, big.n, 16, 2, False), sw,
                                  "k_sweep (one JOR sweep of the whole batch)"),
            "plain_fp32_one_handle_per_graph": {"value": units / (ms_plain / 1e3), "ms_per_step": ms_plain}}


def workload_ba2m(L, dev, stream, steps, warmup, storage="fp32"):
    """Multilevel Alg. 6 on Barabasi-Albert n = 2,000,000, m = 8, lognormal weights,
    R = 16, k = 20, hierarchy to about 1,000 vertices, 40% controlled at the coarse
    third of the levels, through the one-shot call."""
    import torch
    from paper_1601_05527_gb300 import graphgen
    g = graphgen.barabasi_albert(2_000_000, 8, seed=4)
    g = graphgen.with_edge_weights(g, graphgen.lognormal_edge_weights(g.m, seed=4))
    h = L.ad_graph_create(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                          torch.from_numpy(g.weight).to(dev), 0, stream)
    keep = torch.empty(g.m, dtype=torch.uint8, device=dev)
    params = dict(R=16, k=20, omega=OMEGA, seed=SEED, Q=0.5, coarsest_n=1000, mode="local", storage=storage)
    ml = L.ad_ml_build(h, **params)
    lv = L.ad_ml_levels(ml)
    sizes = [L.ad_ml_level_size(ml, l) for l in range(lv)]
    L.ad_ml_destroy(ml)
    ratios = L.ad_ml_segment_ratios(lv, "coarse", max(1, lv // 3), 1.0)[:max(1, lv // 3)]

    def step():
        L.ad_multilevel(h, ratios, 0.4, keep, **params)
    ms = _timed(stream, step, steps, warmup)
    kept = int(keep.sum())
    sw = _sweep_ms(L, h, lambda: L.ad_algebraic_distance(h, 16, 20, OMEGA, SEED, 0, storage, 0, None))
    L.ad_graph_destroy(h)
    units = sum(2 * m_l for _, m_l in sizes) * 16 * 20    # the sweeps of the downward pass
    return {"workload": "multilevel Alg. 6: Barabasi-Albert n=2,000,000 m=8, lognormal(0,1) weights, R=16, k=20, "
                        "Q=0.5, coarsest 1000, 40% controlled at the coarse third of levels (ad_multilevel)",
            "levels": [list(x) for x in sizes], "kept": kept, "value": units / (ms / 1e3), "unit": UNIT,
            "units": "sum over levels of nnz_l*R*k of the downward pass", "ms_per_step": ms,
            "roofline": _roofline(sweep_bytes(g.n, g.nnz, int((g.degrees() > 0).sum()), 16,
                                              4 if storage == "fp32" else 2, True), sw,
                                  "k_sweep (one JOR sweep of the finest level)")}


def workload_rmat22(L, dev, stream, steps, warmup):
    """Reverse mode: R-MAT scale 22 with uniform(0.5, 2) weights, R = 32, k = 30, loss
    over a seeded 1% edge subset, forward keeping its iterates + backward."""
    import torch
    from paper_1601_05527_gb300 import graphgen
    g = graphgen.rmat(22, 16, seed=6)
    ew = graphgen.uniform_edge_weights(g.m, seed=6)
    g = graphgen.with_edge_weights(g, ew)
    S = torch.from_numpy(graphgen.random_edge_subset(g.m, 0.01, seed=6)).to(dev)
    h = L.ad_graph_create(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                          torch.from_numpy(g.weight).to(dev), 0, stream)
    rho = torch.empty(g.m, dtype=torch.float32, device=dev)
    rb = torch.zeros(g.m, dtype=torch.float32, device=dev)
    wb = torch.empty(g.m, dtype=torch.float32, device=dev)

    def fwd():
        L.ad_algebraic_distance(h, 32, 30, OMEGA, SEED, 0, "fp32", L.AD_DIST_KEEP_STATE, rho)

    def step():
        fwd()
        rb.index_copy_(0, S, 2.0 * rho.index_select(0, S))
        L.ad_algebraic_distance_backward(h, rb, wb)
    ms_fwd = _timed(stream, fwd, steps, warmup, mark=False)
    ms = _timed(stream, step, steps, warmup)
    sw = _sweep_ms(L, h, lambda: L.ad_algebraic_distance(h, 32, 30, OMEGA, SEED, 0, "fp32", 0, None))
    L.ad_graph_destroy(h)
    units = g.nnz * 32 * 30
    return {"workload": "reverse mode: R-MAT scale 22, uniform(0.5,2) weights, R=32, k=30, "
                        "loss = sum of rho^2 over a seeded 1% edge subset, every iterate kept (16.6 GB)",
            "n": g.n, "m": g.m, "nnz": g.nnz, "value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "forward_with_checkpoints_ms": ms_fwd, "backward_ms": ms - ms_fwd,
            "roofline": _roofline(sweep_bytes(g.n, g.nnz, int((g.degrees() > 0).sum()), 32, 4, True), sw,
                                  "k_sweep (one forward JOR sweep)")}


WORKLOADS = {"grid64": workload_grid64, "ws512": workload_ws512, "ba2m": workload_ba2m, "rmat22": workload_rmat22}


def run_workload(args):
    """One of the other workloads of the hot path on its own, one JSON line."""
    import torch
    from paper_1601_05527_gb300 import build, _lib as L
    build.build()
    L.load()
    L.use_torch_allocator()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    fn = WORKLOADS[args.workload]
    kw = {} if args.workload in ("grid64", "rmat22") else {"storage": args.storage}
    if args.workload == "ws512":
        kw["graphs_in_batch"] = args.batch_graphs
    res = fn(L, dev, stream, args.steps, args.warmup, **kw)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "value": res.pop("value"), "config": {"workload": res.pop("workload")}, **res}
    print(json.dumps(line), flush=True)
    return 0


def main():
    global SCALE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16", "q16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-graphs", type=int, default=512,
                    help="ws512 workload: run the first N graphs of the 512-graph batch (a smaller profiling case)")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the 16-bit storage comparison")
    ap.add_argument("--workload", default="rmat20", choices=["rmat20", "grid64", "ws512", "ba2m", "rmat22"],
                    help="rmat20 is the benchmark; the others time the latency-bound, batched, multilevel and "
                         "reverse-mode paths (the default line carries them too)")
    ap.add_argument("--no-workloads", dest="workloads", action="store_false",
                    help="leave the other workloads out of the default line")
    ap.add_argument("--scale", type=int, default=SCALE,
                    help="R-MAT scale; values other than 20 are smaller profiling cases, not the benchmark")
    args = ap.parse_args()
    SCALE = args.scale
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args) if args.workload == "rmat20" else run_workload(args)


if __name__ == "__main__":
    sys.exit(main())
