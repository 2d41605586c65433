#!/usr/bin/env python3
"""Benchmark of the edge-partitioned flux kernel on one GB300.

Workload: the 1M-node mesh (1,048,576 points uniform in the unit cube, seed
0, symmetrised k=4 nearest-neighbour graph, ~2.57M tasks in shuffled order),
state x: 5 x fp32 N(0,1), weights w ~ U(0.5, 1.5), explicit steps
x <- x + 1e-3 * flux(x).  One bench step is one explicit step (edge kernel
plus shared-vertex update) on the whole mesh, with L2 flushed (a write and
then a read of scratch buffers twice the L2 size) before every timed step and
outside its events.

Reported (one JSON line on rank 0):
  value        forward edge updates/s, partitioned schedule (C = --C)
  default      the same kernel under the default order (C consecutive tasks)
  fwd_bwd      10 steps forward + backward (checkpoint every 5, recompute
               included) through the autograd function, edge updates/s
  roofline     the forward edge kernel: algorithmic bytes per launch (the cost
               model of Eq. 1, 4*D bytes per vertex load) / its mean duration
  e2e          ep_run_host with one step per call: host x, w (pinned) copied in
               and x read back every step; resident_state = 100 steps per call
  cpu_baseline the FP64 oracle on the host, bounded sample of steps
With --impl reference the oracle itself is timed as the reference arm.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge updates/s, fwd & fwd+bwd, partitioned vs default order; % HBM peak"
UNIT = "edge updates/s"
D = 5
TAU = 1e-3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--C", type=int, default=512)
    ap.add_argument("--threads", type=int, default=None,
                    help="threads per CUDA block (default 256 consumer threads for the mesh, "
                         "192 for the R-MAT SpMV)")
    ap.add_argument("--stages", type=int, default=3, help="0: one CUDA block per schedule block")
    ap.add_argument("--n", type=int, default=1 << 20, help="mesh points (default: the 1M-node mesh)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--sweep", action="store_true", help="also time C in {256, 512, 1024}")
    ap.add_argument("--only", default="", choices=["", "fwd"],
                    help="fwd: time only the forward loops (for profiler runs)")
    ap.add_argument("--workload", default="mesh", choices=["mesh", "rmat", "batch"],
                    help="mesh: 1M-node kNN mesh flux steps; rmat: R-MAT scale-20 SpMV; "
                         "batch: 512 uneven meshes, 100 steps fwd+bwd in one CUDA graph")
    ap.add_argument("--meshes", type=int, default=512, help="batch workload: number of meshes")
    ap.add_argument("--study", default="", choices=["", "cache"],
                    help="cache: shared-memory staging vs read-only data cache, C in {256, 512, 1024}, "
                         "partitioned and default schedules (one JSON line, no bench line)")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(n):
    import workloads as W

    src, dst = W.knn_mesh(n, 4, 0)
    x0 = W.flux_state(n, D, 0)
    w = W.flux_weights(src.size, 0)
    return src, dst, x0, w


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling while the timed loops run."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


class L2Flush:
    """Write a buffer twice the L2 size, then read a second one of that size.

    The write evicts everything the previous step left in L2; the read then
    evicts the write's own dirty lines, so the next timed step starts from a
    cold, clean L2 and does not pay for the flush's write-backs."""

    def __init__(self, torch):
        l2 = torch.cuda.get_device_properties(0).L2_cache_size
        self.bytes = max(2 * l2, 64 << 20)
        self.a = torch.empty(self.bytes // 4, dtype=torch.float32, device="cuda")
        self.b = torch.zeros(self.bytes // 4, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.a.zero_()
        self.b.sum()


def timed_loop(torch, body, steps, warmup, flush):
    """W untimed runs, then `steps` runs each bracketed by events, L2 flushed before each."""
    for _ in range(warmup):
        body()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    barrier(torch)
    for a, b in ev:
        flush()
        a.record()
        body()
        b.record()
    torch.cuda.synchronize()
    barrier(torch)
    return [a.elapsed_time(b) for a, b in ev]


def barrier(torch):
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()


def max_over_ranks(torch, value):
    """Max of a host number over all ranks (NCCL on GPUs, gloo in CPU tests)."""
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return value


def algorithmic_bytes(S, loads, foreign):
    """Cost-model bytes of one forward edge-kernel launch.

    Task stream (16-bit slot pair + weight, 8 B) + block descriptor (32 B) +
    foreign record ids (4 B each) + one gather and one write-back of 4*D bytes
    per vertex load (loads = sum_b |V_b|, Eq. 1)."""
    return 8 * S.m + 32 * S.k + 4 * foreign + 2 * 4 * D * loads


def bench_fwd(torch, E, S, x0, w, steps, warmup, flush):
    x = torch.from_numpy(x0).cuda()
    wt = torch.from_numpy(w).cuda()
    xl = torch.empty(S.layout_floats(D), device="cuda")
    wl = torch.empty(S.weights_floats(), device="cuda")
    S.layout_in(x, xl)
    S.weights_in(wt, wl)
    for _ in range(warmup):
        S.step(D, xl, xl, wl, None, TAU)
    # whole steps without per-kernel instrumentation, then a separate pass
    # with the library's per-kernel events for the kernel times
    ms = timed_loop(torch, lambda: S.step(D, xl, xl, wl, None, TAU), steps, 0, flush)
    S.timing(2)
    n_instr = max(20, steps // 5)
    timed_loop(torch, lambda: S.step(D, xl, xl, wl, None, TAU), n_instr, 0, flush)
    edge_ms, edge_n = S.timing_read(E.T_EDGE_FWD)
    bnd_ms, bnd_n = S.timing_read(E.T_BND)
    S.timing(0)
    per_step = (edge_n + bnd_n) / n_instr  # our kernels per step (edge kernel + fold)
    return dict(ms=ms, edge_ms=edge_ms / max(edge_n, 1), edge_launches=edge_n,
                bnd_ms=bnd_ms / max(bnd_n, 1), bnd_launches=bnd_n,
                launches_timed=int(round(per_step * len(ms))))


def bench_fwd_bwd(torch, S, x0, w, iters, warmup, flush, T=10, every=5):
    from paper_1605_02043_gb300.autograd import flux_steps
    import workloads as W

    x = torch.from_numpy(x0).cuda()
    wt = torch.from_numpy(w).cuda()
    g = torch.from_numpy(W.loss_weights(S.n, D, 1).astype(np.float32)).cuda()

    def body():
        xr = x.clone().requires_grad_(True)
        wr = wt.clone().requires_grad_(True)
        xT = flux_steps(xr, wr, S, T, TAU, every)
        xT.backward(g)

    ms = timed_loop(torch, body, iters, warmup, flush)
    return dict(ms=ms, T=T)


def bench_e2e(torch, S, x0, w, reps=20, T_long=100):
    """End to end through the public host-buffer call (ep_run_host): every step
    copies that step's inputs (state and weights, pinned host memory) to the
    device and reads the new state back.  Also reported: the same call running
    T_long steps per copy-in/copy-out (state resident between steps)."""
    xh = torch.from_numpy(x0.copy()).pin_memory()
    wh = torch.from_numpy(w.copy()).pin_memory()
    for _ in range(3):  # warm-up (allocates workspace)
        S.run_host(xh, wh, None, steps=1, tau=TAU, D=D)
    barrier(torch)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        S.run_host(xh, wh, None, steps=1, tau=TAU, D=D)
        times.append(time.perf_counter() - t0)
    t = max_over_ranks(torch, statistics.median(times))
    long_times = []
    for _ in range(3):
        xh.copy_(torch.from_numpy(x0))
        t0 = time.perf_counter()
        S.run_host(xh, wh, None, steps=T_long, tau=TAU, D=D)
        long_times.append(time.perf_counter() - t0)
    tl = max_over_ranks(torch, statistics.median(long_times))
    return dict(value=S.m / t, unit=UNIT, h2d_bytes_per_step=int(xh.numel() * 4 + wh.numel() * 4),
                d2h_bytes_per_step=int(xh.numel() * 4), steps_per_call=1, seconds_per_step=t,
                resident_state={"steps_per_call": T_long, "value": S.m * T_long / tl, "unit": UNIT,
                                "h2d_bytes_per_call": int(xh.numel() * 4 + wh.numel() * 4),
                                "d2h_bytes_per_call": int(xh.numel() * 4)})


def cpu_baseline(src, dst, x0, w, seconds):
    import oracle as O

    x = x0.astype(np.float64)
    t0 = time.perf_counter()
    steps = 0
    while True:
        x, _ = O.flux_steps(src, dst, x, w, 1, TAU)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return dict(value=src.size * steps / el, unit=UNIT, cores=1, kind="oracle",
                sample=f"{steps} FP64 NumPy flux steps of the full mesh ({src.size} tasks), single thread")


def cpu_fair(src, dst, x0, w, n, seconds):
    """All host cores, FP64 (oracle/cpu_fair.c, OpenMP); None where it cannot be built."""
    import oracle as O

    try:
        F = O.FairCpu(src, dst, n, D)
    except (RuntimeError, ValueError):
        return None
    x = np.ascontiguousarray(x0, np.float64)
    F.steps(x, w, 1, TAU)  # warm-up
    t0 = time.perf_counter()
    steps = used = 0
    while True:
        _, used = F.steps(x, w, 1, TAU)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return dict(value=src.size * steps / el, unit=UNIT, cores=used, kind="openmp-fp64",
                sample=f"{steps} FP64 flux steps of the full mesh on {used} threads (pull form, "
                       f"one vertex per loop iteration)")


def spmv_time(torch, E, sch, x0, w, n, steps, warmup, flush):
    """Mean SpMV kernel time (ms) and step time (ms) on schedule-layout buffers."""
    xl = torch.empty(n, device="cuda")
    wl = torch.empty(sch.weights_floats(), device="cuda")
    yl = torch.empty(n, device="cuda")
    sch.spmv_x_in(torch.from_numpy(x0).cuda(), xl)
    sch.weights_in(torch.from_numpy(w).cuda(), wl)
    for _ in range(warmup):
        sch.spmv(xl, wl, yl)
    sch.timing(2)
    ms = timed_loop(torch, lambda: sch.spmv(xl, wl, yl), steps, 0, flush)
    kms, kn = sch.timing_read(E.T_SPMV)
    sch.timing(0)
    return kms / max(kn, 1), statistics.mean(ms)


def study_cache_spmv(torch, E, args, rows, cols, n, x0, w):
    """EP-smem vs EP-text (Section 5, Fig. 11, Table 3) for the R-MAT SpMV."""
    flush = L2Flush(torch)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    out = []
    for C in (256, 512, 1024):
        for sched, dflt in (("partitioned", False), ("default", True)):
            S = E.Schedule.partition(rows, cols, n, C, bipartite=True, default_order=dflt)
            S.set_threads(args.threads)
            loads, _ = S.cost_host()
            for name, mode in (("smem", E.CACHE_SMEM), ("l1_readonly", E.CACHE_L1)):
                S.set_cache(mode)
                kms, sms = spmv_time(torch, E, S, x0, w, n, max(20, args.steps // 5), args.warmup, flush)
                out.append(dict(C=C, schedule=sched, kernel=name, loads=loads, kernel_us=1e3 * kms,
                                step_us=1e3 * sms, edge_updates_per_s=rows.size / (1e-3 * sms)))
            S.close()
    clk = clocks.stop()
    print(json.dumps({"study": "cache", "workload": "rmat", "n": n, "m": int(rows.size),
                      "threads": args.threads, "rows": out, "clocks": clk}))


def bench_rmat(args):
    """SpMV on the R-MAT scale-20 graph (y_u += w_e x_v), partitioned vs default order."""
    import torch
    import paper_1605_02043_gb300 as E
    import workloads as W

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    rows, cols = W.rmat()
    n, m = 1 << 20, rows.size
    x0, w = W.spmv_inputs(n, m, 0)
    if args.study == "cache":
        study_cache_spmv(torch, E, args, rows, cols, n, x0, w)
        return
    C = args.C if args.C != 256 else 512
    t0 = time.perf_counter()
    S = E.Schedule.partition(rows, cols, n, C, bipartite=True)
    part_s = time.perf_counter() - t0
    Sd = E.Schedule.partition(rows, cols, n, C, bipartite=True, default_order=True)
    flush = L2Flush(torch)
    res = {}
    for name, sch in (("partitioned", S), ("default", Sd)):
        sch.set_threads(args.threads)
        loads, cut = sch.cost()
        xl = torch.empty(n, device="cuda")
        wl = torch.empty(sch.weights_floats(), device="cuda")
        yl = torch.empty(n, device="cuda")
        sch.spmv_x_in(torch.from_numpy(x0).cuda(), xl)
        sch.weights_in(torch.from_numpy(w).cuda(), wl)
        for _ in range(args.warmup):
            sch.spmv(xl, wl, yl)
        ms = timed_loop(torch, lambda: sch.spmv(xl, wl, yl), args.steps, 0, flush)
        sch.timing(2)  # kernel times from a separate, instrumented pass
        n_instr = max(20, args.steps // 5)
        timed_loop(torch, lambda: sch.spmv(xl, wl, yl), n_instr, 0, flush)
        kms, kn = sch.timing_read(E.T_SPMV)
        sch.timing(0)
        kn_timed = int(round(kn / n_instr * len(ms)))
        # cost-model bytes: entry + weight per task, 64-byte descriptor per block,
        # foreign ids, one 4-byte gather (x) or write-back (y) per vertex load
        alg = 8 * m + 64 * sch.k + 4 * cut + 4 * loads
        tot = max_over_ranks(torch, sum(ms))
        res[name] = dict(edge_updates_per_s=ws * m * len(ms) / (1e-3 * tot), ms_per_step=tot / len(ms),
                         kernel_ms=kms / max(kn, 1), loads=loads, vertex_cut=cut, alg_bytes=alg,
                         alg_GBps=alg / (kms / max(kn, 1) * 1e-3) / 1e9, launches=kn_timed)
    if rank != 0:
        return
    import oracle as O

    t0 = time.perf_counter()
    reps = 0
    while True:
        O.spmv(rows, cols, x0, w, n)
        reps += 1
        if time.perf_counter() - t0 >= args.cpu_seconds:
            break
    cpu_v = m * reps / (time.perf_counter() - t0)
    xh = torch.from_numpy(x0.copy()).pin_memory()
    wh = torch.from_numpy(w.copy()).pin_memory()
    yh = torch.zeros(n).pin_memory()
    S.run_host(xh, wh, yh, steps=1, kernel=E.SPMV, D=1)
    times = []
    for _ in range(3):
        t1 = time.perf_counter()
        S.run_host(xh, wh, yh, steps=1, kernel=E.SPMV, D=1)
        times.append(time.perf_counter() - t1)
    peak, peak_kind = peaks()
    p = res["partitioned"]
    print(json.dumps({
        "metric": "edge updates/s (SpMV y_u += w_e x_v), partitioned vs default order; % HBM peak",
        "value": p["edge_updates_per_s"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": p["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"R-MAT scale 20 (n={n}, m={m}), bipartite SpMV", "C": C,
                   "threads_per_block": args.threads,
                   "l2": "flushed before every timed step (write then read of scratch buffers)"},
        "roofline": {"bound": "hbm", "achieved": p["alg_GBps"], "peak": peak, "unit": "GB/s",
                     "frac": p["alg_GBps"] / peak, "traffic": None, "kernel": "spmv_kernel",
                     "algorithmic_bytes_per_launch": p["alg_bytes"], "launch_ms": p["kernel_ms"],
                     "peak_kind": f"{peak_kind} HBM copy"},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{reps} FP64 NumPy SpMV of the full matrix"},
        "e2e": {"value": m / statistics.median(times), "unit": UNIT,
                "h2d_bytes_per_step": int(4 * n + 4 * m), "d2h_bytes_per_step": int(4 * n)},
        "gpu_launches": p["launches"], "partitioned": p, "default": res["default"],
        "partition_s": part_s,
    }))


def bench_batch(args):
    """512 uneven meshes: autotuned C and kernel, one persistent launch per kernel over all
    meshes, 100 steps fwd+bwd (checkpoint every 10) captured in one CUDA graph; against the
    same work launched eagerly and against per-mesh launches."""
    import torch
    import paper_1605_02043_gb300 as E
    import workloads as W
    from paper_1605_02043_gb300 import autotune
    from paper_1605_02043_gb300.autograd import FluxRunner

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    T, every = 100, 10
    t0 = time.perf_counter()
    graphs = W.batch_meshes(args.meshes)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    tuned = autotune.tune(graphs, D=D)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    parts = autotune.partition_many(graphs, tuned["C"])
    part_s = time.perf_counter() - t0
    B = E.Schedule.batch(parts)
    for sch in parts + [B]:
        sch.set_pipeline(tuned["stages"])
        sch.set_threads(tuned["threads"])
    N, M = B.n, B.m
    x0 = torch.from_numpy(W.flux_state(N, D, 0)).cuda()
    w = torch.from_numpy(W.flux_weights(M, 0)).cuda()
    g = torch.from_numpy(W.loss_weights(N, D, 1).astype(np.float32)).cuda()
    R = FluxRunner(B, D, T, TAU, every)
    R.load(x0, w, g)
    R.run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        R.run()
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    reps = max(1, min(args.steps, 5))
    # the batch's state and task data (hundreds of MB) exceed the L2: no flush needed
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    barrier(torch)
    for a, b in ev:
        a.record()
        graph.replay()
        b.record()
    torch.cuda.synchronize()
    barrier(torch)
    g_ms = [a.elapsed_time(b) for a, b in ev]
    g_tot = max_over_ranks(torch, sum(g_ms))
    graph_v = ws * M * T * reps / (1e-3 * g_tot)
    B.check_errors()
    # same work, eager launches from the host
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    R.run()
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    # per-mesh launches (eager)
    offs_n = np.cumsum([0] + [p.n for p in parts])
    offs_m = np.cumsum([0] + [p.m for p in parts])
    runners = []
    for i, p in enumerate(parts):
        r = FluxRunner(p, D, T, TAU, every)
        r.load(x0[:, offs_n[i]:offs_n[i + 1]], w[offs_m[i]:offs_m[i + 1]], g[:, offs_n[i]:offs_n[i + 1]])
        runners.append(r)
    for r in runners[:4]:
        r.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    for r in runners:
        r.run()
    e1.record()
    torch.cuda.synchronize()
    mesh_ms = e0.elapsed_time(e1)
    mesh_wall = time.perf_counter() - t0
    if rank != 0:
        return
    peak, peak_kind = peaks()
    print(json.dumps({
        "metric": "edge updates/s, fwd+bwd (100 steps, checkpoint every 10), batched uneven meshes",
        "value": graph_v, "unit": UNIT, "n_gpus": ws, "steps": reps, "warmup": max(args.warmup, 3),
        "ms_per_step": g_tot / reps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.meshes} kNN k=4 meshes, n log-uniform in [1024, 65536] "
                               f"(N={N}, M={M}), D=5, 100 explicit steps fwd+bwd",
                   "C": tuned["C"], "pipeline_stages": tuned["stages"],
                   "consumer_threads": tuned["threads"], "autotuned": True,
                   "l2": "not flushed: the batch state and task data exceed the L2",
                   "bench_step": "one CUDA-graph replay of the whole fwd+bwd pass"},
        "graph_batched": graph_v,
        "eager_batched": M * T / (1e-3 * eager_ms),
        "per_mesh_launches": M * T / (1e-3 * mesh_ms), "per_mesh_wall_s": mesh_wall,
        "autotune": {k: tuned[k] for k in ("C", "stages", "threads")},
        "autotune_table": tuned.get("table"),
        "gen_s": gen_s, "tune_s": tune_s, "partition_s": part_s, "loads": B.cost_host()[0],
        "cpu_baseline": None, "roofline": None,
        "e2e": None, "gpu_launches": None, "peak_GBps": peak,
    }))


def mesh_config(args, n, m, ws, l2):
    """The `config` object of the mesh workload (both arms)."""
    return {
        "workload": f"kNN mesh n={n} k=4 (m={m}), D=5, one explicit flux step per bench step",
        "schedule": "edge partition (clone-and-connect + recursive bisection)",
        "C": args.C, "consumer_threads": args.threads, "pipeline_stages": args.stages, "tau": TAU,
        "l2": l2, "parallelism": "replicas" if ws > 1 else "single GPU",
    }


def run_reference(args):
    """The oracle as the reference arm (rank 0 only)."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle as O

    src, dst, x0, w = workload(args.n)
    m = src.size
    # every step is a bounded sample: one explicit step over a window of the
    # task list, sized so that all steps together are about 20 full-mesh steps
    ms = max(1, int(m * min(1.0, 20.0 / max(args.steps, 1))))
    x = x0.astype(np.float64)

    def step(i):
        lo = (i * ms) % m
        idx = np.arange(lo, lo + ms) % m
        return x + TAU * O.flux(src[idx], dst[idx], x, w[idx])

    for i in range(max(args.warmup, 3)):
        x = step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        x = step(i)
    el = time.perf_counter() - t0
    v = ms * args.steps / el
    sample = (f"{args.steps} FP64 NumPy oracle steps over windows of {ms} of the {m} tasks "
              f"(about 20 full-mesh steps in all), one thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": mesh_config(args, args.n, m, 1, "not applicable (host cores)"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def study_cache(torch, E, args, src, dst, x0, w, flush):
    """Texture-cache vs software-cache study of Section 5 (Fig. 11, Table 3) on
    GB300: forward edge-kernel time per launch and step time, per C and schedule."""
    n, m = args.n, src.size
    kinds = (("smem_pipelined", E.CACHE_SMEM, args.stages or 3),
             ("smem_block", E.CACHE_SMEM, 0),
             ("l1_readonly", E.CACHE_L1, 0))
    rows = []
    for C in (256, 512, 1024):
        for sched, default_order in (("partitioned", False), ("default", True)):
            S = E.Schedule.partition(src, dst, n, C, default_order=default_order)
            S.set_threads(args.threads)
            loads, _ = S.cost_host()
            for name, cache, stages in kinds:
                S.set_pipeline(stages)
                S.set_cache(cache)
                r = bench_fwd(torch, E, S, x0, w, max(20, args.steps // 5), args.warmup, flush)
                rows.append(dict(C=C, schedule=sched, kernel=name, loads=loads,
                                 edge_kernel_us=1e3 * r["edge_ms"], bnd_kernel_us=1e3 * r["bnd_ms"],
                                 step_us=1e3 * statistics.mean(r["ms"]),
                                 edge_updates_per_s=m * len(r["ms"]) / (1e-3 * sum(r["ms"]))))
            S.close()
    return rows


def main():
    args = parse()
    if args.threads is None:
        args.threads = 192 if args.workload == "rmat" else 256
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "rmat":
        bench_rmat(args)
        return
    if args.workload == "batch":
        bench_batch(args)
        return
    import torch

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    import paper_1605_02043_gb300 as E

    src, dst, x0, w = workload(args.n)
    n, m = args.n, src.size
    t0 = time.perf_counter()
    S = E.Schedule.partition(src, dst, n, args.C)
    part_s = time.perf_counter() - t0
    Sd = E.Schedule.partition(src, dst, n, args.C, default_order=True)
    for s in (S, Sd):
        s.set_threads(args.threads)
        s.set_pipeline(args.stages)
    loads, cut = S.cost()
    loads_d, cut_d = Sd.cost()
    assert (loads, cut) == S.cost_host() and (loads_d, cut_d) == Sd.cost_host()
    flush = L2Flush(torch)
    flush_bytes = flush.bytes

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    if args.study == "cache":
        rows = study_cache(torch, E, args, src, dst, x0, w, flush)
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"study": "cache", "n": n, "m": m, "D": D, "threads": args.threads,
                              "rows": rows, "clocks": clk}))
        return
    fwd = bench_fwd(torch, E, S, x0, w, args.steps, args.warmup, flush)
    fwd_d = bench_fwd(torch, E, Sd, x0, w, args.steps, args.warmup, flush)
    if args.only == "fwd":
        clocks.stop()
        if rank == 0:
            print(json.dumps({"only": "fwd", "n": n, "m": m, "C": args.C, "threads": args.threads,
                              "partitioned_edge_ms": fwd["edge_ms"], "default_edge_ms": fwd_d["edge_ms"],
                              "partitioned_step_ms": statistics.mean(fwd["ms"]),
                              "default_step_ms": statistics.mean(fwd_d["ms"]),
                              "loads": loads, "loads_default": loads_d}))
        return
    iters = max(3, args.steps // 20)
    fb = bench_fwd_bwd(torch, S, x0, w, iters, 3, flush)
    fb_d = bench_fwd_bwd(torch, Sd, x0, w, iters, 3, flush)
    clk = clocks.stop()

    sweep = {}
    if args.sweep:
        for C in (256, 512, 1024):
            Sc = E.Schedule.partition(src, dst, n, C)
            Sc.set_threads(args.threads)
            Sc.set_pipeline(args.stages)
            r = bench_fwd(torch, E, Sc, x0, w, max(10, args.steps // 4), args.warmup, flush)
            sweep[str(C)] = dict(edge_updates_per_s=m * len(r["ms"]) / (1e-3 * sum(r["ms"])),
                                 loads=Sc.cost_host()[0])

    e2e = bench_e2e(torch, S, x0, w)
    e2e["value"] *= ws  # replicas: whole-job aggregate
    e2e["resident_state"]["value"] *= ws
    tot = max_over_ranks(torch, sum(fwd["ms"]))
    value = ws * m * len(fwd["ms"]) / (1e-3 * tot)
    fb_tot = max_over_ranks(torch, sum(fb["ms"]))
    fb_value = ws * m * fb["T"] * len(fb["ms"]) / (1e-3 * fb_tot)

    # every load beyond a vertex's first block is a foreign record id: sum = vertex cut
    alg = algorithmic_bytes(S, loads, cut)
    alg_d = algorithmic_bytes(Sd, loads_d, cut_d)
    peak, peak_kind = peaks()
    achieved = alg / (fwd["edge_ms"] * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            from paper_1605_02043_gb300 import build as B
            import hashlib
            hh = hashlib.sha256()
            for f in ("flux_tma.cu", "kernels.h", "internal.h"):  # the pipelined kernels' sources
                hh.update(open(os.path.join(B.CSRC, f), "rb").read())
            h = hh.hexdigest()[:16]
            ent = tr.get(f"flux_fwd_C{args.C}_n{n}")
            if ent and ent.get("kernel_sources_sha") == h:
                traffic = ent["dram_bytes_per_launch"]
        except Exception:
            traffic = None

    if rank != 0:
        return
    cpu = cpu_baseline(src, dst, x0, w, args.cpu_seconds) if ws == 1 else None
    fair = cpu_fair(src, dst, x0, w, n, min(5.0, args.cpu_seconds)) if ws == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot / len(fwd["ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": mesh_config(args, n, m, ws,
                              f"flushed before every timed step ({flush_bytes >> 20} MiB write then "
                              f"{flush_bytes >> 20} MiB read of scratch buffers, outside the events)"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "flux_fwd_tma_kernel<5>" if args.stages else "flux_fwd_kernel<5>",
                     "algorithmic_bytes_per_launch": alg,
                     "launch_ms": fwd["edge_ms"], "peak_kind": f"{peak_kind} HBM copy"},
        "cpu_baseline": cpu,
        "cpu_all_cores": fair,
        "e2e": e2e,
        "gpu_launches": fwd["launches_timed"],
        "clocks": clk,
        "partitioned": {"edge_updates_per_s": value, "loads": loads, "vertex_cut": cut,
                        "edge_kernel_ms": fwd["edge_ms"], "bnd_kernel_ms": fwd["bnd_ms"],
                        "partition_s": part_s, "alg_bytes": alg,
                        "alg_GBps_edge_kernel": achieved},
        "default": {"edge_updates_per_s": ws * m * len(fwd_d["ms"]) / (1e-3 * sum(fwd_d["ms"])),
                    "loads": loads_d, "vertex_cut": cut_d, "edge_kernel_ms": fwd_d["edge_ms"],
                    "bnd_kernel_ms": fwd_d["bnd_ms"], "alg_bytes": alg_d,
                    "alg_GBps_edge_kernel": alg_d / (fwd_d["edge_ms"] * 1e-3) / 1e9},
        "fwd_bwd": {"partitioned": fb_value,
                    "default": ws * m * fb_d["T"] * len(fb_d["ms"]) / (1e-3 * sum(fb_d["ms"])),
                    "unit": UNIT, "steps": fb["T"], "checkpoint_every": 5, "iterations": len(fb["ms"])},
        "C_sweep": sweep or None,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
