#!/usr/bin/env python3
"""Benchmark of the edge-partitioned flux kernel on one GB300.

Workload: the 1M-node mesh (1,048,576 points uniform in the unit cube, seed
0, symmetrised k=4 nearest-neighbour graph, ~2.57M tasks in shuffled order),
state x: 5 x fp32 N(0,1), weights w ~ U(0.5, 1.5), explicit steps
x <- x + 1e-3 * flux(x).  One bench step is one explicit step of a run of
`--steps` steps on the whole mesh: one launch of the edge kernel (the copies of
shared vertices stay one step behind, ep_step_pending), with the L2 flushed (a
write and then a read of scratch buffers twice the L2 size) before every timed
step and outside its events; the run's final finish (ep_finish) is timed too
and added to the total.

Reported (one JSON line on rank 0):
  value          forward edge updates/s of the run, partitioned schedule (C = --C)
  default        the same under the default order (C consecutive tasks per block)
  complete_step  steps that each finish their state (edge kernel + finish)
  back_to_back   steps without L2 flushes between them (state and tasks stay in L2)
  fwd_bwd        10 steps forward + backward (checkpoint every 5, recompute
                 included) through the autograd function, edge updates/s
  adjoint        the adjoint edge kernel alone: time per launch and its roofline
  roofline       the forward edge kernel: algorithmic bytes per launch (the cost
                 model of Eq. 1, 4*D bytes per vertex load) / its mean duration;
                 traffic = ncu DRAM bytes per launch from profiles/traffic.json
                 while the kernel sources hash to the recorded value
  e2e            ep_run_host with one step per call: host x, w (pinned) read by
                 the layout kernels over the host link and x written back every
                 step; resident_state = 100 steps per call
  C_sweep        C in {256, 512, 1024}: value and roofline of each
  cpu_baseline   the FP64 oracle on the host, bounded sample of steps
  rmat           R-MAT scale-20 SpMV sub-record (partitioned vs default order)
  batch          512 uneven meshes sub-record (100 steps fwd+bwd in a CUDA graph)
With --impl reference the oracle itself is timed as the reference arm.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import platform
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
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--C", type=int, default=512)
    ap.add_argument("--threads", type=int, default=None,
                    help="consumer threads per CUDA block (default 192 for the mesh and the SpMV)")
    ap.add_argument("--stages", type=int, default=3, help="0: one CUDA block per schedule block")
    ap.add_argument("--n", type=int, default=1 << 20, help="mesh points (default: the 1M-node mesh)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--quick", action="store_true",
                    help="mesh line only: no C sweep, R-MAT or batch sub-records")
    ap.add_argument("--only", default="", choices=["", "fwd", "adj"],
                    help="fwd / adj: time only the forward loops / the adjoint steps (profiler runs)")
    ap.add_argument("--workload", default="mesh", choices=["mesh", "rmat", "batch"],
                    help="mesh: 1M-node kNN mesh flux steps (with the sub-records); rmat: R-MAT "
                         "scale-20 SpMV alone; batch: 512 uneven meshes alone")
    ap.add_argument("--meshes", type=int, default=512, help="batch workload: number of meshes")
    ap.add_argument("--study", default="", choices=["", "cache", "autotune"],
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


def cpu_info():
    """Host CPU model and thread count."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return dict(model=model, machine=platform.machine(), threads=os.cpu_count())


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
    cold, clean L2 and does not pay for the flush's write-backs.  (The previous
    step's own dirty lines are written back during the flush, outside the
    events: `back_to_back` times steps without flushes.)"""

    def __init__(self, torch):
        l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
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
        if flush is not None:
            flush()
        a.record()
        body()
        b.record()
    torch.cuda.synchronize()
    barrier(torch)
    return [a.elapsed_time(b) for a, b in ev]


def time_once(torch, body):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    body()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


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


def adjoint_bytes(S, loads, foreign):
    """Cost-model bytes of one adjoint edge-kernel launch: the task stream, the
    descriptor and foreign ids, a gather of x and of lam and a write-back of lam
    (4*D bytes each per vertex load), and the weight gradient (4 B per task)."""
    return 12 * S.m + 32 * S.k + 4 * foreign + 3 * 4 * D * loads


ROOT = os.path.dirname(os.path.abspath(__file__))


def kernel_sources_sha():
    """Hash of the library sources the kernels are built from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1605_02043_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def traffic(key):
    """ncu DRAM bytes (read + write) per launch recorded in profiles/traffic.json
    for this kernel and workload, if recorded from the current sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sources_sha") != kernel_sources_sha():
        return None
    return rec.get("dram_bytes_per_launch")


def roofline(alg_bytes, launch_ms, kernel, peak, peak_kind, traffic=None):
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "algorithmic_bytes_per_launch": alg_bytes,
            "launch_ms": launch_ms, "peak_kind": f"{peak_kind} HBM copy"}


def bench_fwd(torch, S, x0, w, steps, warmup, flush, complete=True, b2b_steps=50):
    """A run of `steps` pending steps (one edge-kernel launch each, L2 flushed
    before each, events around each) and its final finish; steps that finish
    their state each time; and pending steps back to back without flushes."""
    x = torch.from_numpy(x0).cuda()
    wt = torch.from_numpy(w).cuda()
    xl = torch.empty(S.layout_floats(D), device="cuda")
    wl = torch.empty(S.weights_floats(), device="cuda")
    S.layout_in(x, xl)
    S.weights_in(wt, wl)
    pend = lambda: S.step(D, xl, xl, wl, None, TAU, pending=True)  # noqa: E731
    for _ in range(warmup):
        pend()
    S.finish(D, xl, TAU)
    ms = timed_loop(torch, pend, steps, 0, flush)
    fin_ms = time_once(torch, lambda: S.finish(D, xl, TAU))
    res = dict(ms=ms, finish_ms=fin_ms, total_ms=sum(ms) + fin_ms, edge_ms=statistics.mean(ms),
               launches_timed=len(ms) + 1)
    if complete:
        cms = timed_loop(torch, lambda: S.step(D, xl, xl, wl, None, TAU), max(10, steps // 5), 2, flush)
        res["complete_ms"] = cms
    torch.cuda.synchronize()

    def b2b():
        for _ in range(b2b_steps):
            pend()
        S.finish(D, xl, TAU)

    b2b()
    res["b2b_ms_per_step"] = time_once(torch, b2b) / b2b_steps
    S.check_errors()
    return res


def bench_adj(torch, S, x0, w, steps, warmup, flush):
    """Adjoint steps at the state x0 (one edge-kernel launch each, the
    cotangent's shared copies pending between them, L2 flushed before each,
    events around each): mean ms per launch."""
    import workloads as W

    xl = torch.empty(S.layout_floats(D), device="cuda")
    wl = torch.empty(S.weights_floats(), device="cuda")
    lam = torch.empty_like(xl)
    gw = torch.zeros_like(wl)
    S.layout_in(torch.from_numpy(x0).cuda(), xl)
    S.weights_in(torch.from_numpy(w).cuda(), wl)
    S.layout_in(torch.from_numpy(W.loss_weights(S.n, D, 1).astype(np.float32)).cuda(), lam)
    step = lambda: S.adjoint_step(D, xl, wl, lam, gw, TAU, pending=True)  # noqa: E731
    for _ in range(warmup):
        step()
    ms = timed_loop(torch, step, steps, 0, flush)
    S.adjoint_finish(D, lam, TAU)
    S.check_errors()
    return statistics.mean(ms)


def adjoint_record(torch, S, x0, w, args, flush, peak, peak_kind):
    loads, cut = S.cost()
    ms = bench_adj(torch, S, x0, w, max(20, args.steps // 2), args.warmup, flush)
    alg = adjoint_bytes(S, loads, cut)
    return {"edge_kernel_ms": ms, "edge_updates_per_s": S.m / (1e-3 * ms), "alg_bytes": alg,
            "roofline": roofline(alg, ms, "flux_adj_tma_kernel<5>" if args.stages else "flux_adj_kernel<5>",
                                 peak, peak_kind, traffic(f"flux_adj_{S.origin}_C{S.C}_n{S.n}")),
            "note": "adjoint steps with the cotangent's shared copies pending, L2 flushed before each"}


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
    hb, db = int(xh.numel() * 4 + wh.numel() * 4), int(xh.numel() * 4)
    return dict(value=S.m / t, unit=UNIT, h2d_bytes_per_step=hb, d2h_bytes_per_step=db, steps_per_call=1,
                seconds_per_step=t, copy_GBps=(hb + db) / t / 1e9,
                resident_state={"steps_per_call": T_long, "value": S.m * T_long / tl, "unit": UNIT,
                                "h2d_bytes_per_call": hb, "d2h_bytes_per_call": db})


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
    ci = cpu_info()
    return dict(value=src.size * steps / el, unit=UNIT, cores=1, kind="oracle", cpu=ci["model"],
                host_threads=ci["threads"],
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
    return dict(value=src.size * steps / el, unit=UNIT, cores=used, kind="openmp-fp64", cpu=cpu_info()["model"],
                sample=f"{steps} FP64 flux steps of the full mesh on {used} threads (pull form, "
                       f"one vertex per loop iteration)")


# ------------------------------------------------------------------- R-MAT SpMV

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
    return kms / max(kn, 1), ms


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
                                step_us=1e3 * statistics.mean(sms),
                                edge_updates_per_s=rows.size / (1e-3 * statistics.mean(sms))))
            S.close()
    clk = clocks.stop()
    print(json.dumps({"study": "cache", "workload": "rmat", "n": n, "m": int(rows.size),
                      "threads": args.threads, "rows": out, "clocks": clk}))


def rmat_record(torch, E, args, ws, flush, C=512, cpu_seconds=5.0):
    """SpMV on the R-MAT scale-20 graph (y_u += w_e x_v), partitioned vs default order."""
    import workloads as W
    import oracle as O

    rows, cols = W.rmat()
    n, m = 1 << 20, rows.size
    x0, w = W.spmv_inputs(n, m, 0)
    t0 = time.perf_counter()
    S = E.Schedule.partition(rows, cols, n, C, bipartite=True)
    part_s = time.perf_counter() - t0
    Sd = E.Schedule.partition(rows, cols, n, C, bipartite=True, default_order=True)
    peak, peak_kind = peaks()
    res = {}
    steps = max(20, args.steps)
    for name, sch in (("partitioned", S), ("default", Sd)):
        sch.set_threads(args.threads)
        loads, cut = sch.cost()
        kms, ms = spmv_time(torch, E, sch, x0, w, n, steps, args.warmup, flush)
        tot = max_over_ranks(torch, sum(ms))
        # cost-model bytes: entry + weight per task, 64-byte descriptor per block,
        # foreign ids, one 4-byte gather (x) or write-back (y) per vertex load
        alg = 8 * m + 64 * sch.k + 4 * cut + 4 * loads
        res[name] = dict(edge_updates_per_s=ws * m * len(ms) / (1e-3 * tot), ms_per_step=tot / len(ms),
                         kernel_ms=kms, loads=loads, vertex_cut=cut, alg_bytes=alg,
                         roofline=roofline(alg, kms, "spmv_kernel", peak, peak_kind,
                                           traffic(f"spmv_{sch.origin}_C{sch.C}_n{n}")))
    # the oracle on the host, bounded
    t0 = time.perf_counter()
    reps = 0
    while True:
        O.spmv(rows, cols, x0, w, n)
        reps += 1
        if time.perf_counter() - t0 >= cpu_seconds:
            break
    cpu_v = m * reps / (time.perf_counter() - t0)
    xh = torch.from_numpy(x0.copy()).pin_memory()
    wh = torch.from_numpy(w.copy()).pin_memory()
    yh = torch.zeros(n).pin_memory()
    S.run_host(xh, wh, yh, steps=1, kernel=E.SPMV, D=1)
    times = []
    for _ in range(5):
        t1 = time.perf_counter()
        S.run_host(xh, wh, yh, steps=1, kernel=E.SPMV, D=1)
        times.append(time.perf_counter() - t1)
    p = res["partitioned"]
    return {
        "metric": "edge updates/s (SpMV y_u += w_e x_v), partitioned vs default order; % HBM peak",
        "value": p["edge_updates_per_s"], "unit": UNIT, "ms_per_step": p["ms_per_step"],
        "config": {"workload": f"R-MAT scale 20 (n={n}, m={m}), bipartite SpMV", "C": C,
                   "threads_per_block": args.threads,
                   "l2": "flushed before every timed step (write then read of scratch buffers)"},
        "roofline": p["roofline"],
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_info()["model"],
                         "sample": f"{reps} FP64 NumPy SpMV of the full matrix"},
        "e2e": {"value": m / statistics.median(times), "unit": UNIT,
                "h2d_bytes_per_step": int(4 * n + 4 * m), "d2h_bytes_per_step": int(4 * n)},
        "partitioned": p, "default": res["default"], "partition_s": part_s,
        "speedup_vs_default": res["default"]["kernel_ms"] / p["kernel_ms"],
    }


def bench_rmat(args):
    import torch
    import paper_1605_02043_gb300 as E

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    if args.study == "cache":
        import workloads as W
        rows, cols = W.rmat()
        x0, w = W.spmv_inputs(1 << 20, rows.size, 0)
        study_cache_spmv(torch, E, args, rows, cols, 1 << 20, x0, w)
        return
    flush = L2Flush(torch)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    rec = rmat_record(torch, E, args, ws, flush, C=args.C, cpu_seconds=args.cpu_seconds)
    clk = clocks.stop()
    if rank != 0:
        return
    rec.update({"n_gpus": ws, "steps": max(20, args.steps), "warmup": args.warmup, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "gpu_launches": max(20, args.steps), "clocks": clk})
    print(json.dumps(rec))


# ---------------------------------------------------------- 512 uneven meshes

def batch_record(torch, E, args, ws, T=100, every=10, cpu_seconds=5.0):
    """512 uneven meshes: autotuned C and kernel, one persistent launch per kernel over all
    meshes, T steps fwd+bwd (checkpoint every `every`) captured in one CUDA graph; against the
    same work launched eagerly and against per-mesh launches.  The batch's state and task data
    (hundreds of MB) exceed the L2, so no flush is needed."""
    import workloads as W
    import oracle as O
    from paper_1605_02043_gb300 import autotune
    from paper_1605_02043_gb300.autograd import FluxRunner

    t0 = time.perf_counter()
    graphs = W.batch_meshes(args.meshes)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    parts_by_C = {}
    tuned = autotune.tune(graphs, D=D, partitions=parts_by_C)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    parts = parts_by_C.get(tuned["C"]) or autotune.partition_many(graphs, tuned["C"])
    part_s = time.perf_counter() - t0
    B = E.Schedule.batch(parts)
    for sch in parts + [B]:
        sch.set_pipeline(tuned["stages"])
        sch.set_threads(tuned["threads"])
    N, M = B.n, B.m
    x0h = W.flux_state(N, D, 0)
    wh_ = W.flux_weights(M, 0)
    gh = W.loss_weights(N, D, 1).astype(np.float32)
    x0 = torch.from_numpy(x0h).cuda()
    w = torch.from_numpy(wh_).cuda()
    g = torch.from_numpy(gh).cuda()
    R = FluxRunner(B, D, T, TAU, every)
    R.load(x0, w, g)
    R.run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        R.run()
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    reps = 5
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
    eager_ms = time_once(torch, R.run)
    # end to end: inputs copied in from pinned host memory, the replay, gradients read back
    x0p = torch.from_numpy(x0h.copy()).pin_memory()
    wp = torch.from_numpy(wh_.copy()).pin_memory()
    gp = torch.from_numpy(gh.copy()).pin_memory()
    dxp = torch.empty_like(x0p).pin_memory()
    dwp = torch.empty(M).pin_memory()
    e2e_t = []
    for _ in range(3):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        R.load(x0p.cuda(non_blocking=True), wp.cuda(non_blocking=True), gp.cuda(non_blocking=True))
        graph.replay()
        _, dx, dw = R.results(x0, M)
        dxp.copy_(dx, non_blocking=True)
        dwp.copy_(dw, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t1)
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
    mesh_ms = time_once(torch, lambda: [r.run() for r in runners])
    # roofline over the replay: cost-model bytes of every launch in it
    loads, cut = B.cost_host()
    nseg = (T + every - 1) // every
    n_fwd = T + (T - nseg)  # forward steps + recomputed states
    alg = n_fwd * algorithmic_bytes(B, loads, cut) + T * adjoint_bytes(B, loads, cut)
    peak, peak_kind = peaks()
    rl = roofline(alg, g_tot / reps, "flux_fwd_tma_kernel<5> + flux_adj_tma_kernel<5> (whole replay)",
                  peak, peak_kind)
    # the oracle on sampled meshes, bounded
    rng = np.random.default_rng(5)
    done_tasks, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < cpu_seconds:
        i = int(rng.integers(len(graphs)))
        n_i, s_i, d_i = graphs[i]
        xi = x0h[:, offs_n[i]:offs_n[i + 1]]
        wi = wh_[offs_m[i]:offs_m[i + 1]]
        O.flux_steps(s_i, d_i, xi, wi, T, TAU)
        O.flux_adjoint(s_i, d_i, xi, wi, T, TAU, gh[:, offs_n[i]:offs_n[i + 1]])
        done_tasks += s_i.size * T
    cpu_v = done_tasks / (time.perf_counter() - t1)
    e2e = statistics.median(e2e_t)
    return {
        "metric": f"edge updates/s, fwd+bwd ({T} steps, checkpoint every {every}), batched uneven meshes",
        "value": graph_v, "unit": UNIT, "ms_per_step": g_tot / reps, "steps": reps,
        "config": {"workload": f"{args.meshes} kNN k=4 meshes, n log-uniform in [1024, 65536] "
                               f"(N={N}, M={M}), D=5, {T} explicit steps fwd+bwd",
                   "C": tuned["C"], "pipeline_stages": tuned["stages"],
                   "consumer_threads": tuned["threads"], "autotuned": True,
                   "l2": "not flushed: the batch state and task data exceed the L2",
                   "bench_step": "one CUDA-graph replay of the whole fwd+bwd pass"},
        "roofline": rl,
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_info()["model"],
                         "sample": f"FP64 NumPy fwd+bwd ({T} steps) of randomly drawn meshes for "
                                   f"{cpu_seconds:.0f} s, {done_tasks} edge updates"},
        "e2e": {"value": M * T / e2e, "unit": UNIT, "h2d_bytes_per_step": int(4 * (x0h.size + wh_.size + gh.size)),
                "d2h_bytes_per_step": int(4 * (x0h.size + M)), "seconds_per_step": e2e},
        "graph_batched": graph_v, "eager_batched": M * T / (1e-3 * eager_ms),
        "per_mesh_launches": M * T / (1e-3 * mesh_ms),
        "autotune": {k: tuned[k] for k in ("C", "stages", "threads")},
        "autotune_confirmed": tuned.get("confirmed"),
        "gen_s": gen_s, "tune_s": tune_s, "partition_s": part_s, "loads": loads,
    }


def study_autotune(torch, E, args):
    """The autotuner's pick against a full-batch sweep of every candidate
    (every C in DEFAULT_CS x every (stages, threads) in DEFAULT_KERNELS, timed
    the way the autotuner times them: one forward and one adjoint step, L2
    flushed before each of 20 repetitions)."""
    import workloads as W
    from paper_1605_02043_gb300 import autotune

    graphs = W.batch_meshes(args.meshes)
    parts_by_C = {}
    tuned = autotune.tune(graphs, D=D, partitions=parts_by_C, cache=None)
    flush = autotune._Flush(torch)
    full = []
    for C in autotune.DEFAULT_CS:
        parts = parts_by_C.get(C) or autotune.partition_many(graphs, C)
        B = E.Schedule.batch(parts)
        for (st, th), ms in zip(autotune.DEFAULT_KERNELS,
                                autotune._time_configs(torch, B, D, autotune.DEFAULT_KERNELS, 20, TAU, flush)):
            full.append(dict(C=C, stages=st, threads=th, ms=ms))
        B.close()
    best = min(full, key=lambda r: r["ms"])
    pick = next(r for r in full if (r["C"], r["stages"], r["threads"]) ==
                (tuned["C"], tuned["stages"], tuned["threads"]))
    print(json.dumps({"study": "autotune", "meshes": args.meshes, "tuned": {k: tuned[k] for k in
                      ("C", "stages", "threads")}, "screening": tuned["table"], "confirmed": tuned["confirmed"],
                      "sample": tuned["sample"], "full_sweep": full, "best": best,
                      "pick_over_best": pick["ms"] / best["ms"]}))


def bench_batch(args):
    import torch
    import paper_1605_02043_gb300 as E

    if args.study == "autotune":
        study_autotune(torch, E, args)
        return

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    rec = batch_record(torch, E, args, ws, cpu_seconds=args.cpu_seconds)
    clk = clocks.stop()
    if rank != 0:
        return
    rec.update({"n_gpus": ws, "warmup": max(args.warmup, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "clocks": clk,
                "gpu_launches": None})
    print(json.dumps(rec))


# ------------------------------------------------------------------ mesh line

def mesh_config(args, n, m, ws, l2):
    """The `config` object of the mesh workload (both arms)."""
    return {
        "workload": f"kNN mesh n={n} k=4 (m={m}), D=5, one explicit flux step per bench step "
                    f"(a run of {args.steps} steps and its finish)",
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
    ci = cpu_info()
    sample = (f"{args.steps} FP64 NumPy oracle steps over windows of {ms} of the {m} tasks "
              f"(about 20 full-mesh steps in all), one thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": mesh_config(args, args.n, m, 1, "not applicable (host cores)"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": ci["model"], "host_threads": ci["threads"]},
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
                r = bench_fwd(torch, S, x0, w, max(20, args.steps // 5), args.warmup, flush, complete=False)
                rows.append(dict(C=C, schedule=sched, kernel=name, loads=loads,
                                 edge_kernel_us=1e3 * r["edge_ms"], finish_us=1e3 * r["finish_ms"],
                                 edge_updates_per_s=m * len(r["ms"]) / (1e-3 * r["total_ms"])))
            S.close()
    return rows


def mesh_run(torch, E, S, x0, w, args, flush, peak, peak_kind, complete=True):
    """Forward record of one schedule: value, roofline of the edge kernel and the variants."""
    loads, cut = S.cost()
    assert (loads, cut) == S.cost_host()
    r = bench_fwd(torch, S, x0, w, args.steps, args.warmup, flush, complete=complete)
    m = S.m
    alg = algorithmic_bytes(S, loads, cut)
    rec = {"edge_updates_per_s": m * len(r["ms"]) / (1e-3 * r["total_ms"]), "loads": loads, "vertex_cut": cut,
           "edge_kernel_ms": r["edge_ms"], "finish_ms": r["finish_ms"], "alg_bytes": alg,
           "roofline": roofline(alg, r["edge_ms"], "flux_fwd_tma_kernel<5>" if args.stages else
                                "flux_fwd_kernel<5>", peak, peak_kind,
                                traffic(f"flux_fwd_{S.origin}_C{S.C}_n{S.n}")),
           "back_to_back": {"ms_per_step": r["b2b_ms_per_step"],
                            "edge_updates_per_s": m / (1e-3 * r["b2b_ms_per_step"]),
                            "note": "50 pending steps and their finish without L2 flushes"}}
    if "complete_ms" in r:
        rec["complete_step"] = {"ms_per_step": statistics.mean(r["complete_ms"]),
                                "edge_updates_per_s": m / (1e-3 * statistics.mean(r["complete_ms"])),
                                "note": "each step finishes its state (edge kernel + finish)"}
    if args.stages:
        rec["launch_plan"] = S.pipeline_info(D)
    return r, rec


def main():
    args = parse()
    if args.threads is None:
        args.threads = 192
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
    flush = L2Flush(torch)
    flush_bytes = flush.bytes
    peak, peak_kind = peaks()

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    if args.study == "cache":
        rows = study_cache(torch, E, args, src, dst, x0, w, flush)
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"study": "cache", "n": n, "m": m, "D": D, "threads": args.threads,
                              "rows": rows, "clocks": clk}))
        return
    if args.only == "adj":
        rec = adjoint_record(torch, S, x0, w, args, flush, peak, peak_kind)
        clocks.stop()
        if rank == 0:
            print(json.dumps({"only": "adj", "n": n, "m": m, "C": args.C, "threads": args.threads,
                              "partitioned": rec}))
        return
    fwd, p_rec = mesh_run(torch, E, S, x0, w, args, flush, peak, peak_kind)
    fwd_d, d_rec = mesh_run(torch, E, Sd, x0, w, args, flush, peak, peak_kind, complete=False)
    if args.only == "fwd":
        clocks.stop()
        if rank == 0:
            print(json.dumps({"only": "fwd", "n": n, "m": m, "C": args.C, "threads": args.threads,
                              "partitioned": p_rec, "default": d_rec}))
        return
    adj = adjoint_record(torch, S, x0, w, args, flush, peak, peak_kind)
    iters = max(3, args.steps // 20)
    fb = bench_fwd_bwd(torch, S, x0, w, iters, 3, flush)
    fb_d = bench_fwd_bwd(torch, Sd, x0, w, iters, 3, flush)
    tot = max_over_ranks(torch, fwd["total_ms"])
    value = ws * m * len(fwd["ms"]) / (1e-3 * tot)
    fb_tot = max_over_ranks(torch, sum(fb["ms"]))
    fb_value = ws * m * fb["T"] * len(fb["ms"]) / (1e-3 * fb_tot)
    sweep = None
    if not args.quick:
        sweep = {}
        for C in (256, 512, 1024):
            Sc = S if C == args.C else E.Schedule.partition(src, dst, n, C)
            Sc.set_threads(args.threads)
            Sc.set_pipeline(args.stages)
            _, rec = mesh_run(torch, E, Sc, x0, w, args, flush, peak, peak_kind, complete=False)
            sweep[str(C)] = {k: rec[k] for k in ("edge_updates_per_s", "loads", "vertex_cut", "edge_kernel_ms",
                                                 "finish_ms", "roofline", "back_to_back")}
    clk = clocks.stop()

    e2e = bench_e2e(torch, S, x0, w)
    e2e["value"] *= ws  # replicas: whole-job aggregate
    e2e["resident_state"]["value"] *= ws
    rmat = batch = None
    if not args.quick:
        rmat = rmat_record(torch, E, args, ws, flush)
        batch = batch_record(torch, E, args, ws)

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
        "roofline": p_rec["roofline"],
        "cpu_baseline": cpu,
        "cpu_all_cores": fair,
        "e2e": e2e,
        "gpu_launches": fwd["launches_timed"],
        "clocks": clk,
        "partitioned": dict(p_rec, partition_s=part_s),
        "default": d_rec,
        "fwd_bwd": {"partitioned": fb_value,
                    "default": ws * m * fb_d["T"] * len(fb_d["ms"]) / (1e-3 * sum(fb_d["ms"])),
                    "unit": UNIT, "steps": fb["T"], "checkpoint_every": 5, "iterations": len(fb["ms"])},
        "adjoint": adj,
        "C_sweep": sweep,
        "rmat": rmat,
        "batch": batch,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
