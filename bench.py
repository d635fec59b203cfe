"""Throughput of the fractional ABM engine on one synthetic workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fabm|reference]
                    [--workload NAME] [--precision fp64|split]

One "step" is one whole solve of the workload (every block of the history
sums, the recurrence, initial values) through the C ABI.  The default
workload is the largest single-GPU configuration: 256 trajectories of the
3-dim Lorenz-type system, alpha = 0.95, h = 1e-4, N = 2^20 steps, in split
precision (history sums on tensor cores).  The same run times the plain FP64
single-trajectory solve (Lorenz-type, alpha = 0.98, h = 5e-4, N = 2^18) as
``vs_fp64_path``: the batched split path against the plain FP64 path.

Timing: W untimed warm-up solves, then K timed solves, each bracketed by CUDA
events, with a 256 MiB buffer written between them to flush L2.  The library
times its own kernels with CUDA events on the streams they run on (the
history kernel's numbers give the roofline line).  ``e2e`` repeats the solve
with host buffers, the host->device and device->host copies inside the timed
region.  ``cpu_baseline`` times the CPU oracle on a bounded prefix of the same
workload and extrapolates by N^2.

Under torchrun with N > 1 ranks every rank solves its own replica (the method
has no exchange step across trajectories); rank 0 prints the line.
``--impl reference`` times the CPU oracle instead, on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import fabm_workloads as wl  # noqa: E402

WORKLOADS = {
    "lorenz-single": lambda: wl.lorenz_single(),
    "ml-scalar": lambda: wl.ml_scalar(),
    "duffing-sweep": lambda: wl.duffing_sweep(),
    "lorenz-long": lambda: _lorenz_long(),
    "lcr-sweep": lambda: _lcr_sweep(),
}
DEFAULT_WORKLOAD = "lorenz-long"
# arithmetic of the history sum, by the kernel a solve ran: three-term bf16
# split on tensor cores, compensated fp32, double, double-double
DTYPE_OF_HISTORY = {"tensor": "bf16x3", "tensor-wide": "bf16x3", "fp32c": "f32c",
                    "fp64": "f64", "fp64-persist": "f64", "x2": "f64x2"}


def _lorenz_long():
    """256 Lorenz-type trajectories x 2^20 steps, split precision by default."""
    w = wl.lorenz_long()
    w.precision = "split"
    return w


def _lcr_sweep():
    """Sec. 5's forced LCR circuit, 1024 forcing amplitudes in [0, 0.2], split precision."""
    w = wl.lcr_sweep(B=1024, N=2 ** 14)
    w.precision = "split"
    return w
SM_COUNT = 152
FP64_FLOP_PER_CLK_PER_SM = 4  # 2 DFMA per clock per SM on GB300 (1.25 TFLOP/s nominal at 2.07 GHz)
FP32_FLOP_PER_CLK_PER_SM = 256  # 128 FFMA per clock per SM
L2_FLUSH_BYTES = 256 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_max(x: float, device) -> float:
    """Max of x over the ranks of the default process group (x itself when
    there is none): the slowest rank's time is the job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world_size: int, step_ms_max: float) -> float:
    """Whole-job throughput of independent replicas: every rank solves its own
    copy of the workload, so the job processes world_size x units in the
    slowest rank's time."""
    return units_per_rank * world_size / (step_ms_max * 1e-3)


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and local_rank < len(ids) and ids[local_rank].strip().isdigit():
        return int(ids[local_rank])
    return local_rank


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.proc = gpu, None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# Sources each profiled kernel is built from; a committed ncu summary gives its
# traffic only while the sha256 over these files (in this order) still matches.
KERNEL_SOURCES = {
    "history_fp64": ["history_fp64.cu", "history_blocks.cuh", "fabm_internal.cuh"],
    "history_split": ["history_far.cu", "history_split.cu", "sm100_ptx.cuh", "fabm_internal.cuh"],
    "recurrence": ["recurrence.cu", "recurrence.cuh", "rhs.cuh", "fabm_internal.cuh"],
    "recurrence_split": ["recurrence_cols.cu", "recurrence.cuh", "rhs.cuh", "ff.cuh",
                         "fabm_internal.cuh"],
    "history_served": ["serve.cu", "history_blocks.cuh", "recurrence.cuh", "fabm_internal.cuh"],
}


def _code_tokens(src: str) -> str:
    """The source without comments and with whitespace collapsed, so that only
    code changes change a kernel's hash (string and character literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        ch = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif ch in "\"'":
            j = i + 1
            while j < n and src[j] != ch:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(ch)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_sha(key: str) -> str:
    """sha256 over the code (comments and whitespace removed) of the files a
    kernel class is built from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[key]:
        with open(os.path.join(ROOT, "paper_1710_01133_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_tokens(fh.read()).encode())
    return h.hexdigest()


def _profile_traffic(key: str, name: str):
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the current sources of the kernel."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    m_tr = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    if not (m_sha and m_tr):
        return None
    return float(m_tr.group(1)) if kernel_source_sha(key) == m_sha.group(1) else None


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), d.get("bf16_tflops"), "of measured"
    except (OSError, ValueError):
        return 6800.0, 1900.0, "of fallback"


def roofline(kind, ks, precision, clocks, workload, w=None, step_ms=None):
    """Roofline line for the dominant kernel class.

    For the history kernels the headline `achieved` is the algorithmic history
    work of one whole solve (2 N^2 flops per column: the predictor and the
    corrector sum, one multiply-add per past point each) divided by the
    uninstrumented solve time `step_ms`: a lower bound on the kernel's rate,
    since the solve also runs the recurrence and the launches between blocks.
    `in_launch` gives the same work per timed launch divided by the time those
    launches ran (CUDA events on the launching streams, overlaps counted once),
    taken on separate instrumented solves."""
    n, flops = ks["launches"], ks["flops"]
    # time during which the timed launches ran, overlaps counted once (history
    # launches of consecutive blocks overlap on two streams in long FP64 solves)
    ms = ks.get("busy_ms") or ks["ms"]
    avg_us = ks["ms"] * 1e3 / max(n, 1)
    hbm, bf16, src = _measured_peaks()
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    out = {"kernel": f"{kind} ({precision})"}
    tensor = kind == "history" and precision == "split"
    if tensor:
        # 6 bf16 products per algorithmic multiply-add (three-term split, order <= 2)
        mult, unit, scale, peak = 6.0, "TFLOP/s", 1e12, bf16
        out.update({"bound": "tensor",
                    "peak_note": f"dense bf16 burst {src} (MEASURED_PEAKS.json); achieved counts "
                                 "the 6 bf16 products per algorithmic multiply-add"})
    elif kind == "recurrence" and precision == "split":
        # float-float on the FP32 pipe: algorithmic near-field FLOP/s against FP32 FMA
        mult, unit, scale = 1.0, "GFLOP/s", 1e9
        peak = FP32_FLOP_PER_CLK_PER_SM * SM_COUNT * sm_max * 1e6 / 1e9
        out.update({"bound": "alu",
                    "peak_note": "FP32 FMA pipe: 128 FFMA/clk/SM x 152 SMs x max SM clock "
                                 "(probe: 74.7 TFLOP/s); a latency-bound serial chain, each "
                                 "algorithmic multiply-add costs ~15 float-float operations"})
    else:
        mult, unit, scale = 1.0, "GFLOP/s", 1e9
        peak = FP64_FLOP_PER_CLK_PER_SM * SM_COUNT * sm_max * 1e6 / 1e9
        note = ("FP64 FMA pipe: 2 DFMA/clk/SM x 152 SMs x max SM clock "
                "(probe: 1.19 TFLOP/s at 1.96 GHz)")
        if precision == "fp64x2":
            note += ("; achieved counts algorithmic multiply-adds, each of which costs ten "
                     "FP64 operations in double-double")
        out.update({"bound": "alu", "peak_note": note})
    in_launch = mult * flops / (ms * 1e-3) / scale if ms > 0 else 0.0
    out["in_launch"] = {"launches_timed": n, "avg_launch_us": avg_us, "busy_ms": ms,
                        "achieved": in_launch, "frac": in_launch / peak if peak else None,
                        "over": "union of the timed launches' intervals (instrumented solves)"}
    if kind == "history" and w is not None and step_ms:
        solve_flops = 2.0 * w.history_macs()
        achieved = mult * solve_flops / (step_ms * 1e-3) / scale
        out.update({"achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak if peak else None,
                    "work_per_step": mult * solve_flops,
                    "achieved_over": "whole uninstrumented solve: algorithmic history work "
                                     "(2 N^2 flops per column) / ms_per_step"})
    else:
        out.update({"achieved": in_launch, "peak": peak, "unit": unit,
                    "frac": in_launch / peak if peak else None,
                    "achieved_over": out["in_launch"]["over"]})
    key = {"history": f"history_{'split' if precision == 'split' else 'fp64'}",
           "recurrence": "recurrence_split" if precision == "split" else "recurrence"}.get(kind)
    # profiles/<kernel class>_<precision>_<workload>.md, e.g. history_fp64_lorenz-single.md
    traffic = _profile_traffic(key, f"{kind}_{precision}_{workload}") if key else None
    out["traffic"] = traffic
    return out


def fp64_comparator(steps, warmup):
    """The plain FP64 single-trajectory solve (Lorenz-type, alpha 0.98,
    h 5e-4, N 2^18) timed the same way as the headline: the path the batched
    split solve is compared with."""
    import torch

    import paper_1710_01133_gb300 as fabm
    w = wl.lorenz_single()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out_dev = torch.empty((w.B, w.N + 1, w.dim), dtype=torch.float64, device="cuda")
    with fabm.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64") as s:
        for _ in range(warmup):
            s.solve_batch(w.y0, out=out_dev)
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.solve_batch(w.y0, out=out_dev)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    return {"workload": w.name, "precision": "fp64", "trajectories": w.B, "steps_N": w.N,
            "value": w.steps_traj() / (ms * 1e-3), "unit": "steps*traj/s", "ms_per_step": ms,
            "steps": steps, "warmup": warmup}


def cpu_baseline(w, target_s=12.0):
    """The oracle on a prefix of the workload (1 trajectory, or as many
    trajectories as the host has cores), extrapolated to the full workload by
    sum N^2; returns a dict for the JSON line."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    ntraj = 1 if w.B == 1 else min(w.B, cores)
    sub = w.subset(np.arange(ntraj))
    # calibrate on a short prefix, then size the sample for ~target_s
    n0 = min(w.N, 2000)
    t0 = time.perf_counter()
    oracle.solve_batch(sub.rhs, sub.alpha, sub.h, n0, sub.y0, params=sub.params,
                       traj_params=sub.traj_params, threads=ntraj)
    dt0 = max(time.perf_counter() - t0, 1e-4)
    n = int(min(w.N, n0 * np.sqrt(target_s / dt0)))
    t0 = time.perf_counter()
    oracle.solve_batch(sub.rhs, sub.alpha, sub.h, n, sub.y0, params=sub.params,
                       traj_params=sub.traj_params, threads=ntraj)
    dt = time.perf_counter() - t0
    full_time = dt * (w.N / n) ** 2 * (w.B / ntraj)
    line = {"value": w.steps_traj() / full_time, "unit": "steps*traj/s", "cores": ntraj,
            "kind": "oracle",
            "sample": f"{ntraj} trajectory(ies) x first {n} of {w.N} steps in {dt:.2f} s, "
                      f"extrapolated to {w.B} x {w.N} by N^2 (host has {cores} cores)",
            "history_gmac_s": w.history_macs() / full_time / 1e9}
    if w.B == 1 and np.ndim(w.alpha) == 0 and w.alpha <= 1.0 and cores > 1:
        # the paper's Alg. 2 layout for reference: the k-sums of every step split
        # over the host's threads, same sample
        threads = min(cores, 16)
        t0 = time.perf_counter()
        oracle.solve_threaded(sub.rhs, sub.alpha, sub.h, n, sub.y0[0], params=sub.params,
                              threads=threads)
        dtt = time.perf_counter() - t0
        ft = dtt * (w.N / n) ** 2
        line["threaded_k"] = {"value": w.steps_traj() / ft, "threads": threads,
                              "sample": f"first {n} steps in {dtt:.2f} s, extrapolated by N^2"}
    return line


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    ntraj = 1 if w.B == 1 else min(w.B, cores)
    sub = w.subset(np.arange(ntraj))
    n0 = min(w.N, 2000)
    t0 = time.perf_counter()
    oracle.solve_batch(sub.rhs, sub.alpha, sub.h, n0, sub.y0, params=sub.params,
                       traj_params=sub.traj_params, threads=ntraj)
    dt0 = max(time.perf_counter() - t0, 1e-4)
    n = int(min(w.N, n0 * np.sqrt(4.0 / dt0)))  # ~4 s per step
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve_batch(sub.rhs, sub.alpha, sub.h, n, sub.y0, params=sub.params,
                           traj_params=sub.traj_params, threads=ntraj)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    dt = float(np.mean(times))
    full_time = dt * (w.N / n) ** 2 * (w.B / ntraj)
    value = w.steps_traj() / full_time
    line = {
        "impl": "reference", "metric": "steps_traj_per_s", "value": value,
        "unit": "steps*traj/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": full_time * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w, args),
        "history_gmac_s": w.history_macs() / full_time / 1e9,
        "cpu_baseline": {"value": value, "unit": "steps*traj/s", "cores": ntraj,
                         "kind": "oracle",
                         "sample": f"each step: {ntraj} trajectory(ies) x first {n} of {w.N} "
                                   f"steps ({dt:.2f} s), extrapolated by N^2"},
        "e2e": {"value": value, "unit": "steps*traj/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_served(args):
    """Served mixed stream: requests of fabm_workloads.served_stream submitted
    at their arrival times to a fabm server while it steps; throughput over the
    whole stream and arrival-to-result latency percentiles.  The arrival rate is
    0.8 x the capacity measured first with every request queued at t = 0."""
    import torch

    import paper_1710_01133_gb300 as fabm
    fabm.load()
    torch.cuda.set_device(0)
    n = args.n_requests
    k_hi = args.k_max

    def serve(reqs, rate_label):
        with fabm.Server(120 << 30, precision=args.precision) as srv:
            t0 = time.perf_counter()
            pending = list(reqs)
            inflight = {}
            lat = []
            nxt = 0
            while nxt < len(pending) or inflight:
                now = time.perf_counter() - t0
                while nxt < len(pending) and pending[nxt].arrival <= now:
                    r = pending[nxt]
                    tk = srv.submit(r.rhs, r.dim, r.alpha, r.h, r.N, r.y0, r.params)
                    inflight[tk] = r
                    nxt += 1
                if not inflight:
                    time.sleep(max(0.0, pending[nxt].arrival - now))
                    continue
                srv.step()
                now = time.perf_counter() - t0
                done = srv.finished()
                for tk in done:
                    r = inflight.pop(tk)
                    srv.result(tk)
                    lat.append(now - r.arrival)
            wall = time.perf_counter() - t0
            st = srv.stats()
        steps = sum(r.N for r in reqs)
        macs = sum(float(r.N) ** 2 * r.dim for r in reqs)
        return {"rate": rate_label, "wall_s": wall, "steps_traj_per_s": steps / wall,
                "history_gmac_s": macs / wall / 1e9,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "server_steps": st["steps"],
                "gpu_launches": st["launches"]}

    burst = wl.served_stream(n=n, rate=1e12, k_hi=k_hi)
    serve(wl.served_stream(n=min(n, 64), rate=1e12, k_hi=min(k_hi, 12)), "warmup")
    cap = serve(burst, "all at t=0")
    rate = 0.8 * n / cap["wall_s"]
    timed = serve(wl.served_stream(n=n, rate=rate, k_hi=k_hi), f"{rate:.1f}/s")
    line = {
        "metric": "steps_traj_per_s", "value": timed["steps_traj_per_s"], "unit": "steps*traj/s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": timed["wall_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32c" if args.precision == "split" else "f64",
        "data": "synthetic",
        "config": {"workload": f"served-mix-{n}req-k12..{k_hi}", "precision": args.precision,
                   "requests": n, "arrival_rate_per_s": rate, "hbm_budget_gb": 120},
        "history_gmac_s": timed["history_gmac_s"],
        "latency_ms": {"p50": timed["p50_ms"], "p99": timed["p99_ms"]},
        "capacity_run": cap, "gpu_launches": timed["gpu_launches"],
    }
    print(json.dumps(line))


def _config(w, args):
    return {"workload": w.name, "precision": args.precision,
            "history_kernel": getattr(args, "history", "auto"), "rhs": w.rhs, "dim": w.dim,
            "alpha": w.alpha, "h": w.h, "steps_N": w.N, "trajectories": w.B,
            "l2": "flushed between timed solves (256 MiB write)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fabm", choices=["fabm", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + ["served-mix"])
    ap.add_argument("--precision", default=None, choices=["fp64", "split", "fp64x2"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-steps", type=int, default=None,
                    help="override the workload's N (small cases for profiling)")
    ap.add_argument("--n-traj", type=int, default=None,
                    help="keep only the first n trajectories of the workload")
    ap.add_argument("--timing-period", type=int, default=128,
                    help="time the kernel launches of every k-th time block")
    ap.add_argument("--n-requests", type=int, default=2000, help="served-mix: requests")
    ap.add_argument("--autotune", type=int, default=0, metavar="N_PROBE",
                    help="before the warm-up, let the library's autotuner pick the history "
                         "kernel settings on solves truncated to N_PROBE steps (0: off)")
    ap.add_argument("--k-max", type=int, default=14, help="served-mix: N = 2^k, k <= k_max")
    ap.add_argument("--recurrence", default="auto", choices=["auto", "columns", "targets"],
                    help="split precision, tensor history: layout of the recurrence")
    ap.add_argument("--history", default="auto",
                    choices=["auto", "tensor", "tensor-wide", "fp32c", "fp64", "fp64-persist", "x2"],
                    help="history kernel (auto: the library's choice)")
    ap.add_argument("--no-fp64-comparator", action="store_true",
                    help="skip timing the plain FP64 single-trajectory solve (vs_fp64_path)")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="end-to-end solves timed (at most --steps; 0: no end-to-end leg)")
    ap.add_argument("--stat-solves", type=int, default=2,
                    help="instrumented solves for the per-launch kernel statistics (0: none)")
    args = ap.parse_args()
    if args.workload == "served-mix":
        if args.precision is None:
            args.precision = "split"
        run_served(args)
        return
    w = WORKLOADS[args.workload]()
    if args.n_steps is not None or args.n_traj is not None:
        idx = np.arange(min(args.n_traj or w.B, w.B))
        w = w.subset(idx, N=args.n_steps or w.N)
    if args.precision is None:
        args.precision = w.precision
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist

    import paper_1710_01133_gb300 as fabm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fabm.load()
    solver = fabm.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision=args.precision,
                         recurrence=args.recurrence,
                         history=None if args.history == "auto" else args.history)
    wstats = solver.kernel_stats()["weights"]
    tuned = None
    if args.autotune > 0:
        tuned = solver.autotune(w.y0, traj_params=w.traj_params, n_probe=args.autotune)

    out_dev = torch.empty((w.B, w.N + 1, w.dim), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def solve_dev():
        solver.solve_batch(w.y0, traj_params=w.traj_params, N_each=w.N_each, out=out_dev)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # the warm-up runs the launch sequence that is timed (its CUDA graph is
    # built here, not inside the timed region); the timed solves carry no
    # per-launch instrumentation
    solver.set_timing(0)
    for _ in range(args.warmup):
        solve_dev()
    barrier()

    launches = 0
    times = []
    with ClockSampler(_gpu_index(local)) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            solve_dev()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            launches += solver.last_launch_count
    barrier()
    # per-kernel statistics for the roofline: the same solve with CUDA events
    # around the launches of the sampled blocks, run after the timed ones
    stat_solves = min(args.steps, args.stat_solves)
    if stat_solves > 0:
        solver.set_timing(args.timing_period)
        solve_dev()  # builds the instrumented graph
        solver.set_timing(args.timing_period)  # resets the counters
        for _ in range(stat_solves):
            flush.fill_(1.0)
            solve_dev()
    barrier()
    kstats = solver.kernel_stats()
    solver.set_timing(0)
    step_ms = dist_max(float(np.mean(times)), "cuda")

    # end to end: host y0 in, host trajectory out (pinned), copies timed
    e2e_times = []
    e2e_steps = min(args.steps, args.e2e_steps)
    out_host = None
    if e2e_steps > 0:
        out_host = torch.empty((w.B, w.N + 1, w.dim), dtype=torch.float64, pin_memory=True)
        solver.solve_batch(w.y0, traj_params=w.traj_params, N_each=w.N_each, out=out_host)
    barrier()
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        solver.solve_batch(w.y0, traj_params=w.traj_params, N_each=w.N_each, out=out_host)
        e1.record()
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = dist_max(float(np.mean(e2e_times)), "cuda") if e2e_times else None
    finite = bool(torch.isfinite(out_dev).all().item())
    del out_host
    comparator = None
    if not args.no_fp64_comparator and not (args.workload == "lorenz-single"
                                            and args.precision == "fp64"):
        comparator = fp64_comparator(max(3, min(args.steps, 5)), 3)

    if rank == 0:
        units = w.steps_traj() * ws  # replicas: every rank solves its own copy
        clocks = clk.summary()
        # the kinds that do the method's arithmetic (both are timed on the same
        # sampled blocks; combine, slice and init only move or convert data)
        dom = max(("history", "recurrence"), key=lambda k: kstats[k]["busy_ms"] or kstats[k]["ms"])
        line_roof = roofline(dom, kstats[dom], args.precision, clocks, args.workload, w, step_ms)
        h2d = w.B * w.dim * 8 + w.B * 8 * 8 + w.B * 8
        d2h = w.B * (w.N + 1) * w.dim * 8 + 8
        line = {
            "metric": "steps_traj_per_s",
            "value": replica_throughput(w.steps_traj(), ws, step_ms),
            "unit": "steps*traj/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": DTYPE_OF_HISTORY.get(solver.last_history_kernel, "f64"),
            "data": "synthetic",
            "config": _config(w, args),
            "history_gmac_s": w.history_macs() * ws / (step_ms * 1e-3) / 1e9,
            "roofline": line_roof,
            "kernels": {k: {"timed_launches": v["launches"], "ms": round(v["ms"], 3),
                            "busy_ms": round(v["busy_ms"], 3)}
                        for k, v in kstats.items() if k != "weights"},
            "kernel_timing": f"CUDA events around the launches of every "
                             f"{args.timing_period}th time block (of the 8 blocks from it "
                             f"when history launches overlap on two streams), in "
                             f"{min(args.steps, 2)} instrumented solves after the timed ones "
                             f"(the timed solves carry no events)",
            "weights_ms": wstats["ms"],
            "e2e": None if e2e_ms is None else {
                "value": replica_throughput(w.steps_traj(), ws, e2e_ms), "unit": "steps*traj/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks,
            "autotune": None if tuned is None else {
                "n_probe": args.autotune,
                "candidates_predicted_ms_kernel_setting": [[round(m, 3), k, c] for m, k, c in tuned],
                "recurrence_warps": fabm.fabm_get_recurrence_warps(solver.handle)},
            "output_finite": finite,
        }
        if comparator is not None:
            comparator["ratio"] = line["value"] / comparator["value"]
            line["vs_fp64_path"] = comparator
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line))
    solver.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
