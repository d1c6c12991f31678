#!/usr/bin/env python
"""Benchmark: eigvalsh TFLOP/s (nominal 4n^3/3 flops) on one GB300.

Workload (default): n = 16384, mixed precision (FP32 data, tensor-core
trailing update, FP64 Householder norms/tau/beta and FP64 Sturm recurrence),
A = Q diag(D) Q^T with D geometrically spaced over 1e-6..1 in magnitude with
random signs and 16-fold clusters of gap 1e-10, Q from the QR of a seeded
N(0,1) matrix; first half-bandwidth b0 = 128, band schedule from b0 down to 1
chosen by the library's autotuner (sev_autotune, run once before the
warm-up; --no-tune keeps the fixed rule 128 -> 32 -> 16 -> 1).
A step is one sev_eigvalsh call (full-to-band, every band-to-band stage,
bisection).  The FP64 form of the same matrix is timed beside it.

Output: one JSON line on rank 0 (see the keys below).  --impl reference
times the CPU oracle on a bounded sample of the same workload instead.
Multi-GPU (torchrun): independent replicas, one matrix per rank (the
single-matrix path does not shard); value aggregates all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigvalsh TFLOP/s (4n^3/3 nominal) at n=16384, mixed precision"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--b0", type=int, default=128)
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-form timing")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the batched workloads")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the autotuning call: the library's own schedule (a tuned one from SEV_TUNE_CACHE, "
                        "else the fixed rule)")
    p.add_argument("--no-free-b0", action="store_true", help="skip the comparison run at the library's own b0")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock / power / throttle reasons."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def nominal_flops(n):
    return 4.0 * n ** 3 / 3.0


def panel_sizes(n, b):
    out = []
    k = 0
    while True:
        r0 = (k + 1) * b
        if r0 >= n or n - r0 < 2:
            break
        out.append(n - r0)
        k += 1
    return out


def schedule(b0, elem=4):
    """The library's band schedule (see api.cu): b <= 16 -> 1, b >= 128 ->
    32, other multiples of 16 -> 16, else the widest supported divisor."""
    def tri(b):
        return b in (2, 4, 8, 16) or (b == 32 and elem == 4)
    s = [b0]
    while s[-1] > 1:
        b = s[-1]
        nxt = 1 if b % 2 else b // 2
        if b <= 16 and tri(b):
            nxt = 1
        elif b >= 128 and b % 32 == 0:
            nxt = 32
        elif b > 16 and b % 16 == 0:
            nxt = 16
        elif tri(b):
            nxt = 1
        else:
            w = 16
            while w >= 2:
                if tri(w) and b % w == 0 and w < b:
                    nxt = w
                    break
                w //= 2
        s.append(nxt)
    return s


def kernel_model(name, n, b0, elem, sched=None):
    """Algorithmic work of one step for a kernel: (amount, unit, bound).

    syr2k / symm: 2 N^2 b flops per panel (lower triangle, both products).
    band stages b -> h (k = b/h): each of the n/h sweeps reads and writes the
    2b stored diagonals of the columns it passes, ~2 s 2b (n - ih) bytes, so
    2 s k n^2 bytes per stage; the b -> 1 stage is k = b.
    tree-QR nodes: 2(2b)b^2 - (2/3)b^3 flops per stacked-triangle QR (the
    dense count; the kernel skips the structural zeros); leaves of at most
    256 rows, so ceil(N/256) - 1 nodes per panel.
    bisection: n eigenvalues x iterations x n Sturm steps (the per-eigenvalue
    definition; each step is three FP64 instructions, division-free).
    """
    Ns = panel_sizes(n, b0)
    if sched is None:
        sched = schedule(b0, elem)
    if name in ("syr2k", "syr2k_tc"):
        flops = sum(2.0 * N * (N + 1) * b0 for N in Ns)
        return flops, "flop", "tensor" if name.endswith("_tc") else "alu"
    if name == "symm":
        flops = sum(2.0 * N * N * b0 for N in Ns)
        return flops, "flop", "alu"
    if name == "band_tri":
        b1 = sched[-2]
        return 2.0 * elem * b1 * float(n) ** 2, "byte", "hbm"
    if name == "band_chase":
        tot = 0.0
        for b, h in zip(sched[:-1], sched[1:]):
            if h == 1 and (b in (2, 4, 8, 16) or (b == 32 and elem == 4)):
                continue
            tot += 2.0 * elem * (b // h) * float(n) ** 2
        return tot, "byte", "hbm"
    if name == "tsqr_node_qr":
        nodes = sum(max(-(-N // 256) - 1, 0) for N in Ns)
        return nodes * (4.0 * b0 ** 3 - 2.0 * b0 ** 3 / 3.0), "flop", "alu"
    if name == "bisect":
        rtol = 1e-9 if elem == 4 else 1e-14
        iters = math.ceil(math.log2(2.0 / rtol)) + 1
        return float(n) * n * iters, "sturm_step", "alu"
    return None, None, None


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per step of a
# kernel, taken by ncu at this benchmark's configuration (n = 16384, b0 = 128,
# the schedule named) for the kernel as it is built now; a kernel or schedule
# absent here reports null.
MEASURED_TRAFFIC = {
    "band_chase": {"schedule": [128, 32, 8, 1], "bytes_per_step": 16848640 + 5070080 + 5244672 + 1515776,
                   "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the two band_chase launches of one "
                           "eigvalsh (128 -> 32 on clusters: 21.9 MB; 32 -> 8: 6.8 MB), 1 pass, full size: the 16 MB "
                           "band is read about once and stays in L2"},
}


def roofline(name, amount, unit, bound, ms_per_step, peaks, clocks, elem):
    if amount is None or ms_per_step <= 0:
        return None
    sec = ms_per_step / 1e3
    mhz = (clocks or {}).get("sm_mhz") or 1900.0
    if unit == "flop" and bound == "tensor":
        bf16 = peaks.get("bf16_tflops_sustained") or 1713.1
        peak = bf16 / 3.0  # BF16x3: three bf16 products per useful FP32-class product
        ach = amount / sec / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_note": "of measured: bf16 sustained / 3 (BF16x3 useful flops)"}
    if unit == "flop":
        # SIMT FMA: FP32 152 SMs x 128 FMA/clk x 2; FP64 152 x 2 DFMA/clk x 2
        per_clk = 152 * (128 if elem == 4 else 2) * 2
        peak = per_clk * mhz * 1e6 / 1e12
        ach = amount / sec / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_note": "unit counts x median SM clock"}
    if unit == "byte":
        peak = peaks.get("hbm_gbs") or 6762.3
        ach = amount / sec / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_note": "of measured"}
    if unit == "sturm_step":
        # three FP64 instructions per (division-free) Sturm step; the FP64 pipe
        # issues 2 instructions per SM per clock (152 SMs)
        peak = 152 * 2 * mhz * 1e6 / 3.0 / 1e9
        ach = amount / sec / 1e9
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gstep/s", "frac": ach / peak,
                "peak_note": "unit counts x median SM clock: 2 FP64 instructions per SM per clock, 3 per step"}
    return None


# ---------------------------------------------------------------- oracle leg
def host_cores():
    """Cores this process may run on (read at run time)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(A64_host, n, rtol, seconds, steps_cap=None, omp=False):
    """Time the CPU oracle on a bounded sample of the workload and
    extrapolate: the first m Householder steps of the tridiagonalisation of
    A (step j costs ~(n-1-j)^2) and k of the n bisections (equal cost each).
    omp: the oracle's OpenMP build on every core (same results; None if the
    compiler has no OpenMP runtime)."""
    import numpy as np

    import oracle

    oracle.build()
    if omp and oracle.load_omp() is None:
        return None
    budget_tri = 0.8 * seconds
    # per-step estimate from one step
    M = np.asfortranarray(A64_host.T)  # symmetric: the transpose is the same matrix, F-ordered view
    M = np.array(M, order="F", copy=True)
    d = np.zeros(n)
    e = np.zeros(n)
    t0 = time.perf_counter()
    oracle.tridiagonalize_inplace(M, d, e, 1, omp=omp)
    t1 = time.perf_counter() - t0
    m = max(1, min(n - 2, int(budget_tri / max(t1, 1e-6))))
    if steps_cap:
        m = min(m, steps_cap)
    M = np.array(np.asfortranarray(A64_host.T), order="F", copy=True)
    t0 = time.perf_counter()
    oracle.tridiagonalize_inplace(M, d, e, m, omp=omp)
    t_m = time.perf_counter() - t0
    del M
    w = (np.arange(n - 1, 1, -1, dtype=np.float64)) ** 2  # (n-1-j)^2, j = 0..n-3
    t_tri = t_m * w.sum() / w[:m].sum()
    rng = np.random.default_rng(1)
    dd, ee = rng.standard_normal(n), rng.standard_normal(n - 1)
    k = 8
    t0 = time.perf_counter()
    oracle.bisect_range(dd, ee, 0, k, rtol, omp=omp)
    tk = time.perf_counter() - t0
    k = max(8, min(n, int(0.2 * seconds / max(tk / 8, 1e-9))))
    t0 = time.perf_counter()
    oracle.bisect_range(dd, ee, n // 2 - k // 2, n // 2 - k // 2 + k, rtol, omp=omp)
    t_k = time.perf_counter() - t0
    t_bis = t_k * n / k
    total = t_tri + t_bis
    return {
        "cores": host_cores() if omp else 1,
        "seconds_extrapolated": total,
        "value": nominal_flops(n) / total / 1e12,
        "sample": "first %d of %d Householder steps of the oracle tridiagonalisation of the workload matrix "
                  "(%.2f s, extrapolated by (n-1-j)^2) + %d of %d bisections (rtol %.0e, %.2f s, x n/k)"
                  % (m, n - 2, t_m, k, n, rtol, t_k),
        "measured_seconds": t_m + t_k,
    }


def gen_workload(n, device):
    import torch

    from paper_1604_03703_gb300 import inputs as I

    D = I.workload_clustered_d(n)
    A64 = I.qdq_torch(D, I.SEED_BASE + 2, device)
    torch.cuda.synchronize()
    return A64, D


def time_plan(plan, work, orig, reps=3):
    """Device time of plan.run() (CUDA events), median of reps; the inputs
    are restored before every run, outside the events."""
    import torch

    times = []
    for _ in range(reps):
        for w, o in zip(work, orig):
            w.copy_(o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def time_plan_graph(plan, work, orig, reps=20):
    """The plan captured once in a CUDA graph, then replayed reps times: the
    median device time of one replay (CUDA events on the replay stream); the
    inputs are restored before every replay, outside the events."""
    import torch

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture
        plan.run()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        for w, o in zip(work, orig):
            w.copy_(o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    del g
    return statistics.median(times)


def max_over_ranks(ms, world, device):
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def bench_batched(h, device, args, rank=0, world=1):
    """The two batched workloads, FP64 and mixed: matrices per second of one
    plan run (one persistent launch for the small matrices; the SCF-like
    orders run the single-matrix path one after another).  With N ranks each
    takes its LPT shard of the batch (no data-path collective); the time is
    the slowest rank's."""
    import torch

    from paper_1604_03703_gb300 import _lib
    from paper_1604_03703_gb300 import inputs as I
    from paper_1604_03703_gb300 import shard

    out = {}
    host_all = I.batch_small()
    part = shard.lpt_partition([A.shape[0] for A in host_all], world)[rank]
    host = [host_all[i] for i in part]
    del host_all
    sizes = [A.shape[0] for A in host]
    small = {"workload": "4096 symmetric N(0,1)/sqrt(n) matrices, n uniform in 32..512", "count": 4096,
             "sharding": "lpt over %d rank(s)" % world}
    for name, dt, prec in (("mixed", torch.float32, _lib.SEV_MIXED), ("fp64", torch.float64, _lib.SEV_FP64)):
        b = h.batch_autotune(sizes, prec)
        orig = [torch.from_numpy(A).to(dt).to(device) for A in host]
        work = [t.clone() for t in orig]
        outs = [torch.empty(t.shape[0], dtype=torch.float64, device=device) for t in orig]
        plan = h.batch_plan(work, outs, b)
        ms = max_over_ranks(time_plan_graph(plan, work, orig, 20), world, device)
        h.raise_device_error("batched " + name)
        plan.close()
        small[name] = {"ms": ms, "mats_per_s": 4096 / (ms / 1e3), "b": b, "launches": 1,
                       "timing": "median of 20 replays of the plan captured in a CUDA graph"}
        del orig, work, outs
        torch.cuda.empty_cache()
    small["mixed_speedup"] = small["fp64"]["ms"] / small["mixed"]["ms"]
    out["small"] = small
    scf = {"workload": "64 SCF-like matrices A0(n) + 1e-3 E, n uniform in 1024..6144, D uniform in [-10, 10]",
           "count": 64}
    part = shard.lpt_partition([int(m) for m in I.batch_sizes(64, 1024, 6144, I.SEED_BASE + 4)], world)[rank]
    mats = [A for k, A in enumerate(I.batch_scf_torch(64, device=device)) if k in set(part)]
    for name, dt in (("mixed", torch.float32), ("fp64", torch.float64)):
        orig = [A.to(dt) for A in mats]
        work = [t.clone() for t in orig]
        outs = [torch.empty(t.shape[0], dtype=torch.float64, device=device) for t in orig]
        plan = h.batch_plan(work, outs, 0)
        ms = max_over_ranks(time_plan(plan, work, orig, reps=1), world, device)
        h.raise_device_error("scf " + name)
        plan.close()
        scf[name] = {"ms": ms, "mats_per_s": 64 / (ms / 1e3)}
        del orig, work, outs
        torch.cuda.empty_cache()
    scf["mixed_speedup"] = scf["fp64"]["ms"] / scf["mixed"]["ms"]
    out["scf"] = scf
    del mats
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------- arms
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import torch

    n = args.n
    torch.cuda.set_device(local)
    A64, D = gen_workload(n, "cuda:%d" % local)
    A_host = A64.cpu().numpy()
    del A64
    torch.cuda.empty_cache()
    rtol = 1e-9
    per = max(2.0, min(args.cpu_seconds, 20.0) / 3)
    vals, last = [], None
    for s in range(args.warmup + args.steps):
        r = oracle_sample(A_host, n, rtol, per)
        if s >= args.warmup:
            vals.append(r["value"])
            last = r
    value = statistics.median(vals)
    ms = nominal_flops(n) / (value * 1e12) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "eigvalsh n=%d clustered QDQ^T spectrum (CPU oracle, bounded sample)" % n,
                   "n": n, "b0": args.b0},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": last["sample"]},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1604_03703_gb300 import _lib, api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = "cuda:%d" % local
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(device))
    n, b0 = args.n, args.b0
    A64, D = gen_workload(n, device)
    Dmax = float(np.abs(D).max())
    A_host64 = A64.cpu().numpy() if rank == 0 else None
    A0 = A64.float()
    if args.no_fp64:
        del A64
        A64 = None
    torch.cuda.empty_cache()
    A = torch.empty_like(A0)
    h = api.Handle(local)
    lam = torch.empty(n, dtype=torch.float64, device=device)

    def barrier():
        if world > 1:
            dist.barrier()

    # the band schedule: measured per stage at this order by the library's
    # autotuner (untimed, once per process), for the fixed b0 and for a free b0
    tune = None
    if not args.no_tune:
        t0 = time.perf_counter()
        free_bands, free_pred = h.autotune(n, _lib.SEV_MIXED, 0)
        t1 = time.perf_counter()
        fixed_bands, fixed_pred = h.autotune(n, _lib.SEV_MIXED, b0)
        t2 = time.perf_counter()
        h.raise_device_error("autotune")
        tune = {"b0_%d" % b0: {"schedule": fixed_bands, "predicted_ms": fixed_pred, "tuning_s": t2 - t1},
                "free_b0": {"schedule": free_bands, "predicted_ms": free_pred, "tuning_s": t1 - t0}}
    sched = h.eigvalsh_bands(n, b0, _lib.SEV_MIXED)
    sched_free = h.eigvalsh_bands(n, 0, _lib.SEV_MIXED)

    # warm-up
    for _ in range(max(args.warmup, 3)):
        A.copy_(A0)
        h.eigvalsh(A, b0, out=lam)
    torch.cuda.synchronize()
    h.raise_device_error("warm-up")
    # one untimed profiling step: per-kernel totals and launch counts
    h.set_kernel_timing(True)
    A.copy_(A0)
    h.eigvalsh(A, b0, out=lam)
    prof = h.kernel_times()
    h.set_kernel_timing(False)
    launches_per_step = sum(c for _, c in prof.values())
    dominant = max(prof, key=lambda k: prof[k][0])

    # timed region: K steps; only the dominant kernel's launches are bracketed
    h.set_kernel_timing(dominant)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        A.copy_(A0)  # restore the input the previous step overwrote (outside the step's events)
        ev[s][0].record()
        h.eigvalsh(A, b0, out=lam)
        ev[s][1].record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    dom_ms, dom_cnt = h.kernel_times().get(dominant, (0.0, 0))
    h.set_kernel_timing(False)
    h.raise_device_error("timed steps")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_per_step = tot_ms / args.steps
    value = world * nominal_flops(n) / (ms_per_step / 1e3) / 1e12
    lam_np = lam.cpu().numpy()
    err = float(np.abs(np.sort(lam_np) - D).max() / Dmax)

    # the library's own choice of band width (b0 = 0: the tuned b0), same matrix
    auto = None
    if not args.no_free_b0:
        ea = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        A.copy_(A0)
        h.eigvalsh(A, 0, out=lam)
        for e0, e1 in ea:
            A.copy_(A0)
            e0.record()
            h.eigvalsh(A, 0, out=lam)
            e1.record()
        torch.cuda.synchronize()
        h.raise_device_error("default b0")
        a_ms = min(e0.elapsed_time(e1) for e0, e1 in ea)
        a_err = float(np.abs(np.sort(lam.cpu().numpy()) - D).max() / Dmax)
        auto = {"b0": sched_free[0], "schedule": sched_free, "ms_per_step": a_ms,
                "tflops": nominal_flops(n) / (a_ms / 1e3) / 1e12, "max_err_vs_D": a_err}

    # end to end through the host-buffer entry point (H2D + solve + D2H)
    e2e = None
    if not args.no_e2e:
        A_pin = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        A_pin.copy_(A0.cpu())
        out = torch.empty(n, dtype=torch.float64)
        h.eigvalsh_host(A_pin, b0, out=out)  # warm (allocates the staging buffer)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h.eigvalsh_host(A_pin, b0, out=out)
        dt = (time.perf_counter() - t0) / args.steps
        e2e = {"value": world * nominal_flops(n) / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 4 * n * n, "d2h_bytes_per_step": 8 * n, "ms_per_step": dt * 1e3}
        del A_pin

    # the FP64 form on the same matrix (one warm-up + one timed call)
    fp64 = None
    if A64 is not None:
        del A0, A
        torch.cuda.empty_cache()
        A = torch.empty_like(A64)
        A.copy_(A64)
        h.eigvalsh(A, 64, out=lam)
        torch.cuda.synchronize()
        A.copy_(A64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.eigvalsh(A, 64, out=lam)
        e1.record()
        torch.cuda.synchronize()
        h.raise_device_error("fp64")
        f_ms = e0.elapsed_time(e1)
        f_err = float(np.abs(np.sort(lam.cpu().numpy()) - D).max() / Dmax)
        fp64 = {"eigvalsh_s": f_ms / 1e3, "tflops": nominal_flops(n) / (f_ms / 1e3) / 1e12, "b0": 64,
                "max_err_vs_D": f_err, "mixed_speedup": f_ms / ms_per_step}

    batched = None
    if not args.no_batched:
        del A
        torch.cuda.empty_cache()
        batched = bench_batched(h, device, args, rank, world)

    peaks = measured_peaks()
    amount, unit, bound = kernel_model(dominant, n, b0, 4, sched)
    dom_ms_step = dom_ms / args.steps if dom_ms else prof[dominant][0]
    roof = roofline(dominant, amount, unit, bound, dom_ms_step, peaks, clk, 4)
    if roof is not None:
        roof["kernel"] = dominant
        traffic = MEASURED_TRAFFIC.get(dominant) if (n, b0) == (16384, 128) else None
        if traffic and traffic.get("schedule") != list(sched):
            traffic = None
        roof["traffic"] = traffic["bytes_per_step"] if traffic else None
        if traffic:
            roof["traffic_note"] = traffic["note"]
        roof["launches_per_step"] = prof[dominant][1]
        roof["ms_per_step"] = dom_ms_step

    cpu = None
    if rank == 0 and world == 1:
        one = oracle_sample(A_host64, n, 1e-9, args.cpu_seconds / 2)
        allc = oracle_sample(A_host64, n, 1e-9, args.cpu_seconds / 2, omp=True)
        cpu = {"value": one["value"], "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": one["sample"]}
        if allc is not None:
            cpu["all_cores"] = {"value": allc["value"], "unit": "TFLOP/s", "cores": allc["cores"], "kind": "oracle",
                                "sample": allc["sample"] + " (OpenMP build: same results, independent loops on "
                                                           "every core)"}

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16x3+f64", "data": "synthetic",
        "config": {"workload": "eigvalsh n=%d, A = Q diag(D) Q^T, D geometric 1e-6..1 with random signs and "
                               "16-fold clusters (gap 1e-10), FP32 data, bands %s" % (n, "->".join(map(str, sched))),
                   "n": n, "b0": b0, "schedule": sched, "autotune": tune, "parallelism": "replicas" if world > 1 else "single",
                   "precision": "mixed: FP32 data and FP32 arithmetic, BF16x3 tensor-core trailing update "
                                "(FP32 accumulation), pair-float Householder scalars, FP64 Sturm counts",
                   "l2": "inputs larger than L2 (1 GiB matrix per step); input restore excluded from step events"},
        "max_err_vs_D": err,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk,
        "fp64": fp64,
        "default_b0": auto,
        "batched": batched,
        "kernels_ms_per_step": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
