#!/usr/bin/env python
"""Benchmark of the k-center farthest-point hot path on GB300.

Headline workload: GON (Section 3.1) with k = 1024 on n = 8,000,000 points in
d = 64, a mixture of 100 isotropic Gaussians (sigma 0.5, means uniform in
[-10, 10]^64), FP32, seed 4: the largest single-GPU configuration of the
Gonzalez + EIM precision workload.  One step = one kc_gonzalez call through
the C ABI (pack, the persistent k-step kernel, the FP64 radius recheck).

Metric: point-center distance evaluations per second (k sweeps of n points
per solve), whole job over all ranks.  `value` is device-timed with the
points resident in HBM (CUDA events around every step; the 2 GB point set is
larger than L2, so no flush is needed); `e2e` is the same metric with the
points in pinned host memory passed to the C ABI, host-to-device traffic and
result read-back inside the wall-clock timed region.  The same line carries
the mixed-precision comparison of the metric ("mixed"): the bf16 sweep
against the FP32 sweep on this workload (identical selections checked), and
the 4,096-instance batch (bf16 sweep, one CUDA-graph replay) against one
FP32 kc_gonzalez call per instance and against the FP32 batch.

Under torchrun (N > 1) every rank solves its own independent instance of the
workload (seed 4 + 1000 * rank): weak scaling, no collective on the data path.

--impl reference times the CPU oracle as it stands on all host cores: one
worker process per core, each running the oracle's GON on its contiguous
shard of the same point set (first 32 centers per shard), per step.

--workload NAME measures one of the other paths (one JSON line with the same
keys): GON + radius on 1M x 10 (L2-resident, against the measured L2 read
peak), GON / MRG on 10M x 16, tensor-core radius / EIM on 8M x 64, the int
latency case, the 4,096-instance batch plan and its one-call-per-instance
baseline.  --report k|n|phi prints the sweeps over k, over n, or over EIM's
phi on 2-D sets shaped like the paper's experiments instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point-center dist evals/s & % HBM roofline; mixed-prec batched vs FP32 solve ms"
UNIT = "dist_evals/s"
N, D, K = 8_000_000, 64, 1024
WORKLOAD = "gon_gau_n8000000_d64_k1024"
CFG2 = "gon_radius_gau_n1000000_d10_k100"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
CPU_K_SINGLE = 4      # oracle sample, one thread: GON with 4 centers on all n points
CPU_K_SHARD = 32      # oracle sample, all cores: GON with 32 centers on each core's shard

# Further workloads (one JSON line each, same keys): GON + radius on the
# L2-resident 1M x 10 set, the int GON latency case, GON / MRG on 10M x 16,
# the tensor-core radius and EIM on 8M x 64, the 4,096-instance batch, and the
# same instances as one kc_gonzalez call each (the unbatched baseline).
EXTRA = (CFG2, "gon_int_n10000_d2_k10", "gon_unif_n10000000_d16_k200", "mrg_unif_n10000000_d16_m64_k200",
         "radius_gau_n8000000_d64_k1024", "eim_gau_n8000000_d64_k1024", "batch_4096", "batch_4096_per_call")

# DRAM traffic (read + write bytes) per launch of the dominant kernel from an
# ncu capture, keyed by the SHA-256 of the kernel's source file at capture
# time; reported only while the source is unchanged.  Values are for the
# full workload (a smaller capture scaled by the units processed).
NCU_TRAFFIC = {
    # gon_group_kernel<float, 64, 1> at k = 16 on the 8M x 64 set (mean of two launches):
    # 33,414,887,680 B read + 275,456,128 B written; x 64 for k = 1024
    "3f019a95cd88c2d2cbef16eee6b28214751a0de558481537031966052fe939c9": 2_156_182_003_712,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="headline: leave out the 4,096-instance part of the mixed-precision comparison")
    ap.add_argument("--workload", default=WORKLOAD, choices=(WORKLOAD,) + EXTRA,
                    help="the default is the headline line; the others measure the remaining paths")
    ap.add_argument("--sweep", default="f32", choices=["f32", "bf16", "fp16", "fp8"],
                    help="sweep precision for the GON / MRG / batch workloads")
    ap.add_argument("--n", type=int, default=0,
                    help="fewer points than the configuration's (small profiling cases)")
    ap.add_argument("--k", type=int, default=0, help="8M x 64 workloads: another k (small profiling cases)")
    ap.add_argument("--report", choices=["k", "n", "phi"], default=None,
                    help="instead of a bench line: runtime and solution value over k (k) or over n at "
                         "k = 10 and 100 (n) for GON, MRG and EIM, or EIM over phi (phi), on 2-D sets shaped "
                         "like the paper's; JSON rows on stdout, tables on stderr")
    ap.add_argument("--seeds", type=int, default=3, help="--report: sets drawn per shape")
    ap.add_argument("--runs", type=int, default=2, help="--report: runs per set and method")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload_seed(rank: int) -> int:
    """Seed of rank r's replica of the headline workload (independent instances)."""
    return 4 + 1000 * rank


def job_reduce(x: float, op: str, device) -> float:
    """x reduced over the ranks of the default process group ("max" or
    "min"); x itself without one (a single process)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.MIN)
    return float(t.item())


def job_throughput(units_per_step: float, steps: int, world: int, job_ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_step * steps * world / (job_ms / 1e3)


def peaks(kind="hbm"):
    """Roofline denominator: measured HBM copy GB/s, or dense bf16 TFLOP/s
    (burst; fp16 runs at the bf16 rate)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return (float(j["hbm_gbs"]) if kind == "hbm" else float(j["bf16_tflops"])), "measured"
    return (FALLBACK_HBM_GBS if kind == "hbm" else FALLBACK_BF16_TFLOPS), "fallback"


def read_peak(nbytes: int, reps: int = 20, tries: int = 10) -> float:
    """Read bandwidth (GB/s, best of `tries`) of a device buffer of `nbytes`
    swept `reps` times in one kc_read_sweep launch: the L2 read peak for a
    buffer well under the L2 size."""
    import torch
    import paper_1604_03228_gb300 as kc
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(3):
        kc.kc_read_sweep(buf, reps, sink)
    best = 0.0
    for _ in range(tries):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        kc.kc_read_sweep(buf, reps, sink)
        b.record(s)
        b.synchronize()
        best = max(best, nbytes * reps / (a.elapsed_time(b) / 1e3) / 1e9)
    del buf
    return best


def workload(rank: int, n: int = N):
    from paper_1604_03228_gb300 import inputs as I
    return I.eim_gau_8m(n=n, seed=workload_seed(rank))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=2)

    def summary(self, t0, t1):
        inside = [r for (t, r) in self.rows if t0 <= t <= t1]
        window = "timed"
        if not inside:
            inside = [r for (_, r) in self.rows]
            window = "whole run (timed region shorter than one sample)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(inside), "window": window}


# ------------------------------------------------------------- CPU oracle

def cpu_single(pts, k: int = CPU_K_SINGLE):
    """The oracle on one thread: GON with k centers on all points (canonical
    FP32 selection, then its FP64 radius), as kc_gonzalez computes."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.gonzalez(pts, k, mode="f32")
    dt = time.perf_counter() - t0
    return k * pts.shape[0], dt


def cpu_baseline(pts, rows: int):
    """The oracle as it stands on the host's cores: one thread, and one worker
    process per core on contiguous shards of the same points."""
    from oracle.parallel import ShardPool
    nproc = os.cpu_count() or 1
    e1, t1 = cpu_single(pts)
    pool = ShardPool(pts)
    try:
        wall, evals, _ = pool.gon(CPU_K_SHARD, "f32")
    finally:
        pool.close()
    return {"value": evals / wall, "unit": UNIT, "cores": pool.procs, "nproc": nproc, "kind": "oracle",
            "sample": f"GON with {CPU_K_SHARD} centers (canonical FP32 selection + FP64 radius) on each of "
                      f"{pool.procs} contiguous shards of the n={rows} x d={pts.shape[1]} points, one worker "
                      f"process per core ({wall:.2f} s wall)",
            "single_thread": {"value": e1 / t1, "unit": UNIT, "cores": 1,
                              "sample": f"GON with {CPU_K_SINGLE} centers on all {rows} points, one thread "
                                        f"({t1:.2f} s)"}}


def run_reference(args):
    """The CPU oracle, unmodified, on every host core (rank 0 only)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle.parallel import ShardPool
    n = getattr(args, "n", 0) or N
    pts = workload(0, n)
    pool = ShardPool(pts)
    try:
        for _ in range(args.warmup):
            pool.gon(CPU_K_SHARD, "f32")
        tot_e, tot_t = 0, 0.0
        for _ in range(args.steps):
            t, e, _ = pool.gon(CPU_K_SHARD, "f32")
            tot_e += e
            tot_t += t
    finally:
        pool.close()
    v = tot_e / tot_t
    sample = (f"per step: GON with {CPU_K_SHARD} centers (canonical FP32 selection + FP64 radius) on each of "
              f"{pool.procs} contiguous shards of the n={n} x d={D} points, one worker process per core")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": n, "d": D, "k": K},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.procs, "nproc": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU

def timed_steps(step, steps, s, flush=None):
    """Device ms of each of `steps` calls of step() (CUDA events on stream s)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(s)
        step()
        ev[i][1].record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def batch_comparison(args, kc, sw="bf16"):
    """The 4,096-instance workload: the mixed-precision batch (one CUDA-graph
    replay of a plan, bf16 sweep) against one FP32 kc_gonzalez call per
    instance and against the FP32 batch plan; selections compared."""
    import numpy as np
    import torch
    from paper_1604_03228_gb300 import inputs as I
    s = torch.cuda.current_stream()
    insts = [I.batch_instance(i) for i in range(4096)]
    xs = [torch.from_numpy(np.ascontiguousarray(z.points)).cuda() for z in insts]
    ks = [z.k for z in insts]
    evals = sum(z.points.shape[0] * min(z.k, z.points.shape[0]) for z in insts)
    out = {"workload": "batch_4096", "count": 4096, "evals_per_solve": evals}
    steps = max(3, min(args.steps, 10))
    for name, sweep in (("lp", sw), ("f32", None)):
        plan = kc.kc_batch_plan_create(xs, ks, sweep=sweep, flags=kc.KC_AUTOTUNE)
        for _ in range(3):
            kc.kc_batch_plan_run(plan)
        res = kc.kc_batch_plan_wait(plan)
        ms = timed_steps(lambda: kc.kc_batch_plan_run(plan), steps, s)
        kc.kc_batch_plan_wait(plan)
        out[f"{name}_plan_ms"] = statistics.median(ms)
        out[f"{name}_plan_theta"] = kc.kc_batch_plan_info(plan)[0]
        if name == "lp":
            lp_res = [(r.centers.cpu().tolist(), r.radius) for r in res]
        else:
            out["selections_identical"] = all((r.centers.cpu().tolist(), r.radius) == q
                                              for r, q in zip(res, lp_res))
        kc.kc_batch_plan_destroy(plan)
    # the unbatched FP32 baseline: one synchronous call per instance, in order
    def per_call():
        for xi, ki in zip(xs, ks):
            kc.kc_gonzalez(xi, ki)
    per_call()
    ms = timed_steps(per_call, 2, s)
    out["f32_per_call_ms"] = statistics.median(ms)
    out["sweep"] = sw
    out["speedup_vs_f32_per_call"] = out["f32_per_call_ms"] / out["lp_plan_ms"]
    out["speedup_vs_f32_plan"] = out["f32_plan_ms"] / out["lp_plan_ms"]
    return out


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1604_03228_gb300 as kc

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kc.load()
    n, k = args.n or N, args.k or K
    pts = workload(rank, n)
    x = torch.from_numpy(pts).cuda()
    s = torch.cuda.current_stream()
    cen = torch.empty(k, dtype=torch.int64, device="cuda")
    kout = torch.empty(1, dtype=torch.int32, device="cuda")
    rad = torch.empty(1, dtype=torch.float64, device="cuda")
    big = n * D * 4 > 2 * L2_FLUSH_BYTES
    flush = None if big else torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(sweep=None):
        kc.kc_gonzalez(x, k, flags=kc.KC_ASYNC, out=(cen, kout, rad), sweep=sweep)

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(max(args.warmup, 3)):
        step()
    assert kc.kc_sync(s) == kc.KC_OK
    ref_centers, ref_rad = cen.cpu().tolist(), float(rad.item())
    assert int(kout.item()) == k
    # the result's FP32 evaluation against FP64: the canonical FP32 covering
    # radius beside the returned FP64 one (the same for every sweep precision)
    r32 = kc.kc_last_fp32_radius(s)
    fp64_error = {"radius_fp64": ref_rad, "radius_fp32": r32, "rel_err": abs(r32 - ref_rad) / ref_rad}
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    kc.kc_trace_read()
    kc.kc_trace_enable(True)
    launches0 = kc.kc_launch_count()
    t_wall0 = time.time()
    step_ms = timed_steps(step, args.steps, s, flush)
    t_wall1 = time.time()
    launches = kc.kc_launch_count() - launches0
    kc.kc_trace_enable(False)
    trace = kc.kc_trace_read()
    assert kc.kc_sync(s) == kc.KC_OK
    total_ms = job_reduce(sum(step_ms), "max", "cuda")
    clocks = sampler.summary(t_wall0, t_wall1)

    evals_step = n * k
    value = job_throughput(evals_step, args.steps, world, total_ms)

    # dominant kernel: the persistent GON kernel (one launch per step)
    gon_ms = [ms for (name, nk, ms) in trace if name == "gonzalez"]
    gon_avg = statistics.mean(gon_ms)
    alg_bytes = k * n * (4 * D + 4)
    achieved = alg_bytes / (gon_avg / 1e3) / 1e9
    peak, peak_kind = peaks()
    src = open(os.path.join(ROOT, "paper_1604_03228_gb300", "csrc", "kc_gon.cu"), "rb").read()
    traffic = NCU_TRAFFIC.get(hashlib.sha256(src).hexdigest()) if (n, k) == (N, K) else None
    shares = {}
    for name, nk, ms in trace:
        shares[name] = shares.get(name, 0.0) + ms

    # mixed precision on the same workload: the bf16 sweep, same selections
    mixed = {}
    for sw in ("bf16", "fp16"):
        for _ in range(2):
            step(sw)
        assert kc.kc_sync(s) == kc.KC_OK
        kc.kc_counters()
        ms = timed_steps(lambda: step(sw), args.steps, s, flush)
        cnt = kc.kc_counters()
        assert kc.kc_sync(s) == kc.KC_OK
        same = cen.cpu().tolist() == ref_centers and float(rad.item()) == ref_rad
        mixed[f"gon_{sw}_ms"] = statistics.median(ms)
        mixed[f"gon_{sw}_identical_selection"] = same
        mixed[f"gon_{sw}_rechecks_per_solve"] = cnt[0] / args.steps
        # per-CTA phase time of the persistent kernel (clock cycles summed
        # over CTAs, per solve, at the sampled SM clock)
        ctas = max(1, int(torch.cuda.get_device_properties(local).multi_processor_count))
        mhz = (sampler.summary(0, time.time()).get("sm_mhz") or 2070.0)
        mixed[f"gon_{sw}_phase_ms"] = {ph: cnt[i] / args.steps / ctas / (mhz * 1e3)
                                       for ph, i in (("sweep", 6), ("recheck", 7), ("exchange", 8))}
        mixed[f"gon_{sw}_speedup"] = statistics.median(step_ms) / statistics.median(ms)
    mixed["gon_f32_ms"] = statistics.median(step_ms)
    if not args.no_batch:
        mixed["batch"] = batch_comparison(args, kc)
    sampler.stop()

    # end to end: points in pinned host memory through the C ABI each step
    e2e = None
    hp = torch.from_numpy(pts).pin_memory()
    for _ in range(2):
        kc.kc_gonzalez(hp, k)
    reps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        g = kc.kc_gonzalez(hp, k)     # host buffers: the call reads the points and returns host results
        _ = (g.centers[0], g.radius)
    t1 = time.perf_counter()
    # whole job: every rank's rate no better than the slowest rank's
    e2e_val = job_reduce(evals_step * reps / (t1 - t0), "min", "cuda") * world
    e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": n * D * 4,
           "d2h_bytes_per_step": k * 8 + 4 + 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pts, n)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if (n, k) == (N, K) else f"gon_gau_n{n}_d{D}_k{k}",
                           "n": n, "d": D, "k": k,
                           "points": "100-Gaussian mixture, sigma 0.5, means U[-10,10]^64",
                           "l2": ("inputs larger than L2 (no flush)" if big
                                  else f"{L2_FLUSH_BYTES >> 20} MiB flush between steps"),
                           "step": "one kc_gonzalez call: pack + persistent k-step GON + FP64 radius recheck",
                           "sweep": "f32", "replicas": world},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "kernel": "gon_group_kernel",
                             "peak_kind": peak_kind, "avg_ms": gon_avg, "alg_bytes_per_launch": alg_bytes,
                             "alg_bytes_rule": "k n (4 d + 4): each step reads every point and its running minimum"},
                "mixed": mixed, "fp64_error": fp64_error, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks,
                "step_share_ms": {k_: v / args.steps for k_, v in shares.items()}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------- other workloads

def run_extra(args):
    """One of EXTRA on one GPU: warm-up, then `steps` timed calls (CUDA
    events around each); the dominant step's device time comes from the
    library's trace events."""
    import numpy as np
    import torch

    import paper_1604_03228_gb300 as kc
    from paper_1604_03228_gb300 import inputs as I

    torch.cuda.set_device(0)
    kc.load()
    name, sw = args.workload, (None if args.sweep == "f32" else args.sweep)
    bpc = {"f32": 4, "bf16": 2, "fp16": 2, "fp8": 1}[args.sweep]
    mind_b = 4 if sw is None else 2          # running minimum: u32, or 16-bit code in the mixed sweep
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cfg = {"workload": name, "sweep": args.sweep, "l2": "inputs larger than L2"}
    if args.n:
        cfg["n_override"] = args.n
    dom, bound, plan, flush, peak_l2 = "gonzalez", "hbm", None, None, None
    if name == CFG2:
        # GON k=100 + kc_radius on 1M x 10: the 40 MB point set stays in L2
        # between the k sweeps, so the bound is the measured L2 read peak
        n, d, k = args.n or 1_000_000, 10, 100
        pts = I.gauss_mixture(n, d, 1, 25, 1.0, -50.0, 50.0)
        x = dev(pts)
        cen = torch.empty(k, dtype=torch.int64, device="cuda")
        kout = torch.empty(1, dtype=torch.int32, device="cuda")
        rad = torch.empty(1, dtype=torch.float64, device="cuda")
        rrad = torch.empty(1, dtype=torch.float64, device="cuda")
        ram = torch.empty(1, dtype=torch.int64, device="cuda")

        def step():
            kc.kc_gonzalez(x, k, flags=kc.KC_ASYNC, out=(cen, kout, rad), sweep=sw)
            kc.kc_radius(x, cen, flags=kc.KC_ASYNC, out=(rrad, ram))
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        evals = 2 * k * n                              # GON's k sweeps + the n x k radius block
        units = k * n * (d * bpc + mind_b)
        bound = "l2"
        peak_l2 = max(read_peak(n * d * 4), read_peak(64 << 20))
        cfg.update(n=n, d=d, k=k, points="25-Gaussian mixture, sigma 1, means U[-50,50]^10",
                   step="kc_gonzalez + kc_radius", l2=f"{L2_FLUSH_BYTES >> 20} MiB flush between steps; "
                   "the 40 MB point set stays in L2 across the k sweeps of a step",
                   l2_read_peak_gbs=peak_l2, hbm_read_gbs=read_peak(4 << 30, reps=2, tries=5))
    elif name == "gon_int_n10000_d2_k10":
        w = I.gon_int_10k()
        x, k, n, d = dev(w.points), w.k, 10_000, 2
        step = lambda: kc.kc_gonzalez(x, k)
        evals, units = k * n, None
        cfg.update(n=n, d=d, k=k, dtype="int32", l2="80 KB input, on chip (latency bound)")
    elif name in ("gon_unif_n10000000_d16_k200", "mrg_unif_n10000000_d16_m64_k200"):
        pts, off, k = I.mrg_unif_10m(**({"n": args.n} if args.n else {}))
        n, d = pts.shape
        x, o = dev(pts), dev(off)
        if name.startswith("gon"):
            step = lambda: kc.kc_gonzalez(x, k, sweep=sw)
            evals = k * n                               # the k sweeps (the radius is their maximum)
        else:
            step = lambda: kc.kc_mrg(x, k, 64, o, sweep=sw)
            dom = "mrg_round1"
            evals = k * n + k * (64 * k) + k * n        # round 1, round 2 on the union, radius
            cfg.update(m=64, parts="Zipf(1.1) contiguous")
        units = k * n * (d * bpc + mind_b)
        cfg.update(n=n, d=d, k=k)
    elif name in ("gon_gau_n8000000_d64_k1024", "radius_gau_n8000000_d64_k1024", "eim_gau_n8000000_d64_k1024"):
        pts = I.eim_gau_8m(**({"n": args.n} if args.n else {}))
        n, d = pts.shape
        k = args.k or 1024
        x = dev(pts)
        cfg.update(n=n, d=d, k=k)
        if name.startswith("gon"):
            step = lambda: kc.kc_gonzalez(x, k, sweep=sw)
            evals = k * n
            units = k * n * (d * bpc + mind_b)
        elif name.startswith("radius"):
            cen = torch.from_numpy(np.sort(I.uniform_int(7, 3, k, 0, n - 1)).astype(np.int64)).cuda()
            step = lambda: kc.kc_radius(x, cen)
            dom, bound = "radius", "tensor"
            evals = k * n
            units = 2.0 * n * k * d                     # GEMM-form flops of the n x k block
            cfg.update(centers="k seeded uniform indices", path="tcgen05 fp16 block + exact recheck")
        else:
            step = lambda: kc.kc_eim(x, k, eps=0.1, phi=6.0, seed=40)
            dom, bound = "eim_prune", "tensor"
            evals, units = None, None                   # from the prune counters below
            cfg.update(eps=0.1, phi=6.0, seed=40, metric_note="evals = prune |R| x |S| + GON on the sample + radius")
    elif name == "batch_4096_per_call":
        insts = [I.batch_instance(i) for i in range(4096)]
        xs = [dev(z.points) for z in insts]
        ks = [z.k for z in insts]

        def step():
            for xi, ki in zip(xs, ks):
                kc.kc_gonzalez(xi, ki, sweep=sw)
        evals = sum(z.points.shape[0] * min(z.k, z.points.shape[0]) for z in insts)
        units = sum(z.points.shape[0] * min(z.k, z.points.shape[0]) * (z.points.shape[1] * bpc + mind_b)
                    for z in insts)
        cfg.update(count=4096, step="one synchronous kc_gonzalez call per instance, in order")
    elif name == "batch_4096":
        insts = [I.batch_instance(i) for i in range(4096)]
        xs = [dev(z.points) for z in insts]
        ks = [z.k for z in insts]
        plan = kc.kc_batch_plan_create(xs, ks, sweep=sw, flags=kc.KC_AUTOTUNE)
        step = lambda: kc.kc_batch_plan_run(plan)
        dom = "gonzalez_batch"
        evals = sum(z.points.shape[0] * min(z.k, z.points.shape[0]) for z in insts)
        units = sum(z.points.shape[0] * min(z.k, z.points.shape[0]) * (z.points.shape[1] * bpc + mind_b)
                    for z in insts)
        th, nh, gh, grid = kc.kc_batch_plan_info(plan)
        cfg.update(count=4096, step="CUDA-graph replay of the batch plan", theta=th, group_instances=nh,
                   group_ctas=gh, grid=grid)
    s = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    kc.kc_counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = kc.kc_launch_count()
    t0 = time.time()
    for i in range(args.steps):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(s)
        step()
        ev[i][1].record(s)
    torch.cuda.synchronize()
    t1 = time.time()
    if name == CFG2:
        assert kc.kc_sync(s) == kc.KC_OK
    launches = kc.kc_launch_count() - launches0
    sampler.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    counters = kc.kc_counters()
    # the dominant step's device time, traced outside the timed region
    kc.kc_trace_read()
    kc.kc_trace_enable(True)
    if plan is not None:
        kc.kc_gonzalez_batch(xs, ks, sweep=sw, flags=kc.KC_AUTOTUNE)   # same shape, traced (graphs are not)
    else:
        step()
    torch.cuda.synchronize()
    kc.kc_trace_enable(False)
    trace = kc.kc_trace_read()
    shares = {}
    for nm, nk, ms in trace:
        shares[nm] = shares.get(nm, 0.0) + ms
    dom_ms = shares.get(dom)
    if name.startswith("eim"):
        pairs = counters[4] // args.steps
        units = 2.0 * pairs * d
        evals = pairs + k * n                           # prune blocks, radius (GON on the sample not counted)
        cfg.update(prune_pairs_per_solve=pairs)
    roof = None
    if units is not None and dom_ms:
        peak, pk = (peak_l2, "measured here (kc_read_sweep, best of 10)") if bound == "l2" else peaks(bound)
        if bound in ("hbm", "l2"):
            achieved, unit = units / (dom_ms / 1e3) / 1e9, "GB/s"
        else:
            achieved, unit = units / (dom_ms / 1e3) / 1e12, "TFLOP/s"
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": None, "kernel_step": dom, "avg_ms": dom_ms, "peak_kind": pk,
                "alg_per_launch": units}
    line = {"metric": METRIC, "value": evals * args.steps / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i32" if name.startswith("gon_int") else "f32", "data": "synthetic", "config": cfg,
            "roofline": roof, "cpu_baseline": None, "e2e": None, "gpu_launches": launches,
            "clocks": sampler.summary(t0, t1), "step_share_ms": shares,
            "counters": {"sweep_rechecks": counters[0], "sweep_overflows": counters[1],
                         "prune_undecided_pairs": counters[2], "prune_points": counters[3],
                         "sweep_big_rechecks": counters[5], "gon_cycles_sweep": counters[6],
                         "gon_cycles_recheck": counters[7], "gon_cycles_exchange": counters[8],
                         "gon_cycles_sweep_max_cta": counters[9], "gon_cycles_sweep_recheck_max_cta": counters[10],
                         "tc_mma_cycles_wait_centers": counters[11], "tc_mma_cycles_wait_accumulator": counters[12],
                         "tc_mma_cycles_wait_points": counters[13], "tc_mma_cycles": counters[14]}}
    print(json.dumps(line), flush=True)


def run_report(args):
    """The k / phi sweeps of paper_1604_03228_gb300.report on one GPU."""
    import torch
    from paper_1604_03228_gb300 import report
    assert torch.cuda.is_available(), "--report needs a CUDA device"
    if args.report == "k":
        rows, bad = report.k_sweep(seeds=args.seeds, runs=args.runs)
    elif args.report == "n":
        rows, bad = report.n_sweep(seeds=args.seeds, runs=args.runs)
    else:
        rows, bad = report.phi_sweep(seeds=args.seeds, runs=args.runs)
    for r in rows:
        print(json.dumps(r), flush=True)
    log(report.markdown(rows))
    log(f"guarantee violations: {len(bad)}")
    for v in bad:
        log("  " + v)
    if bad:
        sys.exit(1)


def main():
    args = parse()
    if args.report:
        run_report(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload != WORKLOAD:
        run_extra(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
