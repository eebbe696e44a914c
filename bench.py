#!/usr/bin/env python
"""Benchmark of the k-center farthest-point hot path on GB300.

Workload: GON (Section 3.1) with k = 100 followed by the covering radius of
its centers (kc_radius), on n = 1,000,000 points in d = 10, a mixture of 25
isotropic Gaussians (sigma 1, means uniform in [-50, 50]^10), FP32, seed 1.
One step = one kc_gonzalez + one kc_radius call through the C ABI.

Metric: point-center distance evaluations per second (GON: k sweeps of n
points; radius: n x k), whole job over all ranks.  `value` is device-timed
with the points resident in HBM (CUDA events around every step, 256 MiB L2
flush between steps outside the events); `e2e` is the same metric with the
points in pinned host memory passed to the C ABI, host<->device copies and
result read-back inside the wall-clock timed region.

Under torchrun (N > 1) every rank solves its own independent instance of the
workload (seed 1 + 1000 * rank): weak scaling, no collective on the data path.

--impl reference times the CPU oracle (plain C, one thread) on a bounded
sample of the same workload: the first 5 GON steps plus the radius of those 5
centers over all n points per step.

--workload NAME measures one of the other paths (one JSON line with the same
keys): GON / MRG on 10M x 16, GON / tensor-core radius / EIM on 8M x 64, the
int latency case, the 4,096-instance batch plan and its one-call-per-instance
baseline.  --report k|phi prints the sweeps over k (GON, MRG, EIM) or over
EIM's phi on 2-D sets shaped like the paper's experiments instead.
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
N, D, K = 1_000_000, 10, 100
WORKLOAD = "gon_radius_gau_n1000000_d10_k100"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0

# Further workloads (one JSON line each, same keys): the int GON latency case,
# GON / MRG on 10M x 16, GON / tensor-core radius / EIM on 8M x 64, the
# 4,096-instance batch, and the same instances as one kc_gonzalez call each
# (the unbatched baseline of the batch).
EXTRA = ("gon_int_n10000_d2_k10", "gon_unif_n10000000_d16_k200", "mrg_unif_n10000000_d16_m64_k200",
         "gon_gau_n8000000_d64_k1024", "radius_gau_n8000000_d64_k1024", "eim_gau_n8000000_d64_k1024",
         "batch_4096", "batch_4096_per_call")

# DRAM traffic (read + write bytes) per launch of the dominant kernel from an
# ncu capture, keyed by the SHA-256 of the kernel's source file at capture
# time; reported only while the source is unchanged.
NCU_TRAFFIC = {
    # gon_group_kernel<float,10>, n=1e6, d=10, k=100: 40,171,776 B read + 50,176 B written
    "83d6b9d6aa15d5e0bbd6ec721055ace70324555880c49da6f01b4b47d298c92a": 40_221_952,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=(WORKLOAD,) + EXTRA,
                    help="the default is the headline line; the others measure the remaining paths")
    ap.add_argument("--sweep", default="f32", choices=["f32", "bf16", "fp8"],
                    help="sweep precision for the GON / MRG / batch workloads")
    ap.add_argument("--n", type=int, default=0,
                    help="other workloads: fewer points than the configuration's (small profiling cases)")
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
    """Seed of rank r's replica of the workload (independent instances)."""
    return 1 + 1000 * rank


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


def workload(rank: int):
    from paper_1604_03228_gb300 import inputs as I
    return I.gauss_mixture(N, D, workload_seed(rank), 25, 1.0, -50.0, 50.0)


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

def oracle_sample(pts, k_sample=5):
    """Oracle on a bounded sample: first k_sample GON steps + their radius."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    g = O.gonzalez(pts, k_sample, mode="f64")
    O.radius(pts, g.centers, mode="f64")
    dt = time.perf_counter() - t0
    evals = pts.shape[0] * k_sample * 2
    return evals, dt


def cpu_baseline(pts):
    evals, dt = oracle_sample(pts)
    return {"value": evals / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 5 GON steps + radius of those 5 centers, n={N}, d={D}, FP64, "
                      f"one thread ({dt:.2f} s)"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    pts = workload(0)
    for _ in range(args.warmup):
        oracle_sample(pts)
    tot_e, tot_t = 0, 0.0
    for _ in range(args.steps):
        e, t = oracle_sample(pts)
        tot_e += e
        tot_t += t
    v = tot_e / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "d": D, "k": K},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "first 5 GON steps + radius of those 5 centers per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU

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
    pts = workload(rank)
    x = torch.from_numpy(pts).cuda()
    s = torch.cuda.current_stream()
    cen = torch.empty(K, dtype=torch.int64, device="cuda")
    kout = torch.empty(1, dtype=torch.int32, device="cuda")
    rad = torch.empty(1, dtype=torch.float64, device="cuda")
    rrad = torch.empty(1, dtype=torch.float64, device="cuda")
    ram = torch.empty(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        kc.kc_gonzalez(x, K, flags=kc.KC_ASYNC, out=(cen, kout, rad))
        kc.kc_radius(x, cen, flags=kc.KC_ASYNC, out=(rrad, ram))

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    kc.kc_sync(s)
    assert int(kout.item()) == K
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kc.kc_trace_read()
    kc.kc_trace_enable(True)
    launches0 = kc.kc_launch_count()
    t_wall0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(s)
        step()
        ev[i][1].record(s)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    launches = kc.kc_launch_count() - launches0
    kc.kc_trace_enable(False)
    trace = kc.kc_trace_read()
    kc.kc_sync(s)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = job_reduce(sum(step_ms), "max", "cuda")
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)

    evals_step = N * K + N * K
    value = job_throughput(evals_step, args.steps, world, total_ms)

    # dominant kernel: the persistent GON kernel (one launch per step)
    gon_ms = [ms for (name, nk, ms) in trace if name == "gonzalez"]
    gon_avg = statistics.mean(gon_ms)
    alg_bytes = K * N * (4 * D + 4)
    achieved = alg_bytes / (gon_avg / 1e3) / 1e9
    peak, peak_kind = peaks()
    src = open(os.path.join(ROOT, "paper_1604_03228_gb300", "csrc", "kc_gon.cu"), "rb").read()
    traffic = NCU_TRAFFIC.get(hashlib.sha256(src).hexdigest())
    shares = {}
    for name, nk, ms in trace:
        shares[name] = shares.get(name, 0.0) + ms

    # end to end: points in pinned host memory through the C ABI each step
    e2e = None
    if rank == 0 or world > 1:
        hp = torch.from_numpy(pts).pin_memory()
        for _ in range(2):
            g = kc.kc_gonzalez(hp, K)
            kc.kc_radius(hp, g.centers)
        reps = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            g = kc.kc_gonzalez(hp, K)
            r = kc.kc_radius(hp, g.centers)
            _ = (g.radius, r.radius)
        t1 = time.perf_counter()
        # whole job: every rank's rate no better than the slowest rank's
        e2e_val = job_reduce(evals_step * reps / (t1 - t0), "min", "cuda") * world
        h2d = 2 * N * D * 4 + K * 8
        d2h = K * 8 + 4 + 8 + 8 + 8
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pts)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": N, "d": D, "k": K, "points": "25-Gaussian mixture",
                           "l2": f"{L2_FLUSH_BYTES >> 20} MiB flush between steps",
                           "step": "kc_gonzalez + kc_radius", "replicas": world},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "kernel": "gon_kernel",
                             "peak_kind": peak_kind, "avg_ms": gon_avg,
                             "alg_bytes_per_launch": alg_bytes},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
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
    bpc = {"f32": 4, "bf16": 2, "fp8": 1}[args.sweep]
    mind_b = 4 if sw is None else 2          # running minimum: u32, or 16-bit code in the mixed sweep
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cfg = {"workload": name, "sweep": args.sweep, "l2": "inputs larger than L2"}
    if args.n:
        cfg["n_override"] = args.n
    dom, bound, plan = "gonzalez", "hbm", None
    if name == "gon_int_n10000_d2_k10":
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
        ev[i][0].record(s)
        step()
        ev[i][1].record(s)
    torch.cuda.synchronize()
    t1 = time.time()
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
        peak, pk = peaks(bound)
        if bound == "hbm":
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
                         "gon_cycles_sweep_max_cta": counters[9], "gon_cycles_sweep_recheck_max_cta": counters[10]}}
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
