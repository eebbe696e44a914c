"""The multi-process path of bench.py on CPU: two gloo ranks, the max-over-
ranks job time, the whole-job rate, per-rank replica seeds, and the reference
arm running on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank                   # rank 1 is the slow one
        job_ms = bench.job_reduce(local_ms, "max", "cpu")
        rate = bench.job_reduce(100.0 / (1 + rank), "min", "cpu")
        value = bench.job_throughput(2e8, 4, world, job_ms)
        q.put((rank, job_ms, rate, value, bench.workload_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_job_time_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, rate0, v0, s0), (r1, ms1, rate1, v1, s1) = out
    assert ms0 == ms1 == 15.0                          # the slowest rank's time, on every rank
    assert rate0 == rate1 == 50.0                       # the slowest rank's rate
    assert v0 == v1 == pytest.approx(2e8 * 4 * 2 / 0.015)
    assert s0 != s1                                     # independent replicas


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_reduce(3.5, "max", "cpu") == 3.5
    assert bench.job_throughput(10, 3, 1, 1000.0) == 30.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.argparse.Namespace(gpus=2, steps=1, warmup=0, n=20000))
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    # rank 0 prints one JSON line with the keys the benchmark contract names
    sys.path.insert(0, ROOT)
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.run_reference(bench.argparse.Namespace(gpus=1, steps=1, warmup=0, n=20000))
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == bench.UNIT
    assert j["value"] > 0 and j["ms_per_step"] > 0 and j["higher_is_better"] is True
    assert (j["n_gpus"], j["steps"], j["warmup"], j["scaling"], j["data"]) == (1, 1, 0, "weak", "synthetic")
    assert j["config"]["workload"] == bench.WORKLOAD and j["vs_baseline"] is None
    cb = j["cpu_baseline"]
    assert cb["value"] == j["value"] and cb["kind"] == "oracle" and cb["sample"]
    assert cb["cores"] == cb["nproc"] == os.cpu_count()   # one oracle worker per host core
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
