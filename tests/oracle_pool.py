"""The CPU oracle over many independent instances in worker processes
(spawn), for full-size parity of the batched workload.  Test infrastructure:
each worker draws instance i itself from the seeded generator and runs the
unmodified oracle on it."""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor


def _instance_gon(i: int):
    from oracle import oracle as O
    from paper_1604_03228_gb300 import inputs as I
    z = I.batch_instance(i)
    r = O.gonzalez(z.points, z.k, mode="f32")
    return i, [int(c) for c in r.centers], float(r.radius)


def batch_oracle(count: int, procs: int | None = None):
    """{i: (centers, FP64 radius)} of the oracle's GON on instances 0..count-1."""
    procs = procs or os.cpu_count() or 1
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        return {i: (c, r) for i, c, r in ex.map(_instance_gon, range(count), chunksize=8)}
