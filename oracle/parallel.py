"""The CPU oracle on every host core (test and benchmark infrastructure only).

Runs the unmodified oracle (``oracle.gonzalez``, one thread per call) in one
worker process per core, each on its own contiguous shard of one point set
held in shared memory, so the host's cores are timed on the same work a
single oracle call does on the whole set.  Workers are started with the
``spawn`` method, which is safe after the parent has initialised CUDA.
Only ``bench.py``'s CPU-baseline legs use this module.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import shared_memory

import numpy as np

_W = {}


def _attach(name: str, shape, dtype: str) -> None:
    shm = shared_memory.SharedMemory(name=name)
    _W["shm"] = shm
    _W["pts"] = np.ndarray(shape, dtype=np.dtype(dtype), buffer=shm.buf)


def _shard_gon(lo: int, hi: int, k: int, mode: str):
    from oracle import oracle as O
    t0 = time.perf_counter()
    g = O.gonzalez(_W["pts"][lo:hi], k, mode=mode)
    return time.perf_counter() - t0, len(g.centers)


class ShardPool:
    """`procs` worker processes over one shared copy of `pts`."""

    def __init__(self, pts: np.ndarray, procs: int | None = None):
        self.procs = procs or os.cpu_count() or 1
        pts = np.ascontiguousarray(pts)
        self.shape, self.dtype = pts.shape, pts.dtype.str
        self.shm = shared_memory.SharedMemory(create=True, size=max(pts.nbytes, 1))
        np.ndarray(pts.shape, dtype=pts.dtype, buffer=self.shm.buf)[...] = pts
        self.ex = ProcessPoolExecutor(max_workers=self.procs, mp_context=mp.get_context("spawn"),
                                      initializer=_attach, initargs=(self.shm.name, self.shape, self.dtype))
        self.gon(1, "f32", rows=self.procs * 2)   # start every worker and load the oracle

    def gon(self, k: int, mode: str = "f32", rows: int | None = None):
        """GON with k centers on each of `procs` contiguous shards of the
        first `rows` points (all by default), all shards at once.  Returns
        (wall seconds, point-center distance evaluations)."""
        n = min(rows or self.shape[0], self.shape[0])
        bounds = [(i * n // self.procs, (i + 1) * n // self.procs) for i in range(self.procs)]
        t0 = time.perf_counter()
        futs = [self.ex.submit(_shard_gon, lo, hi, k, mode) for lo, hi in bounds if hi > lo]
        res = [f.result() for f in futs]
        wall = time.perf_counter() - t0
        evals = sum(min(k, hi - lo) * (hi - lo) for lo, hi in bounds if hi > lo)
        return wall, evals, res

    def close(self):
        self.ex.shutdown(wait=True)
        self.shm.close()
        self.shm.unlink()
