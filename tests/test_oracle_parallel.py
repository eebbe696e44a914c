"""The all-core oracle pool (oracle/parallel.py) that bench.py's CPU baseline
and reference arm use: every shard runs the oracle (as many centers as the
single-process oracle finds on it), and the evaluation count is k per point."""
import numpy as np

from oracle import oracle as O
from oracle import parallel as P
from paper_1604_03228_gb300 import inputs as I


def test_shard_pool_runs_the_oracle_on_every_shard():
    pts = I.gauss_mixture(4000, 5, 77, 6, 1.0, -10, 10)
    pool = P.ShardPool(pts, procs=3)
    try:
        wall, evals, res = pool.gon(7, "f32")
        assert wall > 0 and evals == 7 * 4000
        bounds = [(i * 4000 // 3, (i + 1) * 4000 // 3) for i in range(3)]
        assert [kout for _, kout in res] == [7, 7, 7]
        # the same shards through the oracle in this process give the same sizes
        for (lo, hi), (_, kout) in zip(bounds, res):
            assert len(O.gonzalez(pts[lo:hi], 7, mode="f32").centers) == kout
        _, ev2, _ = pool.gon(3, "f32", rows=30)
        assert ev2 == 3 * 30
    finally:
        pool.close()
