"""GPU runs of the k / phi sweeps on small sets: every (method, k) row
present, the approximation guarantees hold on every run, and the GON and
MRG radii equal the oracle's on the same sets."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I
from paper_1604_03228_gb300 import report as R

pytestmark = pytest.mark.gpu

SMALL = {"gau": ("gau", 4000, 5), "unif": ("unif", 3000, 0), "unb": ("unb", 3000, 5)}
KS = (2, 5, 25)


def test_k_sweep_small_sets(kc):
    rows, bad = R.k_sweep(sets=SMALL, ks=KS, seeds=1, runs=2, m=10)
    assert bad == []
    assert len(rows) == len(SMALL) * len(KS) * 3
    for name, (kind, n, clusters) in SMALL.items():
        pts = R.point_set(kind, n, clusters, 5000)
        for k in KS:
            cell = {r["method"]: r for r in rows if r["set"] == name and r["k"] == k}
            assert set(cell) == {"gon", "mrg", "eim"} and all(r["runs"] == 2 for r in cell.values())
            g = O.gonzalez(pts, k, mode="f32")
            assert cell["gon"]["radius"] == O.radius(pts, g.centers, mode="f64")[0]
            mr = O.mrg(pts, k, I.even_offsets(n, 10), mode="f32")
            assert cell["mrg"]["radius"] == O.radius(pts, mr.centers, mode="f64")[0]
            assert cell["eim"]["radius"] > 0 and cell["gon"]["ms"] > 0


def test_phi_sweep_small_set(kc):
    rows, bad = R.phi_sweep(phis=(1.0, 6.0), ks=(2, 10), seeds=1, runs=2, set_shape=("gau", 5000, 5))
    assert bad == []
    assert sorted((r["phi"], r["k"]) for r in rows) == [(1.0, 2), (1.0, 10), (6.0, 2), (6.0, 10)]
    assert all(r["radius"] > 0 and r["runs"] == 2 for r in rows)
