"""Host logic of the k / phi sweeps (paper_1604_03228_gb300.report): the
synthetic sets, the guarantee checks and the tables.  No GPU."""
import numpy as np
import pytest

from paper_1604_03228_gb300 import report as R


@pytest.mark.parametrize("kind,clusters", [("unif", 0), ("gau", 25), ("unb", 25)])
def test_point_sets_shape_range_and_determinism(kind, clusters):
    a = R.point_set(kind, 20000, clusters, 5)
    b = R.point_set(kind, 20000, clusters, 5)
    c = R.point_set(kind, 20000, clusters, 6)
    assert a.shape == (20000, 2) and a.dtype == np.float32
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # the [0, 100) scale (Gaussian tails may leave it by a few sigma)
    assert a.min() > -1.0 and a.max() < 101.0


def _largest_block_share(p, cell=2.0):
    # share of the points in the fullest 3 x 3 block of grid cells, so that a
    # cluster of sigma 0.1 on a cell border still counts whole
    h, _, _ = np.histogram2d(p[:, 0], p[:, 1], bins=int(100 / cell), range=[[0, 100], [0, 100]])
    h = np.pad(h, 1)
    s = sum(h[1 + i:h.shape[0] - 1 + i, 1 + j:h.shape[1] - 1 + j] for i in (-1, 0, 1) for j in (-1, 0, 1))
    return s.max() / len(p)


def test_unbalanced_set_puts_about_half_in_one_cluster():
    # UnB (Section 7.2): about half of the points in a single cluster
    share = _largest_block_share(R.point_set("unb", 40000, 25, 7))
    assert 0.45 < share < 0.6
    # Gau: clusters of similar size (1/25 each, so no block holds much more)
    assert _largest_block_share(R.point_set("gau", 40000, 25, 7)) < 0.15


def test_guarantee_checks_flag_each_bound():
    assert R.check_guarantees({"gon": 2.0, "mrg": 1.5, "eim": 1.2}) == []
    # r_GON <= 2 OPT <= 2 r_X
    assert R.check_guarantees({"gon": 10.0, "mrg": 4.0})
    assert R.check_guarantees({"gon": 10.0, "eim": 4.9})
    # r_MRG <= 4 OPT <= 4 r_GON
    assert R.check_guarantees({"gon": 1.0, "mrg": 4.5})
    assert R.check_guarantees({"gon": 1.0, "mrg": 4.0}) == []
    # r_EIM <= 10 r_GON only where the high-probability bound applies
    assert R.check_guarantees({"gon": 1.0, "eim": 11.0}, phi=6.0)
    assert R.check_guarantees({"gon": 1.0, "eim": 11.0}, phi=4.0) == []
    # NaN never passes
    assert R.check_guarantees({"gon": 1.0, "mrg": float("nan")})


def test_n_sweep_table():
    rows = [{"report": "n_sweep", "set": "gau_k25", "n": n, "method": m, "k": k, "m": 50, "ms": n / 1000,
             "radius": 100.0 / n, "runs": 2} for k in (10, 100) for n in (10000, 20000) for m in ("mrg", "gon")]
    md = R.markdown(rows).splitlines()
    assert md[0] == "gau_k25, k = 10: ms per call | radius over n"
    assert md[1] == "| n | mrg ms | gon ms | mrg | gon |"
    assert md[3] == "| 10000 | 10 | 10 | 0.01 | 0.01 |" and md[4] == "| 20000 | 20 | 20 | 0.005 | 0.005 |"
    assert md[6] == "gau_k25, k = 100: ms per call | radius over n"


def test_markdown_tables():
    rows = [{"report": "k_sweep", "set": "s", "n": 10, "method": m, "k": k, "m": 2, "ms": 1.0 + k,
             "radius": 10.0 / k, "runs": 2} for k in (2, 5) for m in ("mrg", "gon")]
    md = R.markdown(rows).splitlines()
    assert md[0].startswith("s:") and md[1] == "| k | mrg | gon | mrg ms | gon ms |"
    assert md[3] == "| 2 | 5 | 5 | 3 | 3 |" and md[4] == "| 5 | 2 | 2 | 6 | 6 |"
    prow = [{"report": "phi_sweep", "set": "g", "n": 10, "phi": p, "k": 2, "ms": p, "radius": 1.0 / p, "runs": 1}
            for p in (1.0, 6.0)]
    md = R.markdown(prow).splitlines()
    assert md[1] == "| k | phi 1 | phi 6 | phi 1 ms | phi 6 ms |" and md[3] == "| 2 | 1 | 0.1667 | 1 | 6 |"


class _Res:
    def __init__(self, radius):
        self.radius = radius


def _oracle_calls(monkeypatch):
    # the sweeps' library calls answered by the oracle, on the CPU
    from oracle import oracle as O
    from paper_1604_03228_gb300 import inputs as I

    def r64(pts, centers):
        return O.radius(pts, centers, mode="f64")[0]

    monkeypatch.setattr(R.B, "kc_gonzalez",
                        lambda x, k: _Res(r64(x.numpy(), O.gonzalez(x.numpy(), k, mode="f32").centers)))
    monkeypatch.setattr(R.B, "kc_mrg",
                        lambda x, k, m: _Res(r64(x.numpy(), O.mrg(x.numpy(), k, I.even_offsets(len(x), m),
                                                                   mode="f32").centers)))
    monkeypatch.setattr(R.B, "kc_eim",
                        lambda x, k, eps, phi, seed: _Res(r64(x.numpy(), O.eim(x.numpy(), k, eps, phi, seed,
                                                                                mode="f32").centers)))


def test_sweeps_on_the_oracle(monkeypatch):
    # every row present and the guarantees hold on the oracle's own GON, MRG
    # and EIM results (Lemmas 1 and 2; EIM's bound at phi = 6)
    _oracle_calls(monkeypatch)
    rows, bad = R.n_sweep(ns=(3000, 6000), ks=(5, 20), seeds=1, runs=2, m=10, device="cpu")
    assert bad == [] and len(rows) == 2 * 2 * 3
    assert {(r["n"], r["k"], r["method"]) for r in rows} == {(n, k, m) for n in (3000, 6000) for k in (5, 20)
                                                             for m in ("mrg", "eim", "gon")}
    assert all(r["report"] == "n_sweep" and r["runs"] == 2 and r["radius"] > 0 for r in rows)
    rows, bad = R.k_sweep({"unb": ("unb", 4000, 5)}, ks=(2, 8), seeds=1, runs=1, m=8, device="cpu")
    assert bad == [] and len(rows) == 6
    rows, bad = R.phi_sweep(phis=(1.0, 6.0), ks=(4,), seeds=1, runs=1, set_shape=("gau", 4000, 5), device="cpu")
    assert bad == [] and len(rows) == 2
