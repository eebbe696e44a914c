"""Mixed-precision sweeps (bf16, fp16 with one power-of-two scale, fp8 e4m3
with per-column scale) must select exactly what the FP32 sweep selects: same
center sequence, same k_out, same FP64 radius.  The FP32 path itself is pinned
to the oracle elsewhere; here a few cases are also compared with the oracle
directly.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SWEEPS = ["bf16", "fp16", "fp8"]


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def same(a, b):
    assert a.k_out == b.k_out
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist()
    assert a.radius == b.radius


@pytest.mark.parametrize("sweep", SWEEPS)
@pytest.mark.parametrize("n,d", [(1, 3), (31, 2), (1000, 10), (50000, 16), (20000, 17), (8000, 64)])
def test_gonzalez_lp_equals_f32(kc, sweep, n, d):
    pts = I.gauss_mixture(n, d, 500 + n + d, 20, 0.5, -10, 10)
    x = _dev(pts)
    for k in sorted({1, 2, min(n, 50), min(n, 300)}):
        same(kc.kc_gonzalez(x, k, sweep=sweep), kc.kc_gonzalez(x, k))


@pytest.mark.parametrize("sweep", SWEEPS)
def test_lp_matches_oracle_directly(kc, sweep):
    pts = I.gauss_mixture(30000, 10, 501, 25, 1.0, -50, 50)
    r = kc.kc_gonzalez(_dev(pts), 100, sweep=sweep)
    ref = O.gonzalez(pts, 100, mode="f32")
    assert np.array_equal(r.centers.cpu().numpy(), ref.centers)
    assert r.radius == O.radius(pts, ref.centers, mode="f64")[0]


@pytest.mark.parametrize("sweep", SWEEPS)
def test_lp_wide_dynamic_range(kc, sweep):
    # tight clusters far from the origin: large quantisation errors relative
    # to the distances, many flagged candidates
    pts = I.gauss_mixture(20000, 8, 502, 10, 1e-2, -1e3, 1e3)
    x = _dev(pts)
    for k in (5, 40, 200):
        same(kc.kc_gonzalez(x, k, sweep=sweep), kc.kc_gonzalez(x, k))


@pytest.mark.parametrize("sweep", SWEEPS)
def test_lp_exact_codes_and_ties(kc, sweep):
    # small integers are exact in bf16 and fp8 (zero error bounds) and tie a lot
    pts = I.int_points(40000, 4, 503, -7, 7).astype(np.float32)
    x = _dev(pts)
    for k in (3, 60, 500):
        same(kc.kc_gonzalez(x, k, sweep=sweep), kc.kc_gonzalez(x, k))
    dup = np.repeat(I.gauss_mixture(11, 5, 504, 3, 1.0, 0, 1), 300, axis=0)
    a = kc.kc_gonzalez(_dev(dup), 30, sweep=sweep)
    assert a.k_out == 11 and a.radius == 0.0
    same(a, kc.kc_gonzalez(_dev(dup), 30))


@pytest.mark.parametrize("sweep", SWEEPS)
def test_mrg_lp_equals_f32(kc, sweep):
    n, m = 200_000, 32
    pts = I.unif_points(n, 16, 505)
    off = I.offsets_from_sizes(I.zipf_partition_sizes(n, m, 1.1))
    same(kc.kc_mrg(_dev(pts), 30, m, off, sweep=sweep), kc.kc_mrg(_dev(pts), 30, m, off))


@pytest.mark.parametrize("sweep", SWEEPS)
def test_eim_lp_equals_f32(kc, sweep):
    pts = I.gauss_mixture(30000, 16, 506, 50, 0.5, -10, 10)
    same(kc.kc_eim(_dev(pts), 4, sweep=sweep), kc.kc_eim(_dev(pts), 4))


def test_batch_bf16_equals_f32(kc):
    insts = [I.batch_instance(i, n_lo=100, n_hi=30_000) for i in range(200)]
    xs = [_dev(z.points) for z in insts]
    ks = [z.k for z in insts]
    a = kc.kc_gonzalez_batch(xs, ks, sweep="bf16")
    b = kc.kc_gonzalez_batch(xs, ks)
    for ra, rb in zip(a, b):
        same(ra, rb)
    for sw in ("fp8", "fp16"):
        with pytest.raises(kc.KCError):
            kc.kc_gonzalez_batch(xs[:3], ks[:3], sweep=sw)


@pytest.mark.parametrize("scale", [1e-15, 1e-3, 1e4, 1e12])
def test_fp16_scale_extremes(kc, scale):
    # the fp16 copy is taken in units of a power of two fitted to the largest
    # magnitude: tiny and huge coordinates select exactly as FP32 does
    pts = (I.gauss_mixture(30000, 12, 507, 15, 0.3, -10, 10) * np.float32(scale)).astype(np.float32)
    x = _dev(pts)
    for k in (7, 90):
        same(kc.kc_gonzalez(x, k, sweep="fp16"), kc.kc_gonzalez(x, k))
    ref = O.gonzalez(pts, 90, mode="f32")
    assert kc.kc_gonzalez(x, 90, sweep="fp16").centers.cpu().tolist() == ref.centers.tolist()


@pytest.mark.parametrize("local_t", ["0", "1"])
@pytest.mark.parametrize("sweep", ["bf16", "fp16"])
def test_lp_group_and_local_bounds(kc, sweep, local_t, monkeypatch):
    # CTA groups filter their exact rechecks against the group's largest lower
    # bound or each CTA's own: both select what FP32 selects
    monkeypatch.setenv("KC_LP_LOCAL_T", local_t)
    pts = I.gauss_mixture(300_000, 64, 508, 40, 0.5, -10, 10)
    x = _dev(pts)
    same(kc.kc_gonzalez(x, 200, sweep=sweep), kc.kc_gonzalez(x, 200))
    n, m = 300_000, 16
    off = I.offsets_from_sizes(I.zipf_partition_sizes(n, m, 1.1))
    same(kc.kc_mrg(x, 40, m, off, sweep=sweep), kc.kc_mrg(x, 40, m, off))


def test_lp_rechecks_read_rows_or_packed_copy(kc):
    # device rows (aligned or not) are read by the exact rechecks; pinned host
    # rows are not (the packed copy is read instead): same selections
    import torch
    pts = I.gauss_mixture(100_000, 32, 509, 30, 0.5, -10, 10)
    ref = kc.kc_gonzalez(_dev(pts), 120)
    unal = torch.from_numpy(np.concatenate([pts[:1].ravel()[:1], pts.ravel()])).cuda()[1:].view(100_000, 32)
    hp = torch.from_numpy(pts).pin_memory()
    for sw in ("bf16", "fp16"):
        same(kc.kc_gonzalez(unal, 120, sweep=sw), ref)
        r = kc.kc_gonzalez(hp, 120, sweep=sw)
        assert r.centers.tolist() == ref.centers.cpu().tolist() and r.radius == ref.radius
