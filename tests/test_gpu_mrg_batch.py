"""GPU parity of kc_mrg (Algorithm 1, two rounds) and kc_gonzalez_batch.

Selections are compared exactly with the oracle taking the same argmax
decisions (canonical FP32 for float points, exact int64 for int32 points);
returned radii equal the oracle's FP64 (or exact) covering radius of the
returned centers.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_mrg(kc, pts, k, off, use_offsets=True):
    is_int = np.issubdtype(pts.dtype, np.integer)
    m = len(off) - 1
    res = kc.kc_mrg(_dev(pts), k, m, _dev(off) if use_offsets else None)
    ref = O.mrg(pts, k, off, mode="i64" if is_int else "f32")
    got = res.centers.cpu().numpy()
    assert np.array_equal(got, ref.centers), (got[:12], ref.centers[:12])
    if is_int:
        assert res.radius == math.sqrt(O.radius(pts, got)[2])
    else:
        assert res.radius == O.radius(pts, got, mode="f64")[0]
    return res


@pytest.mark.parametrize("n,d,m,k", [(5000, 3, 4, 10), (20000, 10, 16, 25), (777, 2, 7, 5), (4096, 17, 3, 40)])
def test_mrg_float_even(kc, n, d, m, k):
    pts = I.gauss_mixture(n, d, 40 + n + d, 8, 1.0, -10, 10)
    check_mrg(kc, pts, k, I.even_offsets(n, m))


def test_mrg_zipf_parts(kc):
    n, m, k = 300_000, 64, 20
    pts = I.unif_points(n, 16, 41)
    off = I.offsets_from_sizes(I.zipf_partition_sizes(n, m, 1.1))
    check_mrg(kc, pts, k, off)


def test_mrg_int_exact(kc):
    pts = I.int_points(30_000, 4, 42, 0, 50)
    check_mrg(kc, pts, 30, I.even_offsets(30_000, 9))
    pts = I.int_points(5000, 2, 43, 1, 4)           # heavy ties
    check_mrg(kc, pts, 12, I.even_offsets(5000, 5))


def test_mrg_default_offsets_balanced(kc):
    n, m = 10_001, 7
    pts = I.gauss_mixture(n, 5, 44, 5, 1.0, 0, 10)
    off = np.array([i * n // m for i in range(m + 1)], dtype=np.int64)
    check_mrg(kc, pts, 9, off, use_offsets=False)


def test_mrg_one_part_is_gon_set(kc):
    pts = I.gauss_mixture(9000, 6, 45, 5, 1.0, -3, 3)
    r = kc.kc_mrg(_dev(pts), 15, 1)
    g = kc.kc_gonzalez(_dev(pts), 15)
    assert sorted(r.centers.cpu().tolist()) == sorted(g.centers.cpu().tolist())
    assert r.radius == g.radius


def test_mrg_singleton_parts_is_gon(kc):
    # every part is one point: the union is V and round 2 is GON(V) itself
    pts = I.gauss_mixture(300, 3, 46, 4, 1.0, 0, 5)
    r = kc.kc_mrg(_dev(pts), 12, 300)
    g = kc.kc_gonzalez(_dev(pts), 12)
    assert r.centers.cpu().tolist() == g.centers.cpu().tolist() and r.radius == g.radius


def test_mrg_small_parts_fewer_than_k(kc):
    pts = I.gauss_mixture(200, 2, 47, 3, 1.0, 0, 5)
    off = I.offsets_from_sizes(np.array([3, 100, 2, 95]))
    check_mrg(kc, pts, 10, off)


def test_mrg_bad_offsets(kc):
    pts = I.gauss_mixture(100, 2, 48, 3, 1.0, 0, 5)
    with pytest.raises(kc.KCError):
        kc.kc_mrg(_dev(pts), 5, 3, np.array([0, 50, 50, 100]))
    with pytest.raises(kc.KCError):
        kc.kc_mrg(_dev(pts), 5, 2, np.array([0, 50, 99]))


# --------------------------------------------------------------- batched

def _check_instance(pts, k, res):
    is_int = np.issubdtype(pts.dtype, np.integer)
    ref = O.gonzalez(pts, k, mode="i64" if is_int else "f32")
    got = res.centers.cpu().numpy() if hasattr(res.centers, "cpu") else res.centers
    assert np.array_equal(got, ref.centers), (got[:10], ref.centers[:10])
    assert res.k_out == len(ref.centers)
    if is_int:
        assert res.radius == math.sqrt(ref.radius2)
    else:
        assert res.radius == O.radius(pts, got, mode="f64")[0]


def test_batch_mixed_instances(kc):
    insts, ks = [], []
    for i in range(60):
        inst = I.batch_instance(i, n_lo=50, n_hi=20_000)
        insts.append(inst.points)
        ks.append(min(inst.k, 64))
    res = kc.kc_gonzalez_batch([_dev(p) for p in insts], ks)
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)


def test_batch_uniform_d_and_host_pointers(kc):
    insts = [I.gauss_mixture(1000 + 37 * i, 8, 50 + i, 5, 0.5, 0, 1) for i in range(20)]
    ks = [1 + (3 * i) % 40 for i in range(20)]
    res = kc.kc_gonzalez_batch(insts, ks)            # numpy (host) in and out
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)


def test_batch_int_and_degenerate(kc):
    insts = [I.int_points(n, 3, 60 + n, 0, 9) for n in (1, 2, 5, 129, 3000)]
    insts.append(np.zeros((50, 3), dtype=np.int32))
    ks = [1, 5, 5, 200, 17, 4]
    res = kc.kc_gonzalez_batch([_dev(p) for p in insts], ks)
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)
    assert res[-1].k_out == 1 and res[-1].radius == 0.0


def test_batch_many_instances_sampled(kc):
    """4,096 instances of the many-instance workload, scaled to n <= 20,000
    so that the oracle can check a seeded sample of them exactly."""
    count = 4096
    insts = [I.batch_instance(i, n_lo=100, n_hi=20_000) for i in range(count)]
    res = kc.kc_gonzalez_batch([_dev(x.points) for x in insts], [x.k for x in insts])
    rng = np.random.default_rng(0)
    for i in rng.choice(count, 24, replace=False):
        _check_instance(insts[i].points, insts[i].k, res[i])
    assert all(r.k_out >= 1 for r in res)
