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


# ------------------------------------------- launch shapes, autotune, plans

def _heavy_batch():
    """Three large instances (heavy under theta <= 8) and 40 small ones."""
    insts = [I.gauss_mixture(150_000 + 7 * i, 8, 90 + i, 25, 0.1, 0, 1) for i in range(3)]
    ks = [64, 40, 90]
    for i in range(40):
        inst = I.batch_instance(i, n_lo=200, n_hi=5_000)
        insts.append(I.gauss_mixture(inst.points.shape[0], 8, 200 + i, 5, 0.2, 0, 1))
        ks.append(min(inst.k, 50))
    return insts, ks


@pytest.mark.parametrize("theta", ["inf", "4", "1", "0.25"])
def test_batch_theta_shapes_exact(kc, monkeypatch, theta):
    monkeypatch.setenv("KC_BATCH_THETA", theta)
    insts, ks = _heavy_batch()
    res = kc.kc_gonzalez_batch([_dev(p) for p in insts], ks)
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)


def test_batch_bf16_groups_exact(kc, monkeypatch):
    monkeypatch.setenv("KC_BATCH_THETA", "1")
    insts, ks = _heavy_batch()
    res = kc.kc_gonzalez_batch([_dev(p) for p in insts], ks, sweep="bf16")
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)


def test_batch_autotune_exact(kc):
    insts, ks = _heavy_batch()
    res = kc.kc_gonzalez_batch([_dev(p) for p in insts], ks, flags=kc.KC_AUTOTUNE)
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)
    again = kc.kc_gonzalez_batch([_dev(p) for p in insts], ks, flags=kc.KC_AUTOTUNE)   # cached shape
    assert [a.centers.cpu().tolist() for a in again] == [a.centers.cpu().tolist() for a in res]


def test_batch_plan_replays_current_points(kc, monkeypatch):
    import torch
    monkeypatch.setenv("KC_BATCH_THETA", "1")
    insts, ks = _heavy_batch()
    xs = [_dev(p) for p in insts]
    plan = kc.kc_batch_plan_create(xs, ks)
    theta, nheavy, gheavy, grid = kc.kc_batch_plan_info(plan)
    assert theta == 1.0 and nheavy >= 1 and gheavy >= 2 * nheavy and grid >= gheavy
    for _ in range(2):
        kc.kc_batch_plan_run(plan)
        res = kc.kc_batch_plan_wait(plan)
        for p, k, r in zip(insts, ks, res):
            _check_instance(p, k, r)
    # new values in the bound buffers: the next replay solves them
    new = [I.gauss_mixture(p.shape[0], p.shape[1], 500 + i, 7, 0.3, -1, 1) for i, p in enumerate(insts)]
    for x, p in zip(xs, new):
        x.copy_(torch.from_numpy(p))
    kc.kc_batch_plan_run(plan)
    res = kc.kc_batch_plan_wait(plan)
    for p, k, r in zip(new, ks, res):
        _check_instance(p, k, r)
    kc.kc_batch_plan_destroy(plan)


def test_batch_plan_autotune_and_stream(kc):
    import torch
    insts, ks = _heavy_batch()
    xs = [_dev(p) for p in insts]
    plan = kc.kc_batch_plan_create(xs, ks, flags=kc.KC_AUTOTUNE)
    theta, nheavy, gheavy, grid = kc.kc_batch_plan_info(plan)
    assert theta in (1e300, 4.0, 2.0, 1.0, 0.5) and grid >= 1
    s = torch.cuda.Stream()
    kc.kc_batch_plan_run(plan, stream=s)
    res = kc.kc_batch_plan_wait(plan)
    for p, k, r in zip(insts, ks, res):
        _check_instance(p, k, r)
    kc.kc_batch_plan_destroy(plan)


def test_batch_plan_rejects_host_memory(kc):
    L = kc.load()
    import ctypes as ct
    pts = np.zeros((10, 2), dtype=np.float32)
    ptrs = (ct.c_void_p * 1)(pts.ctypes.data)
    cen = np.zeros(2, dtype=np.int64)
    cptrs = (ct.c_void_p * 1)(cen.ctypes.data)
    n = np.array([10], dtype=np.int64)
    d = np.array([2], dtype=np.int32)
    k = np.array([2], dtype=np.int32)
    ko = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1, dtype=np.float64)
    h = ct.c_void_p()
    st = L.kc_batch_plan_create(1, ptrs, n.ctypes.data, d.ctypes.data, k.ctypes.data, cptrs, ko.ctypes.data,
                                rr.ctypes.data, None, ct.byref(h))
    assert st == kc.KC_ERR_ARG and b"device memory" in L.kc_last_error()


# ------------------------------------------------ MRG with a capacity

@pytest.mark.parametrize("n,d,k,m,cap", [(30000, 3, 20, 60, 200), (20000, 8, 16, 40, 100), (9000, 5, 7, 90, 14)])
def test_mrg_rounds_exact(kc, n, d, k, m, cap):
    pts = I.gauss_mixture(n, d, 80 + d, 12, 0.4, -4, 4)
    off = I.even_offsets(n, m)
    ref = O.mrg_rounds(pts, k, off, cap, mode="f32")
    got, rounds = kc.kc_mrg_rounds(_dev(pts), k, m, cap, _dev(off))
    assert rounds == ref.rounds and rounds >= 3
    assert got.centers.cpu().tolist() == ref.centers.tolist()
    assert got.radius == O.radius(pts, ref.centers, mode="f64")[0]


def test_mrg_rounds_int_zipf_and_two_round_case(kc):
    pts = I.int_points(50000, 4, 81, 0, 200)
    off = I.offsets_from_sizes(I.zipf_partition_sizes(50000, 32, 1.1))
    ref = O.mrg_rounds(pts, 25, off, 120)
    got, rounds = kc.kc_mrg_rounds(_dev(pts), 25, 32, 120, _dev(off))
    assert rounds == ref.rounds and got.centers.cpu().tolist() == ref.centers.tolist()
    assert got.radius == math.sqrt(ref.radius2)
    # capacity for the whole union: the two-round kc_mrg
    two, r2 = kc.kc_mrg_rounds(_dev(pts), 25, 32, 32 * 25, _dev(off))
    m2 = kc.kc_mrg(_dev(pts), 25, 32, _dev(off))
    assert r2 == 2 and two.centers.cpu().tolist() == m2.centers.cpu().tolist() and two.radius == m2.radius


def test_mrg_rounds_rejects_small_capacity(kc):
    pts = I.gauss_mixture(1000, 3, 82, 3, 1.0, 0, 1)
    with pytest.raises(kc.KCError):
        kc.kc_mrg_rounds(_dev(pts), 10, 4, 19)


def test_mrg_rounds_bf16_first_round(kc):
    pts = I.gauss_mixture(40000, 16, 83, 10, 0.5, -3, 3)
    off = I.even_offsets(40000, 50)
    ref = O.mrg_rounds(pts, 12, off, 100, mode="f32")
    got, rounds = kc.kc_mrg_rounds(_dev(pts), 12, 50, 100, _dev(off), sweep="bf16")
    assert rounds == ref.rounds and got.centers.cpu().tolist() == ref.centers.tolist()
