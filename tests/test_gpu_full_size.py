"""Full-size checks at the benchmark configurations, in the configuration
bench.py times (points resident on the device, default options): sampled
oracle checks (tests/sampled_checks.py) and identities between paths that
must agree exactly (mixed-precision and FP32 sweeps; tensor-core and
CUDA-core radius and prune), and the 4,096-instance plan against the oracle.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle_pool import batch_oracle
from paper_1604_03228_gb300 import inputs as I
from sampled_checks import farthest_steps, radius_checks, sample_rows

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def unif10m():
    """n = 10M, d = 16, U[0,1)^16; 64 Zipf(1.1) parts; k = 200."""
    return I.mrg_unif_10m()


@pytest.fixture(scope="module")
def gau8m():
    """n = 8M, d = 64, 100 clusters."""
    return I.eim_gau_8m()


def _centers(res):
    return res.centers.cpu().numpy()


def test_gon_10m_d16_golden_and_oracle_at_full_n(kc, unif10m):
    """Whole center sequences at full n, element by element: the stored
    oracle record (k = 32) and the oracle run here (k = 16, FP32 sweep and
    bf16 sweep)."""
    pts, _, _ = unif10m
    g = json.load(open(os.path.join(GOLDEN, "gon_unif_n10000000_d16_k32.json")))
    assert hashlib.sha256(pts.tobytes()).hexdigest() == g["points_sha256"]
    x = _dev(pts)
    res = kc.kc_gonzalez(x, g["k"])
    assert _centers(res).tolist() == g["centers"] and res.radius == g["radius"]
    ref = O.gonzalez(pts, 16, mode="f32")
    for sw in (None, "bf16"):
        r16 = kc.kc_gonzalez(x, 16, sweep=sw)
        assert _centers(r16).tolist() == ref.centers.tolist()
        assert r16.radius == ref.radius


def test_mrg_10m_zipf_parts_oracle_at_full_n(kc, unif10m):
    """MRG on the 64 Zipf parts at full n with k = 16 per part: the round-2
    selection and the radius equal the oracle's."""
    pts, off, _ = unif10m
    ref = O.mrg(pts, 16, off, mode="f32")
    x, o = _dev(pts), _dev(off)
    for sw in (None, "bf16"):
        m = kc.kc_mrg(x, 16, len(off) - 1, o, sweep=sw)
        assert _centers(m).tolist() == ref.centers.tolist()
        assert m.radius == ref.radius


def test_gon_8m_d64_oracle_at_full_n(kc, gau8m):
    """The 8M x 64 workload at full n with k = 16: the whole sequence and the
    radius equal the oracle's, for the FP32 and bf16 sweeps."""
    pts = gau8m
    ref = O.gonzalez(pts, 16, mode="f32")
    x = _dev(pts)
    for sw in (None, "bf16"):
        r = kc.kc_gonzalez(x, 16, sweep=sw)
        assert _centers(r).tolist() == ref.centers.tolist()
        assert r.radius == ref.radius


def test_gon_10m_d16_k200(kc, unif10m):
    pts, _, k = unif10m
    x = _dev(pts)
    a = kc.kc_gonzalez(x, k)
    b = kc.kc_gonzalez(x, k, sweep="bf16")
    ca = _centers(a)
    assert ca.tolist() == _centers(b).tolist() and a.radius == b.radius
    assert len(set(ca.tolist())) == k and ca[0] == 0
    s = sample_rows(len(pts), 20000, 11)
    assert farthest_steps(pts, ca, s) == []
    rr = kc.kc_radius(x, a.centers)
    assert rr.radius == a.radius
    assert radius_checks(pts, ca, rr.radius, rr.argmax, s) == []


def test_mrg_10m_zipf_parts(kc, unif10m):
    pts, off, k = unif10m
    x, o = _dev(pts), _dev(off)
    a = kc.kc_mrg(x, k, len(off) - 1, o)
    b = kc.kc_mrg(x, k, len(off) - 1, o, sweep="bf16")
    ca = _centers(a)
    assert ca.tolist() == _centers(b).tolist() and a.radius == b.radius
    assert len(set(ca.tolist())) == k
    rr = kc.kc_radius(x, a.centers)
    assert rr.radius == a.radius
    assert radius_checks(pts, ca, rr.radius, rr.argmax, sample_rows(len(pts), 20000, 12)) == []


def test_gon_8m_d64_k1024(kc, gau8m):
    pts = gau8m
    x = _dev(pts)
    a = kc.kc_gonzalez(x, 1024)
    b = kc.kc_gonzalez(x, 1024, sweep="bf16")
    ca = _centers(a)
    assert ca.tolist() == _centers(b).tolist() and a.radius == b.radius
    assert len(set(ca.tolist())) == 1024
    s = sample_rows(len(pts), 4000, 13)
    assert farthest_steps(pts, ca, s) == []
    rr = kc.kc_radius(x, a.centers)   # tensor-core path (k d >= 8192)
    assert rr.radius == a.radius
    assert radius_checks(pts, ca, rr.radius, rr.argmax, s) == []


def test_radius_8m_tensor_cores_equal_cuda_cores(kc, gau8m, monkeypatch):
    pts = gau8m
    n = len(pts)
    C = np.sort(I.uniform_int(7, 3, 1024, 0, n - 1)).astype(np.int64)   # the bench's center set
    x, c = _dev(pts), _dev(C)
    a = kc.kc_radius(x, c)
    monkeypatch.setenv("KC_RADIUS_TC", "0")
    b = kc.kc_radius(x, c)
    assert a.radius == b.radius and a.argmax == b.argmax
    assert radius_checks(pts, C, a.radius, a.argmax, sample_rows(n, 4000, 14)) == []


def test_eim_8m_tensor_core_prune_equals_cuda_cores(kc, gau8m, monkeypatch):
    pts = gau8m
    x = _dev(pts)
    a = kc.kc_eim(x, 1024, eps=0.1, phi=6.0, seed=40)
    monkeypatch.setenv("KC_PRUNE_TC", "0")
    b = kc.kc_eim(x, 1024, eps=0.1, phi=6.0, seed=40)
    ca = _centers(a)
    assert ca.tolist() == _centers(b).tolist() and a.radius == b.radius
    assert len(set(ca.tolist())) == len(ca) == 1024
    rr = kc.kc_radius(x, a.centers)
    assert rr.radius == a.radius
    assert radius_checks(pts, ca, rr.radius, rr.argmax, sample_rows(len(pts), 4000, 15)) == []


def test_batch_4096_plan(kc):
    insts = [I.batch_instance(i) for i in range(4096)]
    xs = [_dev(z.points) for z in insts]
    ks = [z.k for z in insts]
    plan = kc.kc_batch_plan_create(xs, ks, flags=kc.KC_AUTOTUNE)
    kc.kc_batch_plan_run(plan)
    res = kc.kc_batch_plan_wait(plan)
    lp = kc.kc_gonzalez_batch(xs, ks, sweep="bf16")
    for r, q in zip(res, lp):
        assert r.centers.cpu().tolist() == q.centers.cpu().tolist() and r.radius == q.radius
    # every instance against the oracle, element by element
    ref = batch_oracle(len(insts))
    bad = [i for i in range(len(insts))
           if (res[i].centers.cpu().numpy().tolist(), res[i].radius) != ref[i]]
    assert bad == [], bad[:10]
    kc.kc_batch_plan_destroy(plan)
