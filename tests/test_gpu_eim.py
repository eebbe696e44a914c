"""GPU parity of kc_eim (Algorithms 2 and 3 with phi, then GON on the sample).

The random draws follow one written definition on both sides (counter-based
splitmix64), so the sample, the pivot, the pruned set and the final centers
must all equal the oracle's exactly; the radius equals the oracle's FP64 (or
exact) covering radius of the returned centers.
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


def check_eim(kc, pts, k, eps=0.1, phi=6.0, seed=40, expect_loop=None):
    is_int = np.issubdtype(pts.dtype, np.integer)
    res = kc.kc_eim(_dev(pts), k, eps=eps, phi=phi, seed=seed)
    ref = O.eim(pts, k, eps, phi, seed, mode="i64" if is_int else "f32")
    if expect_loop is not None:
        assert (ref.iterations > 0) == expect_loop
    got = res.centers.cpu().numpy()
    assert np.array_equal(got, ref.centers), (got[:10], ref.centers[:10])
    if is_int:
        assert res.radius == math.sqrt(O.radius(pts, got)[2])
    else:
        assert res.radius == O.radius(pts, got, mode="f64")[0]
    return res, ref


def test_eim_fallback_equals_gon(kc):
    pts = I.gauss_mixture(3000, 4, 70, 10, 0.5, -5, 5)
    res, ref = check_eim(kc, pts, 20, expect_loop=False)
    g = kc.kc_gonzalez(_dev(pts), 20)
    assert res.centers.cpu().tolist() == g.centers.cpu().tolist() and res.radius == g.radius


@pytest.mark.parametrize("seed", [40, 41, 42])
def test_eim_int_loop_exact(kc, seed):
    pts = I.int_points(6000, 2, 18, 0, 3000)
    check_eim(kc, pts, 2, seed=seed, expect_loop=True)


@pytest.mark.parametrize("phi", [1.0, 4.0, 6.0, 8.0])
def test_eim_float_phi_sweep(kc, phi):
    pts = I.gauss_mixture(20000, 3, 71, 25, 0.1, 0, 1)
    check_eim(kc, pts, 3, phi=phi, expect_loop=True)


@pytest.mark.parametrize("n,d,k", [(40000, 16, 4), (30000, 64, 3), (12000, 70, 2), (30000, 13, 4), (30000, 14, 4)])
def test_eim_float_dims(kc, n, d, k):
    pts = I.gauss_mixture(n, d, 72 + d, 100, 0.5, -10, 10)
    check_eim(kc, pts, k, expect_loop=True)


@pytest.mark.parametrize("d", [2, 3, 5, 8, 13])
@pytest.mark.parametrize("tc", ["0", "1"])
def test_eim_prune_paths_small_d(kc, monkeypatch, d, tc):
    # both prune paths where the default is the CUDA cores (d < 16); each
    # CUDA-core width (2, 4, 8, 16 coordinates) and the tensor-core blocks
    monkeypatch.setenv("KC_PRUNE_TC", tc)
    pts = I.gauss_mixture(20000, d, 80 + d, 25, 0.1, 0, 100)
    check_eim(kc, pts, 6, expect_loop=True)


def test_eim_eps_variants(kc):
    pts = I.gauss_mixture(30000, 5, 73, 20, 0.2, -3, 3)
    for eps in (0.05, 0.2):
        check_eim(kc, pts, 3, eps=eps)


def test_eim_bad_eps(kc):
    with pytest.raises(kc.KCError):
        kc.kc_eim(_dev(I.gauss_mixture(100, 2, 1, 2, 1.0, 0, 1)), 2, eps=1.5)


@pytest.mark.parametrize("route", ["default", "pair", "single"])
@pytest.mark.parametrize("cap", [None, "1"])
def test_eim_tc_prune_deferred_pairs(kc, monkeypatch, cap, route):
    # Integer-valued FP32 coordinates on a small grid: many pair distances
    # equal the threshold exactly, so the tensor-core bounds leave pairs
    # undecided and the deferred exact check decides them.  cap=1 overflows
    # the pair buffer at once, so the full-scan route decides those rows.
    pts = I.int_points(40000, 8, 19, 0, 20).astype(np.float32)
    monkeypatch.setenv("KC_PRUNE_TC", "1")   # d = 8 takes the CUDA cores by default
    if route != "default":   # streamed centers, two point tiles per center tile or one
        monkeypatch.setenv("KC_TC_STREAM_CENTERS", "1")
        monkeypatch.setenv("KC_TC_PAIR", "1" if route == "pair" else "0")
    if cap is not None:
        monkeypatch.setenv("KC_PRUNE_PAIR_CAP", cap)
    kc.kc_counters()
    check_eim(kc, pts, 4, expect_loop=True)
    assert kc.kc_counters()[2] > 0


@pytest.mark.parametrize("stream", [None, "1"])
def test_eim_tc_prune_center_ring(kc, monkeypatch, stream):
    # the sample S through the two-stage center ring and resident
    if stream:
        monkeypatch.setenv("KC_TC_STREAM_CENTERS", stream)
    pts = I.gauss_mixture(40000, 24, 77, 60, 0.5, -10, 10)
    check_eim(kc, pts, 5, expect_loop=True)


@pytest.mark.parametrize("n", [90_001, 39_100])
def test_eim_tc_prune_two_point_tiles_per_center_tile(kc, monkeypatch, n):
    # streamed centers: the kernel that feeds each center tile to two point
    # tiles against the one-tile kernel and the oracle, with several pairs
    # per CTA and pairs whose second tile is missing
    pts = I.gauss_mixture(n, 32, 78, 80, 0.5, -10, 10)
    monkeypatch.setenv("KC_TC_STREAM_CENTERS", "1")
    a, _ = check_eim(kc, pts, 6, seed=42, expect_loop=True)
    monkeypatch.setenv("KC_TC_PAIR", "0")
    b = kc.kc_eim(_dev(pts), 6, eps=0.1, phi=6.0, seed=42)
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist() and a.radius == b.radius


def test_eim_tc_prune_matches_cuda_cores(kc, monkeypatch):
    pts = I.gauss_mixture(60000, 32, 75, 100, 0.5, -10, 10)
    a = kc.kc_eim(_dev(pts), 8, eps=0.1, phi=6.0, seed=41)
    monkeypatch.setenv("KC_PRUNE_TC", "0")
    b = kc.kc_eim(_dev(pts), 8, eps=0.1, phi=6.0, seed=41)
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist() and a.radius == b.radius
