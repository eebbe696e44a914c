"""Tensor-core distance blocks against inputs aimed at the FP32 accumulation
of the tensor core: every coordinate is +-A plus a small perturbation, so
each dot product sums d terms of nearly equal magnitude A^2 with random
signs (heavy cancellation), and the squared distances differ only in their
last bits (near-ties everywhere).  The covering radius and its argmax, and
EIM's prune, must come out exactly as on the CUDA cores and as the oracle's.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def cancelling_points(n, d, seed, A=1000.0, delta=1e-3):
    s = (2 * I.uniform_int(seed, 1, n * d, 0, 1) - 1).reshape(n, d).astype(np.float64)
    u = 2.0 * I.uniform01(seed, 2, n * d).reshape(n, d) - 1.0
    return (A * s + delta * u).astype(np.float32)


@pytest.mark.parametrize("d", [16, 64, 125])
def test_radius_with_cancelling_terms(kc, monkeypatch, d):
    n, k = 30_000, max(128, 8192 // d + 1)
    pts = cancelling_points(n, d, 950 + d)
    C = np.sort(I.uniform_int(951 + d, 3, k, 0, n - 1)).astype(np.int64)
    x, c = _dev(pts), _dev(C)
    monkeypatch.setenv("KC_RADIUS_TC", "1")
    a = kc.kc_radius(x, c)
    monkeypatch.setenv("KC_RADIUS_TC", "0")
    b = kc.kc_radius(x, c)
    r64, am, _ = O.radius(pts, C, mode="f64")
    assert a.radius == b.radius == r64
    assert a.argmax == b.argmax == am


def test_eim_prune_with_cancelling_terms(kc, monkeypatch):
    pts = cancelling_points(30_000, 32, 960)
    x = _dev(pts)
    monkeypatch.setenv("KC_PRUNE_TC", "1")
    a = kc.kc_eim(x, 4, eps=0.1, phi=6.0, seed=5)
    monkeypatch.setenv("KC_PRUNE_TC", "0")
    b = kc.kc_eim(x, 4, eps=0.1, phi=6.0, seed=5)
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist() and a.radius == b.radius
    ref = O.eim(pts, 4, 0.1, 6.0, 5, mode="f32")
    assert a.centers.cpu().numpy().tolist() == ref.centers.tolist()


def test_mma_issuer_counters(kc, monkeypatch):
    # the tensor-core MMA issuer's cycle counters: present after a tensor-core
    # radius, each wait within the issuer's total
    pts = cancelling_points(50_000, 64, 970)
    C = np.sort(I.uniform_int(971, 3, 1024, 0, 49_999)).astype(np.int64)
    monkeypatch.setenv("KC_RADIUS_TC", "1")
    kc.kc_counters()
    kc.kc_radius(_dev(pts), _dev(C))
    c = kc.kc_counters()
    assert len(c) == 15
    wait_centers, wait_acc, wait_points, total = c[11:15]
    assert total > 0
    assert 0 <= wait_centers <= total and 0 <= wait_acc <= total and 0 <= wait_points <= total
    assert wait_centers + wait_acc + wait_points <= total
