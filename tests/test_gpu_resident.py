"""The resident single-instance Gonzalez kernel (points held on chip for all
k steps, running minima in registers, candidate coordinates carried in the
exchange slots) against the oracle and against the streaming kernel
(KC_GON_RESIDENT=0), on sizes that use registers only, registers plus shared
memory, and the 1M x 10 workload that fills shared memory; the dimensions
below 8 that stay on the streaming kernel; and the streaming kernel's shared
tail of blocks (KC_GON_TAIL=0 turns it off) on 3M points.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("n", [1, 1025, 4097, 150_001, 600_000])
@pytest.mark.parametrize("d", [2, 3, 8, 10])
def test_resident_equals_oracle(kc, n, d):
    # d = 2 and 3 run the streaming kernel (no resident specialisation)
    pts = I.gauss_mixture(n, d, 900 + d, 12, 1.0, -30.0, 30.0)
    k = min(n, 64)
    r = kc.kc_gonzalez(_dev(pts), k, first=n // 3)
    ref = O.gonzalez(pts, k, first=n // 3, mode="f32")
    assert r.centers.cpu().numpy().tolist() == ref.centers.tolist()
    assert r.radius == ref.radius


def test_resident_equals_streaming_on_the_1m_x_10_workload(kc, monkeypatch):
    pts = I.gauss_mixture(1_000_000, 10, 1, 25, 1.0, -50.0, 50.0)
    x = _dev(pts)
    a = kc.kc_gonzalez(x, 100)
    monkeypatch.setenv("KC_GON_RESIDENT", "0")
    b = kc.kc_gonzalez(x, 100)
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist() and a.radius == b.radius
    ref = O.gonzalez(pts, 100, mode="f32")
    assert a.centers.cpu().numpy().tolist() == ref.centers.tolist() and a.radius == ref.radius


def test_resident_int_ties_and_early_stop(kc):
    # a 7 x 7 integer grid in the first two of ten coordinates: many exact
    # ties (lowest index wins) and an early stop after the 49 distinct points
    pts = np.zeros((300_000, 10), np.int32)
    pts[:, :2] = I.int_points(300_000, 2, 901, 0, 6)
    r = kc.kc_gonzalez(_dev(pts), 80)
    ref = O.gonzalez(pts, 80)
    assert r.centers.cpu().numpy().tolist() == ref.centers.tolist()
    assert r.k_out == len(ref.centers) < 80 and r.radius == 0.0


def test_resident_input_checks(kc):
    pts = I.gauss_mixture(200_000, 8, 902, 5, 1.0, 0.0, 1.0)
    bad = pts.copy()
    bad[123_456, 3] = np.nan
    with pytest.raises(kc.KCError) as e:
        kc.kc_gonzalez(_dev(bad), 10)
    assert e.value.status == kc.KC_ERR_NONFINITE
    big = pts.copy()
    big[7, 0] = 1e17
    with pytest.raises(kc.KCError) as e:
        kc.kc_gonzalez(_dev(big), 10)
    assert e.value.status == kc.KC_ERR_RANGE
    wide = I.int_points(100_000, 10, 903, -30000, 30000)
    with pytest.raises(kc.KCError) as e:
        kc.kc_gonzalez(_dev(wide), 10)
    assert e.value.status == kc.KC_ERR_RANGE
    ok = kc.kc_gonzalez(_dev(pts), 10)   # the status was cleared
    assert ok.k_out == 10


@pytest.mark.parametrize("d", [8, 17])
def test_streaming_shared_tail_equals_oracle(kc, d, monkeypatch):
    # 3M points: too many to stay on chip, and enough blocks per warp that the
    # group shares the last blocks of every step between its CTAs
    pts = I.gauss_mixture(3_000_000, d, 910 + d, 30, 0.7, -10.0, 10.0)
    x = _dev(pts)
    a = kc.kc_gonzalez(x, 64)
    monkeypatch.setenv("KC_GON_TAIL", "0")
    b = kc.kc_gonzalez(x, 64)
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist() and a.radius == b.radius
    ref = O.gonzalez(pts, 64, mode="f32")
    assert a.centers.cpu().numpy().tolist() == ref.centers.tolist() and a.radius == ref.radius
