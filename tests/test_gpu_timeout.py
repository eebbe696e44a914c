"""The abort path of the persistent Gonzalez kernel: a device wait that runs
out of its budget returns KC_ERR_TIMEOUT as a status, the GPU context stays
usable, and the next call is exact again.

The wait is made to run out without any fault: with KC_TEST_WITHHOLD the
last CTA of the launch does not publish its slot for the first step, so the
other CTAs' polls for that step never complete and give up after
timeout_ms (1 ms here).  The group exchange of every step is the wait that
GON (Section 3.1) adds per farthest-point selection.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _pts():
    # 200k points: several CTAs in the launch, so there is an exchange to withhold
    return I.gauss_mixture(200_000, 8, 41, 10, 1.0, -5.0, 5.0)


@pytest.mark.parametrize("sweep", [None, "bf16"])
def test_withheld_slot_times_out_then_next_call_is_exact(kc, sweep):
    import torch
    pts = _pts()
    x = torch.from_numpy(pts).cuda()
    t0 = time.perf_counter()
    with pytest.raises(kc.KCError) as e:
        kc.kc_gonzalez(x, 16, flags=kc.KC_TEST_WITHHOLD, timeout_ms=1, sweep=sweep)
    dt = time.perf_counter() - t0
    assert e.value.status == kc.KC_ERR_TIMEOUT
    assert "GON step exchange (step 0)" in str(e.value)
    assert b"timed out" in kc.load().kc_last_error()
    assert dt < 10.0
    torch.cuda.synchronize()   # the context still answers
    g = kc.kc_gonzalez(x, 16, sweep=sweep)
    ref = O.gonzalez(pts, 16, mode="f32")
    assert g.centers.cpu().numpy().tolist() == ref.centers.tolist()
    assert g.radius == O.radius(pts, ref.centers, mode="f64")[0]


def test_withheld_slot_async_reports_at_sync(kc):
    import torch
    pts = _pts()
    x = torch.from_numpy(pts).cuda()
    s = torch.cuda.current_stream()
    cen = torch.empty(16, dtype=torch.int64, device="cuda")
    kout = torch.empty(1, dtype=torch.int32, device="cuda").fill_(12345)   # stale count: must not be trusted
    rad = torch.empty(1, dtype=torch.float64, device="cuda")
    kc.kc_gonzalez(x, 16, flags=kc.KC_ASYNC | kc.KC_TEST_WITHHOLD, timeout_ms=1, out=(cen, kout, rad))
    with pytest.raises(kc.KCError) as e:
        kc.kc_sync(s)
    assert e.value.status == kc.KC_ERR_TIMEOUT
    assert kc.kc_sync(s) == kc.KC_OK   # the status word was cleared
    kc.kc_gonzalez(x, 16, flags=kc.KC_ASYNC, out=(cen, kout, rad))
    assert kc.kc_sync(s) == kc.KC_OK
    ref = O.gonzalez(pts, 16, mode="f32")
    assert int(kout.item()) == 16
    assert cen.cpu().numpy().tolist() == ref.centers.tolist()


def test_single_cta_launch_has_no_exchange_to_withhold(kc):
    import torch
    pts = I.gauss_mixture(1000, 3, 42, 4, 1.0, 0.0, 1.0)
    x = torch.from_numpy(pts).cuda()
    g = kc.kc_gonzalez(x, 8, flags=kc.KC_TEST_WITHHOLD, timeout_ms=1)
    ref = O.gonzalez(pts, 8, mode="f32")
    assert np.array_equal(g.centers.cpu().numpy(), ref.centers)
