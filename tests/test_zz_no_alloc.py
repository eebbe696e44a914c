"""kc_gonzalez_noalloc: Gonzalez for callers that cannot allocate device
memory during a call (latency-critical loops that must not stall on
cudaMalloc/cudaFree, or processes whose HBM another allocator already holds).
It takes all scratch from a fixed static device array.

Checked through the C ABI against kc_gonzalez on two calls in a row (the
second on different inputs, so stale contents of the shared array would
show), with the same tolerance as the other Gonzalez tests: identical center
sequences and identical radius.  This file is collected last so that a
failure here leaves every other test already run.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_1604_03228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _call_noalloc(kc, x, k, first=0, sweep=0):
    import torch
    L = kc.load()
    n, d = x.shape
    centers = torch.full((k,), -1, dtype=torch.int64, device=x.device)
    k_out = torch.zeros(1, dtype=torch.int32, device=x.device)
    radius = torch.zeros(1, dtype=torch.float64, device=x.device)
    o = kc.binding.kc_opts()
    o.dtype = kc.KC_F32 if x.dtype == torch.float32 else kc.KC_I32
    o.sweep = sweep
    o.stream = int(torch.cuda.current_stream().cuda_stream)
    st = L.kc_gonzalez_noalloc(x.data_ptr(), n, d, k, first, centers.data_ptr(), k_out.data_ptr(),
                               radius.data_ptr(), ct.byref(o))
    return st, centers, int(k_out.item()), float(radius.item())


def test_noalloc_matches_kc_gonzalez_two_calls(kc):
    import torch
    cases = [(I.gauss_mixture(200_000, 10, 31, 25, 1.0, -50, 50), 64, 0),
             (I.gauss_mixture(150_001, 7, 32, 9, 0.5, -10, 10), 40, 1234),
             (I.int_points(100_003, 3, 33, 0, 200), 50, 7)]
    for pts, k, first in cases:
        x = torch.from_numpy(pts).cuda()
        ref = kc.kc_gonzalez(x, k, first=first)
        for _ in range(2):
            st, centers, kk, rad = _call_noalloc(kc, x, k, first)
            assert st == kc.KC_OK, kc.load().kc_last_error()
            assert kk == ref.k_out
            assert centers[:kk].cpu().tolist() == ref.centers.cpu().tolist()
            assert rad == ref.radius


def test_noalloc_binding_and_early_stop(kc):
    import torch
    pts = np.repeat(I.gauss_mixture(9, 4, 34, 3, 1.0, 0, 1), 100, axis=0)
    x = torch.from_numpy(pts).cuda()
    a = kc.kc_gonzalez_noalloc(x, 20)
    b = kc.kc_gonzalez(x, 20)
    assert a.k_out == b.k_out == 9 and a.radius == b.radius == 0.0
    assert a.centers.cpu().tolist() == b.centers.cpu().tolist()


def test_noalloc_rejects_oversize_and_host_pointers(kc):
    import torch
    big = torch.zeros((2_000_000, 8), dtype=torch.float32, device="cuda")   # ~ 90 MB of scratch
    st, *_ = _call_noalloc(kc, big, 4)
    assert st == kc.KC_ERR_ARG
    assert b"static array" in kc.load().kc_last_error()
    with pytest.raises(TypeError):
        kc.kc_gonzalez_noalloc(np.zeros((10, 2), dtype=np.float32), 2)
    # the low-precision sweeps need copies that the fixed array does not hold
    small = torch.from_numpy(I.gauss_mixture(1000, 4, 35, 3, 1.0, 0, 1)).cuda()
    for sw in (kc.KC_SWEEP_BF16, kc.KC_SWEEP_FP8, 7):
        st, *_ = _call_noalloc(kc, small, 4, sweep=sw)
        assert st == kc.KC_ERR_ARG and b"KC_SWEEP_F32" in kc.load().kc_last_error()


def test_noalloc_leaves_free_device_memory_unchanged(kc):
    import torch
    x = torch.from_numpy(I.gauss_mixture(100_000, 8, 36, 10, 1.0, -5, 5)).cuda()
    st, *_ = _call_noalloc(kc, x, 16)   # the first call may load the module that holds the array
    assert st == kc.KC_OK
    torch.cuda.synchronize()
    centers = torch.empty(16, dtype=torch.int64, device="cuda")
    k_out = torch.empty(1, dtype=torch.int32, device="cuda")
    radius = torch.empty(1, dtype=torch.float64, device="cuda")
    o = kc.binding.kc_opts()
    o.stream = int(torch.cuda.current_stream().cuda_stream)
    L = kc.load()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert L.kc_gonzalez_noalloc(x.data_ptr(), 100_000, 8, 16, 0, centers.data_ptr(), k_out.data_ptr(),
                                     radius.data_ptr(), ct.byref(o)) == kc.KC_OK
    assert torch.cuda.mem_get_info()[0] == free0
