"""The checked build (libkcenter_checks.so, compiled with -DKC_CHECKS): its
kernels test the indices they use against the buffers they address and
report KC_ERR_BOUNDS instead of making an out-of-range access.  It stands in
for compute-sanitizer, which this pool does not offer.

A child process loads the checked library (KC_LIBRARY) and runs every entry
point on inputs that take the main kernels (streaming, resident and
mixed-precision GON, MRG, EIM with the tensor-core prune, the tensor-core
radius, the batch, the no-alloc form), each checked against the oracle or the
FP32 path: no check fires.  Then a planted index one past the points (a
testing flag that only the checked build accepts) must come back as
KC_ERR_BOUNDS, found by the check before any access, and the next call must
be exact again.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1604_03228_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import torch
import paper_1604_03228_gb300 as kc
from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

L = kc.load()
assert L._name.endswith("libkcenter_checks.so"), L._name
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

def same_as_oracle(res, pts, k, **kw):
    ref = O.gonzalez(pts, k, mode="f32", **kw)
    assert res.centers.cpu().numpy().tolist() == ref.centers.tolist(), (res.centers[:8], ref.centers[:8])
    assert res.radius == ref.radius

p1 = I.gauss_mixture(3_000_000, 17, 1, 30, 0.7, -10, 10)          # streaming kernel with the shared tail
same_as_oracle(kc.kc_gonzalez(dev(p1), 32), p1, 32)
p2 = I.gauss_mixture(1_000_000, 10, 2, 25, 1.0, -50, 50)          # resident kernel
same_as_oracle(kc.kc_gonzalez(dev(p2), 50), p2, 50)
p3 = I.gauss_mixture(300_000, 64, 3, 40, 0.5, -10, 10)            # mixed-precision sweeps
x3 = dev(p3)
f = kc.kc_gonzalez(x3, 100)
for sw in ("bf16", "fp16", "fp8"):
    r = kc.kc_gonzalez(x3, 100, sweep=sw)
    assert r.centers.cpu().tolist() == f.centers.cpu().tolist() and r.radius == f.radius, sw
off = I.offsets_from_sizes(I.zipf_partition_sizes(200_000, 16, 1.1))
p4 = I.unif_points(200_000, 16, 4)                                 # MRG on uneven parts
m = kc.kc_mrg(dev(p4), 20, 16, dev(off))
mref = O.mrg(p4, 20, off, mode="f32")
assert m.centers.cpu().numpy().tolist() == mref.centers.tolist() and m.radius == mref.radius
p5 = I.gauss_mixture(30_000, 32, 5, 40, 0.5, -10, 10)              # EIM, tensor-core prune
import os
os.environ["KC_PRUNE_TC"] = "1"
e = kc.kc_eim(dev(p5), 4, eps=0.1, phi=6.0, seed=7)
eref = O.eim(p5, 4, 0.1, 6.0, 7, mode="f32")
assert e.centers.cpu().numpy().tolist() == eref.centers.tolist()
C = np.sort(I.uniform_int(6, 3, 300, 0, 29_999)).astype(np.int64)  # tensor-core radius
rr = kc.kc_radius(dev(p5), dev(C))
r64, am, _ = O.radius(p5, C, mode="f64")
assert rr.radius == r64 and rr.argmax == am
insts = [I.batch_instance(i, n_lo=100, n_hi=20_000) for i in range(64)]   # batch
res = kc.kc_gonzalez_batch([dev(z.points) for z in insts], [z.k for z in insts], sweep="bf16")
for z, q in zip(insts, res):
    zr = O.gonzalez(z.points, z.k, mode="f32")
    assert q.centers.cpu().numpy().tolist() == zr.centers.tolist()
na = kc.kc_gonzalez_noalloc(dev(p2[:100_000]), 16)                 # no-alloc form
same_as_oracle(na, p2[:100_000], 16)

# a planted index one past the points: caught, reported, nothing read
x6 = dev(I.gauss_mixture(200_000, 8, 8, 10, 1.0, -5, 5))
try:
    kc.kc_gonzalez(x6, 8, flags=kc.binding.KC_TEST_BAD_INDEX)
    raise SystemExit("the planted index was not caught")
except kc.KCError as err:
    assert err.status == kc.binding.KC_ERR_BOUNDS, err
    assert "GON winner index" in str(err), err
torch.cuda.synchronize()
same_as_oracle(kc.kc_gonzalez(dev(p2), 20), p2, 20)
print("checked build: OK")
'''


def test_checked_build_runs_clean_and_catches_a_planted_index(kc):
    from paper_1604_03228_gb300 import build
    lib = build.build(checks=True)
    env = dict(os.environ, KC_LIBRARY=lib)
    p = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1500)
    assert p.returncode == 0 and "checked build: OK" in p.stdout, p.stdout[-3000:] + p.stderr[-3000:]


def test_regular_build_rejects_the_checked_build_flag(kc):
    import torch
    x = torch.from_numpy(I.gauss_mixture(20_000, 4, 9, 3, 1.0, 0, 1)).cuda()
    with pytest.raises(kc.KCError) as e:
        kc.kc_gonzalez(x, 8, flags=kc.binding.KC_TEST_BAD_INDEX)
    assert e.value.status == kc.KC_ERR_ARG
