"""The sampled full-size checks (tests/sampled_checks.py) pinned on the CPU:
they pass on the oracle's own results and catch a planted mistake."""
import numpy as np

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I
from sampled_checks import farthest_steps, radius_checks, sample_rows


def _case():
    pts = I.gauss_mixture(20000, 6, 91, 12, 1.0, -10, 10)
    g = O.gonzalez(pts, 40, mode="f32")
    r, am, _ = O.radius(pts, g.centers, mode="f64")
    return pts, g.centers, r, am


def test_checks_pass_on_the_oracles_results():
    pts, C, r, am = _case()
    s = sample_rows(len(pts), 3000, 1)
    assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < len(pts)
    assert farthest_steps(pts, C, s) == []
    assert radius_checks(pts, C, r, am, s) == []


def test_checks_catch_planted_mistakes():
    pts, C, r, am = _case()
    s = sample_rows(len(pts), 3000, 2)
    # step 7 takes the sampled point nearest to the centers before it instead
    # of the farthest point
    bad = C.copy()
    near = [x for x in s if x not in set(C[:7])]
    sub = np.unique(np.concatenate([np.array(near), C[:7]]))
    loc = np.searchsorted(sub, C[:7])
    m2 = O.mind(pts[sub], loc, mode="f32")
    cand = [i for i in range(len(sub)) if sub[i] not in set(C[:7])]
    bad[7] = sub[min(cand, key=lambda i: m2[i])]
    assert 7 in farthest_steps(pts, bad, s)
    # a radius slightly below the true one, and a wrong argmax
    assert radius_checks(pts, C, np.nextafter(r, 0.0), am, s)
    other = int(s[0]) if s[0] != am else int(s[1])
    assert radius_checks(pts, C, r, other, s)
