"""Pins for the CPU oracle, each against something other than the oracle itself.

- closed forms: evenly spaced collinear points (Section 3.1 selection rule);
- brute force on tiny inputs: the optimal k-center radius over all subsets,
  giving Lemma 1 (GON <= 2 OPT, also for any subset S) and Lemma 2 (two-round
  MRG <= 4 OPT); full distance matrices for the farthest-point property and
  the covering radius;
- exact arithmetic: the canonical FP32 squared distance checked with
  rational arithmetic and correct rounding;
- special cases: MRG with one part keeps GON's set; EIM whose loop bound is
  at least n is GON (Section 7, Fig. 4 discussion);
- published test vectors: splitmix64 (seed 1234567).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1604_03228_gb300 import inputs as I

SPLITMIX_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                    4593380528125082431, 16408922859458223821]


# ------------------------------------------------------------------ helpers

def brute_d2(pts):
    """Full squared-distance matrix, exact for integers (Python ints)."""
    p = np.asarray(pts)
    if np.issubdtype(p.dtype, np.integer):
        q = p.astype(object)
        n = len(q)
        return np.array([[sum((int(a) - int(b)) ** 2 for a, b in zip(q[i], q[j])) for j in range(n)]
                         for i in range(n)], dtype=object)
    q = p.astype(np.float64)
    return ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)


def brute_opt2(D, k):
    """Optimal k-center squared radius: min over center sets of size <= k."""
    n = D.shape[0]
    best = None
    for r in range(1, min(k, n) + 1):
        for C in itertools.combinations(range(n), r):
            v = max(min(D[x][c] for c in C) for x in range(n))
            if best is None or v < best:
                best = v
    return best


def cover2(D, C, pts_idx=None):
    idx = range(D.shape[0]) if pts_idx is None else pts_idx
    return max(min(D[x][c] for c in C) for x in idx)


# --------------------------------------------------------------- splitmix64

def test_splitmix_published_vector_generator():
    s = np.uint64(1234567)
    i = np.arange(1, 6, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = I.mix64(s + i * I.GOLDEN_GAMMA)
    assert [int(v) for v in out] == SPLITMIX_1234567


def test_splitmix_published_vector_oracle_hash():
    # counter c = it<<33 | x<<1 | stream draws output c+1 of the stream seeded 1234567
    want = [(v >> 11) / 2.0 ** 53 for v in SPLITMIX_1234567]
    got = [O.uniform(1234567, 0, 0, 0), O.uniform(1234567, 0, 0, 1),
           O.uniform(1234567, 0, 1, 0), O.uniform(1234567, 0, 1, 1), O.uniform(1234567, 0, 2, 0)]
    assert got == want


# ---------------------------------------------------------- collinear forms

def collinear_sequence(n):
    """Closed form for x_i = i, n = 2^j + 1, first = 0: 0, n-1, then level by
    level the odd multiples of (n-1)/2^t in increasing order (all tied)."""
    seq = [0, n - 1]
    step = n - 1
    while step > 1:
        half = step // 2
        seq += list(range(half, n, step))
        step = half
    return seq


@pytest.mark.parametrize("j", [3, 4, 6])
def test_collinear_power_of_two_sequence_and_radius(j):
    n = 2 ** j + 1
    pts = I.collinear_points(n, d=2)
    want = collinear_sequence(n)
    for k in range(1, n + 1):
        r = O.gonzalez(pts, k)
        assert list(r.centers) == want[:k]
        if k == 1:
            assert r.radius2 == (n - 1) ** 2
        elif k < n:
            t = int(math.floor(math.log2(k - 1)))
            assert r.radius == pytest.approx((n - 1) / 2 ** (t + 1), rel=0, abs=0)
        else:
            assert r.radius == 0.0


@pytest.mark.parametrize("n", [2, 3, 7, 10, 33, 100])
def test_collinear_k2_radius(n):
    r = O.gonzalez(I.collinear_points(n), 2)
    assert list(r.centers) == [0, n - 1]
    assert r.radius == (n - 1) // 2


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_collinear_float_modes_agree(mode):
    pts = I.collinear_points(17, d=3).astype(np.float32)
    r = O.gonzalez(pts, 9, mode=mode)
    assert list(r.centers) == collinear_sequence(17)[:9]
    assert r.radius == 1.0


# --------------------------------------------------- brute-force invariants

def _tiny_sets():
    for s in range(6):
        yield I.int_points(9 + s, 2, 100 + s, 0, 20)
        yield I.gauss_mixture(10 + s, 3, 200 + s, 3, 0.5, -5, 5)


@pytest.mark.parametrize("idx", range(12))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_gon_two_approximation_lemma1(idx, k):
    pts = list(_tiny_sets())[idx]
    D = brute_d2(pts)
    opt2 = brute_opt2(D, k)
    modes = ["i64"] if np.issubdtype(pts.dtype, np.integer) else ["f64", "f32"]
    for mode in modes:
        for first in (0, len(pts) - 1):
            r = O.gonzalez(pts, k, first=first, mode=mode)
            sol2 = cover2(D, list(r.centers))
            assert sol2 <= 4 * opt2 * (1 + 1e-12)           # radius <= 2 OPT
            assert r.radius ** 2 == pytest.approx(float(sol2), rel=1e-12)


@pytest.mark.parametrize("idx", range(12))
def test_lemma1_any_subset(idx):
    """Lemma 1: GON on any S subset of V covers S within 2 OPT(V)."""
    pts = list(_tiny_sets())[idx]
    D = brute_d2(pts)
    n = len(pts)
    mode = "i64" if np.issubdtype(pts.dtype, np.integer) else "f64"
    for k in (1, 2, 3):
        opt2 = brute_opt2(D, k)
        for s in range(4):
            sub = np.sort(I.uniform_int(7 + s, idx, n, 0, 1).nonzero()[0])
            if len(sub) == 0:
                continue
            r = O.gonzalez(pts, k, mode=mode, subset=sub)
            assert cover2(D, list(r.centers), list(sub)) <= 4 * opt2 * (1 + 1e-12)


@pytest.mark.parametrize("idx", range(12))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_mrg_four_approximation_lemma2(idx, k):
    pts = list(_tiny_sets())[idx]
    D = brute_d2(pts)
    opt2 = brute_opt2(D, k)
    n = len(pts)
    mode = "i64" if np.issubdtype(pts.dtype, np.integer) else "f64"
    for m in (1, 2, 3):
        off = I.even_offsets(n, m)
        r = O.mrg(pts, k, off, mode=mode)
        assert cover2(D, list(r.centers)) <= 16 * opt2 * (1 + 1e-12)   # radius <= 4 OPT
        # every part is covered within 2 OPT by its own round-1 centers
        for i in range(m):
            part = list(range(off[i], off[i + 1]))
            assert cover2(D, list(r.round1[i]), part) <= 4 * opt2 * (1 + 1e-12)


# ------------------------------------------------ multi-round MRG (Lemma 3)

@pytest.mark.parametrize("idx", range(12))
def test_mrg_rounds_lemma3_bound(idx):
    """With capacity c < m k, Algorithm 1 runs extra rounds; after L loop
    rounds and the final GON the radius is at most 2 (L + 1) OPT (Lemma 3:
    each extra round adds two to the factor)."""
    pts = list(_tiny_sets())[idx]
    n = len(pts)
    D = brute_d2(pts)
    mode = "i64" if np.issubdtype(pts.dtype, np.integer) else "f64"
    k = 2
    opt2 = brute_opt2(D, k)
    seen_extra = False
    for m, c in ((7, 4), (6, 5), (5, 4), (7, 6)):
        if m > n:
            continue
        r = O.mrg_rounds(pts, k, I.even_offsets(n, m), c, mode=mode)
        seen_extra |= r.rounds > 2
        factor = 2 * r.rounds            # rounds counts the loop rounds and the final GON
        assert cover2(D, list(r.centers)) <= factor * factor * opt2 * (1 + 1e-12)
    assert seen_extra


def test_mrg_rounds_machine_count_inequality():
    """Machines per round obey inequality (1): m^(i) <= m (k/c)^i + (1 - (k/c)^i) / (1 - k/c),
    and the union shrinks every round."""
    pts = I.unif_points(60000, 3, 21)
    k, m, c = 20, 300, 50
    r = O.mrg_rounds(pts, k, I.even_offsets(len(pts), m), c)
    assert r.rounds >= 5
    q = k / c
    for i, size in enumerate(r.sizes):   # |S| after round i + 1; the next round uses ceil(|S| / c) machines
        if size <= c:
            break
        mi = -(-int(size) // c)
        bound = m * q ** (i + 1) + (1 - q ** (i + 1)) / (1 - q)
        assert mi <= bound + 1e-9
    assert all(int(a) > int(b) for a, b in zip(r.sizes[:-1], r.sizes[1:]))
    assert r.sizes[-1] <= c


def test_mrg_rounds_capacity_cases():
    pts = I.gauss_mixture(3000, 4, 22, 10, 0.5, -5, 5)
    off = I.even_offsets(3000, 12)
    # capacity for the whole union: exactly the two-round algorithm
    two = O.mrg(pts, 15, off)
    r = O.mrg_rounds(pts, 15, off, 12 * 15)
    assert r.rounds == 2 and list(r.centers) == list(two.centers) and r.radius2 == two.radius2
    # a capacity below 2k cannot make progress and is refused
    with pytest.raises(ValueError):
        O.mrg_rounds(pts, 15, off, 29)


@pytest.mark.parametrize("seed", range(5))
def test_farthest_point_property_brute_force(seed):
    """Each selection is the farthest point from the earlier centers, lowest
    index on ties, and its recorded value is that exact distance."""
    pts = I.int_points(40, 3, 300 + seed, 0, 6)       # many ties
    D = brute_d2(pts)
    r = O.gonzalez(pts, 12)
    C = list(r.centers)
    assert len(set(C)) == len(C)
    for j in range(1, len(C)):
        dist = [min(D[x][c] for c in C[:j]) for x in range(len(pts))]
        mx = max(dist)
        assert r.sel2[j] == mx
        assert C[j] == dist.index(mx)
    assert r.radius2 == cover2(D, C)
    # selection values never increase
    assert all(r.sel2[j] >= r.sel2[j + 1] for j in range(1, len(C) - 1))


def test_early_stop_on_duplicates():
    pts = np.array([[1, 1], [1, 1], [5, 5], [5, 5], [1, 1]], dtype=np.int32)
    r = O.gonzalez(pts, 4)
    assert list(r.centers) == [0, 2]
    assert r.radius == 0.0


def test_radius_brute_force_and_argmax():
    pts = I.int_points(60, 4, 11, -30, 30)
    D = brute_d2(pts)
    C = [3, 17, 42]
    rad, am, r2 = O.radius(pts, C)
    dist = [min(D[x][c] for c in C) for x in range(60)]
    assert r2 == max(dist)
    assert am == dist.index(max(dist))
    assert O.mind(pts, C).tolist() == [float(v) for v in dist]


def test_eval_sequence_matches_brute_force():
    pts = I.gauss_mixture(50, 3, 12, 4, 0.3, -3, 3)
    D = brute_d2(pts)
    C = [5, 9, 22, 40]
    sel2, max2 = O.eval_sequence(pts, C)
    for j in range(1, 4):
        dist = [min(D[x][c] for c in C[:j]) for x in range(50)]
        assert max2[j] == pytest.approx(max(dist), rel=1e-12)
        assert sel2[j] == pytest.approx(dist[C[j]], rel=1e-12)
    assert max2[4] == pytest.approx(cover2(D, C), rel=1e-12)


# ------------------------------------------------------ canonical FP32 mode

def _round_to_f32(q: Fraction) -> np.float32:
    """Correctly rounded (ties to even) FP32 of an exact rational."""
    c = np.float32(float(q))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        err = abs(Fraction(float(cand)) - q)
        key = (err, int(np.frombuffer(np.float32(cand).tobytes(), np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return np.float32(best[1])


def _canonical_f32(x, c):
    acc = np.float32(0.0)
    for a, b in zip(x, c):
        t = np.float32(np.float32(a) - np.float32(b))     # one IEEE single subtraction
        acc = _round_to_f32(Fraction(float(t)) * Fraction(float(t)) + Fraction(float(acc)))
    return float(acc)


def test_canonical_f32_distance_exact_rounding():
    pts = I.gauss_mixture(24, 7, 13, 3, 3.0, -1e3, 1e3)
    C = [0, 5, 11]
    got = O.mind(pts, C, mode="f32")
    want = [min(_canonical_f32(pts[x], pts[c]) for c in C) for x in range(len(pts))]
    assert got.tolist() == want


def test_f64_mode_is_exact_for_small_integers_in_float():
    pts = I.int_points(200, 5, 14, -100, 100)
    a = O.mind(pts, [1, 2, 3])
    b = O.mind(pts.astype(np.float32), [1, 2, 3], mode="f64")
    c = O.mind(pts.astype(np.float32), [1, 2, 3], mode="f32")
    assert a.tolist() == b.tolist() == c.tolist()


# -------------------------------------------------------------- MRG special

def test_mrg_one_part_equals_gon_set():
    pts = I.int_points(500, 3, 15, 0, 200)
    g = O.gonzalez(pts, 9)
    r = O.mrg(pts, 9, np.array([0, 500]))
    assert sorted(r.centers) == sorted(g.centers)
    assert r.radius == g.radius
    assert r.centers[0] == 0


def test_mrg_round1_is_gon_per_part():
    pts = I.gauss_mixture(300, 2, 16, 5, 1.0, -10, 10)
    off = I.offsets_from_sizes(np.array([50, 130, 120]))
    r = O.mrg(pts, 6, off)
    for i in range(3):
        sub = np.arange(off[i], off[i + 1])
        assert list(r.round1[i]) == list(O.gonzalez(pts, 6, subset=sub).centers)


# -------------------------------------------------------------- EIM special

def test_eim_falls_back_to_gon_when_bound_exceeds_n():
    # (4/eps) k n^eps ln n >= n: the sampling loop never runs and C = V
    pts = I.int_points(2000, 2, 17, 0, 500)
    e = O.eim(pts, 10, 0.1, 6.0, 40)
    g = O.gonzalez(pts, 10)
    assert e.iterations == 0 and len(e.sample) == 2000
    assert list(e.centers) == list(g.centers) and e.radius == g.radius


@pytest.mark.parametrize("mode", ["i64", "f64"])
def test_eim_loop_brute_force_first_iteration(mode):
    """Loop mechanics of Algorithms 2 and 3 checked by brute force."""
    raw = I.int_points(6000, 2, 18, 0, 3000)
    pts = raw if mode == "i64" else raw.astype(np.float32) * np.float32(0.37)
    n, k, eps, phi, seed = len(pts), 2, 0.1, 6.0, 41
    e = O.eim(pts, k, eps, phi, seed, mode=mode)
    limit = (4 / eps) * k * n ** eps * math.log(n)
    assert limit < n and e.iterations >= 1
    pS, pH, s_size, h_size, v, thr, r_after, p = e.trace[0]
    assert pS == pytest.approx(min(1, 9 * k * n ** eps * math.log(n) / n), rel=1e-12)
    assert pH == pytest.approx(min(1, 4 * n ** eps * math.log(n) / n), rel=1e-12)
    S = [x for x in range(n) if O.uniform(seed, 0, x, 0) < pS]
    H = [x for x in range(n) if O.uniform(seed, 0, x, 1) < pH]
    assert len(S) == s_size and len(H) == h_size
    q = pts.astype(np.float64)
    d2S = ((q[:, None, :] - q[None, S, :]) ** 2).sum(-1).min(1)
    order = sorted(H, key=lambda x: (-d2S[x], x))
    assert p == min(len(H), max(1, math.ceil(phi * math.log(n))))
    assert v == order[int(p) - 1]
    assert thr == pytest.approx(d2S[int(v)], rel=1e-12)
    assert r_after == int((d2S > thr).sum())          # "equal" is removed (Section 4.1)
    # R shrinks every iteration and the loop stops below the bound
    sizes = [n] + [int(t[6]) for t in e.trace]
    assert all(a > b for a, b in zip(sizes, sizes[1:]))
    assert e.r_size <= limit < sizes[-2]
    # the output sample is S u R and contains every sampled point
    assert set(S) <= set(e.sample.tolist())
    assert len(e.sample) == e.s_size + e.r_size


def _brute_gon_from_zero(q, k):
    """GON written out with numpy on rows q (first center q[0]; np.argmax
    takes the first, i.e. lowest, index among equal maxima)."""
    C = [0]
    mind = ((q - q[0]) ** 2).sum(1)
    while len(C) < k:
        j = int(np.argmax(mind))
        if mind[j] == 0:
            break
        C.append(j)
        mind = np.minimum(mind, ((q - q[j]) ** 2).sum(1))
    return C


@pytest.mark.parametrize("mode", ["i64", "f64"])
def test_eim_final_gon_on_brute_force_sample(mode):
    """The last step of Algorithm 2 with Section 4.2: the centers are GON run
    on C = S u R in ascending index order from C's lowest index, where S and R
    are rebuilt by brute force for a set on which the sampling loop runs once."""
    raw = I.int_points(6000, 2, 18, 0, 3000)
    pts = raw if mode == "i64" else raw.astype(np.float32) * np.float32(0.37)
    n, k, eps, phi, seed = len(pts), 6, 0.1, 6.0, 41
    e = O.eim(pts, k, eps, phi, seed, mode=mode)
    assert e.iterations == 1
    pS, pH = e.trace[0][0], e.trace[0][1]
    S = [x for x in range(n) if O.uniform(seed, 0, x, 0) < pS]
    H = [x for x in range(n) if O.uniform(seed, 0, x, 1) < pH]
    q = pts.astype(np.int64 if mode == "i64" else np.float64)
    d2S = ((q[:, None, :] - q[None, S, :]) ** 2).sum(-1).min(1)
    order = sorted(H, key=lambda x: (-d2S[x], x))
    p = min(len(H), max(1, math.ceil(phi * math.log(n))))
    thr = d2S[order[p - 1]]
    R = [x for x in range(n) if d2S[x] > thr]
    C = sorted(set(S) | set(R))
    assert e.sample.tolist() == C
    local = _brute_gon_from_zero(q[C], k)
    want = [C[i] for i in local]
    assert e.centers.tolist() == want
    r2 = ((q[:, None, :] - q[None, want, :]) ** 2).sum(-1).min(1).max()
    assert e.radius == pytest.approx(math.sqrt(r2), rel=0, abs=0)


def test_eim_sampling_rates_statistical():
    n = 20000
    pts = I.int_points(n, 2, 19, 0, 10000)
    e = O.eim(pts, 3, 0.1, 6.0, 42)
    pS, pH, s_size, h_size = e.trace[0][:4]
    for p, cnt in ((pS, s_size), (pH, h_size)):
        mu, sd = n * p, math.sqrt(n * p * (1 - p))
        assert abs(cnt - mu) < 5 * sd


# --------------------------------------------------------- stored goldens

def test_golden_int_10k_reproduces():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gon_int_n10000_d2_k10.json")))
    w = I.gon_int_10k()
    r = O.gonzalez(w.points, w.k)
    assert [int(c) for c in r.centers] == g["centers"] and int(r.radius2) == g["radius2"]


def test_golden_unif_10m_record_is_consistent():
    """The stored 10M x 16 record: its point hash covers the generator (the
    first rows of the stream are the same draws whatever n is), and the stored
    selection has GON's invariants: first center 0, distinct centers, and
    selected distances that never increase (Section 3.1)."""
    import hashlib
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gon_unif_n10000000_d16_k32.json")))
    pre = I.unif_points(g["prefix_rows"], g["d"], 3)
    assert hashlib.sha256(pre.tobytes()).hexdigest() == g["prefix_sha256"]
    c, s2 = g["centers"], g["sel2_f32"]
    assert c[0] == 0 and len(set(c)) == len(c) == g["k"]
    assert all(a >= b for a, b in zip(s2[1:], s2[2:]))
    assert g["radius"] > 0 and g["radius"] ** 2 <= s2[-1] * (1 + 1e-5)
