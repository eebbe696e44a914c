"""Sweeps over k, n and EIM's phi for GON, MRG and EIM through the C ABI, on
2-D synthetic sets shaped like the paper's experiments (Section 7): runtime
curves over k like Figures 2 and 3 and over n like Figure 4, solution-value
tables like Tables 2-4, and the phi trade-off of Tables 6 and 7.

The paper's sets (Section 7.2): Unif, n points uniform in a square; Gau, k'
cluster centers uniform in the square and Gaussian clusters of similar size;
UnB, like Gau with about half of the points in one cluster.  Its printed
radii (about 96 at k = 2) put the coordinates on a [0, 100) scale; the
clusters here have sigma = 0.1 on that scale.  m = 50 machines for MRG and
eps = 0.1, phi = 6 for EIM (Section 7.1).  Each set is drawn with `seeds`
seeds and each method runs `runs` times per set (EIM with a different hash
seed per run), as the paper averages three graphs times two runs.

Guarantees checked per (set, seed, k), with OPT the optimal radius and any
method's radius r_X >= OPT: r_GON <= 2 OPT (Lemma 1) gives r_GON <= 2 r_X;
r_MRG <= 4 OPT (Lemma 2) gives r_MRG <= 4 r_GON; EIM is a 10-approximation
with high probability for phi above the bound of Section 6, so r_EIM <= 10
r_GON is checked there (phi >= 6).
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B
from . import inputs as I

KS = (2, 5, 10, 25, 50, 100)
M = 50
EPS = 0.1
PHI = 6.0
PHIS = (1.0, 4.0, 6.0, 8.0)
SIGMA = 0.1
SCALE = 100.0

# name -> (kind, n, clusters); the figure or table each one mirrors
SETS = {
    "gau_n1000000_k25": ("gau", 1_000_000, 25),   # Table 2, Figure 2(a)
    "unif_n100000": ("unif", 100_000, 0),         # Table 3, Figure 2(b)
    "gau_n1000000_k50": ("gau", 1_000_000, 50),   # Figure 3(a)
    "gau_n50000_k50": ("gau", 50_000, 50),        # Figure 3(b)
    "unb_n200000_k25": ("unb", 200_000, 25),      # Table 4
}
PHI_SET = ("gau", 200_000, 25)                    # Tables 6 and 7
NS = (10_000, 20_000, 50_000, 100_000, 200_000, 500_000, 1_000_000)   # Figure 4
N_KS = (10, 100)
N_SET = ("gau", 25)


def point_set(kind: str, n: int, clusters: int, seed: int) -> np.ndarray:
    """A 2-D set of the paper's three shapes on the [0, 100) scale (FP32)."""
    if kind == "unif":
        return I.unif_points(n, 2, seed, 0.0, SCALE)
    if kind == "gau":
        return I.gauss_mixture(n, 2, seed, clusters, SIGMA, 0.0, SCALE)
    if kind == "unb":
        return I.gauss_mixture(n, 2, seed, clusters, SIGMA, 0.0, SCALE, heavy_frac=0.5)
    raise ValueError(f"unknown set kind {kind!r}")


def _timed(fn):
    t0 = time.perf_counter()
    r = fn()
    return r, (time.perf_counter() - t0) * 1e3


def _solve(method: str, x, k: int, m: int, eps: float, phi: float, run: int):
    if method == "gon":
        return B.kc_gonzalez(x, k)
    if method == "mrg":
        return B.kc_mrg(x, k, m)
    if method == "eim":
        return B.kc_eim(x, k, eps=eps, phi=phi, seed=run)
    raise ValueError(method)


def check_guarantees(radii: dict, phi: float = PHI) -> list:
    """Violations of the bounds above for one (set, seed, k): radii maps a
    method to its radius (one run).  Returns a list of messages."""
    bad = []
    g = radii.get("gon")
    if g is None:
        return bad
    for meth, r in radii.items():
        if meth != "gon" and not g <= 2.0 * r:
            bad.append(f"r_gon {g} > 2 r_{meth} {r}")
    if "mrg" in radii and not radii["mrg"] <= 4.0 * g:
        bad.append(f"r_mrg {radii['mrg']} > 4 r_gon {g}")
    if "eim" in radii and phi >= 6.0 and not radii["eim"] <= 10.0 * g:
        bad.append(f"r_eim {radii['eim']} > 10 r_gon {g}")
    return bad


def k_sweep(sets=None, ks=KS, seeds: int = 3, runs: int = 2, m: int = M, eps: float = EPS, phi: float = PHI,
            methods=("mrg", "eim", "gon"), device: str = "cuda", warmup: bool = True):
    """Mean wall time per call (ms, synchronous C-ABI call, points already on
    the device) and mean radius per (set, method, k).  Returns (rows,
    violations)."""
    import torch
    sets = SETS if sets is None else sets
    rows, violations = [], []
    for name, (kind, n, clusters) in sets.items():
        acc = {}
        for s in range(seeds):
            x = torch.from_numpy(point_set(kind, n, clusters, 5000 + s)).to(device)
            if warmup:
                for meth in methods:
                    _solve(meth, x, ks[0], m, eps, phi, 0)
            for k in ks:
                for run in range(runs):
                    radii = {}
                    for meth in methods:
                        res, ms = _timed(lambda: _solve(meth, x, k, m, eps, phi, run))
                        a = acc.setdefault((meth, k), [0.0, 0.0, 0])
                        a[0] += ms
                        a[1] += res.radius
                        a[2] += 1
                        radii[meth] = res.radius
                    for v in check_guarantees(radii, phi):
                        violations.append(f"{name} seed {s} k {k} run {run}: {v}")
        for (meth, k), (ms, rad, c) in sorted(acc.items(), key=lambda t: (t[0][1], t[0][0])):
            rows.append({"report": "k_sweep", "set": name, "n": n, "method": meth, "k": k, "m": m,
                         "ms": ms / c, "radius": rad / c, "runs": c})
    return rows, violations


def n_sweep(ns=NS, ks=N_KS, seeds: int = 3, runs: int = 2, m: int = M, eps: float = EPS, phi: float = PHI,
            set_shape=N_SET, methods=("mrg", "eim", "gon"), device: str = "cuda"):
    """Mean wall time and radius per (n, method, k) for fixed k over n
    (Figure 4); the guarantees are checked on every run."""
    kind, clusters = set_shape
    rows, violations = [], []
    for n in ns:
        r, bad = k_sweep({f"{kind}_n{n}_k{clusters}": (kind, n, clusters)}, ks=ks, seeds=seeds, runs=runs, m=m,
                         eps=eps, phi=phi, methods=methods, device=device)
        for row in r:
            row["report"] = "n_sweep"
            row["set"] = f"{kind}_k{clusters}"
        rows += r
        violations += bad
    return rows, violations


def phi_sweep(phis=PHIS, ks=KS, seeds: int = 3, runs: int = 2, eps: float = EPS, set_shape=PHI_SET,
              device: str = "cuda"):
    """EIM's mean radius and wall time per (phi, k) (Tables 6 and 7)."""
    import torch
    kind, n, clusters = set_shape
    acc = {}
    violations = []
    for s in range(seeds):
        x = torch.from_numpy(point_set(kind, n, clusters, 6000 + s)).to(device)
        B.kc_eim(x, ks[0], eps=eps, phi=phis[0], seed=0)
        for k in ks:
            g = B.kc_gonzalez(x, k).radius
            for phi in phis:
                for run in range(runs):
                    res, ms = _timed(lambda: B.kc_eim(x, k, eps=eps, phi=phi, seed=run))
                    a = acc.setdefault((phi, k), [0.0, 0.0, 0])
                    a[0] += ms
                    a[1] += res.radius
                    a[2] += 1
                    for v in check_guarantees({"gon": g, "eim": res.radius}, phi):
                        violations.append(f"phi {phi} seed {s} k {k} run {run}: {v}")
    rows = [{"report": "phi_sweep", "set": f"{kind}_n{n}_k{clusters}", "n": n, "phi": phi, "k": k,
             "ms": ms / c, "radius": rad / c, "runs": c}
            for (phi, k), (ms, rad, c) in sorted(acc.items(), key=lambda t: (t[0][1], t[0][0]))]
    return rows, violations


def markdown(rows) -> str:
    """Tables of radius and time over k (one per set), over n (one per k) or
    over phi."""
    out = []
    if not rows:
        return ""
    if rows[0]["report"] == "n_sweep":
        meths = list(dict.fromkeys(r["method"] for r in rows))
        cell = {(r["method"], r["k"], r["n"]): r for r in rows}
        for k in sorted(set(r["k"] for r in rows)):
            out.append(f"{rows[0]['set']}, k = {k}: ms per call | radius over n")
            out.append("| n | " + " | ".join(f"{m} ms" for m in meths) + " | " + " | ".join(meths) + " |")
            out.append("|---" * (1 + 2 * len(meths)) + "|")
            for n in sorted(set(r["n"] for r in rows if r["k"] == k)):
                ms = " | ".join(f"{cell[(m, k, n)]['ms']:.3g}" for m in meths)
                rad = " | ".join(f"{cell[(m, k, n)]['radius']:.4g}" for m in meths)
                out.append(f"| {n} | {ms} | {rad} |")
            out.append("")
    elif rows[0]["report"] == "k_sweep":
        for name in dict.fromkeys(r["set"] for r in rows):
            rs = [r for r in rows if r["set"] == name]
            meths = list(dict.fromkeys(r["method"] for r in rs))
            ks = sorted(set(r["k"] for r in rs))
            cell = {(r["method"], r["k"]): r for r in rs}
            out.append(f"{name}: radius | ms per call")
            out.append("| k | " + " | ".join(meths) + " | " + " | ".join(f"{m} ms" for m in meths) + " |")
            out.append("|---" * (1 + 2 * len(meths)) + "|")
            for k in ks:
                rad = " | ".join(f"{cell[(m, k)]['radius']:.4g}" for m in meths)
                ms = " | ".join(f"{cell[(m, k)]['ms']:.3g}" for m in meths)
                out.append(f"| {k} | {rad} | {ms} |")
            out.append("")
    else:
        phis = sorted(set(r["phi"] for r in rows))
        ks = sorted(set(r["k"] for r in rows))
        cell = {(r["phi"], r["k"]): r for r in rows}
        out.append(f"{rows[0]['set']}: EIM radius | ms per call over phi")
        out.append("| k | " + " | ".join(f"phi {p:g}" for p in phis) + " | " +
                   " | ".join(f"phi {p:g} ms" for p in phis) + " |")
        out.append("|---" * (1 + 2 * len(phis)) + "|")
        for k in ks:
            rad = " | ".join(f"{cell[(p, k)]['radius']:.4g}" for p in phis)
            ms = " | ".join(f"{cell[(p, k)]['ms']:.3g}" for p in phis)
            out.append(f"| {k} | {rad} | {ms} |")
        out.append("")
    return "\n".join(out)
