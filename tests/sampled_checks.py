"""Checks of full-size results that the oracle cannot recompute whole, made on
a seeded sample of the points in the oracle's own modes.

- farthest_steps: every chosen center must be at least as far (canonical FP32
  squared distance to the centers chosen before it) as every sampled point at
  that step, since the selection took the maximum over all points.
- radius_checks: the returned FP64 radius must equal the FP64 nearest-center
  distance of the returned argmax point, and bound that of every sampled point.
"""
import numpy as np

from oracle import oracle as O


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted distinct row indices, seeded."""
    rng = np.random.default_rng(seed)
    return np.unique(rng.integers(0, n, size=min(count, n), dtype=np.int64))


def farthest_steps(pts: np.ndarray, centers: np.ndarray, sample: np.ndarray, mode: str = "f32") -> list:
    """Steps j >= 1 at which a sampled point is farther from centers[0..j-1]
    than centers[j] (empty when the sequence passes)."""
    centers = np.asarray(centers, dtype=np.int64)
    idx = np.unique(np.concatenate([np.asarray(sample, dtype=np.int64), centers]))
    local = np.searchsorted(idx, centers)
    sel2, max2 = O.eval_sequence(pts[idx], local, mode=mode)
    return [j for j in range(1, len(centers)) if not sel2[j] >= max2[j]]


def radius_checks(pts: np.ndarray, centers: np.ndarray, radius: float, argmax: int, sample: np.ndarray) -> list:
    """Failures of the two radius properties (empty when both hold)."""
    bad = []
    r_am = O.radius(pts, centers, mode="f64", subset=np.array([argmax]))[0]
    if r_am != radius:
        bad.append(f"argmax point {argmax}: nearest-center distance {r_am!r} != radius {radius!r}")
    r_s, am_s, _ = O.radius(pts, centers, mode="f64", subset=np.asarray(sample, dtype=np.int64))
    if not r_s <= radius:
        bad.append(f"sampled point {am_s} at {r_s!r} beyond radius {radius!r}")
    return bad
