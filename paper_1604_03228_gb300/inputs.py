"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers; it holds none of the k-center arithmetic, so
both the CUDA path's tests and the CPU oracle can take their inputs from it.

Every random number comes from a counter-based splitmix64 stream (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
output i of the stream with state s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15),
with Stafford's "variant 13" finaliser as mix64.  Integer work is exact in
numpy uint64, so integer inputs are bit-identical on x86 and Arm.  Gaussians
use the Box-Muller transform in FP64 and are then rounded to FP32.

Shapes follow the paper's synthetic sets (Section 7.3, "Data sets"): uniform
points in a box (Unif), k' Gaussian clusters of equal expected size (Gau), and
an unbalanced mixture with a heavy first cluster (UnB).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TAG_MUL = np.uint64(0xD1B54A32D192ED03)


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output finaliser (uint64 in, uint64 out, wraps mod 2**64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _state(seed: int, tag: int) -> np.uint64:
    """Independent stream state for (seed, tag)."""
    with np.errstate(over="ignore"):
        s = mix64(np.array([seed], dtype=np.uint64))[0]
        s = mix64(np.array([s ^ (np.uint64(tag) * _TAG_MUL)], dtype=np.uint64))[0]
    return s


def u64_stream(seed: int, tag: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the stream (seed, tag)."""
    s = _state(seed, tag)
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(s + i * GOLDEN_GAMMA)


def uniform01(seed: int, tag: int, count: int) -> np.ndarray:
    """FP64 uniforms in [0, 1) with 53 random bits."""
    u = u64_stream(seed, tag, count) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_int(seed: int, tag: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on {lo, ..., hi} (inclusive), exact: ((u >> 32) * span) >> 32."""
    span = np.uint64(hi - lo + 1)
    assert 0 < int(span) < (1 << 32)
    u = u64_stream(seed, tag, count) >> np.uint64(32)
    return (u * span >> np.uint64(32)).astype(np.int64) + lo


def normal(seed: int, tag: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller (one cosine branch per pair of uniforms)."""
    u = uniform01(seed, tag, 2 * count)
    u1 = 1.0 - u[0::2]                  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------- point sets

def unif_points(n: int, d: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Unif: n points uniform in [lo, hi)^d, FP32, row-major n x d."""
    u = uniform01(seed, 1, n * d).reshape(n, d)
    return (lo + (hi - lo) * u).astype(np.float32)


def int_points(n: int, d: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Integer coordinates uniform on {lo..hi}, int32, row-major n x d."""
    return uniform_int(seed, 2, n * d, lo, hi).reshape(n, d).astype(np.int32)


def gauss_mixture(n: int, d: int, seed: int, clusters: int, sigma: float,
                  mean_lo: float, mean_hi: float, heavy_frac: float = 0.0) -> np.ndarray:
    """Gau / UnB: isotropic Gaussian clusters, FP32, row-major n x d.

    Means are uniform in [mean_lo, mean_hi)^d.  Each point picks a cluster
    uniformly; with heavy_frac > 0 (UnB) a point first goes to cluster 0 with
    probability heavy_frac and otherwise picks uniformly among the others.
    """
    means = mean_lo + (mean_hi - mean_lo) * uniform01(seed, 3, clusters * d).reshape(clusters, d)
    if heavy_frac > 0.0 and clusters > 1:
        heavy = uniform01(seed, 4, n) < heavy_frac
        other = 1 + uniform_int(seed, 5, n, 0, clusters - 2)
        comp = np.where(heavy, 0, other)
    else:
        comp = uniform_int(seed, 5, n, 0, clusters - 1)
    z = normal(seed, 6, n * d).reshape(n, d)
    return (means[comp] + sigma * z).astype(np.float32)


def collinear_points(n: int, d: int = 1) -> np.ndarray:
    """Points i * e_0 for i = 0..n-1 (int32), the evenly spaced line."""
    p = np.zeros((n, d), dtype=np.int32)
    p[:, 0] = np.arange(n, dtype=np.int32)
    return p


# ------------------------------------------------------------ partitions

def zipf_partition_sizes(n: int, m: int, s: float) -> np.ndarray:
    """Sizes of m contiguous parts with Zipf(s) proportions.

    Part i (1-based) gets floor(n * i**-s / H) points with H = sum_i i**-s;
    the remainder goes one point each to the first parts.
    """
    w = np.arange(1, m + 1, dtype=np.float64) ** (-s)
    h = w.sum()
    sizes = np.floor(n * w / h).astype(np.int64)
    rem = n - int(sizes.sum())
    sizes[:rem] += 1
    return sizes


def offsets_from_sizes(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def even_offsets(n: int, m: int) -> np.ndarray:
    """m contiguous parts, each of size at most ceil(n / m)."""
    q = -(-n // m)
    off = np.minimum(np.arange(m + 1, dtype=np.int64) * q, n)
    return off


# ------------------------------------------------------ named workloads

@dataclass
class Workload:
    name: str
    points: np.ndarray
    k: int
    first: int = 0


def gon_int_10k() -> Workload:
    """n=10,000, d=2, int32 coordinates uniform in [0, 1023], seed 0, k=10."""
    return Workload("gon_int_n10000_d2_k10", int_points(10_000, 2, 0, 0, 1023), 10)


def gon_gau_1m(n: int = 1_000_000, k: int = 100) -> Workload:
    """n=1,000,000, d=10, 25 Gaussians (sigma 1, means U[-50,50]^10), seed 1, k=100."""
    return Workload(f"gon_radius_gau_n{n}_d10_k{k}",
                    gauss_mixture(n, 10, 1, 25, 1.0, -50.0, 50.0), k)


def gon_int13_1m(n: int = 1_000_000, k: int = 100) -> Workload:
    """Integer variant: n=1,000,000, d=10, coordinates uniform on {1..13}, seed 2."""
    return Workload(f"gon_int13_n{n}_d10_k{k}", int_points(n, 10, 2, 1, 13), k)


def mrg_unif_10m(n: int = 10_000_000, m: int = 64, k: int = 200):
    """n=10M, d=16, U[0,1)^16 (seed 3); m Zipf(1.1) contiguous parts; k=200."""
    pts = unif_points(n, 16, 3)
    off = offsets_from_sizes(zipf_partition_sizes(n, m, 1.1))
    return pts, off, k


def eim_gau_8m(n: int = 8_000_000, d: int = 64, seed: int = 4):
    """n=8M, d=64, 100 clusters (sigma 0.5, means U[-10,10]^64), seed 4."""
    return gauss_mixture(n, d, seed, 100, 0.5, -10.0, 10.0)


@dataclass
class Instance:
    points: np.ndarray
    k: int
    kind: str


def batch_instance(i: int, n_lo: int = 1_000, n_hi: int = 200_000) -> Instance:
    """Instance i of the many-instance workload (seed 1000 + i).

    n = round(exp(U[ln n_lo, ln n_hi])), d uniform on {3, 8, 32}, k uniform on
    {8..128}, kind uniform on {unif, gau, unb}: Unif [0,1)^d; Gau 25 clusters,
    sigma 0.1, means U[0,1)^d; UnB the same with 90% of points in cluster 0.
    """
    seed = 1000 + i
    u = uniform01(seed, 10, 1)[0]
    n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
    d = (3, 8, 32)[int(uniform_int(seed, 11, 1, 0, 2)[0])]
    k = int(uniform_int(seed, 12, 1, 8, 128)[0])
    kind = ("unif", "gau", "unb")[int(uniform_int(seed, 13, 1, 0, 2)[0])]
    if kind == "unif":
        pts = unif_points(n, d, seed)
    elif kind == "gau":
        pts = gauss_mixture(n, d, seed, 25, 0.1, 0.0, 1.0)
    else:
        pts = gauss_mixture(n, d, seed, 25, 0.1, 0.0, 1.0, heavy_frac=0.9)
    return Instance(pts, k, kind)
