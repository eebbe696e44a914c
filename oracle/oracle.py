"""Python face of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``kc_oracle.c`` compiled as a
plain shared library (``oracle/build.py``) and converts numpy arrays; every
computation happens in that C file, which shares nothing with the CUDA path.

Modes (see the C file): "f64" (FP32 points widened to double), "f32" (the
canonical FP32 squared distance, used where an argmax must be decided in a
float kernel's precision) and "i64" (int32 points, exact).
"""
from __future__ import annotations

import ctypes as ct
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_MODES = {"f64": 0, "f32": 1, "i64": 2}


class _Metric(ct.Structure):
    _fields_ = [("pts", ct.c_void_p), ("n", ct.c_int64), ("d", ct.c_int32), ("mode", ct.c_int32)]


def lib():
    global _LIB
    if _LIB is None:
        from . import build as _b
        path = _b.build()
        L = ct.CDLL(path)
        P = ct.POINTER
        L.orc_gon.restype = ct.c_int64
        L.orc_gon.argtypes = [P(_Metric), ct.c_void_p, ct.c_int64, ct.c_int64, ct.c_int64,
                              ct.c_void_p, ct.c_void_p, P(ct.c_double)]
        L.orc_radius.restype = ct.c_double
        L.orc_radius.argtypes = [P(_Metric), ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_int64,
                                 P(ct.c_int64)]
        L.orc_eval_sequence.restype = None
        L.orc_eval_sequence.argtypes = [P(_Metric), ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p]
        L.orc_mrg.restype = ct.c_int64
        L.orc_mrg.argtypes = [P(_Metric), ct.c_int64, ct.c_int64, ct.c_void_p, ct.c_void_p,
                              ct.c_void_p, ct.c_void_p, P(ct.c_double)]
        L.orc_mrg_rounds.restype = ct.c_int64
        L.orc_mrg_rounds.argtypes = [P(_Metric), ct.c_int64, ct.c_int64, ct.c_void_p, ct.c_int64, ct.c_int64,
                                     ct.c_void_p, P(ct.c_int64), ct.c_void_p, P(ct.c_double)]
        L.orc_uniform.restype = ct.c_double
        L.orc_uniform.argtypes = [ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_uint64]
        L.orc_eim.restype = ct.c_int64
        L.orc_eim.argtypes = [P(_Metric), ct.c_int64, ct.c_double, ct.c_double, ct.c_uint64,
                              ct.c_void_p, P(ct.c_double), ct.c_void_p, ct.c_void_p,
                              ct.c_void_p, ct.c_int64]
        L.orc_mind.restype = None
        L.orc_mind.argtypes = [P(_Metric), ct.c_void_p, ct.c_int64, ct.c_void_p]
        _LIB = L
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Points:
    """Keeps the (contiguous) coordinate array alive next to its C metric."""

    def __init__(self, pts: np.ndarray, mode: str):
        if mode == "i64":
            arr = np.ascontiguousarray(pts, dtype=np.int32)
            if arr.size:
                span = int(arr.max()) - int(arr.min())
                if arr.shape[1] * span * span >= (1 << 53):
                    raise ValueError("integer range too large for exact comparison in double")
        else:
            arr = np.ascontiguousarray(pts, dtype=np.float32)
        self.arr = arr
        self.m = _Metric(arr.ctypes.data, arr.shape[0], arr.shape[1], _MODES[mode])


def default_mode(pts: np.ndarray) -> str:
    return "i64" if np.issubdtype(pts.dtype, np.integer) else "f64"


@dataclass
class GonResult:
    centers: np.ndarray      # int64 [k_out], global indices in selection order
    sel2: np.ndarray         # squared distance of each center when chosen
    radius2: float           # squared covering radius in the selection metric
    radius: float            # covering radius recomputed in f64 (i64 for ints)


def gonzalez(pts: np.ndarray, k: int, first: int = 0, mode: str | None = None,
             subset: np.ndarray | None = None) -> GonResult:
    """GON (Section 3.1) with lowest-index ties and early stop at radius 0."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    n = P.arr.shape[0] if subset is None else len(subset)
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int64)
    first_pos = first
    C = np.zeros(max(k, 1), dtype=np.int64)
    s2 = np.zeros(max(k, 1), dtype=np.float64)
    r2 = ct.c_double()
    kout = lib().orc_gon(ct.byref(P.m), _ptr(sub), n, k, first_pos, _ptr(C), _ptr(s2), ct.byref(r2))
    C = C[:kout].copy()
    rad = radius(pts, C, mode="i64" if mode == "i64" else "f64", subset=sub)[0]
    return GonResult(C, s2[:kout].copy(), r2.value, rad)


def radius(pts: np.ndarray, centers: np.ndarray, mode: str | None = None,
           subset: np.ndarray | None = None):
    """(radius, argmax point, radius^2): max over points of distance to nearest center."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    C = np.ascontiguousarray(centers, dtype=np.int64)
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int64)
    n = P.arr.shape[0] if sub is None else len(sub)
    am = ct.c_int64()
    r2 = lib().orc_radius(ct.byref(P.m), _ptr(sub), n, _ptr(C), len(C), ct.byref(am))
    return math.sqrt(r2), am.value, r2


def eval_sequence(pts: np.ndarray, centers: np.ndarray, mode: str | None = None):
    """(sel2[k], max2[k+1]) for a given center sequence (see the C file)."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    C = np.ascontiguousarray(centers, dtype=np.int64)
    sel2 = np.zeros(len(C), dtype=np.float64)
    max2 = np.zeros(len(C) + 1, dtype=np.float64)
    lib().orc_eval_sequence(ct.byref(P.m), _ptr(C), len(C), _ptr(sel2), _ptr(max2))
    return sel2, max2


def mind(pts: np.ndarray, centers: np.ndarray, mode: str | None = None) -> np.ndarray:
    """Squared distance of every point to its nearest center."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    C = np.ascontiguousarray(centers, dtype=np.int64)
    out = np.zeros(P.arr.shape[0], dtype=np.float64)
    lib().orc_mind(ct.byref(P.m), _ptr(C), len(C), _ptr(out))
    return out


@dataclass
class MrgResult:
    centers: np.ndarray
    round1: list            # per part: int64 array of its centers (selection order)
    radius2: float
    radius: float


def mrg(pts: np.ndarray, k: int, offsets: np.ndarray, mode: str | None = None) -> MrgResult:
    """Two-round MRG (Algorithm 1) on contiguous parts [off[i], off[i+1])."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    m = len(off) - 1
    r1 = np.full(m * k, -1, dtype=np.int64)
    r1k = np.zeros(m, dtype=np.int64)
    C = np.zeros(k, dtype=np.int64)
    r2 = ct.c_double()
    kout = lib().orc_mrg(ct.byref(P.m), k, m, _ptr(off), _ptr(r1), _ptr(r1k), _ptr(C), ct.byref(r2))
    C = C[:kout].copy()
    rounds = [r1[i * k:i * k + r1k[i]].copy() for i in range(m)]
    rad = radius(pts, C, mode="i64" if mode == "i64" else "f64")[0]
    return MrgResult(C, rounds, r2.value, rad)


@dataclass
class MrgRoundsResult:
    centers: np.ndarray
    rounds: int              # including the final GON
    sizes: np.ndarray        # |S| after each round before the final one
    radius2: float
    radius: float


def mrg_rounds(pts: np.ndarray, k: int, offsets: np.ndarray, capacity: int, mode: str | None = None,
               max_rounds: int = 64) -> MrgRoundsResult:
    """MRG with machine capacity c (Algorithm 1 with its while loop): round 1
    on the given parts, further rounds on ceil(|S|/c) contiguous parts of the
    union until |S| <= c, then GON on S."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    m = len(off) - 1
    C = np.zeros(k, dtype=np.int64)
    sizes = np.zeros(max_rounds, dtype=np.int64)
    rounds = ct.c_int64()
    r2 = ct.c_double()
    kout = lib().orc_mrg_rounds(ct.byref(P.m), k, m, _ptr(off), capacity, max_rounds, _ptr(sizes),
                                ct.byref(rounds), _ptr(C), ct.byref(r2))
    if kout < 0:
        raise ValueError("capacity below 2k or too many rounds")
    C = C[:kout].copy()
    rad = radius(pts, C, mode="i64" if mode == "i64" else "f64")[0]
    return MrgRoundsResult(C, rounds.value, sizes[:rounds.value - 1].copy(), r2.value, rad)


def uniform(seed: int, it: int, x: int, stream: int) -> float:
    return lib().orc_uniform(seed, it, x, stream)


@dataclass
class EimResult:
    centers: np.ndarray
    radius2: float
    radius: float
    iterations: int
    s_size: int
    r_size: int
    sample: np.ndarray       # C = S u R, ascending
    trace: np.ndarray        # [iterations, 8]: pS, pH, |S|, |H|, v, d(v,S)^2, |R| after, p


def eim(pts: np.ndarray, k: int, eps: float, phi: float, seed: int,
        mode: str | None = None) -> EimResult:
    """EIM (Algorithms 2 and 3 with phi) followed by GON on the sample."""
    mode = mode or default_mode(pts)
    P = _Points(pts, mode)
    n = P.arr.shape[0]
    C = np.zeros(k, dtype=np.int64)
    r2 = ct.c_double()
    st = np.zeros(4, dtype=np.int64)
    sample = np.zeros(n, dtype=np.int64)
    cap = 256
    tr = np.zeros(cap * 8, dtype=np.float64)
    kout = lib().orc_eim(ct.byref(P.m), k, eps, phi, seed, _ptr(C), ct.byref(r2), _ptr(st), _ptr(sample),
                         _ptr(tr), cap)
    C = C[:kout].copy()
    rad = radius(pts, C, mode="i64" if mode == "i64" else "f64")[0]
    iters = int(st[0])
    return EimResult(C, r2.value, rad, iters, int(st[1]), int(st[2]), sample[:st[3]].copy(),
                     tr.reshape(cap, 8)[:min(iters, cap)].copy())
