"""Thin Python binding of the C ABI in include/kcenter.h (ctypes).

Each ``kc_*`` function here has the name of the C entry point it calls and
only marshals arguments: it turns torch tensors (CUDA or CPU) or numpy arrays
into pointers and sizes, allocates the output buffers next to the input, and
raises ``KCError`` on a non-zero status.  Every step of the computation runs
in the CUDA library; there is no CPU fallback.  If the library is missing or
fails to build, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

KC_OK, KC_ERR_ARG, KC_ERR_CUDA, KC_ERR_OOM, KC_ERR_TIMEOUT, KC_ERR_RANGE, KC_ERR_NONFINITE, KC_ERR_BOUNDS = range(8)
KC_F32, KC_I32 = 0, 1
KC_ASYNC = 1
KC_AUTOTUNE = 2
KC_TEST_WITHHOLD = 0x80000000
KC_TEST_BAD_INDEX = 0x40000000
STATUS_NAMES = {0: "KC_OK", 1: "KC_ERR_ARG", 2: "KC_ERR_CUDA", 3: "KC_ERR_OOM", 4: "KC_ERR_TIMEOUT",
                5: "KC_ERR_RANGE", 6: "KC_ERR_NONFINITE", 7: "KC_ERR_BOUNDS"}


class KCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class kc_opts(ct.Structure):
    _fields_ = [("dtype", ct.c_int32), ("flags", ct.c_uint32), ("sweep", ct.c_int32),
                ("reserved", ct.c_int32), ("seed", ct.c_uint64), ("phi", ct.c_double),
                ("stream", ct.c_void_p), ("timeout_ms", ct.c_int64)]


KC_SWEEP_F32, KC_SWEEP_BF16, KC_SWEEP_FP8, KC_SWEEP_FP16 = 0, 1, 2, 3
_SWEEPS = {"f32": 0, "bf16": 1, "fp8": 2, "fp16": 3, None: 0, 0: 0, 1: 1, 2: 2, 3: 3}


_LIB = None


def load(path: str | None = None):
    """Build (if stale) and load libkcenter.so (or the library that the
    KC_LIBRARY environment variable names, e.g. the checked build); raises if
    that fails."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or os.environ.get("KC_LIBRARY") or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library missing: {path}")
    L = ct.CDLL(path)
    vp, i64, i32, dbl = ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_double
    popts = ct.POINTER(kc_opts)
    L.kc_gonzalez.restype = ct.c_int
    L.kc_gonzalez.argtypes = [vp, i64, i32, i32, i64, vp, vp, vp, popts]
    L.kc_radius.restype = ct.c_int
    L.kc_radius.argtypes = [vp, i64, i32, vp, i32, vp, vp, popts]
    L.kc_gonzalez_noalloc.restype = ct.c_int
    L.kc_gonzalez_noalloc.argtypes = [vp, i64, i32, i32, i64, vp, vp, vp, popts]
    L.kc_mrg.restype = ct.c_int
    L.kc_mrg.argtypes = [vp, i64, i32, i32, i32, vp, vp, vp, vp, popts]
    L.kc_mrg_rounds.restype = ct.c_int
    L.kc_mrg_rounds.argtypes = [vp, i64, i32, i32, i32, vp, i64, vp, vp, vp, vp, popts]
    L.kc_eim.restype = ct.c_int
    L.kc_eim.argtypes = [vp, i64, i32, i32, dbl, vp, vp, vp, popts]
    L.kc_gonzalez_batch.restype = ct.c_int
    L.kc_gonzalez_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, popts]
    L.kc_batch_plan_create.restype = ct.c_int
    L.kc_batch_plan_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, popts, ct.POINTER(vp)]
    L.kc_batch_plan_run.restype = ct.c_int
    L.kc_batch_plan_run.argtypes = [vp, vp]
    L.kc_batch_plan_wait.restype = ct.c_int
    L.kc_batch_plan_wait.argtypes = [vp]
    L.kc_batch_plan_info.restype = ct.c_int
    L.kc_batch_plan_info.argtypes = [vp, vp, vp, vp, vp]
    L.kc_batch_plan_destroy.restype = ct.c_int
    L.kc_batch_plan_destroy.argtypes = [vp]
    L.kc_sync.restype = ct.c_int
    L.kc_sync.argtypes = [vp]
    L.kc_last_error.restype = ct.c_char_p
    L.kc_release.restype = None
    L.kc_version.restype = ct.c_char_p
    L.kc_trace_enable.restype = None
    L.kc_trace_enable.argtypes = [i32]
    L.kc_trace_read.restype = i32
    L.kc_trace_read.argtypes = [ct.POINTER(kc_trace_rec), i32]
    L.kc_launch_count.restype = i64
    L.kc_counters.restype = i32
    L.kc_counters.argtypes = [vp, i32]
    L.kc_last_fp32_radius.restype = ct.c_int
    L.kc_last_fp32_radius.argtypes = [vp, ct.POINTER(ct.c_double)]
    L.kc_read_sweep.restype = ct.c_int
    L.kc_read_sweep.argtypes = [vp, ct.c_size_t, i32, vp, vp]
    _LIB = L
    return L


def kc_last_fp32_radius(stream=None) -> float:
    """The canonical FP32 covering radius of the last solve or radius call
    on `stream` (default: torch's current stream): with the FP64 radius that
    call returned, the result's FP32 error against FP64."""
    L = load()
    h = None
    if stream is not None:
        h = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    else:
        try:
            h = int(_torch().cuda.current_stream().cuda_stream)
        except Exception:
            h = None
    out = ct.c_double()
    _check(L, L.kc_last_fp32_radius(h, ct.byref(out)))
    return out.value


def kc_read_sweep(buf, reps: int, sink, *, stream=None) -> None:
    """Enqueue one kernel that reads the CUDA tensor `buf` `reps` times
    (16-byte loads, whole GPU) into the 8-byte CUDA tensor `sink`; time it
    with events for a read bandwidth (the L2 roofline denominator)."""
    L = load()
    nbytes = buf.numel() * buf.element_size()
    st = L.kc_read_sweep(_ptr(buf), nbytes, reps, _ptr(sink), _stream_handle(buf, stream))
    _check(L, st)


def kc_counters():
    """Diagnostics since the last call: (sweep exact rechecks, sweep buffer
    overflows, prune undecided pairs, prune points, prune |R| x |S| pairs,
    sweep rechecks with a lagging memo, GON kernel cycles in sweep / recheck /
    exchange summed over CTAs, largest per-CTA sweep and sweep + recheck
    totals, tensor-core MMA issuer cycles waiting for a center tile / a free
    accumulator / a point tile and in all, summed over CTAs)."""
    out = np.zeros(15, dtype=np.int64)
    if load().kc_counters(out.ctypes.data, 15) < 0:
        raise KCError(KC_ERR_CUDA, "kc_counters failed")
    return tuple(int(v) for v in out)


class kc_trace_rec(ct.Structure):
    _fields_ = [("name", ct.c_char * 24), ("kernels", ct.c_int32), ("ms", ct.c_float)]


def kc_trace_enable(on: bool = True) -> None:
    load().kc_trace_enable(1 if on else 0)


def kc_trace_read(cap: int = 65536):
    """[(step name, kernels, device ms)] recorded since the last read."""
    L = load()
    buf = (kc_trace_rec * cap)()
    cnt = L.kc_trace_read(buf, cap)
    return [(buf[i].name.decode(), int(buf[i].kernels), float(buf[i].ms)) for i in range(min(cnt, cap))]


def kc_launch_count() -> int:
    return int(load().kc_launch_count())


def library_path() -> str:
    return _build.LIB


# ----------------------------------------------------------------- helpers

def _torch():
    import torch
    return torch


def _is_torch(x) -> bool:
    try:
        import torch
    except ImportError:
        return False
    return isinstance(x, torch.Tensor)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr()
    return x.ctypes.data


def _points(points):
    """(contiguous points, n, d, dtype code) for a 2-D float32/int32 array."""
    if _is_torch(points):
        torch = _torch()
        if points.dim() != 2:
            raise ValueError("points must be 2-D (n, d)")
        if points.dtype not in (torch.float32, torch.int32):
            raise TypeError("points must be float32 or int32")
        p = points.contiguous()
        code = KC_F32 if p.dtype == torch.float32 else KC_I32
    else:
        p = np.ascontiguousarray(points)
        if p.ndim != 2:
            raise ValueError("points must be 2-D (n, d)")
        if p.dtype == np.float32:
            code = KC_F32
        elif p.dtype == np.int32:
            code = KC_I32
        else:
            raise TypeError("points must be float32 or int32")
    return p, int(p.shape[0]), int(p.shape[1]), code


def _empty_like_place(ref, n, dtype_np, pin=False):
    """Output buffer on the same device as `ref` (torch) or a numpy array."""
    if _is_torch(ref):
        torch = _torch()
        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float64: torch.float64}[dtype_np]
        if ref.is_cuda:
            return torch.empty(n, dtype=tdt, device=ref.device)
        return torch.empty(n, dtype=tdt, pin_memory=pin)
    return np.empty(n, dtype=dtype_np)


def _stream_handle(ref, stream):
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    if _is_torch(ref) and ref.is_cuda:
        return int(_torch().cuda.current_stream(ref.device).cuda_stream)
    return None


def _opts(code, ref, stream, flags, timeout_ms, seed=0, phi=6.0, sweep=None):
    o = kc_opts()
    o.dtype = code
    o.flags = flags
    o.sweep = _SWEEPS[sweep]
    o.seed = seed
    o.phi = phi
    o.stream = _stream_handle(ref, stream)
    o.timeout_ms = timeout_ms
    return o


def _check(L, st):
    if st != KC_OK:
        raise KCError(st, L.kc_last_error().decode(errors="replace"))


def _item(x):
    if _is_torch(x):
        return x[0].item()
    return x[0].item()


@dataclass
class GonResult:
    centers: object        # int64 [k_out] (tensor or ndarray, same place as the input)
    k_out: int
    radius: float


@dataclass
class RadiusResult:
    radius: float
    argmax: int


# --------------------------------------------------------------- entry points

def kc_gonzalez(points, k: int, first: int = 0, *, stream=None, flags: int = 0,
                timeout_ms: int = 0, out=None, sweep=None):
    """GON (Section 3.1) through the C ABI.  With flags=KC_ASYNC returns the
    raw device outputs (centers[k], k_out[1], radius[1]) without waiting."""
    L = load()
    p, n, d, code = _points(points)
    if out is None:
        centers = _empty_like_place(p, k, np.int64)
        k_out = _empty_like_place(p, 1, np.int32)
        radius = _empty_like_place(p, 1, np.float64)
    else:
        centers, k_out, radius = out
    o = _opts(code, p, stream, flags, timeout_ms, sweep=sweep)
    st = L.kc_gonzalez(_ptr(p), n, d, k, first, _ptr(centers), _ptr(k_out), _ptr(radius), ct.byref(o))
    _check(L, st)
    if flags & KC_ASYNC:
        return centers, k_out, radius
    kk = int(_item(k_out))
    return GonResult(centers[:kk], kk, float(_item(radius)))


def kc_gonzalez_noalloc(points, k: int, first: int = 0, *, stream=None, timeout_ms: int = 0,
                        out=None):
    """GON through the entry point that allocates nothing (all scratch in a
    fixed static device array; device tensors only).  For callers that must
    not allocate device memory during a call: see include/kcenter.h."""
    L = load()
    p, n, d, code = _points(points)
    if not (_is_torch(p) and p.is_cuda):
        raise TypeError("kc_gonzalez_noalloc takes CUDA tensors")
    torch = _torch()
    if out is None:
        centers = torch.empty(k, dtype=torch.int64, device=p.device)
        k_out = torch.empty(1, dtype=torch.int32, device=p.device)
        radius = torch.empty(1, dtype=torch.float64, device=p.device)
    else:
        centers, k_out, radius = out
    o = _opts(code, p, stream, 0, timeout_ms)
    st = L.kc_gonzalez_noalloc(_ptr(p), n, d, k, first, _ptr(centers), _ptr(k_out), _ptr(radius),
                               ct.byref(o))
    _check(L, st)
    kk = int(k_out[0].item())
    return GonResult(centers[:kk], kk, float(radius[0].item()))


def kc_radius(points, centers, *, stream=None, flags: int = 0, timeout_ms: int = 0, out=None):
    """Covering radius of a center set through the C ABI."""
    L = load()
    p, n, d, code = _points(points)
    if _is_torch(centers):
        c = centers.to(_torch().int64).contiguous()
    else:
        c = np.ascontiguousarray(centers, dtype=np.int64)
    kc = int(c.shape[0])
    if out is None:
        radius = _empty_like_place(p, 1, np.float64)
        argmax = _empty_like_place(p, 1, np.int64)
    else:
        radius, argmax = out
    o = _opts(code, p, stream, flags, timeout_ms)
    st = L.kc_radius(_ptr(p), n, d, _ptr(c), kc, _ptr(radius), _ptr(argmax), ct.byref(o))
    _check(L, st)
    if flags & KC_ASYNC:
        return radius, argmax
    return RadiusResult(float(_item(radius)), int(_item(argmax)))


def kc_mrg(points, k: int, m: int, offsets=None, *, stream=None, flags: int = 0,
           timeout_ms: int = 0, out=None, sweep=None):
    """Two-round MRG (Algorithm 1) through the C ABI.  offsets: [m+1] part
    boundaries (array/tensor) or None for the balanced split."""
    L = load()
    p, n, d, code = _points(points)
    off = None
    if offsets is not None:
        if _is_torch(offsets):
            off = offsets.to(_torch().int64).contiguous()
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
        if int(off.shape[0]) != m + 1:
            raise ValueError("offsets must have m+1 entries")
    if out is None:
        centers = _empty_like_place(p, k, np.int64)
        k_out = _empty_like_place(p, 1, np.int32)
        radius = _empty_like_place(p, 1, np.float64)
    else:
        centers, k_out, radius = out
    o = _opts(code, p, stream, flags, timeout_ms, sweep=sweep)
    st = L.kc_mrg(_ptr(p), n, d, k, m, _ptr(off), _ptr(centers), _ptr(k_out), _ptr(radius), ct.byref(o))
    _check(L, st)
    if flags & KC_ASYNC:
        return centers, k_out, radius
    kk = int(_item(k_out))
    return GonResult(centers[:kk], kk, float(_item(radius)))


def kc_mrg_rounds(points, k: int, m: int, capacity: int, offsets=None, *, stream=None, timeout_ms: int = 0,
                  sweep=None):
    """MRG with a machine capacity (Algorithm 1 with its while loop) through
    the C ABI.  Returns (GonResult, rounds)."""
    L = load()
    p, n, d, code = _points(points)
    off = None
    if offsets is not None:
        off = offsets.to(_torch().int64).contiguous() if _is_torch(offsets) else np.ascontiguousarray(offsets, dtype=np.int64)
        if int(off.shape[0]) != m + 1:
            raise ValueError("offsets must have m+1 entries")
    centers = _empty_like_place(p, k, np.int64)
    k_out = _empty_like_place(p, 1, np.int32)
    radius = _empty_like_place(p, 1, np.float64)
    rounds = ct.c_int32(0)
    o = _opts(code, p, stream, 0, timeout_ms, sweep=sweep)
    st = L.kc_mrg_rounds(_ptr(p), n, d, k, m, _ptr(off), int(capacity), _ptr(centers), _ptr(k_out), _ptr(radius),
                         ct.byref(rounds), ct.byref(o))
    _check(L, st)
    kk = int(_item(k_out))
    return GonResult(centers[:kk], kk, float(_item(radius))), rounds.value


def kc_eim(points, k: int, eps: float = 0.1, phi: float = 6.0, seed: int = 0, *, stream=None,
           timeout_ms: int = 0, sweep=None):
    """EIM (Algorithms 2 and 3, then GON on the sample) through the C ABI."""
    L = load()
    p, n, d, code = _points(points)
    centers = _empty_like_place(p, k, np.int64)
    k_out = _empty_like_place(p, 1, np.int32)
    radius = _empty_like_place(p, 1, np.float64)
    o = _opts(code, p, stream, 0, timeout_ms, seed=seed, phi=phi, sweep=sweep)
    st = L.kc_eim(_ptr(p), n, d, k, float(eps), _ptr(centers), _ptr(k_out), _ptr(radius), ct.byref(o))
    _check(L, st)
    kk = int(_item(k_out))
    return GonResult(centers[:kk], kk, float(_item(radius)))


def kc_gonzalez_batch(points_list, ks, *, stream=None, flags: int = 0, timeout_ms: int = 0,
                      sweep=None):
    """GON on many independent instances (one persistent launch) through the
    C ABI.  Returns [GonResult] in input order (centers local to each instance)."""
    L = load()
    count = len(points_list)
    if count != len(ks):
        raise ValueError("one k per instance")
    ps = [_points(x) for x in points_list]
    codes = {c for (_, _, _, c) in ps}
    if len(codes) != 1:
        raise TypeError("all instances must share one dtype")
    ref = ps[0][0]
    ptrs = (ct.c_void_p * count)(*[_ptr(p) for (p, _, _, _) in ps])
    ns = np.array([n for (_, n, _, _) in ps], dtype=np.int64)
    ds = np.array([d for (_, _, d, _) in ps], dtype=np.int32)
    kk = np.array([int(k) for k in ks], dtype=np.int32)
    outs = [_empty_like_place(p, max(1, min(int(k), n)), np.int64) for (p, n, _, _), k in zip(ps, ks)]
    cptrs = (ct.c_void_p * count)(*[_ptr(c) for c in outs])
    k_out = _empty_like_place(ref, count, np.int32)
    radii = _empty_like_place(ref, count, np.float64)
    o = _opts(codes.pop(), ref, stream, flags, timeout_ms, sweep=sweep)
    st = L.kc_gonzalez_batch(count, ptrs, ns.ctypes.data, ds.ctypes.data, kk.ctypes.data, cptrs,
                             _ptr(k_out), _ptr(radii), ct.byref(o))
    _check(L, st)
    if flags & KC_ASYNC:
        return outs, k_out, radii
    ko = k_out.cpu().numpy() if _is_torch(k_out) else k_out
    rr = radii.cpu().numpy() if _is_torch(radii) else radii
    return [GonResult(outs[i][:int(ko[i])], int(ko[i]), float(rr[i])) for i in range(count)]


class BatchPlan:
    """A kc_batch_plan handle with the device outputs it is bound to:
    centers (one int64 tensor per instance), k_out and radii."""

    def __init__(self, handle, points, centers, k_out, radii):
        self.handle = handle
        self.points = points      # keeps the bound inputs alive
        self.centers = centers
        self.k_out = k_out
        self.radii = radii

    def results(self):
        ko = self.k_out.cpu().numpy()
        rr = self.radii.cpu().numpy()
        return [GonResult(self.centers[i][:int(ko[i])], int(ko[i]), float(rr[i])) for i in range(len(self.centers))]

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().kc_batch_plan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def kc_batch_plan_create(points_list, ks, *, sweep=None, flags: int = 0, timeout_ms: int = 0) -> BatchPlan:
    """Prepare the batched GON of device tensors `points_list` as a CUDA
    graph (C ABI kc_batch_plan_create); outputs are allocated on the device
    and bound to the plan."""
    L = load()
    torch = _torch()
    count = len(points_list)
    if count != len(ks):
        raise ValueError("one k per instance")
    ps = [_points(x) for x in points_list]
    codes = {c for (_, _, _, c) in ps}
    if len(codes) != 1:
        raise TypeError("all instances must share one dtype")
    ref = ps[0][0]
    if not _is_torch(ref) or not ref.is_cuda:
        raise TypeError("a batch plan takes CUDA tensors")
    ptrs = (ct.c_void_p * count)(*[_ptr(p) for (p, _, _, _) in ps])
    ns = np.array([n for (_, n, _, _) in ps], dtype=np.int64)
    ds = np.array([d for (_, _, d, _) in ps], dtype=np.int32)
    kk = np.array([int(k) for k in ks], dtype=np.int32)
    outs = [torch.empty(max(1, min(int(k), n)), dtype=torch.int64, device=ref.device)
            for (_, n, _, _), k in zip(ps, ks)]
    cptrs = (ct.c_void_p * count)(*[_ptr(c) for c in outs])
    k_out = torch.empty(count, dtype=torch.int32, device=ref.device)
    radii = torch.empty(count, dtype=torch.float64, device=ref.device)
    o = _opts(codes.pop(), ref, None, flags, timeout_ms, sweep=sweep)
    h = ct.c_void_p()
    st = L.kc_batch_plan_create(count, ptrs, ns.ctypes.data, ds.ctypes.data, kk.ctypes.data, cptrs,
                                _ptr(k_out), _ptr(radii), ct.byref(o), ct.byref(h))
    _check(L, st)
    return BatchPlan(h.value, [p for (p, _, _, _) in ps], outs, k_out, radii)


def kc_batch_plan_run(plan: BatchPlan, stream=None) -> None:
    """Enqueue one replay of the plan's graph on `stream` (default: torch's current stream)."""
    L = load()
    _check(L, L.kc_batch_plan_run(plan.handle, _stream_handle(plan.k_out, stream)))


def kc_batch_plan_wait(plan: BatchPlan):
    """Wait for the plan's last run; return its results ([GonResult])."""
    L = load()
    _check(L, L.kc_batch_plan_wait(plan.handle))
    return plan.results()


def kc_batch_plan_info(plan: BatchPlan):
    """(theta, group-solved instances, their CTAs, grid size)."""
    L = load()
    th = ct.c_double()
    nh, gh, gr = ct.c_int32(), ct.c_int32(), ct.c_int32()
    _check(L, L.kc_batch_plan_info(plan.handle, ct.byref(th), ct.byref(nh), ct.byref(gh), ct.byref(gr)))
    return th.value, nh.value, gh.value, gr.value


def kc_batch_plan_destroy(plan: BatchPlan) -> None:
    if plan.handle:
        L = load()
        h, plan.handle = plan.handle, None
        _check(L, L.kc_batch_plan_destroy(h))


def kc_sync(stream=None) -> int:
    """Wait for `stream` and return (and clear) its device status."""
    L = load()
    h = None
    if stream is not None:
        h = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    else:
        try:
            torch = _torch()
            if torch.cuda.is_available():
                h = int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
    st = L.kc_sync(h)
    _check(L, st)
    return st


def kc_release() -> None:
    load().kc_release()


def kc_version() -> str:
    return load().kc_version().decode()
