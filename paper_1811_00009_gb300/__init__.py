"""Python binding of libeik, the GB300 block-based restarted narrow-band fast marching solver.

Argument marshalling only: every step of the solve runs in the CUDA kernels
behind the C ABI of include/eik.h.  Device buffers are torch CUDA tensors
(passed by data_ptr, on torch's current stream); host buffers are numpy arrays.
There is no CPU fallback: if libeik.so is missing or cannot be loaded, every
call raises.

    ctx = eik_create((nx, ny, nz), h, F, precision="fp32")
    eik_add_sources(ctx, [[x, y, z], ...])
    stats = eik_solve(ctx, stride=2 * h)
    psi = eik_result(ctx, out)          # out: torch CUDA tensor or numpy array, shape (nz, ny, nx)
    eik_destroy(ctx)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from typing import Any, Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeik.so")

EIK_OK, EIK_EINVAL, EIK_ENOMEM, EIK_ECUDA, EIK_ETIMEOUT, EIK_ESTATE, EIK_ENOTSUP = range(7)
EIK_FP32, EIK_FP64 = 0, 1
EIK_SCHED_FIXED, EIK_SCHED_LEARNED, EIK_SCHED_RANDOM = 0, 1, 2
SCHED_INPUTS, SCHED_HIDDEN, SCHED_ACTIONS = 10, 32, 12
SCHED_PARAMS = SCHED_HIDDEN * SCHED_INPUTS + SCHED_HIDDEN + SCHED_HIDDEN * SCHED_HIDDEN + SCHED_HIDDEN + \
    SCHED_ACTIONS * SCHED_HIDDEN + SCHED_ACTIONS
STATUS_NAMES = {0: "EIK_OK", 1: "EIK_EINVAL", 2: "EIK_ENOMEM", 3: "EIK_ECUDA", 4: "EIK_ETIMEOUT",
                5: "EIK_ESTATE", 6: "EIK_ENOTSUP"}


class EikError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class eik_params(C.Structure):
    _fields_ = [("stride", C.c_double), ("block_dim", C.c_int32), ("schedule", C.c_int32),
                ("window", C.c_double), ("fallback_tau", C.c_double), ("max_restarts", C.c_int64),
                ("log_restarts", C.c_int32), ("seed", C.c_int32), ("loop_events", C.c_void_p * 2),
                ("switch_margin", C.c_double), ("width", C.c_double), ("wait_polls", C.c_int64)]


class eik_stats(C.Structure):
    _fields_ = [("restarts", C.c_int64), ("marches", C.c_int64), ("accepted", C.c_int64),
                ("solves", C.c_int64), ("updates", C.c_int64), ("fallbacks", C.c_int64),
                ("rounds", C.c_int64), ("device_ms", C.c_double), ("final_bound", C.c_double),
                ("status", C.c_int32), ("block_dim", C.c_int32)]


class eik_restart_rec(C.Structure):
    _fields_ = [("k", C.c_int32), ("active", C.c_int32), ("band", C.c_int64), ("accepted", C.c_int64),
                ("solves", C.c_int64), ("bound", C.c_double), ("stride", C.c_double), ("rmin", C.c_double),
                ("rmax", C.c_double), ("ms", C.c_double), ("block_dim", C.c_int32), ("next_action", C.c_int32),
                ("features", C.c_float * SCHED_INPUTS)]


class eik_batch_item(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("h", C.c_double), ("F", C.c_void_p), ("F_on_device", C.c_int32),
                ("nsrc", C.c_int32), ("xyz", C.POINTER(C.c_double))]


class eik_batch_tile(C.Structure):
    _fields_ = [("block_dim", C.c_int32), ("stride", C.c_double)]


class eik_batch_params(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("window", C.c_double), ("fallback_tau", C.c_double),
                ("max_restarts", C.c_int64), ("loop_events", C.c_void_p * 2)]


class eik_batch_stats(C.Structure):
    _fields_ = [("restarts", C.c_int64), ("marches", C.c_int64), ("accepted", C.c_int64), ("solves", C.c_int64),
                ("updates", C.c_int64), ("fallbacks", C.c_int64), ("rounds", C.c_int64),
                ("device_ms", C.c_double), ("status", C.c_int32), ("ctas", C.c_int32)]


class eik_batch_solve_info(C.Structure):
    _fields_ = [("restarts", C.c_int32), ("block_dim", C.c_int32), ("stride", C.c_double),
                ("done_ms", C.c_double), ("rmin", C.c_double), ("nbricks", C.c_int64)]


_lock = threading.Lock()
_L = None


def lib():
    """Load libeik.so (built by build.py / __graft_entry__.build()).  Raises if absent."""
    global _L
    with _lock:
        if _L is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libeik.so not found at {LIB_PATH}: build it with "
                                  "python -c 'import __graft_entry__ as g; g.build()'")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            L.eik_create.restype = i32
            L.eik_create.argtypes = [C.POINTER(vp), C.POINTER(i32), dbl, vp, C.c_int, C.c_int, vp]
            L.eik_set_speed.restype = i32
            L.eik_set_speed.argtypes = [vp, vp, C.c_int]
            L.eik_source_nodes.restype = i32
            L.eik_source_nodes.argtypes = [C.POINTER(i32), dbl, vp, C.c_int, i32, C.POINTER(C.c_double),
                                           C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int64,
                                           C.POINTER(C.c_int64)]
            L.eik_set_speed_async.restype = i32
            L.eik_set_speed_async.argtypes = [vp, vp, C.c_int]
            L.eik_result_async.restype = i32
            L.eik_result_async.argtypes = [vp, vp, C.c_int]
            L.eik_sync.restype = i32
            L.eik_sync.argtypes = [vp]
            L.eik_add_sources.restype = i32
            L.eik_add_sources.argtypes = [vp, i32, C.POINTER(dbl)]
            L.eik_clear_sources.restype = i32
            L.eik_clear_sources.argtypes = [vp]
            L.eik_params_default.restype = None
            L.eik_params_default.argtypes = [C.POINTER(eik_params)]
            L.eik_solve.restype = i32
            L.eik_solve.argtypes = [vp, dbl, i32, C.POINTER(eik_stats)]
            L.eik_solve_ex.restype = i32
            L.eik_solve_ex.argtypes = [vp, C.POINTER(eik_params), C.POINTER(eik_stats)]
            L.eik_solve_async.restype = i32
            L.eik_solve_async.argtypes = [vp, C.POINTER(eik_params)]
            L.eik_wait.restype = i32
            L.eik_wait.argtypes = [vp, C.POINTER(eik_stats)]
            L.eik_slab_face_bytes.restype = i64
            L.eik_slab_face_bytes.argtypes = [vp]
            L.eik_slab_set.restype = i32
            L.eik_slab_set.argtypes = [vp, i32, i32, i32, i32]
            L.eik_slab_begin.restype = i32
            L.eik_slab_begin.argtypes = [vp, dbl]
            L.eik_slab_restart.restype = i32
            L.eik_slab_restart.argtypes = [vp, C.POINTER(i64)]
            L.eik_slab_export.restype = i32
            L.eik_slab_export.argtypes = [vp, i32, vp]
            L.eik_slab_import.restype = i32
            L.eik_slab_import.argtypes = [vp, i32, vp, C.POINTER(i64)]
            L.eik_slab_end.restype = i32
            L.eik_slab_end.argtypes = [vp, C.POINTER(eik_stats)]
            L.eik_autotune.restype = i32
            L.eik_autotune.argtypes = [vp, i32, C.POINTER(dbl), C.POINTER(i32), C.POINTER(dbl)]
            L.eik_restart_log.restype = i32
            L.eik_restart_log.argtypes = [vp, C.POINTER(eik_restart_rec), i64, C.POINTER(i64)]
            L.eik_result.restype = i32
            L.eik_result.argtypes = [vp, vp, C.c_int]
            L.eik_destroy.restype = None
            L.eik_destroy.argtypes = [vp]
            L.eik_last_error.restype = C.c_char_p
            L.eik_last_error.argtypes = [vp]
            L.eik_version.restype = C.c_char_p
            L.eik_version.argtypes = []
            fp = C.c_void_p
            L.eik_set_schedule.restype = i32
            L.eik_set_schedule.argtypes = [vp, C.POINTER(C.c_float), i32]
            L.eik_sched_actions.restype = i32
            L.eik_sched_actions.argtypes = [C.POINTER(dbl), C.POINTER(i32), i32, C.POINTER(i32)]
            L.eik_mlp_forward.restype = i32
            L.eik_mlp_forward.argtypes = [fp, fp, i32, fp, vp]
            L.eik_mlp_grad.restype = i32
            L.eik_mlp_grad.argtypes = [fp, fp, fp, fp, i32, fp, fp, fp, vp]
            L.eik_mlp_work_floats.restype = i32
            L.eik_mlp_work_floats.argtypes = [i32]
            L.eik_mlp_adam.restype = i32
            L.eik_mlp_adam.argtypes = [fp, fp, fp, fp, i32, C.c_float, C.c_float, C.c_float, C.c_float, i32, vp]
            L.eik_mlp_last_error.restype = C.c_char_p
            L.eik_mlp_last_error.argtypes = []
            L.eik_batch_create.restype = i32
            L.eik_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(eik_batch_item), C.c_int, vp]
            L.eik_batch_params_default.restype = None
            L.eik_batch_params_default.argtypes = [C.POINTER(eik_batch_params)]
            L.eik_batch_solve.restype = i32
            L.eik_batch_solve.argtypes = [vp, C.POINTER(eik_batch_tile), C.POINTER(eik_batch_params),
                                          C.POINTER(eik_batch_stats)]
            L.eik_batch_solve_async.restype = i32
            L.eik_batch_solve_async.argtypes = [vp, C.POINTER(eik_batch_tile), C.POINTER(eik_batch_params)]
            L.eik_batch_wait.restype = i32
            L.eik_batch_wait.argtypes = [vp, C.POINTER(eik_batch_stats)]
            L.eik_batch_info.restype = i32
            L.eik_batch_info.argtypes = [vp, C.POINTER(eik_batch_solve_info), i32]
            L.eik_batch_result.restype = i32
            L.eik_batch_result.argtypes = [vp, i32, vp, C.c_int]
            L.eik_batch_autotune.restype = i32
            L.eik_batch_autotune.argtypes = [vp, i32, C.POINTER(eik_batch_tile), C.POINTER(i32), C.POINTER(dbl)]
            L.eik_batch_size.restype = i32
            L.eik_batch_size.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
            L.eik_batch_destroy.restype = None
            L.eik_batch_destroy.argtypes = [vp]
            L.eik_batch_last_error.restype = C.c_char_p
            L.eik_batch_last_error.argtypes = [vp]
            _L = L
    return _L


def eik_last_error(ctx=None) -> str:
    m = lib().eik_last_error(ctx)
    return m.decode() if m else ""


def _check(status: int, ctx=None):
    if status != EIK_OK:
        raise EikError(status, eik_last_error(ctx))


def _precision(p) -> int:
    if p in ("fp32", EIK_FP32, "float32"):
        return EIK_FP32
    if p in ("fp64", EIK_FP64, "float64"):
        return EIK_FP64
    raise ValueError(f"precision {p!r}")


def _buffer(a, want_dtype):
    """(pointer, on_device, keepalive) for a torch tensor or numpy array of the given element type."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = torch.float32 if want_dtype == np.float32 else torch.float64
            if a.dtype != tdt or not a.is_contiguous():
                raise ValueError(f"tensor must be contiguous {tdt}")
            return C.c_void_p(a.data_ptr()), int(a.is_cuda), a
    except ImportError:
        pass
    arr = np.asarray(a)
    if arr.dtype != want_dtype or not arr.flags.c_contiguous:
        raise ValueError(f"array must be C-contiguous {np.dtype(want_dtype).name}")
    return C.c_void_p(arr.ctypes.data), 0, arr


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def eik_create(dims: Sequence[int], h: float, F, precision="fp32", stream=None):
    """Context for grid dims=(nx, ny, nz), spacing h, speeds F (shape (nz, ny, nx), x fastest)."""
    prec = _precision(precision)
    ptr, on_dev, keep = _buffer(F, np.float32 if prec == EIK_FP32 else np.float64)
    n = int(dims[0]) * int(dims[1]) * int(dims[2])
    if int(np.prod(getattr(keep, "shape", (0,)))) != n:
        raise ValueError("F must hold nx*ny*nz values")
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    out = C.c_void_p()
    _check(lib().eik_create(C.byref(out), d, float(h), ptr, on_dev, prec, _stream_handle(stream)), None)
    return out


def eik_set_speed(ctx, F, precision="fp32") -> None:
    """Replace the context's speed function (same grid and precision)."""
    ptr, on_dev, keep = _buffer(F, np.float32 if _precision(precision) == EIK_FP32 else np.float64)
    _check(lib().eik_set_speed(ctx, ptr, on_dev), ctx)


def eik_set_speed_async(ctx, F, precision="fp32"):
    """Queue the upload of a new speed function; returns F, which must stay alive and unchanged until
    eik_sync(ctx) or the next solve on ctx (host F should be pinned)."""
    ptr, on_dev, keep = _buffer(F, np.float32 if _precision(precision) == EIK_FP32 else np.float64)
    _check(lib().eik_set_speed_async(ctx, ptr, on_dev), ctx)
    return keep


def eik_source_nodes(dims, h, F, sources, precision="fp32"):
    """(linear indices, psi0) of the fixed nodes a solve would start from (host computation, Alg. 1)."""
    prec = _precision(precision)
    arr = np.ascontiguousarray(np.asarray(F, dtype=np.float32 if prec == EIK_FP32 else np.float64))
    xyz = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, 3))
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    n = C.c_int64()
    cap = 8 * max(1, len(xyz))
    idx = np.zeros(cap, np.int64)
    val = np.zeros(cap, np.float64)
    st = lib().eik_source_nodes(d, float(h), C.c_void_p(arr.ctypes.data), prec, len(xyz),
                                xyz.ctypes.data_as(C.POINTER(C.c_double)), idx.ctypes.data_as(C.POINTER(C.c_int64)),
                                val.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(n))
    _check(st, None)
    return idx[:n.value].copy(), val[:n.value].copy()


def eik_add_sources(ctx, xyz) -> None:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    _check(lib().eik_add_sources(ctx, len(a), a.ctypes.data_as(C.POINTER(C.c_double))), ctx)


def eik_clear_sources(ctx) -> None:
    _check(lib().eik_clear_sources(ctx), ctx)


def eik_params_default() -> eik_params:
    p = eik_params()
    lib().eik_params_default(C.byref(p))
    return p


def _stats_dict(s: eik_stats) -> Dict[str, Any]:
    return {k: getattr(s, k) for k, _ in eik_stats._fields_}


def _params(stride: float, **kw) -> eik_params:
    p = eik_params_default()
    p.stride = float(stride)
    for k, v in kw.items():
        if k == "loop_events":
            p.loop_events[0] = C.c_void_p(v[0].cuda_event if hasattr(v[0], "cuda_event") else int(v[0]))
            p.loop_events[1] = C.c_void_p(v[1].cuda_event if hasattr(v[1], "cuda_event") else int(v[1]))
            continue
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def eik_solve(ctx, stride: float, block_dim: int = 8) -> Dict[str, Any]:
    """Solve (Alg. 6) and wait.  stride 0 selects the learned schedule; block_dim 0 lets the schedule or
    eik_autotune pick the block edge."""
    s = eik_stats()
    _check(lib().eik_solve(ctx, float(stride), int(block_dim), C.byref(s)), ctx)
    return _stats_dict(s)


def eik_solve_ex(ctx, stride: float, **kw) -> Dict[str, Any]:
    p = _params(stride, **kw)
    s = eik_stats()
    _check(lib().eik_solve_ex(ctx, C.byref(p), C.byref(s)), ctx)
    return _stats_dict(s)


def eik_solve_async(ctx, stride: float, **kw) -> None:
    p = _params(stride, **kw)
    _check(lib().eik_solve_async(ctx, C.byref(p)), ctx)


def eik_wait(ctx) -> Dict[str, Any]:
    s = eik_stats()
    _check(lib().eik_wait(ctx, C.byref(s)), ctx)
    return _stats_dict(s)


def eik_autotune(ctx, rounds: int = 0) -> Dict[str, Any]:
    """Time the candidate fixed strides and block edges on this context; returns the winner."""
    stride, block, ms = C.c_double(), C.c_int32(), C.c_double()
    _check(lib().eik_autotune(ctx, int(rounds), C.byref(stride), C.byref(block), C.byref(ms)), ctx)
    return {"stride": stride.value, "block_dim": block.value, "ms": ms.value}


def eik_slab_face_bytes(ctx) -> int:
    return int(lib().eik_slab_face_bytes(ctx))


def eik_slab_set(ctx, own_bz0: int, own_bz1: int, zoff: int, nz_all: int) -> None:
    _check(lib().eik_slab_set(ctx, int(own_bz0), int(own_bz1), int(zoff), int(nz_all)), ctx)


def eik_slab_begin(ctx, stride: float) -> None:
    _check(lib().eik_slab_begin(ctx, float(stride)), ctx)


def eik_slab_restart(ctx) -> int:
    n = C.c_int64()
    _check(lib().eik_slab_restart(ctx, C.byref(n)), ctx)
    return n.value


def eik_slab_export(ctx, side: int, buf) -> None:
    """buf: a torch CUDA tensor of eik_slab_face_bytes(ctx) bytes."""
    _check(lib().eik_slab_export(ctx, int(side), _dptr(buf)), ctx)


def eik_slab_import(ctx, side: int, buf) -> int:
    n = C.c_int64()
    _check(lib().eik_slab_import(ctx, int(side), _dptr(buf), C.byref(n)), ctx)
    return n.value


def eik_slab_end(ctx) -> Dict[str, Any]:
    s = eik_stats()
    _check(lib().eik_slab_end(ctx, C.byref(s)), ctx)
    return _stats_dict(s)


def eik_restart_log(ctx, cap: int = 1 << 16) -> List[Dict[str, Any]]:
    recs = (eik_restart_rec * cap)()
    n = C.c_int64()
    _check(lib().eik_restart_log(ctx, recs, cap, C.byref(n)), ctx)
    out = []
    for i in range(n.value):
        d = {k: getattr(recs[i], k) for k, _ in eik_restart_rec._fields_ if k != "features"}
        d["features"] = list(recs[i].features)
        out.append(d)
    return out


# ---- restart-schedule network (no counterpart in the paper) ----

def eik_sched_actions():
    """[(stride in units of h, block edge)] of every action."""
    sh = (C.c_double * SCHED_ACTIONS)()
    bd = (C.c_int32 * SCHED_ACTIONS)()
    n = C.c_int32()
    _check(lib().eik_sched_actions(sh, bd, SCHED_ACTIONS, C.byref(n)))
    return [(sh[i], bd[i]) for i in range(n.value)]


def eik_set_schedule(ctx, weights) -> None:
    """Load the schedule network's weights (host array of SCHED_PARAMS floats) into ctx; None unloads."""
    if weights is None:
        _check(lib().eik_set_schedule(ctx, None, 0), ctx)
        return
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
    _check(lib().eik_set_schedule(ctx, w.ctypes.data_as(C.POINTER(C.c_float)), len(w)), ctx)


def _mlp_check(st):
    if st != EIK_OK:
        raise EikError(st, lib().eik_mlp_last_error().decode())


def _dptr(t):
    return C.c_void_p(t.data_ptr())


def eik_mlp_forward(w, X, Y, stream=None):
    """Y[B, ACTIONS] <- network(X[B, INPUTS]); torch CUDA float32 tensors."""
    _mlp_check(lib().eik_mlp_forward(_dptr(w), _dptr(X), X.shape[0], _dptr(Y), _stream_handle(stream)))


def eik_mlp_grad(w, X, act, tgt, grad, loss, work, stream=None):
    """grad <- d/dw mean (Y[s, act[s]] - tgt[s])^2, loss[0] <- the loss; torch CUDA tensors."""
    _mlp_check(lib().eik_mlp_grad(_dptr(w), _dptr(X), _dptr(act), _dptr(tgt), X.shape[0], _dptr(grad), _dptr(loss),
                                  _dptr(work), _stream_handle(stream)))


def eik_mlp_work_floats(B: int) -> int:
    return int(lib().eik_mlp_work_floats(int(B)))


def eik_mlp_adam(w, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _mlp_check(lib().eik_mlp_adam(_dptr(w), _dptr(grad), _dptr(m), _dptr(v), w.numel(), lr, b1, b2, eps, int(t),
                                  _stream_handle(stream)))


def eik_result(ctx, out):
    """Write psi into `out` (torch CUDA tensor or numpy array, context precision) and return it."""
    for dt in (np.float32, np.float64):
        try:
            ptr, on_dev, keep = _buffer(out, dt)
            break
        except ValueError:
            continue
    else:
        raise ValueError("out must be a contiguous float32/float64 tensor or array")
    _check(lib().eik_result(ctx, ptr, on_dev), ctx)
    return out


def eik_result_async(ctx, out):
    """Queue psi into `out` (as eik_result); complete after eik_sync(ctx).  Host `out` should be pinned."""
    for dt in (np.float32, np.float64):
        try:
            ptr, on_dev, keep = _buffer(out, dt)
            break
        except ValueError:
            continue
    else:
        raise ValueError("out must be a contiguous float32/float64 tensor or array")
    _check(lib().eik_result_async(ctx, ptr, on_dev), ctx)
    return out


def eik_sync(ctx) -> None:
    _check(lib().eik_sync(ctx), ctx)


def eik_destroy(ctx) -> None:
    if ctx:
        lib().eik_destroy(ctx)


def eik_version() -> str:
    return lib().eik_version().decode()


class Solver:
    """Owns one context; convenience wrapper over the functions above."""

    def __init__(self, dims, h, F, precision="fp32", stream=None):
        self.dims = tuple(int(x) for x in dims)
        self.h = float(h)
        self.precision = precision
        self.ctx = eik_create(self.dims, h, F, precision, stream)

    def add_sources(self, xyz):
        eik_add_sources(self.ctx, xyz)

    def clear_sources(self):
        eik_clear_sources(self.ctx)

    def solve(self, stride: float, **kw):
        return eik_solve_ex(self.ctx, stride, **kw)

    def result(self, out=None):
        if out is None:
            dt = np.float32 if _precision(self.precision) == EIK_FP32 else np.float64
            out = np.empty(self.dims[::-1], dtype=dt)
        return eik_result(self.ctx, out)

    def restart_log(self):
        return eik_restart_log(self.ctx)

    def close(self):
        if self.ctx:
            eik_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched solves (many grids, one persistent launch) ----

def _batch_check(status: int, b=None):
    if status != EIK_OK:
        m = lib().eik_batch_last_error(b)
        raise EikError(status, m.decode() if m else "")


def _event_ptr(e):
    return C.c_void_p(e.cuda_event if hasattr(e, "cuda_event") else int(e))


class Batch:
    """Many independent grids solved by one cooperative launch (eik_batch_* of the C ABI).

    grids: sequence of (dims, h, F, sources): dims = (nx, ny, nz), F a numpy
    array or torch CUDA tensor of shape (nz, ny, nx) in the batch precision,
    sources an (n, 3) array of physical coordinates.
    """

    def __init__(self, grids, precision="fp32", stream=None):
        prec = _precision(precision)
        dt = np.float32 if prec == EIK_FP32 else np.float64
        self.precision = precision
        self.dims = []
        items = (eik_batch_item * len(grids))()
        keep = []
        for i, (dims, h, F, src) in enumerate(grids):
            ptr, on_dev, k = _buffer(F, dt)
            n = int(dims[0]) * int(dims[1]) * int(dims[2])
            if int(np.prod(getattr(k, "shape", (0,)))) != n:
                raise ValueError(f"grid {i}: F must hold nx*ny*nz values")
            xyz = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 3))
            keep += [k, xyz]
            items[i].dims[:] = [int(x) for x in dims]
            items[i].h = float(h)
            items[i].F = ptr
            items[i].F_on_device = on_dev
            items[i].nsrc = len(xyz)
            items[i].xyz = xyz.ctypes.data_as(C.POINTER(C.c_double))
            self.dims.append(tuple(int(x) for x in dims))
        self.b = C.c_void_p()
        _batch_check(lib().eik_batch_create(C.byref(self.b), len(grids), items, prec, _stream_handle(stream)))
        self.n = len(grids)

    @staticmethod
    def _tiles(tiles):
        if tiles is None:
            return None
        arr = (eik_batch_tile * len(tiles))()
        for i, (bd, stride) in enumerate(tiles):
            arr[i].block_dim = int(bd)
            arr[i].stride = float(stride)
        return arr

    def _params(self, ctas_per_sm=0, window=0.0, fallback_tau=0.0, max_restarts=0, loop_events=None):
        p = eik_batch_params()
        lib().eik_batch_params_default(C.byref(p))
        p.ctas_per_sm = int(ctas_per_sm)
        if window:
            p.window = float(window)
        if fallback_tau:
            p.fallback_tau = float(fallback_tau)
        if max_restarts:
            p.max_restarts = int(max_restarts)
        if loop_events is not None:
            p.loop_events[0] = _event_ptr(loop_events[0])
            p.loop_events[1] = _event_ptr(loop_events[1])
        return p

    def solve(self, tiles=None, **kw) -> Dict[str, Any]:
        """Solve every grid; tiles = [(block_dim, stride)] per grid or None (tuned, else 8 and 2h)."""
        t = self._tiles(tiles)
        p = self._params(**kw)
        s = eik_batch_stats()
        _batch_check(lib().eik_batch_solve(self.b, t, C.byref(p), C.byref(s)), self.b)
        return {k: getattr(s, k) for k, _ in eik_batch_stats._fields_}

    def solve_async(self, tiles=None, **kw) -> None:
        t = self._tiles(tiles)
        p = self._params(**kw)
        _batch_check(lib().eik_batch_solve_async(self.b, t, C.byref(p)), self.b)

    def wait(self) -> Dict[str, Any]:
        s = eik_batch_stats()
        _batch_check(lib().eik_batch_wait(self.b, C.byref(s)), self.b)
        return {k: getattr(s, k) for k, _ in eik_batch_stats._fields_}

    def info(self) -> List[Dict[str, Any]]:
        recs = (eik_batch_solve_info * self.n)()
        _batch_check(lib().eik_batch_info(self.b, recs, self.n), self.b)
        return [{k: getattr(r, k) for k, _ in eik_batch_solve_info._fields_} for r in recs]

    def result(self, i: int, out=None):
        if out is None:
            dt = np.float32 if _precision(self.precision) == EIK_FP32 else np.float64
            # an index out of range is left to the library to reject
            out = np.empty(self.dims[i][::-1] if 0 <= i < self.n else (1,), dtype=dt)
        for dt in (np.float32, np.float64):
            try:
                ptr, on_dev, keep = _buffer(out, dt)
                break
            except ValueError:
                continue
        else:
            raise ValueError("out must be a contiguous float32/float64 tensor or array")
        _batch_check(lib().eik_batch_result(self.b, int(i), ptr, on_dev), self.b)
        return out

    def autotune(self, rounds: int = 0):
        """Tune tiles and CTAs per SM on the device; returns (tiles, ctas_per_sm, best_ms)."""
        t = (eik_batch_tile * self.n)()
        ctas = C.c_int32()
        ms = C.c_double()
        _batch_check(lib().eik_batch_autotune(self.b, int(rounds), t, C.byref(ctas), C.byref(ms)), self.b)
        return [(t[i].block_dim, t[i].stride) for i in range(self.n)], ctas.value, ms.value

    def size(self):
        """(grids, total 8^3 bricks, most CTAs per SM the launch can use)."""
        n, nb, mc = C.c_int32(), C.c_int64(), C.c_int32()
        _batch_check(lib().eik_batch_size(self.b, C.byref(n), C.byref(nb), C.byref(mc)), self.b)
        return n.value, nb.value, mc.value

    def close(self):
        if getattr(self, "b", None):
            lib().eik_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
