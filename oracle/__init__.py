"""Oracle for the block-based restarted narrow-band fast marching method.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py use it; the product path (paper_1811_00009_gb300) never does.
It shares no code with the CUDA library.

The arithmetic lives in oracle.c (plain FP64 C, compiled with -ffp-contract=off
so that x86 and aarch64 hosts give identical bits).  This module compiles it on
first use and marshals numpy arrays through ctypes.  Arrays are (nz, ny, nx),
x fastest; sources are physical (x, y, z) with the origin at node 0.

Functions and the passages they follow:
  fmm          Sec. 2.1-2.2, Algs. 1-4 (single heap, infinite bound)
  block_fmm    Sec. 2.3-2.6, Alg. 6 with Algs. 1-5
  solve_quadratic  Alg. 3
  jacobi       brute-force fixed point of the same local solve (a pin, not the paper's method)
  residual     Eq. (2.1)-(2.2) evaluated directly
  fix_nodes    Alg. 1, points on or adjacent to Gamma
  mlp_*        (oracle.mlp) FP64 reference of the schedule network
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = float("inf")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, no FP contraction)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            i64p = C.POINTER(C.c_int64)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.orc_fix_nodes.restype = C.c_int64
            L.orc_fix_nodes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int, dp, i64p, dp, C.c_int64]
            L.orc_solve_quadratic.restype = C.c_double
            L.orc_solve_quadratic.argtypes = [C.c_double, dp, ip, C.c_double]
            L.orc_fmm.restype = C.c_int
            L.orc_fmm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int, dp, dp, i64p, dp, C.c_int64, i64p]
            L.orc_jacobi.restype = C.c_int
            L.orc_jacobi.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int, dp, dp, C.c_int64, i64p]
            L.orc_residual.restype = C.c_double
            L.orc_residual.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, dp, i64p, C.c_int64, i64p]
            L.orc_residual_stencils.restype = None
            L.orc_residual_stencils.argtypes = [C.c_int64, dp, dp, C.c_double, dp]
            L.orc_block_fmm.restype = C.c_int
            L.orc_block_fmm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int, dp, C.c_int,
                                        C.c_double, C.c_double, C.c_int, C.c_int64, dp, C.c_void_p]
            _lib = L
    return _lib


class _BlockStats(C.Structure):
    _fields_ = [("nr", C.c_int64), ("marches", C.c_int64), ("exchanges", C.c_int64),
                ("pops", C.c_int64), ("updates", C.c_int64), ("ghost_updates", C.c_int64)]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i64p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _prep(F: np.ndarray, sources) -> Tuple[np.ndarray, np.ndarray, int, int, int]:
    F = np.ascontiguousarray(F, dtype=np.float64)
    if F.ndim != 3:
        raise ValueError("F must be (nz, ny, nx)")
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, 3))
    nz, ny, nx = F.shape
    return F, src, nx, ny, nz


def _check(rc: int, what: str):
    if rc == -1:
        raise ValueError(f"{what}: invalid argument")
    if rc == -2:
        raise MemoryError(what)
    if rc == -3:
        raise RuntimeError(f"{what}: cap reached")
    if rc != 0:
        raise RuntimeError(f"{what}: status {rc}")


def fix_nodes(F: np.ndarray, h: float, sources) -> Tuple[np.ndarray, np.ndarray]:
    """Linear indices and psi0 of the fixed nodes of point sources (Alg. 1)."""
    F, src, nx, ny, nz = _prep(F, sources)
    cap = 8 * max(1, len(src))
    idx = np.zeros(cap, np.int64)
    val = np.zeros(cap)
    n = lib().orc_fix_nodes(nx, ny, nz, h, _dp(F), len(src), _dp(src), _i64p(idx), _dp(val), cap)
    if n < 0:
        _check(int(n), "fix_nodes")
    return idx[:n].copy(), val[:n].copy()


def solve_quadratic(psi_c: float, nbv, nbk, r2: float) -> float:
    """Alg. 3 for one point (neighbour order x-, x+, y-, y+, z-, z+)."""
    v = np.ascontiguousarray(np.asarray(nbv, dtype=np.float64))
    k = (C.c_int * 6)(*[int(bool(b)) for b in nbk])
    return float(lib().orc_solve_quadratic(float(psi_c), _dp(v), k, float(r2)))


def fmm(F: np.ndarray, h: float, sources, log: bool = False):
    """Single-heap fast marching (Algs. 1-4).  Returns psi, or (psi, log_idx, log_val) with log=True."""
    F, src, nx, ny, nz = _prep(F, sources)
    psi = np.empty_like(F)
    npop = np.zeros(1, np.int64)
    if log:
        cap = F.size
        li = np.empty(cap, np.int64)
        lv = np.empty(cap)
        rc = lib().orc_fmm(nx, ny, nz, h, _dp(F), len(src), _dp(src), _dp(psi), _i64p(li), _dp(lv), cap, _i64p(npop))
        _check(rc, "fmm")
        n = int(npop[0])
        return psi, li[:n].copy(), lv[:n].copy()
    rc = lib().orc_fmm(nx, ny, nz, h, _dp(F), len(src), _dp(src), _dp(psi), None, None, 0, _i64p(npop))
    _check(rc, "fmm")
    return psi


def jacobi(F: np.ndarray, h: float, sources, max_sweeps: int = 100000) -> Tuple[np.ndarray, int]:
    """Brute-force Jacobi fixed point of the local solve; returns (psi, sweeps)."""
    F, src, nx, ny, nz = _prep(F, sources)
    psi = np.empty_like(F)
    sw = np.zeros(1, np.int64)
    rc = lib().orc_jacobi(nx, ny, nz, h, _dp(F), len(src), _dp(src), _dp(psi), int(max_sweeps), _i64p(sw))
    _check(rc, "jacobi")
    return psi, int(sw[0])


def residual(F: np.ndarray, h: float, psi: np.ndarray, sources) -> Tuple[float, int]:
    """Max |F^2 * sum max(D^-psi, -D^+psi, 0)^2 - 1| over non-fixed nodes with F > 0, finite psi."""
    F, src, nx, ny, nz = _prep(F, sources)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    idx, _ = fix_nodes(F, h, src)
    idx = np.ascontiguousarray(idx)
    cnt = np.zeros(1, np.int64)
    r = lib().orc_residual(nx, ny, nz, h, _dp(F), _dp(psi), _i64p(idx), len(idx), _i64p(cnt))
    return float(r), int(cnt[0])


def residual_stencils(stencil: np.ndarray, F: np.ndarray, h: float) -> np.ndarray:
    """Residual of Eq. (2.1) at sampled nodes from caller-built 7-point stencils (n, 7)."""
    st = np.ascontiguousarray(stencil, dtype=np.float64).reshape(-1, 7)
    f = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    out = np.empty(len(f))
    lib().orc_residual_stencils(len(f), _dp(st), _dp(f), float(h), _dp(out))
    return out


def block_fmm(F: np.ndarray, h: float, sources, dim_block: int, stride: float,
              width: float = INF, nthreads: int = 0, max_restarts: int = 1 << 40) -> Tuple[np.ndarray, Dict[str, int]]:
    """The paper's block-based restarted narrow-band method (Alg. 6); returns (psi, stats)."""
    F, src, nx, ny, nz = _prep(F, sources)
    psi = np.empty_like(F)
    st = _BlockStats()
    rc = lib().orc_block_fmm(nx, ny, nz, h, _dp(F), len(src), _dp(src), int(dim_block), float(stride),
                             float(width), int(nthreads), int(max_restarts), _dp(psi), C.byref(st))
    _check(rc, "block_fmm")
    return psi, {k: int(getattr(st, k)) for k, _ in _BlockStats._fields_}
