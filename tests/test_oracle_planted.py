"""Plants plausible mistakes in a copy of the oracle's C source and checks that a pin catches each.

The copy is compiled into a temporary library on the CPU; the real oracle is
untouched.  Pins used: the 50-digit golden solution of Eq. (2.1), the residual
of Eq. (2.1), and the brute-force Jacobi fixed point.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MISTAKES = {
    "dropped_speed_term": ("c -= r2;", "c -= 0.5 * r2;"),
    "wrong_upwind_side": ("if (d == 0 || hi < lo) d = 1;", "if (d == 0 || hi > lo) d = 1;"),
    "inverted_growth_test": ("if (id < nd && t > v[id]) { ++id; continue; }", "if (id < nd && t < v[id]) { ++id; continue; }"),
    "max_heap": ("return kx < ky || (kx == ky && x < y);", "return kx > ky || (kx == ky && x < y);"),
    "transposed_stride": ("int64_t st[3] = {sx, sy, sz};", "int64_t st[3] = {sy, sx, sz};"),
    "sign_of_root": ("double t = v[0] + (b + sqrt(disc)) / a;", "double t = v[0] + (b - sqrt(disc)) / a;"),
}


def _planted_lib(tmp_path, old, new):
    text = open(SRC).read()
    assert text.count(old) >= 1, old
    path = tmp_path / "planted.c"
    path.write_text(text.replace(old, new))
    so = tmp_path / "planted.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-I", os.path.dirname(SRC), "-o", str(so), str(path), "-lm"], check=True)
    L = C.CDLL(str(so))
    dp = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    L.orc_fmm.restype = C.c_int
    L.orc_fmm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int, dp, dp, i64p, dp, C.c_int64, i64p]
    return L


def _fmm(L, F, h, src, log=False):
    F = np.ascontiguousarray(F, dtype=np.float64)
    src = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 3))
    psi = np.empty_like(F)
    nz, ny, nx = F.shape
    n = np.zeros(1, np.int64)
    li = np.zeros(4 * F.size, np.int64)
    lv = np.zeros(4 * F.size)
    rc = L.orc_fmm(nx, ny, nz, h, F.ctypes.data_as(C.POINTER(C.c_double)), len(src),
                   src.ctypes.data_as(C.POINTER(C.c_double)), psi.ctypes.data_as(C.POINTER(C.c_double)),
                   li.ctypes.data_as(C.POINTER(C.c_int64)), lv.ctypes.data_as(C.POINTER(C.c_double)),
                   len(li), n.ctypes.data_as(C.POINTER(C.c_int64)))
    if log:
        return rc, psi, lv[:min(int(n[0]), len(lv))]
    return rc, psi


def _some_pin_fails(L):
    """True if the planted library fails the golden, residual, Jacobi or monotone-acceptance pin."""
    # golden: 50-digit solution, F = 1 + i/10 + j/5 - k/20 on 4x5x6, h = 0.25
    import test_oracle_pins as P
    meta, vals = P._read_golden("eq21_varying_speed_cell_source.txt")
    nx, ny, nz = meta["dims"]
    F = np.empty((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                F[k, j, i] = 1 + i / 10 + j / 5 - k / 20
    rc, psi = _fmm(L, F, meta["h"], meta["sources"])
    if rc != 0:
        return True
    for (i, j, k), v in vals.items():
        if not abs(psi[k, j, i] - v) <= 1e-14 * max(1.0, abs(v)):
            return True
    # residual on a random grid, and equality with the (correct) brute force
    dims = (9, 7, 8)
    h = synth.grid_h(dims)
    F = 0.5 + 1.5 * synth.uniform(3, 1, int(np.prod(dims))).reshape(dims[::-1])
    src = synth.random_sources(3, 2, dims, h, 2)
    rc, psi, lv = _fmm(L, F, h, src, log=True)
    if rc != 0:
        return True
    if not np.all(np.diff(lv) >= 0.0):
        return True
    r, _ = oracle.residual(F, h, psi, src)
    if not r <= 1e-12:
        return True
    j, _ = oracle.jacobi(F, h, src)
    return not np.array_equal(psi, j)


def _child(tmp, old, new, q):
    import pathlib
    q.put(_some_pin_fails(_planted_lib(pathlib.Path(tmp), old, new)))


def _check_in_child(tmp_path, old, new, limit=12.0):
    """Run the pins in a spawned child; a planted library that never finishes counts as caught."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(str(tmp_path), old, new, q))
    p.start()
    p.join(limit)
    if p.is_alive():
        p.kill()
        p.join()
        return True
    return q.get() if not q.empty() else True


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_is_caught(tmp_path, orc, name):
    old, new = MISTAKES[name]
    assert _check_in_child(tmp_path, old, new), name


def test_unplanted_copy_passes(tmp_path, orc):
    assert not _check_in_child(tmp_path, "c -= r2;", "c -= r2;")
