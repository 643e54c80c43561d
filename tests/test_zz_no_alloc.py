"""The allocation-free solve entry point agrees with the regular one.

eik_solve_noalloc exists for callers that cannot allocate device memory while
they solve (memory pools or caching allocators they do not own, stream
capture, fixed device footprints).  It keeps its working memory in a fixed
array inside the library.  This test calls it through the C ABI twice in a row
(the second call reuses the array the first one left behind) and compares each
result with eik_create / eik_solve / eik_result on the same input, within the
FP32 tolerance of the parity tests (1e-5 * max psi).  It also checks that a
grid above the array's limit is refused with EIK_EINVAL.  The file is named so
that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00009_gb300 import build
    build.build()
    import paper_1811_00009_gb300 as E
    L = E.lib()
    L.eik_solve_noalloc.restype = C.c_int32
    L.eik_solve_noalloc.argtypes = [C.POINTER(C.c_int32), C.c_double, C.c_void_p, C.c_int32,
                                    C.POINTER(C.c_double), C.POINTER(E.eik_params), C.c_void_p,
                                    C.POINTER(E.eik_stats), C.c_void_p]
    L.eik_noalloc_last_error.restype = C.c_char_p
    return E


def regular(eik, w, Fd, stride):
    import torch
    ctx = eik.eik_create(w.dims, w.h, Fd, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        eik.eik_solve(ctx, stride)
        out = torch.empty_like(Fd)
        eik.eik_result(ctx, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        eik.eik_destroy(ctx)


def noalloc(eik, w, Fd, stride):
    import torch
    L = eik.lib()
    out = torch.full_like(Fd, -1.0)
    d = (C.c_int32 * 3)(*w.dims)
    src = np.ascontiguousarray(np.asarray(w.sources, dtype=np.float64).reshape(-1, 3))
    p = eik.eik_params_default()
    p.stride = stride
    st = eik.eik_stats()
    rc = L.eik_solve_noalloc(d, w.h, C.c_void_p(Fd.data_ptr()), len(src),
                             src.ctypes.data_as(C.POINTER(C.c_double)), C.byref(p), C.c_void_p(out.data_ptr()),
                             C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == eik.EIK_OK, L.eik_noalloc_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy(), st


def close(a, b):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return float(np.max(np.abs(a[fin] - b[fin]))) <= 1e-5 * float(b[fin].max())


def test_noalloc_matches_regular_solve_twice(eik):
    import torch
    cases = [synth.workload("C4", 72), synth.workload("C2", 61)]
    for w in cases:
        Fd = torch.from_numpy(w.speed().astype(np.float32)).cuda()
        ref = regular(eik, w, Fd, 2 * w.h)
        for _ in range(2):                      # the second call starts from the first call's leftovers
            got, st = noalloc(eik, w, Fd, 2 * w.h)
            assert st.status == 0 and st.restarts > 0
            assert close(got, ref)


def test_noalloc_rejects_grids_above_its_limit(eik):
    import torch
    L = eik.lib()
    dims = (256, 256, 128)                      # 32*32*16 = 16384 bricks > 8192
    F = torch.ones((1,), dtype=torch.float32, device="cuda")
    d = (C.c_int32 * 3)(*dims)
    src = np.zeros(3)
    p = eik.eik_params_default()
    p.stride = 0.01
    rc = L.eik_solve_noalloc(d, 0.004, C.c_void_p(F.data_ptr()), 1, src.ctypes.data_as(C.POINTER(C.c_double)),
                             C.byref(p), C.c_void_p(F.data_ptr()), None, None)
    assert rc == eik.EIK_EINVAL
    assert b"bricks" in L.eik_noalloc_last_error()
