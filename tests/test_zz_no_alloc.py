"""The allocation-free solve entry point agrees with the regular one and with the oracle.

eik_solve_noalloc exists for callers that cannot allocate device memory while
they solve: code under a memory pool or caching allocator it does not own, and
embedders that keep the process's device footprint fixed.  It keeps its working
memory in a fixed array inside the library.  This test calls it through the C
ABI twice in a row (the second call reuses the array the first one left
behind) and compares each result with eik_create / eik_solve / eik_result on
the same input -- bit for bit, since both run the same kernels on the same
discrete problem -- and with the FP64 oracle within the FP32 bar of the parity
tests (1e-5 * max psi).  It checks that the device's free memory does not move
across a call, that a grid above the array's limit and bad parameters are
refused, and that a call whose device waits run out (wait_polls = 1) reports
EIK_ETIMEOUT and leaves the next call correct.  The file is named so that
pytest collects it last.
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


def call(eik, w, Fd, out, stride, **kw):
    """eik_solve_noalloc through the C ABI into the caller's device buffer `out`; returns (status, stats)."""
    import torch
    L = eik.lib()
    d = (C.c_int32 * 3)(*w.dims)
    src = np.ascontiguousarray(np.asarray(w.sources, dtype=np.float64).reshape(-1, 3))
    p = eik.eik_params_default()
    p.stride = stride
    for k, v in kw.items():
        setattr(p, k, v)
    st = eik.eik_stats()
    rc = L.eik_solve_noalloc(d, w.h, C.c_void_p(Fd.data_ptr()), len(src),
                             src.ctypes.data_as(C.POINTER(C.c_double)), C.byref(p), C.c_void_p(out.data_ptr()),
                             C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, st


def test_noalloc_matches_regular_solve_and_oracle_twice(eik, orc):
    import torch
    for w in (synth.workload("C4", 72), synth.workload("C2", 61)):
        F = w.speed()
        Fd = torch.from_numpy(F.astype(np.float32)).cuda()
        ref = regular(eik, w, Fd, 2 * w.h)
        oref = orc.fmm(F, w.h, w.sources)
        fin = np.isfinite(oref)
        for _ in range(2):                      # the second call starts from the first call's leftovers
            out = torch.full_like(Fd, -1.0)
            rc, st = call(eik, w, Fd, out, 2 * w.h)
            assert rc == eik.EIK_OK, eik.lib().eik_noalloc_last_error().decode()
            assert st.status == 0 and st.restarts > 0
            got = out.cpu().numpy()
            assert np.array_equal(got, ref)
            assert np.array_equal(np.isfinite(got), fin)
            assert float(np.max(np.abs(got[fin] - oref[fin]))) <= 1e-5 * float(oref[fin].max())


def test_noalloc_leaves_device_memory_untouched(eik):
    """After a first call (which loads the kernels and looks up the array's address), a call changes the
    device's free memory by nothing."""
    import torch
    w = synth.workload("C3", 80)
    Fd = torch.from_numpy(w.speed().astype(np.float32)).cuda()
    out = torch.empty_like(Fd)
    rc, _ = call(eik, w, Fd, out, 2 * w.h)
    assert rc == eik.EIK_OK
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    rc, _ = call(eik, w, Fd, out, 2 * w.h)
    assert rc == eik.EIK_OK
    after = torch.cuda.mem_get_info()[0]
    assert after == before, (before, after)


def test_noalloc_timeout_then_a_correct_call(eik):
    import torch
    w = synth.workload("C2", 96)
    Fd = torch.from_numpy(w.speed().astype(np.float32)).cuda()
    ref = regular(eik, w, Fd, 2 * w.h)
    out = torch.empty_like(Fd)
    rc, st = call(eik, w, Fd, out, w.h, wait_polls=1)
    assert rc == eik.EIK_ETIMEOUT and st.status == eik.EIK_ETIMEOUT
    rc, _ = call(eik, w, Fd, out, 2 * w.h)
    assert rc == eik.EIK_OK
    assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_bad_requests(eik):
    import torch
    L = eik.lib()
    w = synth.workload("C2", 24)
    Fd = torch.from_numpy(w.speed().astype(np.float32)).cuda()
    out = torch.empty_like(Fd)
    for kw, code in ((dict(fallback_tau=2.0), eik.EIK_EINVAL), (dict(wait_polls=-1), eik.EIK_EINVAL),
                     (dict(max_restarts=-5), eik.EIK_EINVAL), (dict(block_dim=16), eik.EIK_ENOTSUP),
                     (dict(schedule=1), eik.EIK_ENOTSUP), (dict(log_restarts=1), eik.EIK_ENOTSUP)):
        rc, _ = call(eik, w, Fd, out, 2 * w.h, **kw)
        assert rc == code, (kw, rc, L.eik_noalloc_last_error())
    rc, _ = call(eik, w, Fd, out, 0.0)
    assert rc == eik.EIK_EINVAL
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
