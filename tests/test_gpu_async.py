"""Asynchronous host I/O (eik_set_speed_async / eik_result_async / eik_sync).

Two contexts used in turn overlap one's host copies with the other's solve.
The answers must be the bits the blocking calls give for the same speeds, and
a bad F queued asynchronously must be reported before any solve uses it.
"""
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
    return E


def pinned_like(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float32 if a.dtype == np.float32 else torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t.numpy()


def blocking(eik, w, F, stride):
    ctx = eik.eik_create(w.dims, w.h, F, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        eik.eik_solve_ex(ctx, stride)
        out = np.empty(F.shape, np.float32)
        eik.eik_result(ctx, out)
        return out
    finally:
        eik.eik_destroy(ctx)


def test_two_context_pipeline_gives_the_blocking_bits(eik):
    w = synth.workload("C4", 70)
    Fa = np.ascontiguousarray(w.speed(), dtype=np.float32)
    Fb = np.ascontiguousarray(Fa[::-1, :, ::-1] * np.float32(1.5))      # another speed field, same grid
    stride = 2 * w.h
    want = {"a": blocking(eik, w, Fa, stride), "b": blocking(eik, w, Fb, stride)}
    ins = {"a": pinned_like(Fa), "b": pinned_like(Fb)}
    seq = ["a", "b", "b", "a", "b"]
    outs = [pinned_like(np.zeros_like(Fa)) for _ in seq]
    import torch
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]      # one stream per context, or nothing overlaps
    ctxs = [eik.eik_create(w.dims, w.h, Fa, "fp32", stream=s) for s in streams]
    try:
        for c in ctxs:
            eik.eik_add_sources(c, w.sources)
        eik.eik_set_speed_async(ctxs[0], ins[seq[0]])
        eik.eik_solve_async(ctxs[0], stride)
        for i in range(len(seq)):
            cur, nxt = ctxs[i % 2], ctxs[(i + 1) % 2]
            if i + 1 < len(seq):
                eik.eik_set_speed_async(nxt, ins[seq[i + 1]])
            eik.eik_wait(cur)
            eik.eik_result_async(cur, outs[i])
            if i + 1 < len(seq):
                eik.eik_solve_async(nxt, stride)
        for c in ctxs:
            eik.eik_sync(c)
    finally:
        for c in ctxs:
            eik.eik_destroy(c)
    for i, k in enumerate(seq):
        assert np.array_equal(outs[i], want[k]), (i, k)


def test_async_result_to_device_and_deferred_speed_errors(eik):
    import torch
    w = synth.workload("C2", 40)
    F = np.ascontiguousarray(w.speed(), dtype=np.float32)
    ref = blocking(eik, w, F, 2 * w.h)
    ctx = eik.eik_create(w.dims, w.h, F, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        bad = pinned_like(F)
        bad[3, 4, 5] = -1.0
        eik.eik_set_speed_async(ctx, bad)
        with pytest.raises(eik.EikError, match="finite and >= 0"):
            eik.eik_solve_ex(ctx, 2 * w.h)
        eik.eik_set_speed_async(ctx, bad)
        with pytest.raises(eik.EikError, match="finite and >= 0"):
            eik.eik_sync(ctx)
        eik.eik_sync(ctx)                                  # reported once
        with pytest.raises(eik.EikError, match="no successful solve"):
            eik.eik_result_async(ctx, np.empty_like(F))
        good = pinned_like(F)
        eik.eik_set_speed_async(ctx, good)
        eik.eik_solve_ex(ctx, 2 * w.h)
        out = torch.empty(F.shape, dtype=torch.float32, device="cuda")
        eik.eik_result_async(ctx, out)
        eik.eik_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        eik.eik_destroy(ctx)


def test_sync_with_a_solve_in_flight(eik):
    """eik_sync waits for a queued solve; its statistics still come from eik_wait, once."""
    w = synth.workload("C2", 48)
    F = np.ascontiguousarray(w.speed(), dtype=np.float32)
    ctx = eik.eik_create(w.dims, w.h, F, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        eik.eik_solve_async(ctx, 2 * w.h)
        eik.eik_sync(ctx)
        st = eik.eik_wait(ctx)
        assert st["restarts"] > 0 and st["status"] == 0
        with pytest.raises(eik.EikError, match="no solve in flight"):
            eik.eik_wait(ctx)
        out = np.empty_like(F)
        eik.eik_result(ctx, out)
        assert np.array_equal(out, blocking(eik, w, F, 2 * w.h))
    finally:
        eik.eik_destroy(ctx)
