"""Blocks of 32^3 nodes (block_dim 32, FP32, fixed stride): one CTA of 1024 threads marches a block.

The paper finds block edge 32 the best for parallel runs (Sec. 3.6).  Through the C ABI this path must
(1) agree with the FP64 oracle within the FP32 bar, on grids that span several 32^3 blocks with a ragged
tail, on the degenerate shapes and on sealed regions; (2) reach the 8^3 solve's result bit for bit (the
root of Alg. 3 is monotone in the neighbour values, so the block edge only schedules work, Sec. 2.4);
(3) refuse what it does not do (FP64, a schedule other than the fixed stride, a restart log); and
(4) give up its waits as a whole CTA and leave the context usable.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_00009_gb300 import build
    build.build()
    import paper_1811_00009_gb300 as E
    return E


def solve(eik, ctx, shape, stride, **kw):
    st = eik.eik_solve_ex(ctx, stride, **kw)
    psi = np.empty(shape, dtype=np.float32)
    eik.eik_result(ctx, psi)
    return psi.astype(np.float64), st


def both(eik, F, h, sources, strides=(2.0,), hs=None):
    """The 32^3 solves at the given strides (multiples of h) and the 8^3 solve at 2h, on one context."""
    Fh = np.ascontiguousarray(F.astype(np.float32))
    nz, ny, nx = F.shape
    ctx = eik.eik_create((nx, ny, nz), h, Fh, "fp32")
    try:
        eik.eik_add_sources(ctx, sources)
        p8, s8 = solve(eik, ctx, F.shape, 2 * h, block_dim=8)
        out = []
        for s in strides:
            out.append(solve(eik, ctx, F.shape, s * h, block_dim=32))
        return p8, s8, out
    finally:
        eik.eik_destroy(ctx)


def assert_fp32_parity(psi, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(psi), fin), "reachable sets differ"
    if fin.any():
        err = float(np.max(np.abs(psi[fin] - ref[fin])))
        assert err <= TOL32 * float(ref[fin].max()), (err, ref[fin].max())


@pytest.mark.parametrize("cfg,n", [("C2", 72), ("C3", 70), ("C4", 80), ("C4", 100)])
def test_parity_and_same_result_as_8_blocks(eik, orc, cfg, n):
    w = synth.workload(cfg, n)
    F = synth.round_to(w.speed(), "fp32")
    ref = orc.fmm(F, w.h, w.sources)
    p8, _, runs = both(eik, F, w.h, w.sources, strides=(0.5, 2.0, 8.0, math.inf))
    for psi, st in runs:
        assert st["status"] == 0 and st["block_dim"] == 32
        assert_fp32_parity(psi, ref)
        assert np.array_equal(psi, p8), int(np.sum(psi != p8))


@pytest.mark.parametrize("dims,src", [
    ((1, 1, 1), [[0.0, 0.0, 0.0]]),
    ((1, 1, 37), [[0.0, 0.0, 0.3]]),
    ((70, 1, 1), [[0.7, 0.0, 0.0]]),
    ((33, 40, 1), [[0.2, 0.45, 0.0]]),
    ((64, 64, 64), [[32 / 63, 32 / 63, 32 / 63]]),         # a node on the faces of eight blocks
    ((33, 33, 33), [[0, 0, 0], [1, 1, 1], [0, 1, 0], [1, 0, 1]]),
    ((65, 31, 97), [[0.3, 0.15, 0.5]]),
])
def test_edge_shapes(eik, orc, dims, src):
    h = synth.grid_h(dims)
    src = np.asarray(src, dtype=np.float64) * (max(dims) - 1) * h if max(dims) > 1 else np.zeros((1, 3))
    F = 0.75 + 0.5 * synth.uniform(5, 1, int(np.prod(dims))).reshape(dims[::-1])
    F = synth.round_to(F, "fp32")
    ref = orc.fmm(F, h, src)
    p8, _, runs = both(eik, F, h, src, strides=(2.0,))
    psi, _ = runs[0]
    assert_fp32_parity(psi, ref)
    assert np.array_equal(psi, p8)


def test_barrier_wall_and_sealed_region(eik, orc):
    n = 72
    h = 1.0 / (n - 1)
    F = np.ones((n, n, n))
    F[:, :, 40] = 0.0
    F[20:60, 20:60, 5] = 0.0                # a box with a sealed interior on the source side, across block faces
    F[20:60, 20:60, 34] = 0.0
    F[20:60, 20, 5:35] = 0.0
    F[20:60, 59, 5:35] = 0.0
    F[20, 20:60, 5:35] = 0.0
    F[59, 20:60, 5:35] = 0.0
    src = [[0.05, 0.05, 0.05]]
    ref = orc.fmm(F, h, src)
    assert np.isinf(ref[40, 40, 20]) and np.isinf(ref[0, 0, 60])
    p8, _, runs = both(eik, F, h, src, strides=(2.0, math.inf))
    for psi, _ in runs:
        assert_fp32_parity(psi, ref)
        assert np.array_equal(psi, p8)


def test_larger_blocks_refresh_less(eik):
    """Sec. 3.5: a larger block carries the front further within a restart, so fewer accepted values are
    refreshed: fewer acceptances and solves per node than with 8^3 blocks, at the same stride."""
    w = synth.workload("C4", 160)
    F = w.speed()
    p8, s8, runs = both(eik, F, w.h, w.sources, strides=(2.0,))
    psi, s32 = runs[0]
    assert np.array_equal(psi, p8)
    assert s32["accepted"] < s8["accepted"] and s32["solves"] < s8["solves"]


def test_full_grid_c2_256(eik):
    """A C2 grid of 256^3 (8^3 blocks of 32^3), several strides: the 8^3 result bit for bit."""
    import torch
    w = synth.workload("C2", 256)
    Fd = torch.from_numpy(w.speed().astype(np.float32)).cuda()
    ctx = eik.eik_create(w.dims, w.h, Fd, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        out = torch.empty_like(Fd)
        eik.eik_solve_ex(ctx, 2 * w.h, block_dim=8)
        eik.eik_result(ctx, out)
        p8 = out.clone()
        for s in (1.0, 4.0):
            st = eik.eik_solve_ex(ctx, s * w.h, block_dim=32)
            eik.eik_result(ctx, out)
            assert st["status"] == 0
            assert torch.equal(out, p8), int((out != p8).sum())
    finally:
        eik.eik_destroy(ctx)


def test_new_speed_and_sources_between_solves(eik, orc):
    """The 32^3 layout of h/F follows eik_set_speed, and the result follows the last solve's block edge."""
    w = synth.workload("C4", 64)
    F1 = synth.round_to(w.speed(), "fp32")
    F2 = synth.round_to(np.where(F1 > 0, 1.0 + 0.5 * synth.uniform(9, 1, F1.size).reshape(F1.shape), 0.0),
                        "fp32")
    Fh = np.ascontiguousarray(F1.astype(np.float32))
    ctx = eik.eik_create(w.dims, w.h, Fh, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        a32, _ = solve(eik, ctx, F1.shape, 2 * w.h, block_dim=32)
        eik.eik_set_speed(ctx, np.ascontiguousarray(F2.astype(np.float32)))
        b32, _ = solve(eik, ctx, F1.shape, 2 * w.h, block_dim=32)
        b8, _ = solve(eik, ctx, F1.shape, 2 * w.h, block_dim=8)
        eik.eik_clear_sources(ctx)
        eik.eik_add_sources(ctx, [[0.0, 0.0, 0.0]])
        c32, _ = solve(eik, ctx, F1.shape, 3 * w.h, block_dim=32)
    finally:
        eik.eik_destroy(ctx)
    assert_fp32_parity(a32, orc.fmm(F1, w.h, w.sources))
    assert_fp32_parity(b32, orc.fmm(F2, w.h, w.sources))
    assert np.array_equal(b32, b8)
    assert_fp32_parity(c32, orc.fmm(F2, w.h, [[0.0, 0.0, 0.0]]))


def test_refused_uses(eik):
    w = synth.workload("C2", 40)
    F = w.speed()
    ctx = eik.eik_create(w.dims, w.h, np.ascontiguousarray(F), "fp64")
    try:
        eik.eik_add_sources(ctx, w.sources)
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve_ex(ctx, 2 * w.h, block_dim=32)
        assert e.value.status == eik.EIK_ENOTSUP
    finally:
        eik.eik_destroy(ctx)
    ctx = eik.eik_create(w.dims, w.h, np.ascontiguousarray(F.astype(np.float32)), "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        for kw in (dict(schedule=eik.EIK_SCHED_LEARNED), dict(schedule=eik.EIK_SCHED_RANDOM, seed=1),
                   dict(log_restarts=1)):
            with pytest.raises(eik.EikError) as e:
                eik.eik_solve_ex(ctx, 2 * w.h, block_dim=32, **kw)
            assert e.value.status == eik.EIK_ENOTSUP, kw
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve_ex(ctx, 2 * w.h, block_dim=24)
        assert e.value.status == eik.EIK_ENOTSUP
    finally:
        eik.eik_destroy(ctx)


def test_waits_give_up_and_the_context_stays_usable(eik, orc):
    """With a limit of one poll the grid barrier's wait runs out; the CTA leaves as a whole, the solve
    reports EIK_ETIMEOUT, and the next solve on the context is correct."""
    w = synth.workload("C2", 96)
    F = synth.round_to(w.speed(), "fp32")
    Fh = np.ascontiguousarray(F.astype(np.float32))
    ctx = eik.eik_create(w.dims, w.h, Fh, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve_ex(ctx, w.h, block_dim=32, wait_polls=1)
        assert e.value.status == eik.EIK_ETIMEOUT
        assert "wait limit" in str(e.value)
        with pytest.raises(eik.EikError, match="no successful solve"):
            eik.eik_result(ctx, np.empty_like(Fh))
        psi, _ = solve(eik, ctx, F.shape, 2 * w.h, block_dim=32)
    finally:
        eik.eik_destroy(ctx)
    assert_fp32_parity(psi, orc.fmm(F, w.h, w.sources))


@pytest.mark.parametrize("frac", [0.3, 0.7])
def test_width_band(eik, orc, frac):
    """width_band (Alg. 6) with 32^3 blocks: exact (the 8^3 full solve's values, bit for bit) wherever the
    solution is at most the width, tentative upper bounds above it."""
    w = synth.workload("C4", 80)
    F = synth.round_to(w.speed(), "fp32")
    full = orc.fmm(F, w.h, w.sources)
    width = frac * float(full[np.isfinite(full)].max())
    Fh = np.ascontiguousarray(F.astype(np.float32))
    ctx = eik.eik_create(w.dims, w.h, Fh, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        p8, _ = solve(eik, ctx, F.shape, 2 * w.h, block_dim=8)
        for s in (1.0, 4.0, math.inf):
            psi, st = solve(eik, ctx, F.shape, s * w.h, block_dim=32, width=width)
            assert st["final_bound"] <= width
            low = p8 <= width
            assert np.array_equal(psi[low], p8[low]), s
            assert np.all(psi[~low] >= p8[~low]), s
    finally:
        eik.eik_destroy(ctx)


def test_async_solve_and_result(eik):
    """eik_solve_async / eik_wait / eik_result_async with 32^3 blocks: the same psi as the synchronous calls,
    with a 32^3 solve and an 8^3 solve on the same context in turn."""
    import torch
    w = synth.workload("C2", 72)
    F = np.ascontiguousarray(w.speed().astype(np.float32))
    ctx = eik.eik_create(w.dims, w.h, F, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        ref, _ = solve(eik, ctx, F.shape, 2 * w.h, block_dim=32)
        outs = [torch.empty(F.shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        for i, bd in enumerate((32, 8)):
            eik.eik_solve_async(ctx, 3 * w.h, block_dim=bd)
            st = eik.eik_wait(ctx)
            assert st["block_dim"] == bd
            eik.eik_result_async(ctx, outs[i].numpy())
            eik.eik_sync(ctx)
        for o in outs:
            assert np.array_equal(o.numpy().astype(np.float64), ref)
    finally:
        eik.eik_destroy(ctx)


def test_restart_cap(eik, orc):
    """max_restarts ends a 32^3 solve with EIK_ETIMEOUT (CTAs in an early march of the next restart finish
    it and leave); the next solve on the context is correct."""
    w = synth.workload("C4", 96)
    F = synth.round_to(w.speed(), "fp32")
    Fh = np.ascontiguousarray(F.astype(np.float32))
    ctx = eik.eik_create(w.dims, w.h, Fh, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        for cap in (1, 3):
            with pytest.raises(eik.EikError) as e:
                eik.eik_solve_ex(ctx, w.h, block_dim=32, max_restarts=cap)
            assert e.value.status == eik.EIK_ETIMEOUT and "restart cap" in str(e.value)
        psi, st = solve(eik, ctx, F.shape, 2 * w.h, block_dim=32)
        assert st["status"] == 0
    finally:
        eik.eik_destroy(ctx)
    assert_fp32_parity(psi, orc.fmm(F, w.h, w.sources))
