"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (from the method's statement of accuracy and Sec. 3.2): FP64 mode max-rel
<= 1e-12 over nodes with psi > 0, exact agreement on +inf and 0; FP32 mode
max-abs <= 1e-5 * max(psi) over finite nodes.  Inputs are seeded synthetic grids
from synth/, generated on the host and uploaded, sized so the oracle finishes in
seconds while spanning several 8^3 bricks and a ragged tail.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
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


def run(eik, F, h, sources, precision, stride, device_io=True, **kw):
    import torch
    dt = np.float32 if precision == "fp32" else np.float64
    Fh = np.ascontiguousarray(F.astype(dt))
    nz, ny, nx = F.shape
    if device_io:
        Fd = torch.from_numpy(Fh).cuda()
        ctx = eik.eik_create((nx, ny, nz), h, Fd, precision)
    else:
        ctx = eik.eik_create((nx, ny, nz), h, Fh, precision)
    try:
        eik.eik_add_sources(ctx, sources)
        st = eik.eik_solve_ex(ctx, stride, **kw)
        if device_io:
            out = torch.empty((nz, ny, nx), dtype=torch.float32 if precision == "fp32" else torch.float64,
                              device="cuda")
            eik.eik_result(ctx, out)
            torch.cuda.synchronize()
            psi = out.cpu().numpy()
        else:
            psi = np.empty((nz, ny, nx), dtype=dt)
            eik.eik_result(ctx, psi)
        return psi.astype(np.float64), st
    finally:
        eik.eik_destroy(ctx)


def assert_parity(psi, ref, precision):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(psi), fin), "reachable sets differ"
    if not fin.any():
        return 0.0
    if precision == "fp64":
        zero = ref == 0.0
        assert np.all(psi[zero] == 0.0)
        pos = fin & ~zero
        err = float(np.max(np.abs(psi[pos] - ref[pos]) / ref[pos])) if pos.any() else 0.0
        assert err <= TOL64, err
    else:
        err = float(np.max(np.abs(psi[fin] - ref[fin])))
        assert err <= TOL32 * float(ref[fin].max()), (err, ref[fin].max())
    return err


def test_c1_full_size_fp64(eik, orc):
    """64^3, h = 1/63, F = 1, centre source, stride 2h, FP64."""
    w = synth.workload("C1")
    F = w.speed()
    ref = orc.fmm(F, w.h, w.sources)
    psi, st = run(eik, F, w.h, w.sources, "fp64", 2 * w.h)
    assert_parity(psi, ref, "fp64")
    assert st["restarts"] >= math.ceil(np.max(ref) / (2 * w.h))


@pytest.mark.parametrize("trial", range(8))
def test_random_ragged_grids_fp64(eik, orc, trial):
    u = synth.uniform(9100 + trial, 1, 4)
    dims = tuple(5 + int(x * 36) for x in u[:3])            # 5..40 per axis, ragged against 8
    h = synth.grid_h(dims)
    F = 0.5 + 1.5 * synth.uniform(trial, 21, int(np.prod(dims))).reshape(dims[::-1])
    if trial % 2:
        F[synth.uniform(trial, 22, F.size).reshape(F.shape) < 0.1] = 0.0
    src = synth.random_sources(trial, 23, dims, h, 1 + trial % 3)
    ref = orc.fmm(F, h, src)
    for bd in (8, 16):
        for s in (0.5, 2.0, 8.0, math.inf):
            psi, _ = run(eik, F, h, src, "fp64", s * h, block_dim=bd)
            assert_parity(psi, ref, "fp64")


@pytest.mark.parametrize("cfg,n", [("C2", 72), ("C3", 64), ("C4", 80)])
def test_families_fp32(eik, orc, cfg, n):
    """The three speed families at reduced size, FP32, fixed-stride sweep {1, 2, 4, 8} h."""
    w = synth.workload(cfg, n)
    F = w.speed()
    ref = orc.fmm(F, w.h, w.sources)
    for bd in (8, 16):
        for s in (1.0, 2.0, 4.0, 8.0):
            psi, st = run(eik, F, w.h, w.sources, "fp32", s * w.h, block_dim=bd)
            assert_parity(psi, ref, "fp32")
            assert st["fallbacks"] == 0


@pytest.mark.parametrize("cfg,n", [("C2", 56), ("C4", 48)])
def test_families_fp64(eik, orc, cfg, n):
    w = synth.workload(cfg, n)
    F = synth.round_to(w.speed(), "fp64")
    ref = orc.fmm(F, w.h, w.sources)
    psi, _ = run(eik, F, w.h, w.sources, "fp64", 2 * w.h)
    assert_parity(psi, ref, "fp64")


def test_host_and_device_buffers_agree(eik, orc):
    w = synth.workload("C2", 33)
    F = w.speed()
    a, _ = run(eik, F, w.h, w.sources, "fp32", 2 * w.h, device_io=True)
    b, _ = run(eik, F, w.h, w.sources, "fp32", 2 * w.h, device_io=False)
    assert np.array_equal(a, b)


def test_deterministic(eik):
    w = synth.workload("C4", 64)
    F = w.speed()
    a, sa = run(eik, F, w.h, w.sources, "fp32", 2 * w.h)
    b, sb = run(eik, F, w.h, w.sources, "fp32", 2 * w.h)
    assert np.array_equal(a, b)
    assert sa["restarts"] == sb["restarts"] and sa["accepted"] == sb["accepted"]


@pytest.mark.parametrize("dims,src", [
    ((1, 1, 1), [[0.0, 0.0, 0.0]]),
    ((1, 1, 37), [[0.0, 0.0, 0.3]]),
    ((29, 1, 1), [[0.7, 0.0, 0.0]]),
    ((17, 23, 1), [[0.2, 0.45, 0.0]]),
    ((24, 24, 24), [[8 / 23, 8 / 23, 8 / 23]]),           # a node on three brick faces
    ((16, 16, 16), [[0, 0, 0], [1, 1, 1], [0, 1, 0], [1, 0, 1]]),
    ((9, 9, 9), [[0.5, 0.5, 0.5]]),
])
def test_edge_shapes(eik, orc, dims, src):
    h = synth.grid_h(dims)
    src = np.asarray(src, dtype=np.float64) * (max(dims) - 1) * h if max(dims) > 1 else np.zeros((1, 3))
    F = 0.75 + 0.5 * synth.uniform(5, 1, int(np.prod(dims))).reshape(dims[::-1])
    ref = orc.fmm(F, h, src)
    for prec in ("fp64", "fp32"):
        Fp = synth.round_to(F, prec)
        refp = orc.fmm(Fp, h, src)
        for bd in (8, 16):
            psi, _ = run(eik, Fp, h, src, prec, 2 * h, block_dim=bd)
            assert_parity(psi, refp, prec)


def test_barrier_wall_and_sealed_region(eik, orc):
    n = 40
    h = 1.0 / (n - 1)
    F = np.ones((n, n, n))
    F[:, :, 20] = 0.0
    F[10:30, 10:30, 5] = 0.0                # a box with a sealed interior on the source side
    F[10:30, 10:30, 14] = 0.0
    F[10:30, 10, 5:15] = 0.0
    F[10:30, 29, 5:15] = 0.0
    F[10, 10:30, 5:15] = 0.0
    F[29, 10:30, 5:15] = 0.0
    src = [[0.05, 0.05, 0.05]]
    ref = orc.fmm(F, h, src)
    assert np.isinf(ref[20, 20, 10]) and np.isinf(ref[0, 0, 30])
    for prec in ("fp64", "fp32"):
        for bd in (8, 16):
            psi, _ = run(eik, F, h, src, prec, 2 * h, block_dim=bd)
            assert_parity(psi, ref, prec)


def test_group_blocks_cut_refreshes(eik, orc):
    """16^3 blocks (2x2x2 bricks marched by one CTA) see more of the front per restart: fewer
    acceptances and solves per node than 8^3 blocks (the paper's Sec. 3.5 block-size effect)."""
    w = synth.workload("C4", 96)
    F = w.speed()
    ref = orc.fmm(F, w.h, w.sources)
    p8, s8 = run(eik, F, w.h, w.sources, "fp32", 2 * w.h, block_dim=8)
    p16, s16 = run(eik, F, w.h, w.sources, "fp32", 2 * w.h, block_dim=16)
    assert_parity(p8, ref, "fp32")
    assert_parity(p16, ref, "fp32")
    assert s16["accepted"] < s8["accepted"] and s16["solves"] < s8["solves"]


@pytest.mark.parametrize("cfg,n", [("C3", 64), ("C4", 96), ("C2", 128), ("C4", 192)])
def test_schedule_does_not_change_the_solution(eik, cfg, n):
    """Sec. 2.4: the stride only schedules work.  The root of Alg. 3 is evaluated as a monotone function of
    the neighbour values, so every stride, block edge, schedule and acceptance window reaches the same
    discrete solution bit for bit."""
    w = synth.workload(cfg, n)
    F = w.speed()
    base, _ = run(eik, F, w.h, w.sources, "fp32", 2 * w.h)
    variants = [dict(stride=s * w.h, block_dim=bd) for s, bd in
                ((0.5, 8), (1.0, 8), (1.5, 8), (4.0, 8), (16.0, 8), (math.inf, 8), (1.0, 16), (2.0, 16), (8.0, 16))]
    variants += [dict(stride=2 * w.h, window=1 / math.sqrt(3)), dict(stride=2 * w.h, window=4.0),
                 dict(stride=0.0, block_dim=0),                                  # the learned schedule
                 dict(stride=2 * w.h, schedule=eik.EIK_SCHED_RANDOM, seed=11)]   # 8^3 and 16^3 restarts mixed
    for v in variants:
        kw = dict(v)
        stride = kw.pop("stride")
        psi, _ = run(eik, F, w.h, w.sources, "fp32", stride, **kw)
        assert np.array_equal(psi, base), (v, int(np.sum(psi != base)))


def test_fp64_schedule_does_not_change_the_solution(eik):
    w = synth.workload("C4", 72)
    F = synth.round_to(w.speed(), "fp64")
    base, _ = run(eik, F, w.h, w.sources, "fp64", 2 * w.h)
    for s, bd in ((0.5, 8), (4.0, 8), (math.inf, 8), (2.0, 16)):
        psi, _ = run(eik, F, w.h, w.sources, "fp64", s * w.h, block_dim=bd)
        assert np.array_equal(psi, base), (s, bd)


def test_stride_zero_is_the_learned_schedule(eik, orc):
    """eik_solve(ctx, 0, 0): the learned schedule with the weights a new context holds, picking stride and
    block edge per restart; same solution as the oracle within the FP32 bar, and as a fixed stride bit for bit."""
    import torch
    w = synth.workload("C3", 96)
    F = w.speed()
    ref = orc.fmm(F, w.h, w.sources)
    Fd = torch.from_numpy(F.astype(np.float32)).cuda()
    ctx = eik.eik_create(w.dims, w.h, Fd, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        st = eik.eik_solve(ctx, 0.0, 0)
        out = torch.empty_like(Fd)
        eik.eik_result(ctx, out)
        learned = out.double().cpu().numpy()
        st_f = eik.eik_solve(ctx, 2 * w.h, 8)
        eik.eik_result(ctx, out)
        fixed = out.double().cpu().numpy()
        eik.eik_set_schedule(ctx, None)                     # unloaded weights: stride 0 is refused
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve(ctx, 0.0, 0)
        assert e.value.status == eik.EIK_ESTATE
    finally:
        eik.eik_destroy(ctx)
    assert st["status"] == 0 and st["restarts"] != st_f["restarts"]
    assert_parity(learned, ref, "fp32")
    assert np.array_equal(learned, fixed)


def test_window_zero_is_the_papers_order(eik, orc):
    """omega = 0 accepts one value level per round (the heap order of Alg. 4); same solution."""
    w = synth.workload("C2", 30)
    F = w.speed()
    ref = orc.fmm(F, w.h, w.sources)
    psi, st0 = run(eik, F, w.h, w.sources, "fp64", 2 * w.h, window=1e-300)
    assert_parity(psi, ref, "fp64")
    _, st1 = run(eik, F, w.h, w.sources, "fp64", 2 * w.h)
    assert st0["rounds"] > st1["rounds"]


def test_restart_count_tracks_the_cpu_block_solver(eik, orc):
    """nr of the GPU run vs the paper's Alg. 6 on the CPU with the same block edge and stride."""
    for cfg, n in (("C1", 48), ("C2", 48)):
        w = synth.workload(cfg, n)
        F = synth.round_to(w.speed(), "fp64")
        for s in (1.0, 2.0):
            _, cpu = orc.block_fmm(F, w.h, w.sources, 8, s * w.h)
            _, st = run(eik, F, w.h, w.sources, "fp64", s * w.h)
            assert abs(st["restarts"] - cpu["nr"]) <= 1, (cfg, s, st["restarts"], cpu["nr"])


def test_error_paths(eik):
    import torch
    F = torch.ones((9, 9, 9), dtype=torch.float32, device="cuda")
    ctx = eik.eik_create((9, 9, 9), 0.125, F, "fp32")
    try:
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve(ctx, 0.25)
        assert e.value.status == eik.EIK_ESTATE
        with pytest.raises(eik.EikError) as e:
            eik.eik_result(ctx, torch.empty_like(F))
        assert e.value.status == eik.EIK_ESTATE
        with pytest.raises(eik.EikError) as e:
            eik.eik_add_sources(ctx, [[0.5, 0.5, 1.5]])
        assert e.value.status == eik.EIK_EINVAL
        eik.eik_add_sources(ctx, [[0.5, 0.5, 0.5]])
        for bad in (-1.0, float("nan"), -float("inf")):
            with pytest.raises(eik.EikError) as e:
                eik.eik_solve(ctx, bad)
            assert e.value.status == eik.EIK_EINVAL
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve_ex(ctx, 0.25, max_restarts=2)
        assert e.value.status == eik.EIK_ETIMEOUT
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve(ctx, 0.25, 12)
        assert e.value.status == eik.EIK_ENOTSUP
        st = eik.eik_solve(ctx, 0.25)
        assert st["status"] == 0
    finally:
        eik.eik_destroy(ctx)
    bad = torch.ones((9, 9, 9), dtype=torch.float32, device="cuda")
    bad[3, 3, 3] = -1.0
    with pytest.raises(eik.EikError) as e:
        eik.eik_create((9, 9, 9), 0.125, bad, "fp32")
    assert e.value.status == eik.EIK_EINVAL
    bad[3, 3, 3] = float("nan")
    with pytest.raises(eik.EikError):
        eik.eik_create((9, 9, 9), 0.125, bad, "fp32")


def test_fallback_counter_fires_on_underflowing_speed_ratio(eik, orc):
    """FP32: when (h/F)^2 underflows the root is taken in double (the counter records it)."""
    n = 12
    h = 1e-3
    F = np.full((n, n, n), 1e17)           # h/F = 1e-20, (h/F)^2 below FLT_MIN
    psi, st = run(eik, F, h, [[0.0, 0.0, 0.0]], "fp32", 1e-19)
    assert st["fallbacks"] > 0
    ref = orc.fmm(synth.round_to(F, "fp32"), h, [[0.0, 0.0, 0.0]])
    assert_parity(psi, ref, "fp32")


def test_full_size_c2_256_fp32(eik, orc):
    """256^3 workload at full size and the benchmark's launch configuration, every node vs the oracle."""
    w = synth.workload("C2")
    F = w.speed()
    ref = orc.fmm(F, w.h, w.sources)
    for s in (1.0, 2.0, 4.0, 8.0):
        psi, st = run(eik, F, w.h, w.sources, "fp32", s * w.h)
        assert_parity(psi, ref, "fp32")


def sampled_local_check(orc, w, psi_d, F_d, nsamp, seed):
    """At nsamp random reachable nodes away from the sources: the largest relative gap between the GPU
    value and the upwind update (Alg. 3 in FP64, the oracle's) of its six GPU neighbours."""
    import torch
    nz, ny, nx = psi_d.shape
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, nsamp)
    k, j, i = idx // (nx * ny), (idx // nx) % ny, idx % nx
    pts = np.stack([i, j, k], 1) * w.h
    away = np.min(np.linalg.norm(pts[:, None, :] - np.asarray(w.sources)[None], axis=2), axis=1) > 2 * w.h
    idx, i, j, k = idx[away], i[away], j[away], k[away]
    flat = psi_d.reshape(-1)

    def take(q):
        return flat[torch.from_numpy(q).to(flat.device)].double().cpu().numpy()

    def nb(di, dj, dk):
        ii, jj, kk = i + di, j + dj, k + dk
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
        q = (np.clip(kk, 0, nz - 1) * ny + np.clip(jj, 0, ny - 1)) * nx + np.clip(ii, 0, nx - 1)
        v = take(q)
        v[~ok] = np.inf
        return v

    nbv = np.stack([nb(-1, 0, 0), nb(1, 0, 0), nb(0, -1, 0), nb(0, 1, 0), nb(0, 0, -1), nb(0, 0, 1)], 1)
    psi = take(idx)
    f = F_d.reshape(-1)[torch.from_numpy(idx).to(F_d.device)].double().cpu().numpy()
    assert np.all(np.isfinite(psi)) and np.all(f > 0)
    u = np.array([orc.solve_quadratic(math.inf, nbv[s], [1] * 6, (w.h / f[s]) ** 2) for s in range(len(idx))])
    return float(np.max(np.abs(psi - u) / psi)), len(idx)


@pytest.mark.parametrize("cfg,n", [("C3", 512), ("C4", 1024)])
def test_full_size_local_equation_on_samples(eik, orc, cfg, n):
    """The full-size workloads in the configuration the benchmark times (FP32, learned schedule, 8^3
    blocks): the oracle cannot solve them, but every reachable non-source node of the discrete solution
    equals the upwind update of its neighbours (Eqs. (2.1)-(2.2)).  At 20,000 sampled nodes the GPU value
    and the FP64 update of its six GPU neighbours agree to 8 ulps of FP32 (the FP32 root's own rounding;
    about one ulp is seen), far inside the 1e-5 x max psi bar."""
    import torch
    from paper_1811_00009_gb300.train_schedule import load_weights
    w = synth.workload(cfg, n)
    F = w.speed_torch(torch.device("cuda"))
    ctx = eik.eik_create(w.dims, w.h, F, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        weights, _ = load_weights()
        eik.eik_set_schedule(ctx, weights)
        st = eik.eik_solve_ex(ctx, 2 * w.h, schedule=eik.EIK_SCHED_LEARNED)
        assert st["status"] == 0 and st["fallbacks"] == 0
        psi = torch.empty_like(F)
        eik.eik_result(ctx, psi)
        torch.cuda.synchronize()
    finally:
        eik.eik_destroy(ctx)
    gap, m = sampled_local_check(orc, w, psi, F, 20000, 1811 + n)
    print(f"{cfg} {n}^3: largest relative gap to the local update {gap:.3e} over {m} nodes")
    assert m > 19000
    assert gap <= 8 * 2.0 ** -24, gap


@pytest.mark.parametrize("kw", [dict(block_dim=8), dict(block_dim=16),
                                dict(block_dim=8, schedule=1), dict(block_dim=8, schedule=2, seed=3)],
                         ids=["blocks8", "blocks16", "learned", "random"])
def test_device_waits_give_up_and_the_context_stays_usable(eik, orc, kw):
    """Failure detection without a GPU fault: with a limit of one poll, the device-side waits (the grid
    barrier, a neighbour's march, a work-list entry, the group-list barrier) run out; the kernel records it,
    every warp returns -- on the 16^3 path a CTA leaves as a whole, after a vote at the start of the restart --
    the solve reports EIK_ETIMEOUT, and the next solve on the same context is correct."""
    w = synth.workload("C2", 96)
    F = w.speed()
    Fh = np.ascontiguousarray(F.astype(np.float32))
    ctx = eik.eik_create(w.dims, w.h, Fh, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve_ex(ctx, w.h, wait_polls=1, **kw)
        assert e.value.status == eik.EIK_ETIMEOUT
        assert "wait limit" in str(e.value)
        with pytest.raises(eik.EikError, match="no successful solve"):
            eik.eik_result(ctx, np.empty_like(Fh))
        eik.eik_solve_ex(ctx, 2 * w.h, **kw)
        psi = np.empty_like(Fh)
        eik.eik_result(ctx, psi)
    finally:
        eik.eik_destroy(ctx)
    assert_parity(psi.astype(np.float64), orc.fmm(F.astype(np.float32).astype(np.float64), w.h, w.sources), "fp32")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_many_sources(eik, orc, precision):
    """200 random point sources on a ragged grid: many bricks and 32^3 blocks hold several fixed nodes, some
    source cells overlap (the smaller distance wins, Alg. 1); every block edge gives the oracle's solution."""
    dims = (67, 45, 53)
    h = synth.grid_h(dims)
    F = synth.round_to(0.5 + synth.uniform(41, 1, int(np.prod(dims))).reshape(dims[::-1]), precision)
    src = synth.random_sources(77, 3, dims, h, 200)
    ref = orc.fmm(F, h, src)
    blocks = (8, 16, 32) if precision == "fp32" else (8, 16)
    outs = []
    for bd in blocks:
        psi, st = run(eik, F, h, src, precision, 2 * h, block_dim=bd)
        assert st["status"] == 0
        assert_parity(psi, ref, precision)
        outs.append(psi)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
