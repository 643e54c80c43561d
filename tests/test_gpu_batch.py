"""Batched solves (eik_batch_* of the C ABI): many grids in one persistent launch.

Every grid of a batch must get the discrete solution of its own problem, so the
bar is the one-grid bar against the FP64 oracle (FP64: max-rel <= 1e-12, FP32:
max-abs <= 1e-5 * max psi), whatever block edge and stride each grid runs with.
Grids are ragged against the 8^3 bricks, mix the speed families and 1-4
sources, and include the degenerate cases (a single node; a source inside a
cell of barrier nodes, so that the grid never becomes active).
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


def assert_parity(psi, ref, precision, what=""):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(psi), fin), f"{what}: reachable sets differ"
    if not fin.any():
        return 0.0
    if precision == "fp64":
        zero = ref == 0.0
        assert np.all(psi[zero] == 0.0), what
        pos = fin & ~zero
        err = float(np.max(np.abs(psi[pos] - ref[pos]) / ref[pos])) if pos.any() else 0.0
        assert err <= TOL64, (what, err)
    else:
        err = float(np.max(np.abs(psi[fin] - ref[fin])))
        assert err <= TOL32 * float(ref[fin].max()), (what, err, ref[fin].max())
    return err


def small_grids(seed, count, precision):
    """Ragged grids 5..40 per axis, speed families of the paper's cases, 1-4 sources."""
    u = synth.uniform(seed, 1, 6 * count).reshape(count, 6)
    fams = ["const", "sines", "layers", "grf"]
    out = []
    for i in range(count):
        dims = tuple(5 + int(x * 36) for x in u[i, :3])
        h = synth.grid_h(dims)
        fam = fams[int(u[i, 3] * 4) % 4]
        w = synth.Workload(f"S{i}", dims, h, fam, seed * 100 + i,
                           synth.random_sources(seed * 100 + i, 7, dims, h, 1 + int(u[i, 4] * 4) % 4),
                           precision=precision)
        F = w.speed()
        if i % 3 == 2:                                   # barrier nodes (F = 0) in some grids
            F = F.copy()
            F[synth.uniform(seed * 100 + i, 8, F.size).reshape(F.shape) < 0.1] = 0.0
        F = np.ascontiguousarray(F, dtype=np.float32 if precision == "fp32" else np.float64)
        out.append((dims, h, F, w.sources))
    return out


def tiles_mixed(grids, seed):
    u = synth.uniform(seed, 2, 2 * len(grids)).reshape(-1, 2)
    strides = [0.5, 1.0, 2.0, 3.0, 8.0]
    return [(8 if u[i, 0] < 0.5 else 16, strides[int(u[i, 1] * 5) % 5] * g[1]) for i, g in enumerate(grids)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_batch_matches_oracle(eik, orc, precision):
    grids = small_grids(4101 if precision == "fp64" else 4102, 14, precision)
    # degenerate members: one node; a grid whose only source lies inside a cell
    # of barrier nodes (no node can be fixed, so the grid never becomes active)
    dt = np.float32 if precision == "fp32" else np.float64
    grids.append(((1, 1, 1), 1.0, np.ones((1, 1, 1), dt), np.array([[0.0, 0.0, 0.0]])))
    Fb = np.ones((9, 10, 11), dt)
    Fb[:2, :2, :2] = 0.0
    grids.append(((11, 10, 9), 0.1, Fb, np.array([[0.05, 0.05, 0.05]])))
    tiles = tiles_mixed(grids, 17)
    with eik.Batch(grids, precision) as B:
        st = B.solve(tiles)
        info = B.info()
        assert st["status"] == 0
        for i, (dims, h, F, src) in enumerate(grids):
            ref = orc.fmm(F.astype(np.float64), h, src)
            psi = B.result(i).astype(np.float64)
            assert_parity(psi, ref, precision, f"grid {i} {dims} tile {tiles[i]}")
            assert info[i]["block_dim"] == tiles[i][0]
        # the barrier-source grid never gets work, the others finish by the last restart
        assert info[-1]["restarts"] == 0
        assert max(r["restarts"] for r in info) == st["restarts"]
        assert all(r["done_ms"] <= st["device_ms"] + 1e-3 for r in info)


def test_batch_equals_single_grid_path(eik):
    """A grid solved inside a batch gives what eik_solve gives it with the same tile (FP64)."""
    import torch
    grids = small_grids(4103, 6, "fp64")
    tiles = tiles_mixed(grids, 18)
    with eik.Batch(grids, "fp64") as B:
        B.solve(tiles)
        for i, (dims, h, F, src) in enumerate(grids):
            with eik.Solver(dims, h, np.ascontiguousarray(F), "fp64") as S:
                S.add_sources(src)
                S.solve(tiles[i][1], block_dim=tiles[i][0])
                one = S.result()
            got = B.result(i)
            assert np.array_equal(got, one)
    torch.cuda.synchronize()


def test_batch_repeatable_and_device_io(eik):
    """Two solves of one batch give the same bits (every march reads the state
    of the previous restart only), and device-resident speeds and outputs work."""
    import torch
    grids = small_grids(4104, 8, "fp32")
    dev = [(d, h, torch.from_numpy(np.ascontiguousarray(F)).cuda(), s) for d, h, F, s in grids]
    with eik.Batch(dev, "fp32") as B:
        B.solve(tiles_mixed(grids, 19))
        first = [B.result(i).copy() for i in range(len(grids))]
        B.solve(tiles_mixed(grids, 19))
        for i, (d, h, F, s) in enumerate(grids):
            out = torch.empty(d[::-1], dtype=torch.float32, device="cuda")
            B.result(i, out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), first[i], equal_nan=True)


def test_batch_errors(eik):
    grids = small_grids(4105, 2, "fp32")
    with eik.Batch(grids, "fp32") as B:
        with pytest.raises(eik.EikError, match="no successful solve"):
            B.result(0)
        with pytest.raises(eik.EikError, match="tile 1"):
            B.solve([(8, grids[0][1]), (12, grids[1][1])])
        with pytest.raises(eik.EikError, match="tile 0"):
            B.solve([(8, math.inf), (8, grids[1][1])])
        with pytest.raises(eik.EikError, match="ctas_per_sm"):
            B.solve(None, ctas_per_sm=99)
        B.solve()
        with pytest.raises(eik.EikError, match="out of range"):
            B.result(5)
    bad = [((8, 8, 8), 0.1, np.ones((8, 8, 8), np.float32), np.array([[0.0, 0.0, 5.0]]))]
    with pytest.raises(eik.EikError, match="item 0: source 0 lies outside"):
        eik.Batch(bad, "fp32")
    neg = [((8, 8, 8), 0.1, -np.ones((8, 8, 8), np.float32), np.array([[0.0, 0.0, 0.0]]))]
    with pytest.raises(eik.EikError, match="finite and >= 0"):
        eik.Batch(neg, "fp32")


def test_autotune_small_batch(eik, orc):
    """The autotuner returns tiles from its candidate table (one policy for the
    batch, and a longer stride, by one factor, for the grids that finish last),
    keeps them for later solves, and the tuned solve still matches the oracle."""
    grids = small_grids(4106, 10, "fp32")
    with eik.Batch(grids, "fp32") as B:
        _, _, max_ctas = B.size()
        tiles, ctas, ms = B.autotune(rounds=2)
        assert 1 <= ctas <= max_ctas and ms > 0
        B.solve()                                # tuned tiles and CTAs per SM
        info = B.info()
        factors = {0.5, 0.75, 1.0, 1.5, 2.0}
        per_h = {1.25, 1.5, 1.75, 2.0, 2.5, 3.0, 4.0}
        f_used, c_used = [], []
        for i, (bd, stride) in enumerate(tiles):
            assert bd in (8, 16)
            assert info[i]["block_dim"] == bd and info[i]["stride"] == stride
            r = info[i]["rmin"]
            if math.isfinite(r):
                f_used.append(round(stride / (bd * r), 6))
            c_used.append(round(stride / grids[i][1], 6))

        def one_policy(vals, table):
            vs = sorted(set(vals))
            if len(vs) == 1:
                return round(vs[0], 4) in table
            if len(vs) != 2:
                return False
            ratio = round(vs[1] / vs[0], 4)
            return ((round(vs[0], 4) in table and ratio in (1.25, 1.5, 2.0)) or             # the last grids longer
                    (round(vs[1], 4) in table and round(vs[0] / vs[1], 4) in (0.5, 0.75)))   # the first shorter
        # a multiple of h, or of edge * min h/F, the same for the batch up to the one boost factor
        assert one_policy(c_used, per_h) or one_policy(f_used, factors), (c_used, f_used)
        for i, (dims, h, F, src) in enumerate(grids):
            ref = orc.fmm(F.astype(np.float64), h, src)
            assert_parity(B.result(i).astype(np.float64), ref, "fp32", f"grid {i}")


def test_full_size_batch_64(eik, orc):
    """The 64-grid batch (edges 32..192 per axis, 1-4 sources, sines / layers /
    GRF speeds, FP32): every grid against the one-grid GPU path, and the
    smallest, a middle and the largest grid against the FP64 oracle."""
    import torch
    ws = synth.batch_workloads(64)
    grids = [(w.dims, w.h, w.speed_torch("cuda"), w.sources) for w in ws]
    with eik.Batch(grids, "fp32") as B:
        st = B.solve()
        assert st["status"] == 0
        info = B.info()
        lat = sorted(r["done_ms"] for r in info)
        assert lat[-1] <= st["device_ms"] + 1e-3 and lat[0] > 0
        order = sorted(range(64), key=lambda i: ws[i].npoints)
        for i in (order[0], order[32], order[-1]):
            F = ws[i].speed().astype(np.float64)
            ref = orc.fmm(F, ws[i].h, ws[i].sources)
            assert_parity(B.result(i).astype(np.float64), ref, "fp32", ws[i].name)
        for i, w in enumerate(ws):
            out = torch.empty(w.dims[::-1], dtype=torch.float32, device="cuda")
            B.result(i, out)
            with eik.Solver(w.dims, w.h, grids[i][2], "fp32") as S:
                S.add_sources(w.sources)
                S.solve(2 * w.h)
                one = torch.empty_like(out)
                eik.eik_result(S.ctx, one)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), one.cpu().numpy()
            assert np.array_equal(a, b), w.name
