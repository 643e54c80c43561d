"""Pins for the FP64 oracle, independent of the oracle itself.

Each test checks the oracle against something the paper or the mathematics
fixes: exact solutions of Eq. (2.1) computed in 50-digit arithmetic by a
different method (golden fixtures), closed forms, a brute-force fixed point,
the residual of Eq. (2.1), monotone acceptance, symmetry, and first-order
convergence to the Euclidean distance.  Plausible mistakes (a dropped term in
the quadratic, a wrong sign, a transposed axis, a heap bug) fail at least one.
"""
import math
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_golden(name):
    meta = {"sources": []}
    vals = {}
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            if line.startswith("#"):
                parts = line[1:].split()
                if parts and parts[0] == "dims":
                    meta["dims"] = tuple(int(p) for p in parts[1:4])
                elif parts and parts[0] == "h":
                    meta["h"] = float(parts[1])
                elif parts and parts[0] == "F":
                    meta["F"] = line.split(None, 2)[2].strip()
                elif parts and parts[0] == "source":
                    meta["sources"].append([float(p) for p in parts[1:4]])
                continue
            i, j, k, v = line.split()
            vals[(int(i), int(j), int(k))] = float(v)
    return meta, vals


@pytest.mark.parametrize("name", ["eq21_unit_node_source.txt", "eq21_varying_speed_cell_source.txt",
                                  "eq21_barrier_two_sources.txt"])
def test_oracle_matches_exact_eq21(orc, name):
    """Golden: 50-digit solution of Eq. (2.1) (Sec. 2.1) on tiny grids; FP64 agrees to rounding."""
    meta, vals = _read_golden(name)
    nx, ny, nz = meta["dims"]
    F = np.empty((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                F[k, j, i] = eval(meta["F"], {}, {"i": float(i), "j": float(j), "k": float(k)})
    psi = orc.fmm(F, meta["h"], meta["sources"])
    for (i, j, k), v in vals.items():
        got = psi[k, j, i]
        if math.isinf(v):
            assert math.isinf(got), (i, j, k, got)
        else:
            assert abs(got - v) <= 1e-14 * max(1.0, abs(v)), (i, j, k, got, v)


def test_closed_forms_node_source(orc):
    """F = 1, source on a node: axis nodes k*h; (1,1,0): h(1 + 1/sqrt2); (1,1,1): h(1 + 1/sqrt2 + 1/sqrt3)."""
    n = 9
    h = 0.125
    F = np.ones((n, n, n))
    psi = orc.fmm(F, h, [[0.0, 0.0, 0.0]])
    for k in range(n):
        assert abs(psi[0, 0, k] - k * h) <= 4 * k * np.finfo(float).eps * h + 0.0
        assert abs(psi[0, k, 0] - k * h) <= 4 * k * np.finfo(float).eps * h
        assert abs(psi[k, 0, 0] - k * h) <= 4 * k * np.finfo(float).eps * h
    a = h * (1 + 1 / math.sqrt(2))
    assert psi[0, 1, 1] == pytest.approx(a, rel=1e-15)
    assert psi[1, 0, 1] == pytest.approx(a, rel=1e-15)
    assert psi[1, 1, 0] == pytest.approx(a, rel=1e-15)
    assert psi[1, 1, 1] == pytest.approx(h * (1 + 1 / math.sqrt(2) + 1 / math.sqrt(3)), rel=1e-15)


def test_plane_sources_give_exact_distance(orc):
    """Sources covering the plane z = 0: psi = z (one-dimensional characteristics)."""
    nx, ny, nz = 6, 5, 12
    h = 1.0 / 11
    F = np.ones((nz, ny, nx))
    src = [[i * h, j * h, 0.0] for j in range(ny) for i in range(nx)]
    psi = orc.fmm(F, h, src)
    for k in range(nz):
        assert np.all(np.abs(psi[k] - k * h) <= 8 * (k + 1) * np.finfo(float).eps), k


def test_speed_scaling(orc):
    """F = c everywhere: psi(F=c) = psi(F=1)/c (Eq. (2.1) is homogeneous in h/F)."""
    w = synth.workload("C1", 20)
    F1 = np.ones(w.dims[::-1])
    p1 = orc.fmm(F1, w.h, w.sources)
    for c in (0.5, 3.0):
        pc = orc.fmm(F1 * c, w.h, w.sources)
        np.testing.assert_allclose(pc, p1 / c, rtol=2e-15, atol=0)


def test_source_cells(orc):
    """Alg. 1 reading: 1 node on a node, 2 on an edge, 4 on a face, 8 inside a cell; out of range rejected."""
    F = np.ones((5, 5, 5))
    h = 0.25
    for src, count in (([0.5, 0.5, 0.5], 1), ([0.6, 0.5, 0.5], 2), ([0.6, 0.7, 0.5], 4), ([0.6, 0.7, 0.1], 8)):
        idx, val = orc.fix_nodes(F, h, [src])
        assert len(idx) == count
        for t, v in zip(idx, val):
            i, j, k = t % 5, (t // 5) % 5, t // 25
            d = math.dist((i * h, j * h, k * h), src)
            assert v == pytest.approx(d, rel=1e-15, abs=0)
    with pytest.raises(ValueError):
        orc.fix_nodes(F, h, [[1.2, 0.5, 0.5]])


def test_fmm_equals_bruteforce_jacobi(orc):
    """(a) Single-heap FMM equals the Jacobi fixed point of the same local solve, on random tiny grids."""
    for trial in range(12):
        u = synth.uniform(7000 + trial, 1, 4)
        dims = tuple(2 + int(x * 11) for x in u[:3])
        h = synth.grid_h(dims)
        F = 0.5 + 1.5 * synth.uniform(trial, 1, int(np.prod(dims))).reshape(dims[::-1])
        if trial % 3 == 2:
            F[synth.uniform(trial, 9, F.size).reshape(F.shape) < 0.15] = 0.0   # barrier nodes
        src = synth.random_sources(trial, 2, dims, h, 1 + trial % 3)
        p = orc.fmm(F, h, src)
        j, sweeps = orc.jacobi(F, h, src)
        assert np.array_equal(p, j), (dims, np.nanmax(np.abs(p - j)))


def test_residual_eq21(orc):
    """(b) The discrete upwind residual of Eq. (2.1) is <= 1e-12 (relative to 1/F^2) at every non-source node."""
    cases = [synth.workload("C1"), synth.workload("C2", 40), synth.workload("C3", 40), synth.workload("C4", 40)]
    for w in cases:
        F = w.speed()
        psi = orc.fmm(F, w.h, w.sources)
        r, n = orc.residual(F, w.h, psi, w.sources)
        assert n > 0.99 * F.size - 16
        assert r <= 1e-12, (w.name, r)


def test_monotone_acceptance(orc):
    """(c) Heap pops come out in non-decreasing psi order, and every reachable node is popped."""
    for w in (synth.workload("C2", 32), synth.workload("C4", 32)):
        F = w.speed()
        psi, li, lv = orc.fmm(F, w.h, w.sources, log=True)
        assert np.all(np.diff(lv) >= 0.0)
        assert len(np.unique(li)) == np.isfinite(psi).sum()


def test_first_order_convergence(orc):
    """(d) F = 1, centred source: max |psi - |x - x_s|| shrinks at first order (up to a log factor)."""
    errs = []
    for n in (17, 33, 65, 129):
        h = 1.0 / (n - 1)
        F = np.ones((n, n, n))
        s = np.array([0.5 + 0.3 * h, 0.5 + 0.1 * h, 0.5 + 0.2 * h])
        psi = orc.fmm(F, h, [s])
        c = np.arange(n) * h
        d = np.sqrt((c[None, None, :] - s[0]) ** 2 + (c[None, :, None] - s[1]) ** 2 + (c[:, None, None] - s[2]) ** 2)
        errs.append(np.max(np.abs(psi - d)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(e > 0 for e in errs)
    assert all(1.3 < r < 2.2 for r in ratios), (errs, ratios)
    # first order with a logarithmic factor: error * n / log n roughly constant
    scaled = [e * (n - 1) / math.log(n - 1) for e, n in zip(errs, (17, 33, 65, 129))]
    assert max(scaled) / min(scaled) < 1.6, scaled


def test_cube_symmetry(orc):
    """Centred source, F = 1: the solution has the 48 symmetries of the cube, bit for bit."""
    w = synth.workload("C1", 24)
    psi = orc.fmm(np.ones(w.dims[::-1]), w.h, w.sources)
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        q = np.transpose(psi, perm)
        for flips in range(8):
            r = q
            for a in range(3):
                if flips >> a & 1:
                    r = np.flip(r, axis=a)
            assert np.array_equal(r, psi)


def test_barriers_and_unreachable(orc):
    """F = 0 nodes are never solved and stay +inf (Sec. 3.3); a sealed region stays +inf."""
    n = 20
    h = 1.0 / (n - 1)
    F = np.ones((n, n, n))
    F[:, :, 10] = 0.0              # a full wall x = 10
    psi = orc.fmm(F, h, [[0.2, 0.3, 0.4]])
    assert np.all(np.isinf(psi[:, :, 10:]))
    assert np.all(np.isfinite(psi[:, :, :10]))
    F[:, 5:15, 10] = 1.0           # open a window: everything reachable except the wall itself
    psi = orc.fmm(F, h, [[0.2, 0.3, 0.4]])
    assert np.all(np.isinf(psi[F == 0.0]))
    assert np.all(np.isfinite(psi[F > 0.0]))


def test_one_dimensional_reduction(orc):
    """A 1 x 1 x n grid is the 1-D problem: psi_k = |k h - s| / F for constant F, up to rounding."""
    n = 50
    h = 0.02
    F = np.full((n, 1, 1), 2.0)
    s = 0.37
    psi = orc.fmm(F, h, [[0.0, 0.0, s]])
    ref = np.abs(np.arange(n) * h - s) / 2.0
    np.testing.assert_allclose(psi[:, 0, 0], ref, rtol=1e-13, atol=1e-16)
