"""Eq. (2.1) solved in 50-digit arithmetic on tiny grids: a pin for the FP64 oracle.

TEST INFRASTRUCTURE ONLY.  Independent of oracle.c: the local equation
    sum_axes max(x - m_a, 0)^2 = h^2 / F^2,
with m_a the smaller of the two neighbours along axis a (Eq. (2.1) with the
one-sided differences of Eq. (2.2)), is solved by bisection instead of the
sorted-root formula of Alg. 3, and the global system by Jacobi sweeps from +inf
(fixed nodes held) until no value moves by more than 1e-40.  Point sources fix
the nodes of the cell that contains them, psi0 = distance / F (Alg. 1).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import mpmath as mp

mp.mp.dps = 50
INF = mp.inf


def _cell_nodes(s, h, n) -> List[int]:
    t = s / h
    tn = mp.floor(t + mp.mpf("0.5"))
    if abs(t - tn) <= mp.mpf("1e-9"):
        return [int(min(max(tn, 0), n - 1))]
    i0 = int(mp.floor(t))
    i0 = min(max(i0, 0), n - 2)
    return [i0, i0 + 1]


def _local_root(m: Sequence, r) -> mp.mpf:
    lo = min(m)
    if lo == INF:
        return INF
    a, b = lo, lo + r          # f(lo) = -r^2 < 0, f(lo + r) >= 0
    for _ in range(200):
        c = (a + b) / 2
        f = sum((max(c - v, 0) if v != INF else 0) ** 2 for v in m) - r * r
        if f > 0:
            b = c
        else:
            a = c
        if b - a < mp.mpf("1e-45") * (1 + abs(b)):
            break
    return (a + b) / 2


def solve(dims: Tuple[int, int, int], h, F, sources) -> dict:
    """Return {(i, j, k): psi} for the grid dims=(nx, ny, nz); F(i, j, k) -> mpf speed."""
    nx, ny, nz = dims
    h = mp.mpf(h)
    psi = {(i, j, k): INF for k in range(nz) for j in range(ny) for i in range(nx)}
    fixed = {}
    for s in sources:
        s = [mp.mpf(c) for c in s]
        for k in _cell_nodes(s[2], h, nz):
            for j in _cell_nodes(s[1], h, ny):
                for i in _cell_nodes(s[0], h, nx):
                    d = mp.sqrt((i * h - s[0]) ** 2 + (j * h - s[1]) ** 2 + (k * h - s[2]) ** 2)
                    f = F(i, j, k)
                    if d == 0:
                        v = mp.mpf(0)
                    elif f > 0:
                        v = d / f
                    else:
                        continue
                    fixed[(i, j, k)] = min(fixed.get((i, j, k), INF), v)
    psi.update(fixed)
    for _ in range(10000):
        new = dict(psi)
        moved = mp.mpf(0)
        for (i, j, k), p in psi.items():
            if (i, j, k) in fixed:
                continue
            f = F(i, j, k)
            if not f > 0:
                continue
            m = []
            for a, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                lo = psi.get((i - di, j - dj, k - dk), INF)
                hi = psi.get((i + di, j + dj, k + dk), INF)
                m.append(min(lo, hi))
            x = _local_root(m, h / f)
            if x < p:
                new[(i, j, k)] = x
                moved = max(moved, (p - x) if p != INF else mp.mpf(1))
        psi = new
        if moved < mp.mpf("1e-40"):
            break
    return psi
