"""Writes tests/golden/eq21_*.txt: exact solutions of the Godunov upwind system.

Source of truth: Eq. (2.1) with the differences of Eq. (2.2) (Sec. 2.1), point
sources fixed on the nodes of their cell (Alg. 1).  The values are computed by
oracle/exact.py in 50-digit arithmetic (bisection of the local equation and
Jacobi sweeps to a fixed point), which shares nothing with oracle.c, and are
stored with 30 significant digits.  Run: python tests/golden/make_eq21.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import mpmath as mp  # noqa: E402

from oracle import exact  # noqa: E402

CASES = [
    # name, dims (nx, ny, nz), h, F as text (i, j, k -> value), sources
    ("unit_node_source", (5, 5, 5), "1", "1", [("0", "0", "0")]),
    ("varying_speed_cell_source", (4, 5, 6), "0.25", "1 + i/10 + j/5 - k/20", [("0.3", "0.55", "0.8")]),
    ("barrier_two_sources", (6, 5, 2), "0.2", "0 if (i == 2 and j <= 2) else 1 + (i + j) / 8",
     [("0", "0", "0"), ("1.0", "0.8", "0.2")]),
]


def main():
    for name, dims, h, ftxt, srcs in CASES:
        def F(i, j, k, _t=ftxt):
            return mp.mpf(eval(_t, {}, {"i": mp.mpf(i), "j": mp.mpf(j), "k": mp.mpf(k)}))
        psi = exact.solve(dims, mp.mpf(h), F, [[mp.mpf(c) for c in s] for s in srcs])
        path = os.path.join(HERE, f"eq21_{name}.txt")
        with open(path, "w") as fh:
            fh.write("# Exact solution of Eq. (2.1)-(2.2), Sec. 2.1; point sources fix their cell's nodes (Alg. 1).\n")
            fh.write("# Written by tests/golden/make_eq21.py with oracle/exact.py (50-digit bisection + Jacobi).\n")
            fh.write(f"# dims {dims[0]} {dims[1]} {dims[2]}\n# h {h}\n# F {ftxt}\n")
            for s in srcs:
                fh.write(f"# source {s[0]} {s[1]} {s[2]}\n")
            fh.write("# i j k psi\n")
            for (i, j, k), v in sorted(psi.items(), key=lambda t: (t[0][2], t[0][1], t[0][0])):
                fh.write(f"{i} {j} {k} {'inf' if v == exact.INF else mp.nstr(v, 30)}\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
