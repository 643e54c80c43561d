"""width_band (Alg. 6) on the GPU: a partial solve that is exact up to the width.

Nodes with psi <= width must match the FP64 oracle's full solution (FP64: max-rel <= 1e-12, FP32:
max-abs <= 1e-5 * max psi); nodes above it hold tentative values that are no smaller than the exact ones
(or +inf), whatever the stride, block edge or schedule.
"""
import math

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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("frac", [0.1, 0.45, 0.8])
def test_width_band_partial_solve(eik, orc, precision, frac):
    w = synth.workload("C4", 56)
    F = synth.round_to(w.speed(), precision)
    full = orc.fmm(F, w.h, w.sources)
    width = frac * float(full[np.isfinite(full)].max())
    dt = np.float32 if precision == "fp32" else np.float64
    for bd in (8, 16):
        for s in (1.0, 2.0, math.inf):
            with eik.Solver(w.dims, w.h, np.ascontiguousarray(F.astype(dt)), precision) as S:
                S.add_sources(w.sources)
                st = S.solve(s * w.h, block_dim=bd, width=width)
                psi = S.result().astype(np.float64)
            assert st["final_bound"] <= width
            low = full <= width
            if precision == "fp64":
                err = np.max(np.abs(psi[low] - full[low]) / np.maximum(full[low], 1e-300))
                assert err <= 1e-12, (bd, s, err)
            else:
                tol = 1e-5 * float(full[np.isfinite(full)].max())
                assert np.max(np.abs(psi[low] - full[low])) <= tol, (bd, s)
            high = ~low & np.isfinite(full)
            slack = 0.0 if precision == "fp64" else 1e-5 * float(full[np.isfinite(full)].max())
            assert np.all(psi[high] >= full[high] * (1 - 1e-12) - slack), (bd, s)


def test_width_band_learned_schedule(eik, orc):
    """The bound cap also holds under a schedule that changes the stride (random actions)."""
    w = synth.workload("C2", 64)
    F = synth.round_to(w.speed(), "fp32")
    full = orc.fmm(F, w.h, w.sources)
    width = 0.5 * float(full.max())
    with eik.Solver(w.dims, w.h, np.ascontiguousarray(F.astype(np.float32)), "fp32") as S:
        S.add_sources(w.sources)
        S.solve(2 * w.h, schedule=eik.EIK_SCHED_RANDOM, seed=3, width=width)
        psi = S.result().astype(np.float64)
    low = full <= width
    assert np.max(np.abs(psi[low] - full[low])) <= 1e-5 * float(full.max())
    assert np.all(psi[~low] >= full[~low] - 1e-5 * float(full.max()))
