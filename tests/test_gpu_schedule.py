"""The per-restart schedule inside the restart loop: logged decisions, features, and invariance of psi."""
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


def solve(eik, w, F, **kw):
    import torch
    Fd = torch.from_numpy(F.astype(np.float32)).cuda()
    ctx = eik.eik_create(w.dims, w.h, Fd, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        weights = kw.pop("weights", None)
        if weights is not None:
            eik.eik_set_schedule(ctx, weights)
        st = eik.eik_solve_ex(ctx, 2 * w.h, log_restarts=1, **kw)
        log = eik.eik_restart_log(ctx)
        out = torch.empty_like(Fd)
        eik.eik_result(ctx, out)
        torch.cuda.synchronize()
        return out.double().cpu().numpy(), st, log
    finally:
        eik.eik_destroy(ctx)


def features_from_record(r, h, nmax):
    """The documented schedule features, restated from a restart record."""
    x = [math.log1p(r["active"]) / 16, math.log1p(r["band"]) / 20, math.log1p(r["accepted"]) / 20,
         math.log(h / r["rmin"]) if 0 < r["rmin"] < 1e300 else 0.0,
         math.log(h / r["rmax"]) if 0 < r["rmax"] < 1e300 else 0.0,
         r["bound"] / (h * nmax), math.log1p(r["k"]) / 8, r["stride"] / h / 4,
         1.0 if r["block_dim"] == 16 else 0.0, math.log1p(r["solves"]) / 20]
    return np.clip(np.array(x), -10, 10)


def test_random_schedule_follows_its_actions_and_keeps_psi(eik, orc):
    w = synth.workload("C4", 88)
    F = synth.round_to(w.speed(), "fp32")
    ref = orc.fmm(F, w.h, w.sources)
    fixed, _, _ = solve(eik, w, F)
    acts = eik.eik_sched_actions()
    psi, st, log = solve(eik, w, F, schedule=eik.EIK_SCHED_RANDOM, seed=5)
    assert len(log) == st["restarts"]
    modes = {r["block_dim"] for r in log}
    assert modes <= {8, 16} and len(modes) == 2
    # restarts 1 and 2 take the initial stride and block edge; the action chosen
    # after restart k applies to restart k+2 (chosen one restart ahead)
    assert log[0]["stride"] == 2 * w.h and log[1]["stride"] == 2 * w.h
    assert log[0]["block_dim"] == 8 and log[1]["block_dim"] == 8
    for a, b in zip(log[:-2], log[2:]):
        sh, bd = acts[a["next_action"]]
        assert b["block_dim"] == bd and abs(b["stride"] - sh * w.h) <= 1e-15
    for a, b in zip(log[:-1], log[1:]):
        assert b["bound"] == a["bound"] + b["stride"]
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(psi), fin)
    assert np.max(np.abs(psi[fin] - ref[fin])) <= 1e-5 * ref[fin].max()
    assert np.array_equal(psi, fixed)


def test_logged_features_match_their_definition(eik):
    w = synth.workload("C2", 72)
    F = synth.round_to(w.speed(), "fp32")
    _, _, log = solve(eik, w, F, schedule=eik.EIK_SCHED_RANDOM, seed=2)
    for r in log:
        np.testing.assert_allclose(np.array(r["features"]), features_from_record(r, w.h, max(w.dims)),
                                   rtol=2e-6, atol=2e-6)


def test_learned_schedule_needs_weights(eik):
    """A new context holds the shipped weights; once they are unloaded the learned schedule is refused."""
    import torch
    w = synth.workload("C2", 24)
    Fd = torch.from_numpy(w.speed().astype(np.float32)).cuda()
    ctx = eik.eik_create(w.dims, w.h, Fd, "fp32")
    try:
        eik.eik_add_sources(ctx, w.sources)
        assert eik.eik_solve_ex(ctx, 2 * w.h, schedule=eik.EIK_SCHED_LEARNED)["status"] == 0
        eik.eik_set_schedule(ctx, None)
        with pytest.raises(eik.EikError) as e:
            eik.eik_solve_ex(ctx, 2 * w.h, schedule=eik.EIK_SCHED_LEARNED)
        assert e.value.status == eik.EIK_ESTATE
        with pytest.raises(eik.EikError):
            eik.eik_set_schedule(ctx, np.zeros(5, np.float32))
    finally:
        eik.eik_destroy(ctx)


def test_learned_schedule_decides_from_the_network(eik, orc):
    """With a given network (and no switching margin) the schedule chooses, after every restart, the
    action of lowest output (for the restart after the next one)."""
    from oracle import mlp
    w = synth.workload("C3", 80)
    F = synth.round_to(w.speed(), "fp32")
    ref = orc.fmm(F, w.h, w.sources)
    weights = (synth.normal(77, 1, mlp.n_params()) * 0.5).astype(np.float32)
    psi, st, log = solve(eik, w, F, schedule=eik.EIK_SCHED_LEARNED, weights=weights, switch_margin=0.0)
    for r in log[:-1]:
        y, _, _ = mlp.forward(weights.astype(np.float64), np.array([r["features"]], dtype=np.float64))
        assert y[0][r["next_action"]] <= y[0].min() + 1e-4     # the lowest output, up to FP32 rounding
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(psi), fin)
    assert np.max(np.abs(psi[fin] - ref[fin])) <= 1e-5 * ref[fin].max()
