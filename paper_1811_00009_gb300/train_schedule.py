"""Train the restart-schedule network from the solver's own per-restart timings.

Data: solves of seeded synthetic grids of the three speed families (seeds
distinct from the evaluation workloads), each run with every fixed action of
the table (stride x block edge) and with the seeded random schedule, recording
per-restart logs (features after restart k, device time of each restart).
Sample for restart k: input = features after k, action = the one chosen then
(it runs in restart k+2), target = log of the cost rate of the `horizon`
restarts from k+2
(device ms per unit h of bound advance).  Training runs on the GPU with the
library's own kernels (eik_mlp_grad / eik_mlp_adam), full batch, Adam.

    python -m paper_1811_00009_gb300.train_schedule --out weights.json [--eval]

--eval then times the 512^3 layered workload (16 z-layers, source at
(0.5, 0.5, 0.1)) with every fixed action and with the learned schedule.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WEIGHTS = os.path.join(HERE, "schedule_weights.json")


def load_weights(path: str = DEFAULT_WEIGHTS):
    with open(path) as fh:
        d = json.load(fh)
    return np.asarray(d["weights"], dtype=np.float32), d


def _solve(eik, ctx, stride, **kw):
    st = eik.eik_solve_ex(ctx, stride, log_restarts=1, **kw)
    return st, eik.eik_restart_log(ctx)


def collect(eik, grids, actions, random_runs=3, log=print):
    """Per-restart records of fixed-action and random-schedule runs on each grid."""
    import torch
    import synth
    runs = []
    for (fam, n, seed) in grids:
        w = synth.workload({"sines": "C2", "layers": "C3", "grf": "C4"}[fam], n)
        w.seed = seed
        w.sources = synth.random_sources(seed, 40, w.dims, w.h, 1 + seed % 2)
        F = w.speed_torch(torch.device("cuda")).float().contiguous()
        ctx = eik.eik_create(w.dims, w.h, F, "fp32")
        eik.eik_add_sources(ctx, w.sources)
        eik.eik_solve_ex(ctx, 2 * w.h)                        # warm-up
        for a, (sh, bd) in enumerate(actions):
            st, recs = _solve(eik, ctx, sh * w.h, block_dim=bd)
            runs.append({"grid": (fam, n, seed), "h": w.h, "fixed": a, "recs": recs, "ms": st["device_ms"]})
        for r in range(random_runs):
            st, recs = _solve(eik, ctx, 2 * w.h, schedule=eik.EIK_SCHED_RANDOM, seed=1000 * seed + r)
            runs.append({"grid": (fam, n, seed), "h": w.h, "fixed": -1, "recs": recs, "ms": st["device_ms"]})
        eik.eik_destroy(ctx)
        log(f"collected {fam} {n}^3 seed {seed}: {len(runs)} runs")
    return runs


def dataset(runs, horizon=2, fixed_only=False):
    X, A, Y = [], [], []
    for run in runs:
        if fixed_only and run["fixed"] < 0:
            continue
        recs, h = run["recs"], run["h"]
        for i in range(len(recs) - 1):
            # the action chosen after restart i runs in restart i+2 (one restart ahead)
            a = run["fixed"] if run["fixed"] >= 0 else recs[i]["next_action"]
            nxt = recs[i + 2:i + 2 + horizon]
            ms = sum(r["ms"] for r in nxt)
            adv = sum(r["stride"] for r in nxt) / h
            if ms <= 0 or not (adv > 0) or not math.isfinite(adv):
                continue
            X.append(recs[i]["features"])
            A.append(a)
            Y.append(math.log(ms / adv))
    return np.asarray(X, np.float32), np.asarray(A, np.int32), np.asarray(Y, np.float32)


def dataset_curves(runs, delta_h=8.0):
    """Every logged state labelled for every action.

    For each grid, the fixed-action runs give T_a(b), the device time until the
    bound reaches b under action a.  A state logged at bound b (in any of the
    grid's runs) gets, for every action a, the target log of the local cost rate
    (T_a(b + delta) - T_a(b)) / (delta / h): what a would cost from this phase
    of the front on.  One sample per (state, action).
    """
    import collections
    by = collections.defaultdict(dict)
    states = collections.defaultdict(list)
    for run in runs:
        g = tuple(run["grid"])
        if run["fixed"] >= 0:
            by[g][run["fixed"]] = run
        states[g].extend(run["recs"])
    X, A, Y = [], [], []
    for g, fixed in by.items():
        h = next(iter(fixed.values()))["h"]
        curves = {}
        for a, run in fixed.items():
            b = np.array([r["bound"] for r in run["recs"]], dtype=np.float64)
            t = np.cumsum([r["ms"] for r in run["recs"]])
            ok = np.isfinite(b)
            curves[a] = (b[ok], t[ok])
        d = delta_h * h
        for rec in states[g]:
            b0 = rec["bound"]
            if not math.isfinite(b0):
                continue
            rates = {}
            for a, (b, t) in curves.items():
                if len(b) < 2 or b0 + 0.5 * d > b[-1]:
                    continue
                t0 = np.interp(b0, b, t)
                t1 = np.interp(min(b0 + d, b[-1]), b, t)
                adv = (min(b0 + d, b[-1]) - b0) / h
                if t1 > t0 and adv > 0:
                    rates[a] = math.log((t1 - t0) / adv)
            if len(rates) < len(curves):
                continue
            for a, y in rates.items():
                X.append(rec["features"])
                A.append(a)
                Y.append(y)
    return np.asarray(X, np.float32), np.asarray(A, np.int32), np.asarray(Y, np.float32)


def dataset_rollout(runs, relative=False):
    """Every logged state labelled for every action with the time to finish.

    For each grid, the fixed-action runs give T_a(b) (device time until the
    bound reaches b under action a) and T_a(end).  A state logged at bound b in
    any of the grid's runs gets, for every action a, the target
    log(T_a(end) - T_a(b) + 0.01 ms): the measured cost of finishing the solve
    from this phase of the front with a.  Taking the lowest at every restart is
    one step of policy improvement over the fixed-stride schedules (a rollout
    policy), so it can only beat the best of them to the extent that these
    values hold for the states it visits.
    """
    import collections
    by = collections.defaultdict(dict)
    states = collections.defaultdict(list)
    for run in runs:
        g = tuple(run["grid"])
        if run["fixed"] >= 0:
            by[g][run["fixed"]] = run
        states[g].extend(run["recs"])
    X, A, Y = [], [], []
    for g, fixed in by.items():
        curves = {}
        for a, run in fixed.items():
            b = np.array([r["bound"] for r in run["recs"]], dtype=np.float64)
            t = np.cumsum([r["ms"] for r in run["recs"]])
            ok = np.isfinite(b)
            curves[a] = (b[ok], t[ok], t[-1])
        for rec in states[g]:
            b0 = rec["bound"]
            if not math.isfinite(b0):
                continue
            ys = {a: math.log(max(tend - (np.interp(b0, b, t) if len(b) else 0.0), 0.0) + 0.01)
                  for a, (b, t, tend) in curves.items()}
            # relative: each action against the mean over actions at this state (the decision only
            # compares actions, and the level, which depends on the grid's size, is left out)
            base = float(np.mean(list(ys.values()))) if relative else 0.0
            for a, y in ys.items():
                X.append(rec["features"])
                A.append(a)
                Y.append(y - base)
    return np.asarray(X, np.float32), np.asarray(A, np.int32), np.asarray(Y, np.float32)


def train(eik, X, A, Y, steps=3000, lr=3e-3, seed=1811, batch=32768, log=print):
    import torch
    import synth
    n = eik.SCHED_PARAMS
    rng = synth.normal(seed, 1, n)
    # layer-wise scaled initial weights, zero biases
    w = np.zeros(n, np.float32)
    o = 0
    for rows, cols in ((eik.SCHED_HIDDEN, eik.SCHED_INPUTS), (eik.SCHED_HIDDEN, 0), (eik.SCHED_HIDDEN, eik.SCHED_HIDDEN),
                       (eik.SCHED_HIDDEN, 0), (eik.SCHED_ACTIONS, eik.SCHED_HIDDEN), (eik.SCHED_ACTIONS, 0)):
        cnt = rows * max(cols, 1) if cols else rows
        if cols:
            w[o:o + cnt] = rng[o:o + cnt] / math.sqrt(cols)
        o += cnt
    w[o - eik.SCHED_ACTIONS:o] = float(np.mean(Y))            # output biases start at the mean target
    perm = np.argsort(synth.uniform(seed, 2, len(Y)))
    nval = max(1, len(Y) // 10)
    val, tr = perm[:nval], perm[nval:]
    dev = torch.device("cuda")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    wd = T(w)
    Xt, At, Yt = T(X[tr]), T(A[tr]), T(Y[tr])
    Xv, Av, Yv = T(X[val]), T(A[val]), T(Y[val])
    nb = min(batch, len(tr))
    order = torch.from_numpy(np.argsort(synth.uniform(seed, 3, len(tr)))).to(dev)
    g = torch.zeros(n, dtype=torch.float32, device=dev)
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.zeros(eik.eik_mlp_work_floats(max(nb, nval)), dtype=torch.float32, device=dev)
    hist = []
    pos = 0
    for t in range(1, steps + 1):
        if pos + nb > len(tr):
            pos = 0
        idx = order[pos:pos + nb]
        pos += nb
        xb, ab, yb = Xt[idx].contiguous(), At[idx].contiguous(), Yt[idx].contiguous()
        eik.eik_mlp_grad(wd, xb, ab, yb, g, loss, work)
        eik.eik_mlp_adam(wd, g, m, v, t, lr=lr if t < steps // 2 else lr / 3)
        if t % 500 == 0 or t == 1:
            tl = loss.item()
            eik.eik_mlp_grad(wd, Xv, Av, Yv, g, loss, work)
            hist.append((t, tl, loss.item()))
            log(f"step {t}: train {tl:.4f} val {loss.item():.4f}")
    return wd.cpu().numpy(), hist


def evaluate(eik, weights, n=512, reps=3, log=print, cfg="C3"):
    """Device time of a workload under every fixed action and under the learned schedule."""
    import torch
    import synth
    w = synth.workload(cfg, n)
    F = w.speed_torch(torch.device("cuda")).float().contiguous()
    ctx = eik.eik_create(w.dims, w.h, F, "fp32")
    eik.eik_add_sources(ctx, w.sources)
    eik.eik_set_schedule(ctx, weights)
    res = {}
    def t(**kw):
        eik.eik_solve_ex(ctx, **kw)
        best = math.inf
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = eik.eik_solve_ex(ctx, **kw)
            best = min(best, time.perf_counter() - t0)
        return best * 1e3, st
    for a, (sh, bd) in enumerate(eik.eik_sched_actions()):
        ms, st = t(stride=sh * w.h, block_dim=bd)
        res[f"fixed_{sh:g}h_b{bd}"] = ms
        log(f"fixed {sh:g}h b{bd}: {ms:.2f} ms, {st['restarts']} restarts")
    for mg in (0.0, 0.02, 0.05):
        ms, st = t(stride=2 * w.h, block_dim=8, schedule=eik.EIK_SCHED_LEARNED, switch_margin=mg)
        res[f"learned_margin_{mg:g}"] = ms
        log(f"learned (margin {mg:g}): {ms:.2f} ms, {st['restarts']} restarts")
    res["learned"] = res["learned_margin_0.02"]
    eik.eik_destroy(ctx)
    best_fixed = min(v for k, v in res.items() if k.startswith("fixed"))
    res["best_fixed"] = best_fixed
    res["learned_over_best_fixed"] = res["learned"] / best_fixed
    res["learned_over_2h"] = res["learned"] / res["fixed_2h_b8"]
    return res


def evaluate_all(eik, weights, log=print, big=False):
    """Held-out 512^3 workloads of the three families (their seeds are not in the training grids) and,
    with big, the 1024^3 GRF workload."""
    out = {}
    keys = ["C3", "C4", "C2"]
    for cfg in keys:
        out[cfg] = evaluate(eik, weights, cfg=cfg, log=log)
    if big:
        out["C4_1024"] = evaluate(eik, weights, n=1024, reps=2, cfg="C4", log=log)
        keys.append("C4_1024")
    out["mean_learned_over_best_fixed"] = float(np.mean([out[c]["learned_over_best_fixed"] for c in keys]))
    out["mean_learned_over_2h"] = float(np.mean([out[c]["learned_over_2h"] for c in keys]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--horizon", type=int, default=8)
    ap.add_argument("--eval", action="store_true")
    ap.add_argument("--eval-1024", action="store_true", help="also evaluate on the 1024^3 GRF workload")
    ap.add_argument("--quick", action="store_true", help="small data set (tests)")
    ap.add_argument("--sizes", default="192,256,320,384,448,512,640,768,1024",
                    help="grid edges of the training grids")
    ap.add_argument("--seeds", type=int, default=2, help="seeds per family and edge (at most 10)")
    ap.add_argument("--runs-out", default=None, help="save the collected per-restart records (JSON)")
    ap.add_argument("--runs-in", default=None,
                    help="train from saved records instead of collecting (comma-separated files are merged)")
    ap.add_argument("--collect-grids", default=None,
                    help="collect these grids (family:edge:seed, comma-separated) and add them to --runs-in")
    ap.add_argument("--variants", default=None,
                    help="comma list N:rollout|rollout_rel|curves|fixed|all (rollout: every action labelled with "
                         "the time its fixed-action run needed to finish from the state's bound; rollout_rel: the "
                         "same relative to the mean over actions; curves: the local cost "
                         "rate over N h; fixed/all: the taken action over the next N restarts); trains and "
                         "evaluates each, keeps the fastest")
    args = ap.parse_args()
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1811_00009_gb300 as eik
    torch.cuda.set_device(0)
    actions = eik.eik_sched_actions()
    if args.quick:
        grids = [("grf", 96, 21), ("layers", 96, 22)]
    else:
        sizes = [int(v) for v in args.sizes.split(",")]
        k = max(1, min(10, args.seeds))
        grids = [(fam, n, 100 + 100 * i + k * j + r if k != 2 else 100 + 20 * i + 2 * j + r)
                 for i, fam in enumerate(("sines", "layers", "grf")) for j, n in enumerate(sizes) for r in range(k)]
    t0 = time.time()
    if args.runs_in:
        runs = []
        for path in args.runs_in.split(","):
            with open(path) as fh:
                runs += json.load(fh)
        if args.collect_grids:
            extra = [(f, int(n), int(sd)) for f, n, sd in (g.split(":") for g in args.collect_grids.split(","))]
            runs += collect(eik, extra, actions)
            grids = grids + extra
    else:
        runs = collect(eik, grids, actions)
    if args.runs_out:
        with open(args.runs_out, "w") as fh:
            json.dump(runs, fh)
    print(f"{len(runs)} runs in {time.time() - t0:.1f} s", flush=True)
    variants = [(0, "rollout")]
    if args.variants:
        variants = [(int(v.split(":")[0]), v.split(":")[1]) for v in args.variants.split(",")]
    best = None
    for hz, fo in variants:
        if fo == "curves":
            X, A, Y = dataset_curves(runs, delta_h=float(hz))
        elif fo == "rollout":
            X, A, Y = dataset_rollout(runs)
        elif fo == "rollout_rel":
            X, A, Y = dataset_rollout(runs, relative=True)
        else:
            X, A, Y = dataset(runs, horizon=hz, fixed_only=(fo == "fixed"))
        print(f"variant {hz} {fo}: {len(Y)} samples", flush=True)
        w, hist = train(eik, X, A, Y, steps=args.steps)
        ev = evaluate_all(eik, w, big=args.eval_1024) if (args.eval or args.variants) else None
        if ev is not None:
            print(json.dumps({"horizon": hz, "labels": fo, "C3": ev["C3"]["learned_over_best_fixed"],
                              "C4": ev["C4"]["learned_over_best_fixed"], "C2": ev["C2"]["learned_over_best_fixed"],
                              "C4_1024": ev.get("C4_1024", {}).get("learned_over_best_fixed"),
                              "mean_vs_best": ev["mean_learned_over_best_fixed"],
                              "mean_vs_2h": ev["mean_learned_over_2h"]}), flush=True)
        score = ev["mean_learned_over_best_fixed"] if ev else 0.0
        if best is None or score < best[0]:
            best = (score, w, hist, hz, fo, ev, len(Y))
    _, w, hist, hz, fo, ev, nsamp = best
    meta = {"weights": [float(v) for v in w], "samples": int(nsamp), "runs": len(runs), "horizon": hz,
            "labels": fo, "grids": grids, "history": hist, "actions": actions,
            "features": ["log1p(active bricks)/16", "log1p(band)/20", "log1p(accepted)/20", "log F_max",
                         "log F_min", "bound/(h*nmax)", "log1p(k)/8", "stride/h/4", "16^3 blocks",
                         "log1p(solves)/20"],
            "target": {"rollout": "log(device ms to finish the solve from the state's bound with the action, from "
                                  "the fixed-action runs) + 0.01 ms",
                       "rollout_rel": "the rollout target minus its mean over the actions at the same state",
                       "curves": f"log(device ms per h of bound advance over the next {hz} h, every action)"}.get(
                           fo, f"log(device ms per h of bound advance over the next {hz} restarts, taken action)")}
    if ev is not None:
        meta["eval_512"] = ev
    with open(args.out, "w") as fh:
        json.dump(meta, fh)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
