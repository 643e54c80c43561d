"""Benchmark: Eikonal solves per second on one GB300, as Mpoints/s and HBM roofline fraction.

One step = one full solve of the block-based restarted narrow-band method
(initialisation, every restart's march and exchange, activation) on the 1024^3
workload: node grid h = 1/1023, F = exp(g) with g a Gaussian random field (white
noise smoothed on the grid by a Gaussian; std 0.5, correlation length 0.05),
point source at the centre, FP32 storage with the FP64 root fallback.  Inputs are resident in HBM when the timed region
starts; they are larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own instance of the workload
(independent problems, no collective on the data path: weak scaling); rank 0
prints one JSON line with the whole-job throughput.  --impl reference times
the FP64 CPU oracle on a bounded sample of the same workload family.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Eikonal Mpoints/s at 512^3/1024^3 + HBM roofline %; learned vs fixed stride"
ALGO_BYTES_PER_POINT = {"fp32": 8, "fp64": 16}      # read F once + write psi once
KERNELS_PER_SOLVE = 4                                # gather_r, init_sources, restart_loop, restore_r
# DRAM bytes and warp instructions per node of k_restart_loop (fixed stride 2h, 8^3 blocks, FP32) from an ncu
# capture of the same workload family at 512^3 (dram__bytes_read.sum + dram__bytes_write.sum = 9.387 GB +
# 4.636 GB; smsp__inst_executed.sum = 23.517 G over 512^3 nodes), scaled to the launch by its node count;
# profiles/k_restart_loop_c4_512_fixed2h.md gives the command.
NCU_TRAFFIC_PER_NODE = {"fp32": (9.436e9 + 4.657e9) / 512 ** 3}
NCU_INST_PER_NODE = {"fp32": 23.852e9 / 512 ** 3}
ISSUE_PER_SM_CYCLE = 4          # warp schedulers per SM, one warp instruction per cycle each


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def rank_workload(n: int, rank: int):
    """The 1024^3-family workload of one rank: every rank solves its own instance (its own random field),
    so ranks share no data and need no collective on the data path (weak scaling)."""
    import synth
    w = synth.workload("C4", n)
    if rank:
        w.seed += 1000 * rank
    return w


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over the ranks (the job is as slow as its slowest rank); x itself when the
    process group is absent or has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points_per_rank: int, steps: int, ranks: int, seconds: float) -> float:
    """Whole-job throughput in Mpoints/s: the points every rank solved over the slowest rank's time."""
    return points_per_rank * steps * ranks / seconds / 1e6


def setup_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(n: int, seed_cfg: str = "C4"):
    """Time the single-heap FP64 oracle (one thread) on the workload family at n^3."""
    import oracle
    import synth
    w = synth.workload(seed_cfg, n)
    F = w.speed()
    oracle.build()
    t0 = time.perf_counter()
    psi = oracle.fmm(F, w.h, w.sources)
    dt = time.perf_counter() - t0
    return w, F, psi, dt


def cpu_block_sample(w, F):
    """Time the CPU form of the paper's method (the oracle's Alg. 6, OpenMP over blocks, FP64) on all host
    cores, block edge 32 and stride 2h (the paper's parallel optimum), on workload w with speeds F (host,
    float64).  Returns the baseline record and the oracle's psi (the oracle tests pin the block solver to the
    single-heap one: identical with one block, equal to machine accuracy with many)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    psi, st = oracle.block_fmm(F, w.h, w.sources, 32, 2.0 * w.h, nthreads=cores)
    dt = time.perf_counter() - t0
    n = w.dims[0]
    return {"value": w.npoints / dt / 1e6, "unit": "Mpoints/s", "cores": cores,
            "kind": "oracle block solver (Alg. 6 with OpenMP)",
            "sample": f"one full solve of the benchmark's workload ({n}^3, the same F), block 32, stride 2h, FP64, "
                      f"{dt:.2f} s, {st['nr']} restarts"}, psi


def max_abs_error(psi32, ref) -> float:
    """max |psi - ref| over the finite nodes of ref, in chunks (the full-size arrays are GiB-sized);
    inf if the sets of unreachable nodes differ."""
    import numpy as np
    a, b = psi32.reshape(-1), ref.reshape(-1)
    err = 0.0
    step = 1 << 26
    for lo in range(0, a.size, step):
        x, y = a[lo:lo + step].astype(np.float64), b[lo:lo + step]
        m = np.isfinite(y)
        if not np.array_equal(np.isfinite(x), m):
            return float("inf")
        if m.any():
            err = max(err, float(np.max(np.abs(x[m] - y[m]))))
    return err


def run_reference(args):
    ws, rank, _ = setup_dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    n = args.ref_n
    w = synth.workload("C4", n)
    F = w.speed()
    oracle.build()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.fmm(F, w.h, w.sources)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = w.npoints * len(times) / total / 1e6
    sample = (f"C4 family (same F recipe) at {n}^3, h=1/{n - 1}, centre source; single-heap FP64 fast "
              f"marching oracle, one thread, one full solve per step")
    line = {"metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"C4-family {n}^3 sample of the 1024^3 GRF workload (oracle)",
                       "grid": [n, n, n]},
            "cpu_baseline": {"value": value, "unit": "Mpoints/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batch_bench(eik, synth, steps: int, warmup: int, tune_rounds: int, dev):
    """The batched launch: 64 grids (edges 32..192 per axis, 1-4 sources, sines /
    layers / GRF speeds, FP32) solved together; solves/s and per-solve latency
    percentiles with the autotuned tiles, and with the untuned default tiles
    (8^3 blocks, stride 2h) beside them."""
    import numpy as np
    import torch
    ws = synth.batch_workloads(64)
    grids = [(w.dims, w.h, w.speed_torch(dev), w.sources) for w in ws]
    stream = torch.cuda.current_stream()
    B = eik.Batch(grids, "fp32", stream=stream)
    try:
        t0 = time.perf_counter()
        if tune_rounds >= 0:
            tiles, ctas, tune_ms = B.autotune(rounds=tune_rounds)
        else:                                        # untuned: the default tiles
            tiles, ctas, tune_ms = [(8, 2.0 * w.h) for w in ws], 0, None
        tune_s = time.perf_counter() - t0

        def timed(tl, ctas_per_sm):
            for _ in range(warmup):
                B.solve(tl, ctas_per_sm=ctas_per_sm)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            lat, ms, restarts = [], [], 0
            for a, b in ev:
                a.record(stream)
                B.solve_async(tl, ctas_per_sm=ctas_per_sm)
                b.record(stream)
                st = B.wait()
                restarts = st["restarts"]
                lat += [r["done_ms"] for r in B.info()]
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in ev]
            lat = np.array(lat)
            return {"solves_per_s": 64 * steps / (sum(ms) * 1e-3), "ms_per_batch": sum(ms) / steps,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "mpoints_per_s": sum(w.npoints for w in ws) * steps / (sum(ms) * 1e-3) / 1e6,
                    "restarts": restarts}

        tuned = timed(None, 0)
        default = timed([(8, 2.0 * w.h) for w in ws], 0)
        info = B.info()
    finally:
        B.close()
    e8 = sum(1 for t in tiles if t[0] == 8)
    sh = sorted({round(t[1] / w.h, 3) for t, w in zip(tiles, ws)})
    return {"grids": 64, "points": int(sum(w.npoints for w in ws)), "autotuned": tuned,
            "default_8_2h": default, "tuned_over_default_ms": tuned["ms_per_batch"] / default["ms_per_batch"],
            "tiles": {"ctas_per_sm": ctas, "blocks_8": e8, "blocks_16": 64 - e8,
                      "stride_h": sh if len(sh) <= 4 else [sh[0], sh[-1]],
                      "tune_seconds": tune_s, "tune_best_ms": tune_ms},
            "latency": "per grid: device time from the start of the launch to the end of its last restart"}


def run_batch(args):
    """--workload batch: the 64-grid batched launch alone (one line; solves/s)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1811_00009_gb300 as eik
    import synth
    rounds = -1 if args.no_tune else args.tune_rounds
    with ClockSampler(0) as clk:
        b = batch_bench(eik, synth, args.steps, args.warmup, rounds, dev)
    peak, peak_kind = measured_peaks()
    tuned = b["autotuned"]
    achieved = ALGO_BYTES_PER_POINT["fp32"] * b["points"] / (tuned["ms_per_batch"] * 1e-3) / 1e9
    line = {"metric": "batched solves/s (64 grids, edges 32-192, FP32)", "value": tuned["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tuned["ms_per_batch"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 grids, per-axis edges from {32,48,...,192}, 1-4 random sources, sines / "
                                   "layers / GRF speeds, one persistent launch",
                       "l2": "working set above L2 (about 0.7 GB of h/F and psi copies), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_batch_loop", "peak_kind": peak_kind},
            "gpu_launches": 3 * args.steps, "clocks": clk.summary(), "batch": b}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = setup_dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    __graft_entry__.build()
    import paper_1811_00009_gb300 as eik
    import synth

    n = args.n
    w = rank_workload(n, rank)                          # independent instance per rank
    prec = args.precision
    Fd = w.speed_torch(dev)
    if prec == "fp64":
        Fd = Fd.double()

    # CPU baseline first (rank 0, N = 1), before the timed GPU work: the single-heap oracle on one core on a
    # 160^3 sample of the family, and the oracle's block solver on every host core on the benchmark's own
    # workload (the same F), whose result also gives the element-wise error of the timed solve at full size
    cpu = None
    full_ref = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        w_s, F_s, psi_s, dt = cpu_oracle_sample(args.cpu_n)
        cpu = {"value": w_s.npoints / dt / 1e6, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
               "sample": f"one full solve of the C4 family at {args.cpu_n}^3 (same F recipe, h=1/{args.cpu_n - 1}, "
                         f"centre source) by the single-heap FP64 fast marching oracle, one thread, {dt:.1f} s"}
        if not args.no_cpu_block:
            cpu["block_solver"], full_ref = cpu_block_sample(w, Fd.double().cpu().numpy())
    ctx = eik.eik_create(w.dims, w.h, Fd, prec)
    eik.eik_add_sources(ctx, w.sources)
    stride = args.stride_h * w.h
    kw = {"window": args.window} if args.window else {}
    if args.schedule == "learned":
        from paper_1811_00009_gb300.train_schedule import load_weights
        weights, _ = load_weights()
        eik.eik_set_schedule(ctx, weights)
        kw["schedule"] = eik.EIK_SCHED_LEARNED

    for _ in range(args.warmup):
        st = eik.eik_solve_ex(ctx, stride, **kw)

    stream = torch.cuda.current_stream()
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in pairs:                   # torch creates the CUDA event on first record; the library re-records it
        a.record(stream)
        b.record(stream)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stats = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_start.record(stream)
        for i in range(args.steps):
            eik.eik_solve_async(ctx, stride, loop_events=pairs[i], **kw)
            stats.append(eik.eik_wait(ctx))
        t_end.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)
    loop_ms = [a.elapsed_time(b) for a, b in pairs]
    value = job_rate(w.npoints, args.steps, ws, elapsed_ms * 1e-3)

    # the same workload with the fixed stride (the method without the schedule network)
    sched_cmp = None
    if args.schedule == "learned":
        # the same workload under each fixed stride of the action table's 8^3 range around the optimum
        kf = {k: v for k, v in kw.items() if k != "schedule"}
        fixed = {}
        for sh in (1.5, 2.0, 2.5, 3.0):
            fixed[f"{sh:g}h"] = min(eik.eik_solve_ex(ctx, sh * w.h, **kf)["device_ms"] for _ in range(2))
        ln = min(s_["device_ms"] for s_ in stats)
        best = min(fixed, key=fixed.get)
        sched_cmp = {"learned_device_ms": ln, "fixed_device_ms": fixed, "best_fixed": best,
                     "learned_over_best_fixed": ln / fixed[best], "learned_over_fixed_2h": ln / fixed["2h"],
                     "learned_restarts": stats[-1]["restarts"]}

    # roofline of the dominant kernel (the restart loop), algorithmic bytes per launch
    peak, peak_kind = measured_peaks()
    algo_bytes = ALGO_BYTES_PER_POINT[prec] * w.npoints
    loop_avg_ms = sum(loop_ms) / len(loop_ms)
    achieved = algo_bytes / (loop_avg_ms * 1e-3) / 1e9
    traffic = NCU_TRAFFIC_PER_NODE.get(prec)
    traffic_b = traffic * w.npoints if traffic else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_b,
            "traffic_source": ("ncu DRAM capture of the 512^3 launch of the same family (fixed 2h), per node x nodes"
                               if traffic else None),
            "dram_gbs": traffic_b / (loop_avg_ms * 1e-3) / 1e9 if traffic_b else None,
            "dram_frac": traffic_b / (loop_avg_ms * 1e-3) / 1e9 / peak if traffic_b else None,
            "kernel": "k_restart_loop", "peak_kind": peak_kind,
            "algo_bytes_per_launch": algo_bytes, "launch_ms": loop_avg_ms}

    # end to end through the public API with host buffers (pinned): every step uploads its F, solves and
    # reads psi back.  Two contexts, each on its own stream, take the steps in turn, so that one's host
    # copies (copy engines) overlap the other's solve (eik_set_speed_async / eik_result_async).
    e2e = None
    if not args.no_e2e:
        Fh = torch.empty(Fd.shape, dtype=Fd.dtype, pin_memory=True)
        Fh.copy_(Fd)
        outs = [torch.empty(Fd.shape, dtype=Fd.dtype, pin_memory=True) for _ in range(2)]
        streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
        ctx2 = eik.eik_create(w.dims, w.h, Fd, prec, stream=streams[1])
        eik.eik_add_sources(ctx2, w.sources)
        ctx1 = eik.eik_create(w.dims, w.h, Fd, prec, stream=streams[0])
        eik.eik_add_sources(ctx1, w.sources)
        if args.schedule == "learned":
            eik.eik_set_schedule(ctx1, weights)
            eik.eik_set_schedule(ctx2, weights)
        ctxs = [ctx1, ctx2]
        torch.cuda.synchronize()

        def pipeline(steps, marks):
            eik.eik_set_speed_async(ctxs[0], Fh.numpy(), prec)
            eik.eik_solve_async(ctxs[0], stride, **kw)
            for i in range(steps):
                cur, nxt = ctxs[i % 2], ctxs[(i + 1) % 2]
                if i + 1 < steps:
                    eik.eik_set_speed_async(nxt, Fh.numpy(), prec)
                eik.eik_wait(cur)
                marks.append(time.perf_counter())
                eik.eik_result_async(cur, outs[i % 2].numpy())
                if i + 1 < steps:
                    eik.eik_solve_async(nxt, stride, **kw)
            for c in ctxs:
                eik.eik_sync(c)

        pipeline(2, [])
        marks = []
        t0 = time.perf_counter()
        pipeline(args.e2e_steps, marks)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e_s = max_over_ranks(t1 - t0, dev)
        gaps = np.diff(np.array(marks)) * 1e3
        for c in ctxs:
            eik.eik_destroy(c)
        nb = Fd.element_size() * w.npoints
        # the copy engines alone: one plain pinned upload and download of the same bytes
        cps = {}
        for name, dst, src in (("h2d", Fd, Fh), ("d2h", outs[0], Fd)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            cps[name] = nb / (a.elapsed_time(b) * 1e-3) / 1e9
        e2e = {"value": job_rate(w.npoints, args.e2e_steps, ws, e2e_s), "unit": "Mpoints/s",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "steps": args.e2e_steps,
               "pipeline": "two contexts on two streams: host copies of one overlap the other's solve",
               "first_solve_ms": (marks[0] - t0) * 1e3 if marks else None,
               "step_ms_median": float(np.median(gaps)) if len(gaps) else None,
               "step_ms": [round(float(g), 1) for g in gaps],
               "h2d_gbs": cps["h2d"], "d2h_gbs": cps["d2h"],
               "last_copy_ms": (t1 - marks[-1]) * 1e3 if marks else None}

    # accuracy of this run's path against the FP64 oracle: the timed solve itself, every node, against the
    # block oracle at full size; and the same path on the single-heap oracle's 160^3 sample
    err = None
    if full_ref is not None:
        o = torch.empty_like(Fd)
        eik.eik_result(ctx, o)
        torch.cuda.synchronize()
        e_full = max_abs_error(o.cpu().numpy(), full_ref)
        top = float(np.max(full_ref[np.isfinite(full_ref)]))
        del o
        err = {"max_abs_over_max_psi": e_full / top, "grid": [n, n, n], "nodes": "every node",
               "oracle": "block solver (Alg. 6, FP64, OpenMP), pinned to the single-heap oracle",
               "tolerance": 1e-5 if prec == "fp32" else None}
        full_ref = None
    if cpu is not None:
        Fs = torch.from_numpy(F_s.astype(np.float32 if prec == "fp32" else np.float64)).to(dev)
        c2 = eik.eik_create(w_s.dims, w_s.h, Fs, prec)
        eik.eik_add_sources(c2, w_s.sources)
        if args.schedule == "learned":
            eik.eik_set_schedule(c2, weights)
        eik.eik_solve_ex(c2, args.stride_h * w_s.h, **kw)
        o = torch.empty_like(Fs)
        eik.eik_result(c2, o)
        eik.eik_destroy(c2)
        p = o.double().cpu().numpy()
        fin = np.isfinite(psi_s)
        small = {"max_abs_over_max_psi": float(np.max(np.abs(p[fin] - psi_s[fin])) / psi_s[fin].max()),
                 "grid": [args.cpu_n] * 3, "oracle": "single-heap FMM (Algs. 1-4, FP64)",
                 "tolerance": 1e-5 if prec == "fp32" else None}
        if err is None:
            err = small
        else:
            err["sample_single_heap"] = small

    eik.eik_destroy(ctx)
    # the FP64 production variant of the whole pipeline on the same workload (one warm-up, one timed solve)
    fp64 = None
    if not args.no_fp64 and prec == "fp32" and rank == 0:
        F64 = Fd.double()
        c64 = eik.eik_create(w.dims, w.h, F64, "fp64")
        eik.eik_add_sources(c64, w.sources)
        eik.eik_solve_ex(c64, 2.0 * w.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)                # torch creates the CUDA events on first record; the library re-records them
        e1.record(stream)
        st64 = eik.eik_solve_ex(c64, 2.0 * w.h, loop_events=(e0, e1))
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        eik.eik_destroy(c64)
        del F64
        fp64 = {"mpoints_per_s": w.npoints / (ms64 * 1e-3) / 1e6, "loop_ms": ms64, "restarts": st64["restarts"],
                "config": "FP64 storage and arithmetic, fixed stride 2h, 8^3 blocks, same workload"}
    # 32^3 blocks (one CTA of 1024 threads per block, FP32, fixed stride) on the same workload, beside the
    # 8^3 solve: one warm-up, one timed solve, and the result against the 8^3 solve's bit for bit
    b32 = None
    if not args.no_block32 and prec == "fp32" and rank == 0:
        c32 = eik.eik_create(w.dims, w.h, Fd, "fp32")
        eik.eik_add_sources(c32, w.sources)
        eik.eik_solve_ex(c32, 1.5 * w.h, block_dim=8)
        o8 = torch.empty_like(Fd)
        eik.eik_result(c32, o8)
        kw32 = dict(block_dim=32, window=4.0)
        eik.eik_solve_ex(c32, 4.0 * w.h, **kw32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e1.record(stream)
        st32 = eik.eik_solve_ex(c32, 4.0 * w.h, loop_events=(e0, e1), **kw32)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1)
        o32 = torch.empty_like(Fd)
        eik.eik_result(c32, o32)
        same = bool(torch.equal(o8, o32))
        eik.eik_destroy(c32)
        del o8, o32
        b32 = {"mpoints_per_s": w.npoints / (ms32 * 1e-3) / 1e6, "loop_ms": ms32, "restarts": st32["restarts"],
               "accepted_per_node": st32["accepted"] / w.npoints, "solves_per_node": st32["solves"] / w.npoints,
               "bitwise_equal_to_8": same,
               "config": "32^3 blocks, one CTA of 1024 threads each, fixed stride 4h, window 4, same workload"}
    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_bench(eik, synth, args.batch_steps, 3, args.tune_rounds, dev)
    clocks = clk.summary()
    # the bound the kernel actually meets: instruction issue (warp instructions per launch from the ncu
    # capture over the launch time, against every scheduler issuing every cycle at the sampled SM clock)
    inst = NCU_INST_PER_NODE.get(prec)
    if inst is not None and roof is not None:
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ach = inst * w.npoints / (roof["launch_ms"] * 1e-3)
        pk = sms * ISSUE_PER_SM_CYCLE * mhz * 1e6
        roof["issue"] = {"achieved": ach, "peak": pk, "unit": "warp instructions/s", "frac": ach / pk,
                         "inst_per_node": inst, "sms": sms, "sm_mhz": mhz,
                         "source": "ncu smsp__inst_executed.sum of the 512^3 launch of the same family (fixed 2h), "
                                   "per node x nodes"}
    s0 = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": (f"C4: {n}^3 node grid, h=1/{n - 1}, F=exp(g), g white noise smoothed by a Gaussian, std 0.5 corr 0.05, "
                                    f"centre source, {prec.upper()} (FP64 root fallback), "
                                    + ("learned stride/block schedule" if args.schedule == "learned" else
                                       f"fixed stride {args.stride_h:g}h, 8^3 blocks")),
                       "grid": [n, n, n], "stride_h": args.stride_h, "block": 8, "schedule": args.schedule,
                       "l2": "inputs larger than L2 (F and psi copies are GiB-sized), no flush",
                       "parallelism": "independent solve per GPU" if ws > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "schedule": sched_cmp,
            "gpu_launches": KERNELS_PER_SOLVE * args.steps, "clocks": clocks,
            "solve": {"restarts": s0["restarts"], "marches": s0["marches"], "accepted": s0["accepted"],
                      "solves": s0["solves"], "updates": s0["updates"], "fallbacks": s0["fallbacks"],
                      "rounds": s0["rounds"], "loop_ms": loop_avg_ms},
            "error_vs_oracle": err, "fp64_solve": fp64, "block32_solve": b32, "batch": batch}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1024, help="grid edge of the workload (default 1024)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--stride-h", type=float, default=2.0, help="fixed stride, and restart 1 of the learned schedule")
    ap.add_argument("--schedule", choices=["learned", "fixed"], default="learned")
    ap.add_argument("--window", type=float, default=0.0)
    ap.add_argument("--cpu-n", type=int, default=160)
    ap.add_argument("--no-cpu-block", action="store_true",
                    help="skip the multi-core CPU block solver on the full workload (and the full-size error)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 solve of the same workload")
    ap.add_argument("--no-block32", action="store_true", help="skip the 32^3-block solve of the same workload")
    ap.add_argument("--ref-n", type=int, default=128)
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-grid batched launch")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--tune-rounds", type=int, default=0, help="autotuner rounds (0: until one candidate is left)")
    ap.add_argument("--no-tune", action="store_true", help="batched launch with the default tiles (8^3, 2h)")
    ap.add_argument("--workload", choices=["c4", "batch"], default="c4",
                    help="c4: the 1024^3 solve (default); batch: the 64-grid batched launch alone")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
