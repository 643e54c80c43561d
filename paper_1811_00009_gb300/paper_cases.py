"""The paper's experiment matrix on one GPU: Cases 1-4 of Sec. 3.1 on the cell-centred grid.

Two studies, both through the library's C ABI:

* restarts and device time (the paper's Figs. 5-6 and its block-size study, Secs. 3.4-3.6): every case,
  grid edge, stride and block edge asked for; nr = number of restarts of Alg. 6, device time of the
  restart loop (%globaltimer), and whether psi equals the 8^3 / 2h solve of the same grid bit for bit;
* accuracy (the paper's Sec. 3.2): Case 1 (F = 1, the source at the domain's centre) against the exact
  distance, max and mean absolute error at every grid edge asked for, FP32 and FP64, with the observed
  order of convergence between successive edges.

    python -m paper_1811_00009_gb300.paper_cases [--sizes 128,256,512,1024] [--out results.json]

F is built plane slab by plane slab on the host (`synth.speed_paper_case_slab`, the same values as the
tests' `synth.speed_paper_case`) and assembled on the device, so a 1024^3 grid needs no 8 GB host array.
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


def speed_on_device(case: int, n: int, dtype, slab: int = 64):
    """F of Case `case` on an n^3 cell-centred grid, in `dtype` on the current CUDA device."""
    import torch
    import synth
    F = torch.empty((n, n, n), dtype=dtype, device="cuda")
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        F[z0:z1].copy_(torch.from_numpy(synth.speed_paper_case_slab(case, n, z0, z1)).to(dtype))
    return F


def exact_case1(n: int, dtype):
    """The exact distance from the centre source at every grid point (Case 1, F = 1), on the device."""
    import torch
    h = 1.0 / n
    c = (torch.arange(n, dtype=torch.float64, device="cuda") - 0.5 * (n - 1)) * h
    return torch.sqrt(c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2).to(dtype)


def restarts_and_time(eik, cases, sizes, strides, blocks, log=print):
    import torch
    rows = []
    for n in sizes:
        h = 1.0 / n
        src = np.array([[0.5 - 0.5 * h] * 3])
        for case in cases:
            F = speed_on_device(case, n, torch.float32)
            ctx = eik.eik_create((n, n, n), h, F, "fp32")
            try:
                eik.eik_add_sources(ctx, src)
                eik.eik_solve_ex(ctx, 2 * h, block_dim=8)                       # warm-up, and the reference psi
                ref = torch.empty_like(F)
                eik.eik_result(ctx, ref)
                out = torch.empty_like(F)
                for bd in blocks:
                    if bd == 16 and n > 512:
                        continue                                                 # (16^3 blocks: 3-4x slower)
                    for sh in strides:
                        st = None
                        for _ in range(2):
                            s = eik.eik_solve_ex(ctx, sh * h, block_dim=bd)
                            if st is None or s["device_ms"] < st["device_ms"]:
                                st = s
                        eik.eik_result(ctx, out)
                        same = bool(torch.equal(out, ref))
                        row = {"case": case, "n": n, "block": bd, "stride_h": sh, "restarts": st["restarts"],
                               "device_ms": st["device_ms"], "mpoints_per_s": n ** 3 / st["device_ms"] / 1e3,
                               "same_as_8_2h": same}
                        rows.append(row)
                        log(json.dumps(row))
            finally:
                eik.eik_destroy(ctx)
            del F
            torch.cuda.empty_cache()
    return rows


def accuracy(eik, sizes, precisions=("fp32", "fp64"), log=print):
    import torch
    rows = []
    for prec in precisions:
        dt = torch.float32 if prec == "fp32" else torch.float64
        prev = None
        for n in sizes:
            h = 1.0 / n
            F = torch.ones((n, n, n), dtype=dt, device="cuda")
            ctx = eik.eik_create((n, n, n), h, F, prec)
            try:
                eik.eik_add_sources(ctx, np.array([[0.5 - 0.5 * h] * 3]))
                eik.eik_solve_ex(ctx, 2 * h)
                psi = torch.empty_like(F)
                eik.eik_result(ctx, psi)
            finally:
                eik.eik_destroy(ctx)
            d = (psi.double() - exact_case1(n, torch.float64)).abs()
            row = {"precision": prec, "n": n, "max_abs": float(d.max()), "mean_abs": float(d.mean())}
            if prev is not None:
                row["order_max"] = math.log2(prev["max_abs"] / row["max_abs"]) / math.log2(n / prev["n"])
                row["order_mean"] = math.log2(prev["mean_abs"] / row["mean_abs"]) / math.log2(n / prev["n"])
            rows.append(row)
            log(json.dumps(row))
            prev = row
            del F, psi, d
            torch.cuda.empty_cache()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="128,256,512,1024")
    ap.add_argument("--cases", default="1,2,3,4")
    ap.add_argument("--strides", default="0.5,1.5,2,2.5,3.5,inf", help="strides in units of h")
    ap.add_argument("--blocks", default="8,16,32")
    ap.add_argument("--accuracy-sizes", default="64,128,256,512,1024")
    ap.add_argument("--out", default=None, help="write every row as JSON")
    args = ap.parse_args()
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1811_00009_gb300 as eik
    torch.cuda.set_device(0)
    t0 = time.time()
    sizes = [int(v) for v in args.sizes.split(",") if v]
    cases = [int(v) for v in args.cases.split(",") if v]
    strides = [float(v) for v in args.strides.split(",") if v]
    blocks = [int(v) for v in args.blocks.split(",") if v]
    acc_sizes = [int(v) for v in args.accuracy_sizes.split(",") if v]
    res = {"restarts": restarts_and_time(eik, cases, sizes, strides, blocks),
           "accuracy": accuracy(eik, acc_sizes) if acc_sizes else []}
    print(f"done in {time.time() - t0:.1f} s", flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh)


if __name__ == "__main__":
    main()
