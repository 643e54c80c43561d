"""Builds libeik.so (the C ABI of include/eik.h) in this package directory with nvcc.

Translation units compile in parallel, for sm_103a only, without FP contraction
(-fmad=false) so that every code path evaluates the upwind root with the same
roundings.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from typing import List, Optional

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libeik.so")
SOURCES = ["eik_kernels.cu", "eik_runtime.cu", "eik_batch.cu", "eik_noalloc.cu", "eik_mlp.cu", "eik_block32.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
         "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


WEIGHTS = os.path.join(PKG, "schedule_weights.json")


def _inputs() -> List[str]:
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "eik.h"))
    files.append(WEIGHTS)
    return files


def write_weights_include(bdir: str) -> None:
    """The shipped schedule-network weights as a C array (every new context starts with them)."""
    import json
    with open(WEIGHTS) as fh:
        w = json.load(fh)["weights"]
    body = ",\n".join(", ".join(repr(float(v)) + "f" for v in w[i:i + 6]) for i in range(0, len(w), 6))
    text = ("// Written by build.py from schedule_weights.json: the shipped weights of the\n"
            "// restart-schedule network (EIK_SCHED_PARAMS floats).\n"
            f"#define EIK_SCHED_DEFAULT_COUNT {len(w)}\n"
            "static const float kSchedDefault[EIK_SCHED_DEFAULT_COUNT] = {\n" + body + "\n};\n")
    path = os.path.join(bdir, "eik_sched_weights.inc")
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as fh:
            fh.write(text)


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose_ptxas: bool = False, extra: Optional[List[str]] = None) -> str:
    if not force and not stale():
        return LIB
    cc = nvcc()
    bdir = os.path.join(PKG, "_build")
    os.makedirs(bdir, exist_ok=True)
    write_weights_include(bdir)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, "-I" + bdir, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
        if extra:
            cmd[1:1] = extra
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if out.strip():
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
