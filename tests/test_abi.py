"""The C ABI library loads and exports every entry point include/eik.h declares (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:eik_status|void|const\s+char\s*\*)\s*\**\s*(eik_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def eik():
    from paper_1811_00009_gb300 import build
    build.build()
    import paper_1811_00009_gb300 as E
    return E


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("eik_create", "eik_add_sources", "eik_solve", "eik_result", "eik_destroy", "eik_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(eik):
    L = eik.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_entry_points(eik):
    assert "sm_103a" in eik.eik_version()
    p = eik.eik_params_default()
    assert p.block_dim == 8 and p.window == 2.0 and p.fallback_tau == 0.125
    # the later fields too: a layout mismatch between eik.h and the binding would garble them
    assert p.max_restarts == 1 << 24 and p.switch_margin == 0.02 and p.width == 0.0 and p.wait_polls == 0
    assert C.sizeof(eik.eik_params) % 8 == 0
    bp = eik.eik_batch_params()
    eik.lib().eik_batch_params_default(C.byref(bp))
    assert bp.ctas_per_sm == 0 and bp.window == 2.0 and bp.fallback_tau == 0.125 and bp.max_restarts == 1 << 24


@pytest.mark.parametrize("dims,h", [((0, 4, 4), 0.1), ((4, 4, -1), 0.1), ((4, 4, 4), 0.0),
                                    ((4, 4, 4), float("nan")), ((4, 4, 4), float("inf")),
                                    ((2048, 2048, 1024), 0.1)])
def test_create_rejects_bad_arguments_before_touching_the_device(eik, dims, h):
    L = eik.lib()
    out = C.c_void_p()
    d = (C.c_int32 * 3)(*dims)
    F = np.ones(8, np.float32)
    st = L.eik_create(C.byref(out), d, h, C.c_void_p(F.ctypes.data), 0, 0, None)
    assert st == eik.EIK_EINVAL
    assert not out.value
    assert eik.eik_last_error(None)


def test_null_context_calls_fail_cleanly(eik):
    L = eik.lib()
    assert L.eik_solve(None, 1.0, 8, None) == eik.EIK_EINVAL
    assert L.eik_result(None, None, 0) == eik.EIK_EINVAL
    assert L.eik_add_sources(None, 0, None) == eik.EIK_EINVAL
    assert L.eik_set_speed_async(None, None, 0) == eik.EIK_EINVAL
    assert L.eik_result_async(None, None, 0) == eik.EIK_EINVAL
    assert L.eik_sync(None) == eik.EIK_EINVAL
    assert L.eik_wait(None, None) == eik.EIK_EINVAL
    L.eik_destroy(None)


@pytest.mark.parametrize("case", ["n0", "dims", "h", "nosrc", "outside"])
def test_batch_create_rejects_bad_items_before_touching_the_device(eik, case):
    L = eik.lib()
    F = np.ones(64, np.float32)
    xyz = np.zeros(3)
    items = (eik.eik_batch_item * 2)()
    for it in items:
        it.dims[:] = [4, 4, 4]
        it.h = 0.1
        it.F = C.c_void_p(F.ctypes.data)
        it.F_on_device = 0
        it.nsrc = 1
        it.xyz = xyz.ctypes.data_as(C.POINTER(C.c_double))
    n = 2
    if case == "n0":
        n = 0
    elif case == "dims":
        items[1].dims[:] = [4, 0, 4]
    elif case == "h":
        items[1].h = float("nan")
    elif case == "nosrc":
        items[1].nsrc = 0
    else:
        far = np.array([0.0, 0.0, 1.0])
        items[1].xyz = far.ctypes.data_as(C.POINTER(C.c_double))
    out = C.c_void_p()
    st = L.eik_batch_create(C.byref(out), n, items, 0, None)
    assert st == eik.EIK_EINVAL
    assert not out.value
    msg = L.eik_batch_last_error(None).decode()
    assert msg and (case == "n0" or "item 1" in msg)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_source_nodes_match_the_oracle(eik, orc, precision):
    """The fixed nodes of Alg. 1 (reading: the nodes of each source's cell, psi0 = distance / F, the
    smallest over sources, none on a barrier node unless the source sits on it), as the solve computes
    them on the host, against the oracle's: same nodes; psi0 equal up to the rounding of h/F (FP32: h and
    h/F rounded to single precision, a few 1e-7 relative)."""
    import synth
    u = synth.uniform(77, 1, 4000)
    tol = 4e-7 if precision == "fp32" else 4e-16
    dt = np.float32 if precision == "fp32" else np.float64
    for trial in range(20):
        v = u[trial * 40:(trial + 1) * 40]
        dims = (1 + int(v[0] * 20), 1 + int(v[1] * 20), 1 + int(v[2] * 20))
        h = 0.01 + v[3]
        F = (0.3 + 2.0 * synth.uniform(100 + trial, 1, dims[0] * dims[1] * dims[2])).reshape(dims[::-1])
        F[synth.uniform(200 + trial, 1, F.size).reshape(F.shape) < 0.2] = 0.0        # barrier nodes
        F = F.astype(dt)
        ns = 1 + int(v[4] * 4)
        src = []
        for s in range(ns):
            p = []
            for a in range(3):
                ext = (dims[a] - 1) * h
                w = v[5 + 3 * s + a]
                # on a node, on a cell edge or face, or inside a cell
                p.append(min(ext, round(w * (dims[a] - 1)) * h) if w < 0.3 else w * ext)
            src.append(p)
        src = np.array(src)
        idx, val = eik.eik_source_nodes(dims, h, F, src, precision)
        ridx, rval = orc.fix_nodes(F.astype(np.float64), h, src)
        o, ro = np.argsort(idx), np.argsort(ridx)
        assert np.array_equal(idx[o], ridx[ro]), trial
        if len(val):
            den = np.where(rval[ro] > 0, rval[ro], 1.0)
            assert np.all(np.abs(val[o] - rval[ro]) <= tol * den), trial
    with pytest.raises(eik.EikError, match="outside"):
        eik.eik_source_nodes((4, 4, 4), 0.1, np.ones((4, 4, 4), dt), [[0.0, 0.0, 0.5]], precision)


def test_binding_argument_counts_match_the_header(eik):
    """Every entry point the binding types (argtypes) takes as many arguments as eik.h declares."""
    text = ""
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text += open(os.path.join(ROOT, "include", hdr)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"(?:eik_status|void|const\s+char\s*\*|int32_t|int64_t)\s*\**\s*(eik_\w+)\s*\(([^)]*)\)\s*;",
                        text)
    L = eik.lib()
    checked = 0
    for name, args in protos:
        fn = getattr(L, name, None)
        types = getattr(fn, "argtypes", None) if fn is not None else None
        if not types:
            continue
        a = args.strip()
        n = 0 if a in ("", "void") else len(a.split(","))
        assert len(types) == n, (name, len(types), n)
        checked += 1
    assert checked >= 20
