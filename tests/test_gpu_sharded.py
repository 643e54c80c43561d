"""One grid sharded in z across GPUs (eik_slab_* of the C ABI), run as slabs in turn on one GPU.

Each slab is a context over its brick planes plus one ghost plane beyond each cut; the restarts run in
lockstep, the face layers at the cuts are exported, handed over and merged into the neighbours' ghost
planes between restarts (Alg. 5 across the cut), and the solve ends when no slab lists a brick.  The
result must equal the one-grid solve bit for bit (the update is monotone, so the order of work does not
change the fixed point) and the oracle within the parity bar.  Kernels of different slabs never wait on
one another: each launch runs one restart and ends by itself.
"""
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


def one_grid(eik, w, F, stride, precision):
    import torch
    ctx = eik.eik_create(w.dims, w.h, F, precision)
    try:
        eik.eik_add_sources(ctx, w.sources)
        st = eik.eik_solve(ctx, stride, 8)
        out = torch.empty_like(F)
        eik.eik_result(ctx, out)
        torch.cuda.synchronize()
        return out.cpu().numpy(), st
    finally:
        eik.eik_destroy(ctx)


@pytest.mark.parametrize("cfg,n,nranks,precision", [("C4", 80, 2, "fp32"), ("C3", 96, 3, "fp32"),
                                                    ("C2", 61, 4, "fp32"), ("C4", 48, 2, "fp64")])
def test_sharded_equals_one_grid_and_oracle(eik, orc, cfg, n, nranks, precision):
    import torch
    from paper_1811_00009_gb300.sharded import solve_sharded_local
    w = synth.workload(cfg, n)
    F = synth.round_to(w.speed(), precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Fd = torch.from_numpy(F).to("cuda", dt)
    ref_gpu, st = one_grid(eik, w, Fd, 2 * w.h, precision)
    psi, k = solve_sharded_local(eik, w.dims, w.h, Fd, w.sources, nranks, 2 * w.h, precision)
    got = psi.cpu().numpy()
    assert np.array_equal(got, ref_gpu)
    ref = orc.fmm(F, w.h, w.sources)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    if precision == "fp32":
        assert np.max(np.abs(got[fin] - ref[fin])) <= 1e-5 * ref[fin].max()
    else:
        pos = fin & (ref > 0)
        assert np.max(np.abs(got[pos] - ref[pos]) / ref[pos]) <= 1e-12
    assert k >= st["restarts"] - 1


def test_sharded_sources_on_and_across_the_cut(eik, orc):
    """Sources in a ghost plane, on a cut between slabs, and none at all in some slabs."""
    import torch
    from paper_1811_00009_gb300.sharded import solve_sharded_local
    n = 40
    dims = (n, n, n)
    h = synth.grid_h(dims)
    F = synth.round_to(0.6 + synth.uniform(31, 1, n ** 3).reshape(n, n, n), "fp32")
    src = np.array([[0.3, 0.4, 16 * h], [0.7, 0.2, 15.5 * h], [0.1, 0.9, 23.9 * h]])
    Fd = torch.from_numpy(F).to("cuda", torch.float32)
    ctx = eik.eik_create(dims, h, Fd, "fp32")
    try:
        eik.eik_add_sources(ctx, src)
        eik.eik_solve(ctx, 2 * h, 8)
        ref_gpu = torch.empty_like(Fd)
        eik.eik_result(ctx, ref_gpu)
    finally:
        eik.eik_destroy(ctx)
    for nranks in (2, 5):
        psi, _ = solve_sharded_local(eik, dims, h, Fd, src, nranks, 2 * h)
        assert np.array_equal(psi.cpu().numpy(), ref_gpu.cpu().numpy()), nranks
    ref = orc.fmm(F, h, src)
    fin = np.isfinite(ref)
    assert np.max(np.abs(ref_gpu.cpu().numpy()[fin] - ref[fin])) <= 1e-5 * ref[fin].max()


def test_slab_calls_out_of_order(eik):
    import torch
    F = torch.ones((24, 16, 16), dtype=torch.float32, device="cuda")
    ctx = eik.eik_create((16, 16, 24), 0.1, F, "fp32")
    try:
        with pytest.raises(eik.EikError) as e:
            eik.eik_slab_begin(ctx, 0.2)
        assert e.value.status == eik.EIK_ESTATE
        with pytest.raises(eik.EikError) as e:
            eik.eik_slab_set(ctx, 2, 1, 0, 24)
        assert e.value.status == eik.EIK_EINVAL
        with pytest.raises(eik.EikError) as e:
            eik.eik_slab_set(ctx, 0, 2, 4, 24)            # the offset must be whole brick planes
        assert e.value.status == eik.EIK_EINVAL
        eik.eik_slab_set(ctx, 0, 2, 0, 24)
        with pytest.raises(eik.EikError) as e:
            eik.eik_slab_restart(ctx)
        assert e.value.status == eik.EIK_ESTATE
        eik.eik_slab_begin(ctx, 0.2)
        buf = torch.empty(eik.eik_slab_face_bytes(ctx), dtype=torch.uint8, device="cuda")
        with pytest.raises(eik.EikError) as e:
            eik.eik_slab_import(ctx, 0, buf)              # no ghost plane below plane 0
        assert e.value.status == eik.EIK_EINVAL
        eik.eik_slab_restart(ctx)
        eik.eik_slab_end(ctx)
    finally:
        eik.eik_destroy(ctx)


def _rank_main(rank, world, port, n, q):
    import os
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1811_00009_gb300 as E
        from paper_1811_00009_gb300.sharded import DistTransport, Slab, run_rank, slab_parts
        w = synth.workload("C4", n)
        F = torch.from_numpy(synth.round_to(w.speed(), "fp32")).to("cuda", torch.float32)
        part = slab_parts(n, world)[rank]
        slab = Slab(E, w.dims, w.h, F[part.zlo:part.zhi].contiguous(), part, w.sources)
        try:
            k = run_rank(slab, DistTransport(rank, world, staging=True), 2 * w.h)
            q.put((rank, slab.result_own().cpu().numpy(), k))
        finally:
            slab.close()
    finally:
        dist.destroy_process_group()


def test_sharded_ranks_as_processes(eik):
    """Two processes, one slab each (on this one GPU), faces exchanged by torch.distributed through host
    memory: the lockstep of sharded.run_rank with real slabs; the result equals the one-grid solve bit for
    bit.  (The slab launches never wait on one another: each restart's launch ends by itself, and the two
    processes' launches share the GPU in turn.)"""
    import socket
    import torch
    import torch.multiprocessing as mp
    n, world = 64, 2
    w = synth.workload("C4", n)
    F = torch.from_numpy(synth.round_to(w.speed(), "fp32")).to("cuda", torch.float32)
    ref, st = one_grid(eik, w, F, 2 * w.h, "fp32")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = np.concatenate([r[1] for r in res], axis=0)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
    assert res[0][2] == res[1][2] and res[0][2] >= st["restarts"] - 1
