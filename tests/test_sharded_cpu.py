"""Host side of the sharded solve on the CPU: the z-slab partition, the sources each slab keeps, and the
lockstep exchange protocol over torch.distributed with gloo ranks (world sizes 2 and 3).

The protocol test drives `sharded.run_rank` with a stand-in slab that has the same interface as the GPU one
(restart / export / import / end and a pending count) but solves a 1-D distance problem on the host: each
restart relaxes its own cells once from their neighbours, the boundary cells travel to the neighbouring
rank, and a lowered ghost cell counts as pending work.  It checks that the faces go to the right ranks and
that the loop ends exactly when no rank has work left, with the serial answer.  The GPU slabs themselves are
tested against the one-grid solve in tests/test_gpu_sharded.py.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1811_00009_gb300.sharded import BRICK, DistTransport, local_sources, run_rank, slab_parts


@pytest.mark.parametrize("nz", [8, 9, 40, 61, 200, 1024])
def test_slab_parts_cover_the_grid(nz):
    BZ = (nz + BRICK - 1) // BRICK
    for nr in range(1, min(9, BZ) + 1):
        parts = slab_parts(nz, nr)
        assert parts[0].z0 == 0 and parts[-1].z1 == nz and parts[0].bz0 == 0 and parts[-1].bz1 == BZ
        for a, b in zip(parts, parts[1:]):
            assert a.z1 == b.z0 and a.bz1 == b.bz0
        sizes = [p.bz1 - p.bz0 for p in parts]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
        for p in parts:
            assert p.z0 == BRICK * p.bz0 and p.z0 % BRICK == 0
            assert p.zlo == (p.z0 - BRICK if p.has_lower else 0)
            assert p.zhi == (min(nz, p.z1 + BRICK) if p.has_upper else nz)
            assert p.zlo + BRICK * p.own_bz0 == p.z0 and p.own_bz1 - p.own_bz0 == p.bz1 - p.bz0
            assert (p.own_bz0 == 1) == p.has_lower
    with pytest.raises(ValueError):
        slab_parts(nz, BZ + 1)


def test_local_sources_keep_what_touches_the_slab():
    h = 0.1
    parts = slab_parts(40, 2)                       # own z: [0, 16) and [16, 40); held: [0, 24) and [8, 40)
    src = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, 1.55], [0.0, 0.0, 2.0], [0.0, 0.0, 3.9]])
    s0 = local_sources(src, parts[0], h)
    s1 = local_sources(src, parts[1], h)
    assert np.array_equal(s0[:, 2], [0.5, 1.55, 2.0])  # 3.9 lies beyond rank 0's ghost plane
    assert np.array_equal(s1[:, 2], [1.55, 2.0, 3.9])  # 0.5 lies below rank 1's ghost plane; whole-grid z kept


class LineSlab:
    """A stand-in slab: cells [z0, z1) of a 1-D distance problem (unit steps, sources at given cells)."""

    def __init__(self, part, n, sources):
        self.part = part
        self.own = np.full(part.z1 - part.z0, np.inf)
        for s in sources:
            if part.z0 <= s < part.z1:
                self.own[s - part.z0] = 0.0
        self.below = np.inf                            # ghost cells beyond the cuts
        self.above = np.inf
        self.log = []

    def begin(self, stride):
        self.log.append(("begin", stride))

    def restart(self):
        u = np.concatenate([[self.below], self.own, [self.above]])
        new = np.minimum(u[1:-1], np.minimum(u[:-2], u[2:]) + 1.0)
        changed = int(np.sum(new < self.own))
        self.own = new
        self.last_changed = changed
        return changed

    def export(self, side):
        return torch.tensor([self.own[0] if side == 0 else self.own[-1]], dtype=torch.float64)

    def import_(self, side, buf):
        v = float(buf[0])
        if side == 0 and v < self.below:
            self.below = v
            self.last_changed += 1
        if side == 1 and v < self.above:
            self.above = v
            self.last_changed += 1
        return self.last_changed

    def end(self):
        self.log.append(("end",))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, sources, out, staging=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = slab_parts(n, world)[rank]
        slab = LineSlab(part, n, sources)
        k = run_rank(slab, DistTransport(rank, world, staging=staging), stride=1.0)
        out.put((rank, part.z0, slab.own.tolist(), k, slab.log))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,sources,staging", [(2, 40, [3], False), (3, 61, [0, 50], False),
                                                     (2, 17, [16], False), (3, 61, [0, 50], True)])
def test_lockstep_exchange_over_gloo(world, n, sources, staging):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, sources, q, staging)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([np.array(r[2]) for r in res])
    want = np.min(np.abs(np.arange(n)[:, None] - np.array(sources)[None, :]), axis=1).astype(float)
    assert np.array_equal(got, want)
    ks = {r[3] for r in res}
    assert len(ks) == 1                               # every rank ran the same restarts
    for r in res:
        assert r[4][0] == ("begin", 1.0) and r[4][-1] == ("end",)
