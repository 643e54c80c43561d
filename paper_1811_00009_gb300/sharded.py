"""One grid sharded across GPUs: z-slabs of brick planes, one per rank.

The blocks of the method (Sec. 2.3) are the library's 8^3 bricks; a grid of
ceil(nz/8) brick planes is cut into contiguous runs of planes, one run per
rank.  Each rank holds its run plus one ghost brick plane beyond each cut, as
an ordinary context over that extended part of the grid.  The restarts of
Alg. 6 run in lockstep on every rank: march the own active bricks up to the
common bound (preset by the stride, so it needs no exchange), send the face
layer of the boundary planes to the rank across each cut, merge the received
faces into the ghost planes (Alg. 5 across the cut: a lowered face lists the
adjacent brick for the next restart), and stop when no rank has a brick
listed (an all-reduce of the counts).  The result equals one GPU's, bit for
bit: the update is monotone, so the order of work does not change the fixed
point.

Everything numeric runs in the library's kernels (eik_slab_* of the C ABI);
this module is the host side: the partition, the buffers and the exchange.
`Transport` is what moves the faces between processes: `DistTransport` uses
torch.distributed (NCCL between GPUs, or gloo); `run_local` runs every slab in
one process instead (one GPU, slabs in turn).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

BRICK = 8


@dataclass(frozen=True)
class SlabPart:
    """Rank r's part of a grid with nz node planes: own node planes [z0, z1) (own brick planes [bz0, bz1)),
    held as the extended node planes [zlo, zhi) (one ghost brick plane beyond each cut); in the local grid
    the own brick planes are [own_bz0, own_bz1)."""
    rank: int
    nranks: int
    bz0: int
    bz1: int
    z0: int
    z1: int
    zlo: int
    zhi: int
    own_bz0: int
    own_bz1: int

    @property
    def has_lower(self) -> bool:
        return self.rank > 0

    @property
    def has_upper(self) -> bool:
        return self.rank < self.nranks - 1

    @property
    def nz_local(self) -> int:
        return self.zhi - self.zlo


def slab_parts(nz: int, nranks: int) -> List[SlabPart]:
    """Contiguous runs of brick planes, as even as possible (runs differ by at most one plane)."""
    BZ = (nz + BRICK - 1) // BRICK
    if nranks < 1 or nranks > BZ:
        raise ValueError(f"need 1 <= ranks <= {BZ} brick planes")
    parts = []
    for r in range(nranks):
        bz0 = (r * BZ) // nranks
        bz1 = ((r + 1) * BZ) // nranks
        z0, z1 = BRICK * bz0, min(BRICK * bz1, nz)
        zlo = BRICK * (bz0 - 1) if r > 0 else 0
        zhi = min(BRICK * (bz1 + 1), nz) if r < nranks - 1 else nz
        own0 = (z0 - zlo) // BRICK
        parts.append(SlabPart(r, nranks, bz0, bz1, z0, z1, zlo, zhi, own0, own0 + (bz1 - bz0)))
    return parts


def local_sources(sources, part: SlabPart, h: float) -> np.ndarray:
    """The sources a part needs, in the whole grid's coordinates: those within a node of its extended planes
    (a source whose cell touches the own planes always lies inside them, the ghost plane being a whole brick
    deep).  The library keeps the whole grid's coordinates for the distances at the fixed nodes, so every part
    computes them exactly as one grid would."""
    src = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    keep = (src[:, 2] >= (part.zlo - 1) * h) & (src[:, 2] <= part.zhi * h)
    return src[keep].copy()


class Slab:
    """One rank's context: the extended part of the grid, its sources, the eik_slab_* calls."""

    def __init__(self, eik, dims: Sequence[int], h: float, F_local, part: SlabPart, sources, precision="fp32",
                 stream=None):
        import torch
        self.eik, self.part, self.h = eik, part, float(h)
        nx, ny, nz = (int(d) for d in dims)
        self.dims_local = (nx, ny, part.nz_local)
        self.ctx = eik.eik_create(self.dims_local, h, F_local, precision, stream)
        eik.eik_slab_set(self.ctx, part.own_bz0, part.own_bz1, part.zlo, nz)
        src = local_sources(sources, part, h)
        if len(src):
            eik.eik_add_sources(self.ctx, src)
        self.has_sources = len(src) > 0
        nbytes = eik.eik_slab_face_bytes(self.ctx)
        dev = F_local.device if hasattr(F_local, "device") and F_local.device.type == "cuda" else torch.device("cuda")
        self.out_faces = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.precision = precision

    def begin(self, stride: float) -> None:
        self.eik.eik_slab_begin(self.ctx, stride)

    def restart(self) -> int:
        return self.eik.eik_slab_restart(self.ctx)

    def export(self, side: int):
        self.eik.eik_slab_export(self.ctx, side, self.out_faces[side])
        return self.out_faces[side]

    def import_(self, side: int, buf) -> int:
        return self.eik.eik_slab_import(self.ctx, side, buf)

    def end(self):
        return self.eik.eik_slab_end(self.ctx)

    def result_own(self):
        """psi of the own node planes (torch tensor on the device, shape (z1 - z0, ny, nx))."""
        import torch
        nx, ny, nzl = self.dims_local
        dt = torch.float32 if self.precision == "fp32" else torch.float64
        out = torch.empty((nzl, ny, nx), dtype=dt, device=self.out_faces[0].device)
        self.eik.eik_result(self.ctx, out)
        a = self.part.z0 - self.part.zlo
        return out[a:a + (self.part.z1 - self.part.z0)]

    def close(self):
        if self.ctx:
            self.eik.eik_destroy(self.ctx)
            self.ctx = None


class Transport:
    """Moves the face records between the ranks of a sharded solve."""

    def exchange(self, down, up) -> Tuple[Optional[object], Optional[object]]:
        """Send `down` to the rank below and `up` to the rank above (None: no such rank); return what the rank
        below and the rank above sent (None where there is no rank)."""
        raise NotImplementedError

    def allreduce_sum(self, x: int) -> int:
        raise NotImplementedError


class DistTransport(Transport):
    """torch.distributed point-to-point sends to the neighbouring ranks and an all-reduce (one process per
    GPU with NCCL).  With `staging`, device buffers travel through host memory (gloo) and arrive back on
    the device they left."""

    def __init__(self, rank: int, nranks: int, device=None, staging: bool = False):
        self.rank, self.nranks, self.device, self.staging = rank, nranks, device, staging

    def exchange(self, down, up):
        import torch
        import torch.distributed as dist
        home = None
        if self.staging:
            home = (down if down is not None else up).device
            down = down.cpu() if down is not None else None
            up = up.cpu() if up is not None else None
        ops, got_below, got_above = [], None, None
        if self.rank > 0:
            got_below = torch.empty_like(down)
            ops += [dist.P2POp(dist.isend, down, self.rank - 1), dist.P2POp(dist.irecv, got_below, self.rank - 1)]
        if self.rank < self.nranks - 1:
            got_above = torch.empty_like(up)
            ops += [dist.P2POp(dist.isend, up, self.rank + 1), dist.P2POp(dist.irecv, got_above, self.rank + 1)]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if self.staging:
            got_below = got_below.to(home) if got_below is not None else None
            got_above = got_above.to(home) if got_above is not None else None
        return got_below, got_above

    def allreduce_sum(self, x: int) -> int:
        import torch
        import torch.distributed as dist
        t = torch.tensor([int(x)], dtype=torch.int64, device="cpu" if self.staging else self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return int(t.item())


def run_rank(slab, transport: Transport, stride: float, max_restarts: int = 1 << 24) -> int:
    """The lockstep restarts of one rank (every rank calls this with its own slab); returns the restart count."""
    p = slab.part
    slab.begin(stride)
    k = 0
    while True:
        k += 1
        pending = slab.restart()
        down = slab.export(0) if p.has_lower else None
        up = slab.export(1) if p.has_upper else None
        below, above = transport.exchange(down, up)
        if below is not None:
            pending = slab.import_(0, below)
        if above is not None:
            pending = slab.import_(1, above)
        if transport.allreduce_sum(pending) == 0 or k >= max_restarts:
            break
    slab.end()
    return k


def run_local(slabs: List, stride: float, max_restarts: int = 1 << 24) -> int:
    """Every slab in this process, in turn (one GPU): the same lockstep as run_rank, the faces handed over
    directly.  Kernels of different slabs never wait on one another (each launch ends by itself)."""
    for s in slabs:
        s.begin(stride)
    k = 0
    while True:
        k += 1
        pending = [s.restart() for s in slabs]
        downs = [s.export(0) if s.part.has_lower else None for s in slabs]
        ups = [s.export(1) if s.part.has_upper else None for s in slabs]
        for i, s in enumerate(slabs):
            if s.part.has_lower:
                pending[i] = s.import_(0, ups[i - 1])
            if s.part.has_upper:
                pending[i] = s.import_(1, downs[i + 1])
        if sum(pending) == 0 or k >= max_restarts:
            break
    for s in slabs:
        s.end()
    return k


def solve_sharded_local(eik, dims, h, F, sources, nranks: int, stride: float, precision="fp32"):
    """Solve one grid as `nranks` slabs on this GPU (tests and demonstration); returns psi (nz, ny, nx) on the
    device and the restart count."""
    import torch
    nx, ny, nz = (int(d) for d in dims)
    parts = slab_parts(nz, nranks)
    slabs = [Slab(eik, dims, h, F[p.zlo:p.zhi].contiguous(), p, sources, precision) for p in parts]
    try:
        k = run_local(slabs, stride)
        psi = torch.cat([s.result_own() for s in slabs], dim=0)
    finally:
        for s in slabs:
            s.close()
    return psi, k
