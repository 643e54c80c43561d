"""Seeded synthetic inputs for the Eikonal solvers: speed functions, point sources, workloads.

This module is shared by the oracle side and the CUDA side and holds none of the
method's arithmetic: it only produces the speed function F on a node-centred
uniform grid and the physical coordinates of point sources (the data of the
boundary value problem |grad psi| F = 1, psi = 0 on Gamma, Sec. 1 Eq. (1.1)).

Grid convention (one reading of Sec. 2.1 / Sec. 3.1): node
(i, j, k) sits at x = (i*h, j*h, k*h); arrays have shape (nz, ny, nx) with x
fastest; the unit cube has h = 1/(n-1).

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
value for (seed, stream, counter) is the SplitMix64 output function applied to
key + (counter+1)*gamma.  It is written with numpy uint64 arithmetic, so every
machine (x86 here, aarch64 on the GPU host) draws the same numbers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "splitmix64", "uniform", "normal", "grid_h", "node_coords",
    "speed_const", "speed_sines", "speed_layers", "speed_grf", "grf_field", "speed_grf_torch",
    "speed_paper_case", "speed_paper_case_slab", "round_to", "Workload", "workload", "batch_workloads",
    "random_sources",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n SplitMix64 outputs for counters start..start+n-1 of (seed, stream)."""
    with np.errstate(over="ignore"):
        key = np.uint64((seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF)
        z = key + (np.arange(start, start + n, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform on [0, 1) (top 53 bits of each SplitMix64 output)."""
    return (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform of paired uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]                      # (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:n]


def grid_h(dims: Sequence[int]) -> float:
    """Spacing of a node-centred grid whose longest axis spans [0, 1]."""
    n = max(int(d) for d in dims)
    return 1.0 / (n - 1) if n > 1 else 1.0


def node_coords(n: int, h: float) -> np.ndarray:
    return np.arange(n, dtype=np.float64) * h


def speed_const(dims: Sequence[int], c: float = 1.0) -> np.ndarray:
    nx, ny, nz = (int(d) for d in dims)
    return np.full((nz, ny, nx), float(c))


def speed_sines(dims: Sequence[int], h: float, amp: float = 0.5, freq: float = 1.0) -> np.ndarray:
    """F = 1 + amp*sin(2 pi f x) sin(2 pi f y) sin(2 pi f z) on the node grid."""
    nx, ny, nz = (int(d) for d in dims)
    sx = np.sin(2.0 * math.pi * freq * node_coords(nx, h))
    sy = np.sin(2.0 * math.pi * freq * node_coords(ny, h))
    sz = np.sin(2.0 * math.pi * freq * node_coords(nz, h))
    return 1.0 + amp * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def speed_layers(dims: Sequence[int], seed: int, nlayers: int = 16,
                 lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Piecewise-constant F in nlayers z-slabs; layer of node k is floor(nlayers*k/nz)."""
    nx, ny, nz = (int(d) for d in dims)
    vals = lo + (hi - lo) * uniform(seed, 3, nlayers)
    layer = (nlayers * np.arange(nz)) // nz
    return np.broadcast_to(vals[layer][:, None, None], (nz, ny, nx)).copy()


def _gauss_multiplier(n: int, h: float, s: float, real: bool = False) -> np.ndarray:
    """Fourier multiplier of a periodic smoothing by a Gaussian of std s (physical units) along an axis of
    n nodes with spacing h: exp(-2 pi^2 s^2 f^2) at the FFT frequencies f (rfft frequencies if real)."""
    f = np.fft.rfftfreq(n, d=h) if real else np.fft.fftfreq(n, d=h)
    return np.exp(-2.0 * (math.pi * s * f) ** 2)


def grf_field(dims: Sequence[int], h: float, seed: int, std: float = 0.5, ell: float = 0.05) -> np.ndarray:
    """g: white N(0, 1) noise from this module's generator on the node grid (stream 5), convolved
    periodically with a separable Gaussian of std ell/sqrt(2) per axis -- so that its covariance is
    proportional to exp(-|r|^2 / (2 ell^2)), a Gaussian of the std of two such kernels -- then set to mean 0
    and standard deviation `std` over the realisation.  Shape (nz, ny, nx)."""
    nx, ny, nz = (int(d) for d in dims)
    w = normal(seed, 5, nx * ny * nz).reshape(nz, ny, nx)
    s = ell / math.sqrt(2.0)
    W = np.fft.rfftn(w)
    W *= (_gauss_multiplier(nz, h, s)[:, None, None] * _gauss_multiplier(ny, h, s)[None, :, None]
          * _gauss_multiplier(nx, h, s, real=True)[None, None, :])
    g = np.fft.irfftn(W, s=(nz, ny, nx), axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g *= std / sd
    return g


def speed_grf(dims: Sequence[int], h: float, seed: int, std: float = 0.5, ell: float = 0.05) -> np.ndarray:
    """F = exp(g), g the Gaussian random field of grf_field (std `std`, correlation length `ell`)."""
    return np.exp(grf_field(dims, h, seed, std, ell))


# ---- the same generators with torch (on a GPU for grids too large for the host's numpy) ----

def _i64(c: int) -> int:
    """An unsigned 64-bit constant as the signed int64 with the same bits."""
    c &= 0xFFFFFFFFFFFFFFFF
    return c - (1 << 64) if c >= (1 << 63) else c


def splitmix64_torch(seed: int, stream: int, n: int, start: int, device):
    """splitmix64's outputs as int64 tensors with the same bits (integer arithmetic wraps modulo 2^64;
    the right shifts are made logical by masking)."""
    import torch
    key = _i64(seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D)
    z = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    z = z * _i64(0x9E3779B97F4A7C15) + key
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * _i64(0x94D049BB133111EB)
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def normal_torch(seed: int, stream: int, n: int, device, chunk: int = 1 << 25):
    """normal(seed, stream, n) computed with torch in float64 on `device` (the same uniforms, bit for bit;
    the Box-Muller transform agrees to rounding)."""
    import torch
    m = (n + 1) // 2
    out = torch.empty(2 * m, dtype=torch.float64, device=device)
    for p0 in range(0, m, chunk):
        p1 = min(m, p0 + chunk)
        z = splitmix64_torch(seed, stream, 2 * (p1 - p0), 2 * p0, device)
        u = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        del z
        u1 = 1.0 - u[0::2]
        u2 = u[1::2]
        rad = torch.sqrt(-2.0 * torch.log(u1))
        out[2 * p0:2 * p1:2] = rad * torch.cos(2.0 * math.pi * u2)
        out[2 * p0 + 1:2 * p1:2] = rad * torch.sin(2.0 * math.pi * u2)
    return out[:n]


def speed_grf_torch(dims: Sequence[int], h: float, seed: int, device, std: float = 0.5, ell: float = 0.05,
                    dtype=None):
    """speed_grf computed with torch on `device` (float64 arithmetic, the result in `dtype`, float32 by
    default).  Values agree with speed_grf to rounding; tests that compare against the oracle generate F
    with one of the two and hand the same values to both sides."""
    import torch
    nx, ny, nz = (int(d) for d in dims)
    s = ell / math.sqrt(2.0)
    w = normal_torch(seed, 5, nx * ny * nz, device).reshape(nz, ny, nx)
    W = torch.fft.rfftn(w)
    del w
    mult = lambda n, real=False: torch.from_numpy(_gauss_multiplier(n, h, s, real)).to(device)
    W *= mult(nz)[:, None, None] * mult(ny)[None, :, None] * mult(nx, True)[None, None, :]
    g = torch.fft.irfftn(W, s=(nz, ny, nx))
    del W
    g -= g.mean()
    sd = g.std(unbiased=False)
    if float(sd) > 0:
        g *= std / sd
    out = torch.exp(g).to(torch.float32 if dtype is None else dtype)
    del g
    if out.is_cuda:
        torch.cuda.empty_cache()
    return out


def speed_paper_case(case: int, n: int) -> Tuple[np.ndarray, float, np.ndarray]:
    """The paper's Cases 1-4 (Sec. 3.1, Eqs. (3.1)-(3.4)) on its cell-centred grid.

    Domain [-0.5, 0.5]^3 with n cells per axis; the grid point of cell i is at
    -0.5 + (i + 0.5)/n.  Returns (F, h, source) with the source at the centre,
    expressed in this module's node convention (origin at grid point 0).
    """
    h = 1.0 / n
    F = speed_paper_case_slab(case, n, 0, n)
    src = np.array([[0.5 - 0.5 * h] * 3])    # the centre, measured from grid point 0
    return F, h, src


def speed_paper_case_slab(case: int, n: int, z0: int, z1: int) -> np.ndarray:
    """Planes z0 <= k < z1 of speed_paper_case(case, n)'s F (same values), shape (z1 - z0, n, n)."""
    h = 1.0 / n
    c = -0.5 + (np.arange(n) + 0.5) * h
    X = c[None, None, :]
    Y = c[None, :, None]
    Z = c[z0:z1, None, None]
    m = z1 - z0
    if case == 1:
        F = np.ones((m, n, n))
    elif case == 2:
        F = 1.0 + 0.5 * np.sin(20 * math.pi * X) * np.sin(20 * math.pi * Y) * np.sin(20 * math.pi * Z)
    elif case == 3:
        F = 1.0 - 0.99 * np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y) * np.sin(2 * math.pi * Z)
    elif case == 4:
        F = np.ones((m, n, n))
        R = np.sqrt(X * X + Y * Y + Z * Z)
        r = np.sqrt(X * X + Y * Y) + 0.0 * Z
        w = 1.0 / 24.0
        shells = [(0.15, 0.05, -1), (0.25, 0.10, +1), (0.35, 0.10, -1), (0.45, 0.10, +1)]
        for R0, rh, side in shells:
            shell = (R > R0) & (R < R0 + w)
            hole = (r < rh) & ((Z < 0) if side < 0 else (Z > 0))
            F[shell & ~hole] = 0.0
    else:
        raise ValueError("case must be 1..4")
    return np.ascontiguousarray(np.broadcast_to(F, (m, n, n)))


def round_to(F: np.ndarray, precision: str) -> np.ndarray:
    """F rounded to the solver's storage precision and widened back to float64."""
    if precision == "fp32":
        return F.astype(np.float32).astype(np.float64)
    if precision == "fp64":
        return np.asarray(F, dtype=np.float64)
    raise ValueError(precision)


def random_sources(seed: int, stream: int, dims: Sequence[int], h: float, count: int) -> np.ndarray:
    """`count` physical points uniform in the grid's box [0,(n-1)h]^3."""
    u = uniform(seed, stream, 3 * count).reshape(count, 3)
    ext = np.array([(int(d) - 1) * h for d in dims])
    return u * ext[None, :]


@dataclass
class Workload:
    """One solve: grid, speed function, sources and solver settings."""
    name: str
    dims: Tuple[int, int, int]
    h: float
    family: str
    seed: int
    sources: np.ndarray
    precision: str = "fp32"
    block: int = 8
    strides_h: List[float] = field(default_factory=lambda: [2.0])
    note: str = ""

    @property
    def npoints(self) -> int:
        return self.dims[0] * self.dims[1] * self.dims[2]

    def speed(self) -> np.ndarray:
        if self.family == "const":
            F = speed_const(self.dims)
        elif self.family == "sines":
            F = speed_sines(self.dims, self.h)
        elif self.family == "layers":
            F = speed_layers(self.dims, self.seed)
        elif self.family == "grf":
            F = speed_grf(self.dims, self.h, self.seed)
        else:
            raise ValueError(self.family)
        return round_to(F, self.precision)

    def speed_torch(self, device):
        """F generated on `device` (large grids); same formulas as speed()."""
        import torch
        if self.family == "grf":
            dt = torch.float32 if self.precision == "fp32" else torch.float64
            return speed_grf_torch(self.dims, self.h, self.seed, device, dtype=dt)
        F = self.speed()
        dt = torch.float32 if self.precision == "fp32" else torch.float64
        return torch.from_numpy(F).to(device=device, dtype=dt)


SEED = 1811


def workload(name: str, n: Optional[int] = None) -> Workload:
    """The five named workloads; `n` overrides the edge for a reduced-size copy of the same family."""
    if name == "C1":
        n = n or 64
        h = 1.0 / (n - 1)
        return Workload("C1", (n, n, n), h, "const", SEED + 1, np.array([[0.5, 0.5, 0.5]]),
                        precision="fp64", block=16, strides_h=[2.0],
                        note="F=1, centre source, FP64")
    if name == "C2":
        n = n or 256
        h = 1.0 / (n - 1)
        return Workload("C2", (n, n, n), h, "sines", SEED + 2, np.array([[0.0, 0.0, 0.0]]),
                        precision="fp32", block=16, strides_h=[1.0, 2.0, 4.0, 8.0],
                        note="F=1+0.5 sin sin sin, corner source, FP32")
    if name == "C3":
        n = n or 512
        h = 1.0 / (n - 1)
        return Workload("C3", (n, n, n), h, "layers", SEED + 3, np.array([[0.5, 0.5, 0.1]]),
                        precision="fp32", block=16, strides_h=[1.0, 2.0, 4.0, 8.0],
                        note="16 z-layers U[0.5,2], source (0.5,0.5,0.1), FP32")
    if name == "C4":
        n = n or 1024
        h = 1.0 / (n - 1)
        return Workload("C4", (n, n, n), h, "grf", SEED + 4, np.array([[0.5, 0.5, 0.5]]),
                        precision="fp32", block=16, strides_h=[2.0],
                        note="F=exp(g), GRF std 0.5, ell 0.05, centre source, FP32")
    raise ValueError(name)


def batch_workloads(count: int = 64, seed: int = SEED + 5,
                    edges: Sequence[int] = tuple(range(32, 193, 16))) -> List[Workload]:
    """The batched workload: `count` grids with per-axis edges drawn from `edges`,
    1-4 random point sources each, F from the sines / layers / GRF families, FP32."""
    out = []
    fams = ["sines", "layers", "grf"]
    u = uniform(seed, 11, 5 * count).reshape(count, 5)
    for s in range(count):
        dims = tuple(int(edges[min(len(edges) - 1, int(u[s, a] * len(edges)))]) for a in range(3))
        h = grid_h(dims)
        fam = fams[min(2, int(u[s, 3] * 3))]
        nsrc = 1 + min(3, int(u[s, 4] * 4))
        src = random_sources(seed + s, 12, dims, h, nsrc)
        out.append(Workload(f"B{s}", dims, h, fam, seed * 1000 + s, src, precision="fp32",
                            block=8, strides_h=[2.0]))
    return out
