"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the Ohta--Kawasaki method: it only draws
random numbers and names workload parameters.  Both the CUDA path and the
CPU oracle receive the arrays it returns as plain inputs.

Generator (counter based, so any entry can be recomputed on its own):
    key      = mix64(seed + GOLDEN)
    bits(k)  = mix64(key + (k + 1) * GOLDEN)          (mod 2**64)
    U01(k)   = (bits(k) >> 11) * 2**-53               in [0, 1)
where mix64 is the SplitMix64 output function (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014):
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
Normals use the Box--Muller transform of the pair (U01(2i), U01(2i+1)):
    N(i) = sqrt(-2 ln(1 - U01(2i))) * cos(2 pi U01(2i+1)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    """SplitMix64 output function on uint64 scalars or arrays (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def bits(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """64 random bits for counters offset .. offset+count-1 of stream `seed`."""
    with np.errstate(over="ignore"):
        key = mix64(np.uint64(seed) + GOLDEN)
        k = np.arange(offset, offset + count, dtype=np.uint64) + np.uint64(1)
        return mix64(key + k * GOLDEN)


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1), 53 random bits each."""
    b = bits(seed, count, offset) >> np.uint64(11)
    return b.astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count)


def normal(seed: int, count: int) -> np.ndarray:
    u = uniform01(seed, 2 * count).reshape(count, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    return r * np.cos(2.0 * math.pi * u[:, 1])


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: grid, physical parameters and initial noise."""
    name: str
    dim: int            # 2: unit square of right triangles, 3: unit cube of Kuhn tetrahedra
    n: int              # cells per side
    eps: float
    sigma: float
    m: float
    theta: float
    dt: float
    steps: int          # timesteps of the full run
    noise: str          # "uniform": m + a*U(-1,1); "normal": m + a*N(0,1);
                        # "cos": m + a*prod_k cos(2 pi x_k) (the paper's Sec. 4 start, a = 1/50)
    amp: float
    seed: int
    restart: int        # (F)GMRES restart length
    gmres_rtol: float
    newton_atol: float

    @property
    def n_vertices(self) -> int:
        return (self.n + 1) ** self.dim

    @property
    def dofs(self) -> int:
        return 2 * self.n_vertices

    @property
    def newton_tols(self):
        """(atol, rtol) of the Newton stop test ||F||_2 <= max(atol, rtol ||F_0||_2).

        The 32x32 case states 1e-10 absolute.  The others scale that absolute
        level by h^d sqrt(N_v) (the size of a weak-form vector of O(1)
        nodal values) and add a relative floor of 1e-12.
        """
        if self.name == "2d_n32":
            return self.newton_atol, 0.0
        h = 1.0 / self.n
        return self.newton_atol * h ** self.dim * math.sqrt(self.n_vertices), 1e-12


def initial_u(w: Workload) -> np.ndarray:
    """Nodal u0 in compact lexicographic order (x fastest)."""
    nv = w.n_vertices
    if w.noise == "uniform":
        return w.m + w.amp * uniform(w.seed, nv, -1.0, 1.0)
    if w.noise == "normal":
        return w.m + w.amp * normal(w.seed, nv)
    if w.noise == "cos":
        x = nodal_coords(w.dim, w.n)
        return w.m + w.amp * np.prod(np.cos(2.0 * np.pi * x), axis=1)
    raise ValueError(w.noise)


def nodal_coords(dim: int, n: int) -> np.ndarray:
    """Vertex coordinates (N_v, dim) of the uniform grid, x fastest."""
    g = np.arange(n + 1, dtype=np.float64) / n
    if dim == 2:
        y, x = np.meshgrid(g, g, indexing="ij")
        return np.stack([x.ravel(), y.ravel()], axis=1)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


# The five workloads: the CPU-sized 2D case, the 2D 1024^2 case timed by the
# benchmark, the 3D 128^3 and 512^3 Kuhn cases, and (serving) a request mix.
SMALL_2D = Workload("2d_n32", 2, 32, 0.04, 100.0, 0.0, 1.0, 1e-4, 5,
                    "uniform", 0.01, 0, 30, 1e-10, 1e-10)
LARGE_2D = Workload("2d_n1024", 2, 1024, 0.02, 200.0, 0.1, 0.5, 2e-5, 20,
                    "normal", 0.05, 1, 30, 1e-8, 1e-10)
CUBE_128 = Workload("3d_n128", 3, 128, 0.03, 100.0, -0.2, 1.0, 5e-5, 10,
                    "uniform", 0.02, 2, 30, 1e-8, 1e-10)
CUBE_512 = Workload("3d_n512", 3, 512, 0.01, 1000.0, 0.0, 0.5, 1e-5, 3,
                    "normal", 0.01, 3, 20, 1e-8, 1e-10)

# The 512^3 workload's parameters on 256^3 (its float32 multigrid vectors of
# 67 MB still exceed L2 together): the size at which the 3D kernels are
# profiled with every counter.
CUBE_256 = Workload("3d_n256", 3, 256, 0.01, 1000.0, 0.0, 0.5, 1e-5, 3,
                    "normal", 0.01, 3, 20, 1e-8, 1e-10)

WORKLOADS = {w.name: w for w in (SMALL_2D, LARGE_2D, CUBE_128, CUBE_512, CUBE_256)}

# The paper's own experiment (Sec. 4): unit cube, m = 0.4, eps = 0.02,
# sigma = 100, theta = 0.5, dt = eps^2, u0 = m + cos(2 pi x) cos(2 pi y) cos(2 pi z) / 50,
# on meshes of 50 2^k cells per side (scaled() picks the size).
PAPER_3D = Workload("paper_3d", 3, 50, 0.02, 100.0, 0.4, 0.5, 4e-4, 300,
                    "cos", 1.0 / 50.0, 0, 30, 1e-8, 1e-10)


def scaled(w: Workload, n: int, **kw) -> Workload:
    """Same parameters on another grid size (parity cases at oracle sizes)."""
    return dataclasses.replace(w, name=f"{w.name}_as_n{n}", n=n, **kw)


def serving_requests(count: int = 256, seed: int = 5, rate: float = 40.0):
    """Request mix of the serving stream: Poisson arrivals at `rate` req/s.

    Half 2D grids from {64,128,256,512}^2, half 3D from {32,48,64,96}^3;
    eps~U(0.01,0.05), sigma~logU(10,1000), m~U(-0.3,0.3), theta in {0.5,1},
    dt = 0.25 eps^2, 5..50 timesteps, u0 noise amplitude 0.01.
    """
    u = uniform01(seed, 8 * count).reshape(count, 8)
    arrivals = np.cumsum(-np.log1p(-u[:, 0]) / rate)
    out = []
    for i in range(count):
        is3d = u[i, 1] >= 0.5
        sizes = (32, 48, 64, 96) if is3d else (64, 128, 256, 512)
        n = sizes[min(3, int(u[i, 2] * 4))]
        eps = 0.01 + 0.04 * u[i, 3]
        sigma = 10.0 ** (1.0 + 2.0 * u[i, 4])
        m = -0.3 + 0.6 * u[i, 5]
        theta = 0.5 if u[i, 6] < 0.5 else 1.0
        steps = 5 + min(45, int(u[i, 7] * 46))
        wl = Workload(f"req{i}", 3 if is3d else 2, n, eps, sigma, m, theta,
                      0.25 * eps * eps, steps, "uniform", 0.01, 1000 + i,
                      30, 1e-8, 1e-10)
        out.append((float(arrivals[i]), wl))
    return out
