"""Seeded synthetic inputs for the LJ workloads (no arithmetic of the method).

Both the CUDA path and the CPU oracle read their inputs from here, so this
module holds only input generation: lattices, random positions, random
velocities and the parameter sets of the workloads.  Nothing here evaluates
Eq. 1, a force, a neighbor list or a time step.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out below with numpy
uint64 arithmetic so that the integer stream is identical on every machine.
Normal deviates use the Box-Muller transform; their last bits follow the
platform's log/cos/sin, so a stored value must never depend on them bit for
bit (tests always generate inputs and evaluate both sides on one machine).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of SplitMix64 started from state `seed`."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """Uniform deviates in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller from one SplitMix64 stream."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def fcc_constant(density: float) -> float:
    """Cubic fcc lattice constant for a number density (4 atoms per cell)."""
    return (4.0 / density) ** (1.0 / 3.0)


def fcc(n: int, density: float = 0.8442):
    """fcc crystal of n^3 cubic cells in a periodic cube.

    Atom order i = ((ix*n + iy)*n + iz)*4 + b with the basis
    (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2).  Returns (x, box, a)."""
    a = fcc_constant(density)
    g = np.arange(n, dtype=np.float64)
    ix, iy, iz = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
    x = ((cells[:, None, :] + FCC_BASIS[None, :, :]) * a).reshape(-1, 3)
    L = n * a
    return np.ascontiguousarray(x), np.array([L, L, L]), a


def maxwell_boltzmann(masses: np.ndarray, T: float, seed: int) -> np.ndarray:
    """Velocities drawn at temperature T (k_B = 1), zero total momentum, then
    scaled so that sum(m v^2) = (3N - 3) T exactly (up to rounding)."""
    masses = np.asarray(masses, dtype=np.float64)
    n = len(masses)
    v = normal(seed, 3 * n).reshape(n, 3) * np.sqrt(T / masses)[:, None]
    p = (masses[:, None] * v).sum(axis=0) / masses.sum()
    v -= p
    if n > 1 and T > 0:
        two_ke = float((masses[:, None] * v * v).sum())
        v *= np.sqrt((3 * n - 3) * T / two_ke)
    else:
        v[:] = 0.0
    return np.ascontiguousarray(v)


def random_positions(n: int, box, seed: int) -> np.ndarray:
    box = np.asarray(box, dtype=np.float64)
    return np.ascontiguousarray(uniform(seed, 3 * n).reshape(n, 3) * box[None, :])


@dataclass
class LJParams:
    """Per-type-pair Eq. 1 coefficients and run settings (reduced LJ units)."""
    eps: np.ndarray
    sigma: np.ndarray
    rc: np.ndarray
    mass: np.ndarray
    skin: float = 0.3
    dt: float = 0.005
    rebuild_every: int = 20

    @property
    def ntypes(self) -> int:
        return len(self.mass)

    @property
    def rlist(self) -> float:
        return float(np.max(self.rc)) + self.skin


def lj_single(eps=1.0, sigma=1.0, rc=2.5, mass=1.0, **kw) -> LJParams:
    one = lambda v: np.full((1, 1), float(v))
    return LJParams(one(eps), one(sigma), one(rc), np.array([float(mass)]), **kw)


@dataclass
class System:
    """One periodic box: positions, velocities, types, box edges, parameters."""
    x: np.ndarray
    v: np.ndarray
    type: np.ndarray
    box: np.ndarray
    params: LJParams
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.x)


def fcc_liquid(n: int, density: float = 0.8442, T: float = 1.44, seed: int | None = None,
               **kw) -> System:
    """The LJ melt / scaling workload: fcc n^3 cells, Maxwell-Boltzmann at T,
    eps = sigma = m = 1, rc = 2.5, skin 0.3, dt 0.005, rebuild every 20.
    The default seed is 1000 + n."""
    x, box, a = fcc(n, density)
    p = lj_single(**kw)
    t = np.zeros(len(x), dtype=np.int32)
    seed = 1000 + n if seed is None else seed
    v = maxwell_boltzmann(p.mass[t], T, seed)
    return System(x, v, t, box, p, dict(kind="fcc", n_cells=n, density=density, T=T,
                                        seed=seed, a=a))


def binary_mixture_params(**kw) -> LJParams:
    """80:20 binary LJ mixture coefficients: eps_AA=1, eps_AB=1.5, eps_BB=0.5,
    sigma_AA=1, sigma_AB=0.8, sigma_BB=0.88, rc = 2.5 sigma_ab, m = 1."""
    eps = np.array([[1.0, 1.5], [1.5, 0.5]])
    sigma = np.array([[1.0, 0.8], [0.8, 0.88]])
    return LJParams(eps, sigma, 2.5 * sigma, np.array([1.0, 1.0]), **kw)


def binary_mixture(n: int = 64000, frac_a: float = 0.8, density: float = 1.2,
                   seed: int = 42, T: float = 1.0) -> System:
    """Random uniform positions (not yet relaxed) of an A:B mixture in a cube:
    the first round(frac_a*n) atoms are type A (0), the rest type B (1)."""
    L = (n / density) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    x = random_positions(n, box, seed)
    na = int(round(frac_a * n))
    t = np.zeros(n, dtype=np.int32)
    t[na:] = 1
    p = binary_mixture_params()
    v = maxwell_boltzmann(p.mass[t], T, seed + 1)
    return System(x, v, t, box, p, dict(kind="mixture", n=n, density=density, seed=seed, T=T))


def replica_cells(R: int = 512, lo: int = 3, hi: int = 20, seed: int = 7) -> np.ndarray:
    """Replica sizes n_r drawn uniformly from {lo..hi} (fcc n_r^3 cells each)."""
    u = uniform(seed, R)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def replica_temperatures(R: int = 512, lo: float = 0.7, hi: float = 1.5, seed: int = 8):
    return lo + uniform(seed, R) * (hi - lo)


def replicas(R: int = 512, seed: int = 7, lo: int = 3, hi: int = 20,
             density: float = 0.8442) -> list[System]:
    """Batched workload: R independent fcc boxes of uneven size, T uniform in
    [0.7, 1.5], replica r seeded 10000 + r."""
    ns = replica_cells(R, lo, hi, seed)
    Ts = replica_temperatures(R, seed=seed + 1)
    return [fcc_liquid(int(ns[r]), density, float(Ts[r]), seed=10000 + r) for r in range(R)]
