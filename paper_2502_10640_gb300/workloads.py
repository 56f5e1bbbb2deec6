"""Seeded synthetic electron bunches (inputs only).

This module draws initial conditions; it holds none of the force or push arithmetic and
is shared by the tests, the benchmark and the oracle checks only as a source of inputs.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a
counter-based generator: draw k of stream s is mix(s * 2^32 + k), so any subset of draws
can be regenerated without the others.  Uniform doubles take the top 53 bits; Gaussians
use the Box-Muller transform; uniform-sphere points use r = R u^(1/3) with an isotropic
direction.

The paper's own workload (Sec. 2.1) is a cube of side l = 0.1 mm with number density
n0 = 5e16 m^-3 sampled by an exact lattice of Np = 16^3 macro-particles, each of weight
w = n0 l^3 / Np, at rest, stepped with dt = 1e-13 s.  The lattice is read as
cell-centred: coordinate (a + 1/2) l / n - l/2 for a = 0..n-1, which gives the stated
inter-particle spacing l/n (12.5 um for 8^3 in Sec. 3.2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 (SI).  Used here only to turn a bunch charge into a macro-particle weight
# and to bound the time step of generated workloads.
E_CHARGE = 1.602176634e-19
M_ELECTRON = 9.1093837015e-31
EPS0 = 8.8541878128e-12

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value (vectorised, wrapping uint64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(counters, dtype=np.uint64) * _GOLDEN + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream `stream` of seed `seed`."""
    base = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(40)) + (np.uint64(stream & 0xFF) << np.uint64(32))
    k = base + np.arange(n, dtype=np.uint64)
    return (splitmix64(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _open_uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in (0, 1]."""
    return 1.0 - uniform(seed, stream, n)


def gaussian(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal deviates by Box-Muller."""
    m = (n + 1) // 2
    u1 = _open_uniform(seed, stream, m)
    u2 = uniform(seed, stream + 1, m)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    return np.concatenate([r * np.cos(t), r * np.sin(t)])[:n]


def _recentre(pos: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(pos - pos.mean(axis=0, keepdims=True))


def gaussian_bunch(n: int, sigma: float, seed: int) -> np.ndarray:
    """[n][3] positions, each coordinate N(0, sigma^2), re-centred to zero mean."""
    if n == 0:
        return np.zeros((0, 3))
    g = gaussian(seed, 0, 3 * n).reshape(3, n).T * sigma
    return _recentre(g)


def uniform_sphere(n: int, radius: float, seed: int, recentre: bool = True) -> np.ndarray:
    """[n][3] positions uniform in a ball of the given radius."""
    if n == 0:
        return np.zeros((0, 3))
    u = uniform(seed, 0, n)
    cz = 2.0 * uniform(seed, 1, n) - 1.0
    ph = 2.0 * math.pi * uniform(seed, 2, n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    r = radius * np.cbrt(u)
    pos = np.stack([r * sz * np.cos(ph), r * sz * np.sin(ph), r * cz], axis=1)
    return _recentre(pos) if recentre else np.ascontiguousarray(pos)


def cube_lattice(n_side: int, side: float) -> np.ndarray:
    """[n_side^3][3] cell-centred lattice filling a cube of edge `side` centred at 0."""
    a = (np.arange(n_side, dtype=np.float64) + 0.5) * (side / n_side) - side / 2.0
    x, y, z = np.meshgrid(a, a, a, indexing="ij")
    return np.ascontiguousarray(np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1))


def lattice_weight(n0: float, side: float, n_particles: int) -> float:
    """Macro-particle weight w = n0 l^3 / Np of a uniform cube (Sec. 2.1)."""
    return n0 * side ** 3 / n_particles


def weight_for_charge(total_charge: float, n: int) -> float:
    """Weight that makes n macro-electrons carry |total_charge| coulombs."""
    return total_charge / (E_CHARGE * n)


def coulomb_k() -> float:
    return 1.0 / (4.0 * math.pi * EPS0)


def explosion_rate(n: int, w: float, radius: float) -> float:
    """K = k e^2 N w / (m_e R^3) [1/s^2]: the shell-expansion constant of a cold uniform ball.

    sqrt(2K) dt measures how far one step moves a bunch of this size; it sets the
    time-step bound of generated workloads.
    """
    return coulomb_k() * E_CHARGE ** 2 * n * w / (M_ELECTRON * radius ** 3)


@dataclasses.dataclass(frozen=True)
class Bunch:
    """One expansion run: n macro-electrons of weight w, softening eps [m], step dt [s]."""
    name: str
    n: int
    w: float
    eps: float
    dt: float
    steps: int
    profile: str          # "gaussian" | "sphere" | "lattice"
    scale: float          # sigma (gaussian), radius (sphere) or edge (lattice) [m]
    seed: int

    def positions(self) -> np.ndarray:
        if self.profile == "gaussian":
            return gaussian_bunch(self.n, self.scale, self.seed)
        if self.profile == "sphere":
            return uniform_sphere(self.n, self.scale, self.seed)
        if self.profile == "lattice":
            side_n = round(self.n ** (1.0 / 3.0))
            if side_n ** 3 != self.n:
                raise ValueError("lattice bunch needs a cube number of particles")
            return cube_lattice(side_n, self.scale)
        raise ValueError(f"unknown profile {self.profile!r}")

    def velocities(self) -> np.ndarray:
        return np.zeros((self.n, 3))                     # cold bunches

    def pairs_per_step(self) -> int:
        return self.n * self.n                           # all-pairs convention


# The five workloads and the paper's own.
COLD_GAUSSIAN_2048 = Bunch("cold Gaussian, N=2048 real electrons, sigma=1 um, no softening",
                           2048, 1.0, 0.0, 1e-16, 200, "gaussian", 1e-6, 1)
GAUSSIAN_65536 = Bunch("cold Gaussian, N=65536 macro-electrons (1e8 e), sigma=10 um, eps=1 nm",
                       65536, 1e8 / 65536, 1e-9, 1e-14, 2000, "gaussian", 1e-5, 2)
SPHERE_1M = Bunch("cold uniform sphere, N=2^20, R=50 um, Q=1 nC, eps=5 nm",
                  1 << 20, weight_for_charge(1e-9, 1 << 20), 5e-9, 2e-14, 500, "sphere", 5e-5, 3)
PAPER_LATTICE = Bunch("cube lattice 16^3, l=0.1 mm, n0=5e16 m^-3 (Sec. 2.1)",
                      4096, lattice_weight(5e16, 1e-4, 4096), 0.0, 1e-13, 100000, "lattice", 1e-4, 0)

WORKLOADS = {
    "gaussian2048": COLD_GAUSSIAN_2048,
    "gaussian65536": GAUSSIAN_65536,
    "sphere1m": SPHERE_1M,
    "paper_lattice": PAPER_LATTICE,
}


def batch_mix(count: int = 64, seed: int = 4, n_min: int = 1024, n_max: int = 131072,
              steps: int = 1000) -> list[Bunch]:
    """Independent cold bunches of uneven size (the batched workload).

    N log-uniform in [n_min, n_max]; Gaussian or uniform sphere 50/50; radius log-uniform
    1-50 um; total charge log-uniform 1 fC - 1 nC; dt log-uniform in [1e-15, 5e-14] s,
    clipped to 0.1 / sqrt(2K); softening 1e-4 R.  Bunch b draws from seed 1000 seed + b.
    """
    out = []
    for b in range(count):
        s = 1000 * seed + b
        u = uniform(s, 7, 6)
        n = int(round(math.exp(math.log(n_min) + u[0] * (math.log(n_max) - math.log(n_min)))))
        profile = "gaussian" if u[1] < 0.5 else "sphere"
        radius = math.exp(math.log(1e-6) + u[2] * (math.log(50e-6) - math.log(1e-6)))
        charge = math.exp(math.log(1e-15) + u[3] * (math.log(1e-9) - math.log(1e-15)))
        dt = math.exp(math.log(1e-15) + u[4] * (math.log(5e-14) - math.log(1e-15)))
        w = weight_for_charge(charge, n)
        dt = min(dt, 0.1 / math.sqrt(2.0 * explosion_rate(n, w, radius)))
        out.append(Bunch(f"batch[{b}]", n, w, 1e-4 * radius, dt, steps, profile, radius, s))
    return out


@dataclasses.dataclass(frozen=True)
class Request:
    """One served expansion run arriving at `arrival` seconds."""
    rid: int
    arrival: float
    bunch: Bunch


def serve_trace(count: int, rate: float = 20.0, seed: int = 5, n_min: int = 4096,
                n_max: int = 524288, steps_min: int = 100, steps_max: int = 5000) -> list[Request]:
    """Poisson arrivals (mean `rate` per second) of uniform-sphere runs.

    N log-uniform in [n_min, n_max], steps uniform in [steps_min, steps_max], weight,
    radius, softening and dt as the 2^20-particle sphere.
    """
    u_gap = _open_uniform(seed, 0, count)
    u_n = uniform(seed, 1, count)
    u_s = uniform(seed, 2, count)
    t = 0.0
    out = []
    for r in range(count):
        t += -math.log(u_gap[r]) / rate
        n = int(round(math.exp(math.log(n_min) + u_n[r] * (math.log(n_max) - math.log(n_min)))))
        steps = steps_min + int(u_s[r] * (steps_max - steps_min + 1))
        b = Bunch(f"req[{r}]", n, SPHERE_1M.w, SPHERE_1M.eps, SPHERE_1M.dt, steps, "sphere",
                  SPHERE_1M.scale, 100000 * seed + r)
        out.append(Request(r, t, b))
    return out
