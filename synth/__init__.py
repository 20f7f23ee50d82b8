"""Seeded synthetic bead systems shaped like the paper's workloads (Sec. 4.3).

This module only draws random numbers: positions, forces, radii and system
sizes.  It holds none of the RPY or FMM arithmetic, so both the CPU oracle
and the CUDA path can take their inputs from here without sharing any of the
method.

Every generator returns plain numpy arrays (float64):
    pos  (N, 3)  bead centres
    f    (N, 3)  forces
    a    float   bead radius
    s    float   kT/eta (the RPY tensor is linear in it)

Positions are always drawn before forces from one ``numpy.random.default_rng``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class BeadSystem:
    pos: np.ndarray
    f: np.ndarray
    a: float
    s: float          # kT / eta
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _sphere_surface(rng: np.random.Generator, n: int, radius: float, centre) -> np.ndarray:
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return np.asarray(centre, dtype=np.float64) + radius * g


def _plummer(rng: np.random.Generator, n: int, b: float) -> np.ndarray:
    """Plummer-like cluster (density ~ (1 + r^2/b^2)^(-5/2)) centred at 0.5,
    kept inside the unit cube by rejection."""
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 64
        u = rng.random(m)
        u = np.clip(u, 1e-12, 1.0)
        r = b / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = 0.5 + r[:, None] * d
        ok = np.all((p >= 0.0) & (p < 1.0), axis=1)
        out = np.concatenate([out, p[ok]])
    return out[:n]


def uniform_cube(n: int, seed: int, a: float, s: float | None = None) -> BeadSystem:
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3))
    f = rng.standard_normal((n, 3))
    return BeadSystem(pos, f, a, 6 * math.pi * a if s is None else s, f"cube{n}")


def config1() -> BeadSystem:
    """N=4096 uniform in the unit cube, seed 0, a=0.004, kT/(6 pi eta a)=1."""
    return uniform_cube(4096, 0, 0.004)


def sphere_plus_cube(n: int, seed: int, a: float, frac_cube: float = 0.1) -> BeadSystem:
    """Uniform on the sphere of radius 0.5 centred in the unit cube, plus a
    fraction of beads uniform in the enclosing cube."""
    rng = np.random.default_rng(seed)
    n_cube = int(round(frac_cube * n))
    n_sph = n - n_cube
    p1 = _sphere_surface(rng, n_sph, 0.5, (0.5, 0.5, 0.5))
    p2 = rng.random((n_cube, 3))
    pos = np.concatenate([p1, p2])
    f = rng.standard_normal((n, 3))
    return BeadSystem(pos, f, a, 6 * math.pi * a, f"sphere{n}")


def config2(n: int = 1_000_000) -> BeadSystem:
    """N=1,000,000: 90% on the sphere surface, 10% uniform in the cube, seed 2, a=1e-4."""
    return sphere_plus_cube(n, 2, 1e-4)


def config3(n: int = 15_000_000) -> BeadSystem:
    """N=15,000,000 uniform in the unit cube, seed 3, a=2e-5."""
    return uniform_cube(n, 3, 2e-5)


def sphere8m(n: int = 8_000_000) -> BeadSystem:
    """N=8,000,000 uniform on the sphere of radius 0.5 centred in the unit cube
    (the paper's sphere workload), seed 6, a=1e-4."""
    return sphere_plus_cube(n, 6, 1e-4, frac_cube=0.0)


def config4(nsys: int = 256, seed: int = 4, lo: float = 1e3, hi: float = 2e5):
    """Many independent systems of log-uniform size, each a uniform cube or a
    Plummer-like cluster (coin flip), a_s = 0.5 / N_s^(1/3)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), nsys))).astype(np.int64)
    kinds = rng.random(nsys) < 0.5
    out = []
    for i in range(nsys):
        n = int(sizes[i])
        if kinds[i]:
            pos = rng.random((n, 3))
        else:
            pos = _plummer(rng, n, 0.1)
        f = rng.standard_normal((n, 3))
        a = 0.5 / n ** (1.0 / 3.0)
        out.append(BeadSystem(pos, f, a, 6 * math.pi * a, ("cube" if kinds[i] else "plummer") + str(n)))
    return out


def config5(nsys: int = 64, seed: int = 5, lo: float = 1e4, hi: float = 2e6):
    """Resident serving systems: log-uniform sizes, half uniform cube, half
    sphere surface, a_s = 0.5 / N_s^(1/3).  Returns the base systems and a
    per-request generator of (jittered positions, fresh forces)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), nsys))).astype(np.int64)
    out = []
    for i in range(nsys):
        n = int(sizes[i])
        if i % 2 == 0:
            pos = rng.random((n, 3))
        else:
            pos = _sphere_surface(rng, n, 0.5, (0.5, 0.5, 0.5))
        f = rng.standard_normal((n, 3))
        a = 0.5 / n ** (1.0 / 3.0)
        out.append(BeadSystem(pos, f, a, 6 * math.pi * a, ("cube" if i % 2 == 0 else "sphere") + str(n)))
    return out


def jitter(rng: np.random.Generator, pos: np.ndarray, sigma: float = 1e-3) -> np.ndarray:
    return pos + sigma * rng.standard_normal(pos.shape)


def sample_targets(n: int, k: int = 2000, seed: int = 12345) -> np.ndarray:
    """Target beads for large-N error checks: k of n, uniformly without replacement."""
    if n <= k:
        return np.arange(n, dtype=np.int64)
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False)).astype(np.int64)
