"""Seeded synthetic inputs for the Lennard-Jones workloads.

This module is shared by the CUDA path and the oracle, so it holds none of
the method's arithmetic: only lattice sites, random numbers and the named
workload shapes.  Random numbers come from numpy's PCG64 generator seeded
explicitly; the same arrays are fed to both sides of every comparison.

Workloads (reduced LJ units, eps = sigma = m = 1, rc = 2.5):
  fluid-2k   N = 2,048     FCC 4*8^3,   rho 0.8442, T 0.728, 100 steps
  fluid-131k N = 131,072   FCC 4*32^3,  rho 0.8442, T 0.728, 1000 steps
  fluid-4m   N = 4,000,000 FCC 4*100^3, rho 0.8442, T 1.0,   200 steps
  fm-32k     N = 32,000    FCC 4*20^3,  rho 0.8442, T 1.0,   50 steps
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n_fcc: int          # FCC unit cells per dimension (N = 4 n^3)
    rho: float
    temperature: float
    steps: int
    dt: float = 0.005
    rc: float = 2.5
    seed: int = 12345

    @property
    def n(self) -> int:
        return 4 * self.n_fcc ** 3

    @property
    def box(self) -> float:
        return box_side(self.n, self.rho)


WORKLOADS = {
    "fluid-2k": Workload("fluid-2k", 8, 0.8442, 0.728, 100),
    "fluid-131k": Workload("fluid-131k", 32, 0.8442, 0.728, 1000),
    "fluid-4m": Workload("fluid-4m", 100, 0.8442, 1.0, 200),
    "fm-32k": Workload("fm-32k", 20, 0.8442, 1.0, 50),
}


def box_side(n: int, rho: float) -> float:
    """Cubic box side L = (N / rho)^(1/3)."""
    return float((n / rho) ** (1.0 / 3.0))


def fcc(n_fcc: int, rho: float) -> tuple[np.ndarray, float]:
    """FCC lattice of 4 n^3 sites filling a cubic box at density rho.

    Lattice constant a = L / n; basis a*{(0,0,0), (1/2,1/2,0), (1/2,0,1/2),
    (0,1/2,1/2)}; every site shifted by a/4 along each axis so that no site
    sits on a cell face.  Returns (x (N, 3) float64, L)."""
    n = 4 * n_fcc ** 3
    L = box_side(n, rho)
    a = L / n_fcc
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(n_fcc, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    x = (cells[:, None, :] + basis[None, :, :] + 0.25) * a
    return np.ascontiguousarray(x.reshape(n, 3)), L


def velocities(n: int, temperature: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """Gaussian velocities with zero total momentum, rescaled so that
    m sum v^2 / (3N - 3) equals the target temperature (k_B = 1)."""
    v = np.random.default_rng(seed).standard_normal((n, 3))
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
        dof = 3 * n - 3
        t_now = mass * float(np.sum(v * v)) / dof
        v *= np.sqrt(temperature / t_now)
    else:
        v[:] = 0.0
    return np.ascontiguousarray(v)


def uniform(n: int, L: float, seed: int) -> np.ndarray:
    """Uniform random positions in [0, L)^3."""
    return np.ascontiguousarray(np.random.default_rng(seed).random((n, 3)) * L)


def jittered_fcc(n_fcc: int, rho: float, amplitude: float, seed: int) -> tuple[np.ndarray, float]:
    """FCC lattice with every coordinate displaced uniformly in
    [-amplitude, amplitude) -- a liquid-like but overlap-free configuration."""
    x, L = fcc(n_fcc, rho)
    x += (np.random.default_rng(seed).random(x.shape) * 2.0 - 1.0) * amplitude
    return np.ascontiguousarray(x), L


def lattice_gas(n: int, rho: float, seed: int, jitter: float = 0.1) -> tuple[np.ndarray, float]:
    """n random positions without overlaps at density rho: the smallest FCC
    lattice of 4 m^3 >= n sites in the box L = (n/rho)^(1/3), with n sites
    kept at random (random vacancies), each coordinate displaced uniformly
    by +-jitter lattice constants."""
    L = box_side(n, rho)
    m = 1
    while 4 * m ** 3 < n:
        m += 1
    a = L / m
    sites, _ = fcc(m, 4 * m ** 3 / L ** 3)
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.choice(sites.shape[0], n, replace=False))
    x = sites[keep] + (rng.random((n, 3)) * 2.0 - 1.0) * jitter * a
    return np.ascontiguousarray(x), L


@dataclass(frozen=True)
class Ensemble:
    """Independent replicas: N_r uniform in [n_lo, n_hi], rho_r uniform in
    [rho_lo, rho_hi], T_r uniform in [t_lo, t_hi], all drawn from one seed."""
    n: np.ndarray
    rho: np.ndarray
    temperature: np.ndarray
    box: np.ndarray
    seed: int


def ensemble(nrep: int = 256, seed: int = 2024, n_lo: int = 500, n_hi: int = 50000, rho_lo: float = 0.7,
             rho_hi: float = 0.9, t_lo: float = 0.7, t_hi: float = 1.5) -> Ensemble:
    rng = np.random.default_rng(seed)
    n = rng.integers(n_lo, n_hi + 1, nrep)
    rho = rng.uniform(rho_lo, rho_hi, nrep)
    temp = rng.uniform(t_lo, t_hi, nrep)
    box = np.array([box_side(int(a), float(b)) for a, b in zip(n, rho)])
    return Ensemble(n, rho, temp, box, seed)


def ensemble_state(ens: Ensemble):
    """Per-replica starting positions (lattice_gas) and velocities."""
    xs, vs = [], []
    for r in range(len(ens.n)):
        x, _ = lattice_gas(int(ens.n[r]), float(ens.rho[r]), ens.seed + 7919 * r)
        xs.append(x)
        vs.append(velocities(int(ens.n[r]), float(ens.temperature[r]), ens.seed + 104729 * r))
    return xs, vs


def workload_state(name: str) -> tuple[np.ndarray, np.ndarray, float, Workload]:
    """(x, v, L, workload) of a named workload's starting state."""
    w = WORKLOADS[name]
    x, L = fcc(w.n_fcc, w.rho)
    v = velocities(w.n, w.temperature, w.seed)
    return x, v, L, w
