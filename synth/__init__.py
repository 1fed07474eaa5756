"""Seeded synthetic particle sets shared by the oracle tests, the GPU tests and the benchmark.

This module only draws inputs; it holds none of the tree method's arithmetic.  The three
distributions stand in for the paper's benchmark sets (Sec. 3: a Sobol sphere and two SPH
snapshots that are not available here):

* ``plummer``  -- Plummer sphere, scale radius 1, total mass 1 (G = 1), radii drawn by the
  inverse of the enclosed-mass fraction X(r) = r^3 / (r^2 + 1)^(3/2) with X uniform on
  (0, 0.999], so the sphere is truncated at r_c = (0.999^(-2/3) - 1)^(-1/2) ~ 38.7.
* ``sphere``   -- uniform-density unit sphere (rejection from the cube [-1, 1]^3).
* ``cube``     -- uniform unit cube [0, 1)^3.

Masses are either equal (1/N) or ``loguniform10``: m ~ 10^U, U ~ U[0, 1), normalised to a
total of 1.  Smoothing lengths are set from the analytic number density n(r) so that a
kernel support of radius 2h holds ``n_neigh`` particles on average:
h = 0.5 * (3 n_neigh / (4 pi n(r)))^(1/3).
"""
from __future__ import annotations

import math

import numpy as np

PLUMMER_XMAX = 0.999
SEED_BASE = 20110728


def seed_for(config: int, case: int = 0) -> int:
    """Seed of a workload: 20110728 + 1000 * config + case."""
    return SEED_BASE + 1000 * int(config) + int(case)


def plummer_rc() -> float:
    return (PLUMMER_XMAX ** (-2.0 / 3.0) - 1.0) ** -0.5


def _directions(rng: np.random.Generator, n: int) -> np.ndarray:
    z = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def number_density(kind: str, r: np.ndarray, n: int) -> np.ndarray:
    """Analytic number density of the distribution at radius r (per unit volume)."""
    if kind == "plummer":
        return n * (3.0 / (4.0 * math.pi)) * (1.0 + r * r) ** -2.5 / PLUMMER_XMAX
    if kind == "sphere":
        return np.full_like(r, 3.0 * n / (4.0 * math.pi))
    if kind == "cube":
        return np.full_like(r, float(n))
    raise ValueError(kind)


def make_particles(kind: str, n: int, seed: int, mass_mode: str = "equal",
                   n_neigh: float = 50.0):
    """Return (x[n,3], m[n], h[n]) as float64 numpy arrays, particles in random order."""
    if n < 0:
        raise ValueError("n must be >= 0")
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "plummer":
        X = PLUMMER_XMAX * (1.0 - rng.random(n))          # (0, 0.999]
        r = (X ** (-2.0 / 3.0) - 1.0) ** -0.5
        x = _directions(rng, n) * r[:, None]
    elif kind == "sphere":
        out = np.empty((0, 3))
        while out.shape[0] < n:
            c = 2.0 * rng.random((max(1024, int(1.95 * (n - out.shape[0]))), 3)) - 1.0
            c = c[np.einsum("ij,ij->i", c, c) < 1.0]
            out = np.concatenate([out, c], axis=0)
        x = out[:n].copy()
    elif kind == "cube":
        x = rng.random((n, 3))
    else:
        raise ValueError(f"unknown distribution {kind!r}")
    x = np.ascontiguousarray(x, dtype=np.float64) + 0.0       # no negative zeros
    if mass_mode == "equal":
        m = np.full(n, 1.0 / max(n, 1))
    elif mass_mode == "loguniform10":
        m = 10.0 ** rng.random(n)
        m = m / m.sum()
    else:
        raise ValueError(f"unknown mass mode {mass_mode!r}")
    r = np.sqrt(np.einsum("ij,ij->i", x, x))
    dens = number_density(kind, r, n)
    h = 0.5 * np.cbrt(3.0 * n_neigh / (4.0 * math.pi * dens))
    return x, np.ascontiguousarray(m), np.ascontiguousarray(h)


def jitter(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Positions displaced by independent N(0, sigma^2) offsets (for the gradient workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return x + sigma * rng.standard_normal(x.shape)


def random_unit_vectors(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(shape)
    return v / np.linalg.norm(v)
