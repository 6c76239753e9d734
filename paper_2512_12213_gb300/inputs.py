"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only draws random numbers and marks solid nodes; it holds none of
the lattice Boltzmann arithmetic, so both the CUDA library and the CPU oracle
can be fed from it without sharing any of the method.

Geometry arrays are ``uint8`` shaped ``(nz, ny, nx)``: 0 marks a fluid node and
k > 0 a solid node belonging to wall k.  Per-population arrays are shaped
``(Q, nz, ny, nx)``.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int = 12345) -> np.random.Generator:
    return np.random.default_rng(seed)


def empty_mask(nx: int, ny: int, nz: int = 1) -> np.ndarray:
    """All-fluid domain (walls, if any, are the closed faces of the box)."""
    return np.zeros((nz, ny, nx), dtype=np.uint8)


def sphere_mask(nx, ny, nz, center, radius, wall=1) -> np.ndarray:
    """Staircase sphere: solid where |x - c| <= r at node centres."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[r2 <= radius * radius] = wall
    return m


def cylinder_mask(nx, ny, center, radius, wall=1) -> np.ndarray:
    """Staircase circular cylinder of a 2-D domain (nz = 1)."""
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2
    m = np.zeros((1, ny, nx), dtype=np.uint8)
    m[0][r2 <= radius * radius] = wall
    return m


def block_mask(nx, ny, nz, lo, hi, wall=1, base=None) -> np.ndarray:
    """Axis-aligned solid block lo <= (x, y, z) < hi, optionally added to `base`."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8) if base is None else base.copy()
    m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = wall
    return m


def random_solids(nx, ny, nz, fraction, n_walls=1, seed=7) -> np.ndarray:
    """Scattered solid nodes with wall ids 1..n_walls (stress test of boundary handling)."""
    g = rng(seed)
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    hit = g.random((nz, ny, nx)) < fraction
    m[hit] = g.integers(1, n_walls + 1, size=int(hit.sum()), dtype=np.uint8)
    return m


def noise(q, nx, ny, nz=1, amplitude=1e-3, seed=12345) -> np.ndarray:
    """Relative population perturbation xi ~ amplitude * U(-1, 1), shape (Q, nz, ny, nx)."""
    return amplitude * rng(seed).uniform(-1.0, 1.0, size=(q, nz, ny, nx))


def smooth_fields(nx, ny, nz=1, rho_amplitude=0.02, u_amplitude=0.05, dims=2, seed=99, modes=3):
    """Smooth periodic density and velocity fields built from a few random
    Fourier modes.  Returns rho (nz, ny, nx) around 1 and u (3, nz, ny, nx)."""
    g = rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def field():
        s = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky = g.integers(0, 3, size=2)
            kz = g.integers(0, 3) if dims == 3 else 0
            ph = g.uniform(0, 2 * np.pi)
            s += np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / max(nz, 1)) + ph)
        return s / modes

    rho = 1.0 + rho_amplitude * field()
    u = np.zeros((3, nz, ny, nx))
    for k in range(dims):
        u[k] = u_amplitude * field()
    return rho, u
