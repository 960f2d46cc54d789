"""Seeded synthetic inputs (target clouds and parameter sweeps).

This module holds no arithmetic of the method: it only draws points and
parameters with NumPy's PCG64, so that the CUDA path and the CPU oracle can be
fed identical inputs.  Shapes and distributions follow the workloads the
method is meant for (uniform clouds over one period cell and the slab
|x_last| <= 1, optionally with a fraction clustered around lattice points).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def _lattice_distance_3d(x: np.ndarray) -> np.ndarray:
    # distance to the nearest lattice point (2 pi m1, 2 pi m2, 0)
    d1 = x[:, 0] - TWO_PI * np.round(x[:, 0] / TWO_PI)
    d2 = x[:, 1] - TWO_PI * np.round(x[:, 1] / TWO_PI)
    return np.sqrt(d1 * d1 + d2 * d2 + x[:, 2] * x[:, 2])


def _lattice_distance_2d(x: np.ndarray) -> np.ndarray:
    d1 = x[:, 0] - TWO_PI * np.round(x[:, 0] / TWO_PI)
    return np.sqrt(d1 * d1 + x[:, 1] * x[:, 1])


def targets_3d(n: int, seed: int = 0, exclude: float = 1e-3, zmax: float = 1.0) -> np.ndarray:
    """n points, x1, x2 ~ U[0, 2 pi), x3 ~ U[-zmax, zmax], redrawn while within
    `exclude` of a lattice point.  Returns float64 (n, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((n, 3))
    x[:, 0] = rng.uniform(0.0, TWO_PI, n)
    x[:, 1] = rng.uniform(0.0, TWO_PI, n)
    x[:, 2] = rng.uniform(-zmax, zmax, n)
    bad = _lattice_distance_3d(x) < exclude
    while bad.any():
        m = int(bad.sum())
        x[bad, 0] = rng.uniform(0.0, TWO_PI, m)
        x[bad, 1] = rng.uniform(0.0, TWO_PI, m)
        x[bad, 2] = rng.uniform(-zmax, zmax, m)
        bad = _lattice_distance_3d(x) < exclude
    return x


def targets_2d(n: int, seed: int = 0, exclude: float = 1e-3, zmax: float = 1.0) -> np.ndarray:
    """n points, x1 ~ U[0, 2 pi), x2 ~ U[-zmax, zmax], lattice exclusion."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((n, 2))
    x[:, 0] = rng.uniform(0.0, TWO_PI, n)
    x[:, 1] = rng.uniform(-zmax, zmax, n)
    bad = _lattice_distance_2d(x) < exclude
    while bad.any():
        m = int(bad.sum())
        x[bad, 0] = rng.uniform(0.0, TWO_PI, m)
        x[bad, 1] = rng.uniform(-zmax, zmax, m)
        bad = _lattice_distance_2d(x) < exclude
    return x


def targets_3d_clustered(n: int, seed: int = 0, frac: float = 0.1, rmin: float = 1e-3,
                         rmax: float = 0.05) -> np.ndarray:
    """(1 - frac) n uniform points as targets_3d, plus frac n points uniform in
    the shell rmin <= r <= rmax (isotropic, radius ~ u^(1/3)) around one of the
    four lattice points at the corners of [0, 2 pi]^2, shuffled."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nc = int(round(frac * n))
    xu = targets_3d(n - nc, seed=seed + 1)
    u = rng.uniform(0.0, 1.0, nc)
    r = (rmin**3 + u * (rmax**3 - rmin**3)) ** (1.0 / 3.0)
    d = rng.standard_normal((nc, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    corner = rng.integers(0, 2, (nc, 2)) * TWO_PI
    xc = np.empty((nc, 3))
    xc[:, :2] = corner + r[:, None] * d[:, :2]
    xc[:, 2] = r * d[:, 2]
    x = np.concatenate([xu, xc])
    return x[rng.permutation(n)]


def sweep_pairs(n_pairs: int, seed: int = 0, kmin: float = 0.5, kmax: float = 5.0,
                wood_gap: float = 1e-3):
    """(alpha1, alpha2, k) triples: k ~ U[kmin, kmax], alpha ~ U[-1/2, 1/2]^2,
    redrawn while some in-plane wave vector |alpha + n| lies within wood_gap of k
    (|n_i| <= ceil(k) + 1).  Returns float64 (n_pairs, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n_pairs, 3))
    i = 0
    while i < n_pairs:
        k = rng.uniform(kmin, kmax)
        a = rng.uniform(-0.5, 0.5, 2)
        R = int(np.ceil(k)) + 1
        n = np.arange(-R, R + 1)
        A = np.sqrt((a[0] + n)[:, None] ** 2 + (a[1] + n)[None, :] ** 2)
        if np.abs(A - k).min() < wood_gap:
            continue
        out[i] = (a[0], a[1], k)
        i += 1
    return out
