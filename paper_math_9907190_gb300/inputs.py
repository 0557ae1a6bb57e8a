"""Seeded synthetic inputs shaped like the paper's unit-square / unit-cube runs.

This module only draws inputs; it holds none of the method's arithmetic.  It
serves both the CUDA path and the CPU oracle (which never import each other).
All arrays are float64 full grids (Dirichlet ring included), C order, x the
last axis.  The paper uses no dataset: its experiments are Poisson problems on
the unit square (65x65 grid) and unit cube (17^3 grid) with a zero Dirichlet
boundary; the recipes below follow those shapes at the sizes benchmarked.
"""

from __future__ import annotations

import math

import numpy as np


def coords(dim: int, n: int):
    x = np.linspace(0.0, 1.0, n + 2)
    return np.meshgrid(*([x] * dim), indexing="ij")  # (Y, X) or (Z, Y, X)


def manufactured_2d(n: int):
    """u = sin(pi x) sin(2 pi y), f = Laplacian(u) = -5 pi^2 u (exact, continuous)."""
    Y, X = coords(2, n)
    u = np.sin(math.pi * X) * np.sin(2 * math.pi * Y)
    return np.ascontiguousarray(-5 * math.pi**2 * u), np.ascontiguousarray(u)


def manufactured_3d(n: int):
    """u = sin(pi x) sin(pi y) sin(2 pi z), f = -6 pi^2 u."""
    Z, Y, X = coords(3, n)
    u = np.sin(math.pi * X) * np.sin(math.pi * Y) * np.sin(2 * math.pi * Z)
    return np.ascontiguousarray(-6 * math.pi**2 * u), np.ascontiguousarray(u)


def uniform_f(dim: int, n: int, seed: int) -> np.ndarray:
    """f ~ U[-1, 1] on the full grid (ring included, read only by order 4)."""
    return np.ascontiguousarray(np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n + 2,) * dim))


def square_small(n: int = 63, seed: int = 0) -> np.ndarray:
    """2D h = 1/64 case: manufactured f plus 1e-3 * U[-1, 1] noise."""
    f, _ = manufactured_2d(n)
    return np.ascontiguousarray(f + 1e-3 * np.random.default_rng(seed).uniform(-1.0, 1.0, size=f.shape))


def square_large(n: int = 4095, kind: str = "uniform", seed: int = 1) -> np.ndarray:
    """2D h = 1/4096: 'uniform' f ~ U[-1,1] (seed 1) or 'manufactured' (as square_small, seed 0)."""
    if kind == "uniform":
        return uniform_f(2, n, seed)
    return square_small(n, seed=0)


def cube(n: int = 255, seed: int = 2) -> np.ndarray:
    """3D h = 1/256: manufactured f plus N(0, 1e-3^2) noise."""
    f, _ = manufactured_3d(n)
    return np.ascontiguousarray(f + np.random.default_rng(seed).normal(0.0, 1e-3, size=f.shape))


def batch_sides(count: int = 512, seed: int = 3, kmin: int = 5, kmax: int = 10) -> list[int]:
    """Sides n_b = 2^k - 1 with k ~ U{kmin..kmax}: 2^k intervals per side."""
    ks = np.random.default_rng(seed).integers(kmin, kmax + 1, size=count)
    return [int(2**k - 1) for k in ks]


def batch_f(n: int, b: int) -> np.ndarray:
    """Problem b of the batch: f ~ U[-1, 1] with seed 4 + b."""
    return uniform_f(2, n, 4 + b)


def grad_f(n: int, b: int) -> np.ndarray:
    """Problem b of the differentiable 3D batch: f ~ N(0, 1), seed (5, b)."""
    return np.ascontiguousarray(np.random.default_rng([5, b]).normal(0.0, 1.0, size=(n + 2,) * 3))


def grad_target(n: int, seed: int = 6) -> np.ndarray:
    """Smooth target: sum over k in {1,2,3}^3 of a_k sin(k1 pi x) sin(k2 pi y) sin(k3 pi z), a ~ N(0,1)."""
    Z, Y, X = coords(3, n)
    a = np.random.default_rng(seed).normal(0.0, 1.0, size=(3, 3, 3))
    out = np.zeros_like(X)
    for k1 in range(3):
        for k2 in range(3):
            for k3 in range(3):
                out += a[k1, k2, k3] * (np.sin((k1 + 1) * math.pi * X) * np.sin((k2 + 1) * math.pi * Y)
                                        * np.sin((k3 + 1) * math.pi * Z))
    return np.ascontiguousarray(out)


def grad_coords(n: int, count: int = 8, seed: int = 7):
    """Interior coordinates (k, j, i) for the finite-difference gradient check."""
    rng = np.random.default_rng(seed)
    return [tuple(int(x) for x in rng.integers(1, n + 1, size=3)) for _ in range(count)]


def zero_ring(a: np.ndarray) -> np.ndarray:
    out = a.copy()
    m = np.ones_like(out, dtype=bool)
    m[(slice(1, -1),) * out.ndim] = False
    out[m] = 0.0
    return out
