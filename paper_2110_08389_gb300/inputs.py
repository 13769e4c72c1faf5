"""Seeded synthetic inputs shared by the tests, the oracle and the benchmark.

This module holds no arithmetic of the multigrid method: it only produces the
problems the method is run on -- grid coordinates from the paper's stretching
maps (Sec. 5, Eqs. tanh and tanh_inv) and right-hand sides drawn from a seeded
NumPy ``Generator(PCG64(seed))`` (the paper's experiments use random
right-hand sides, Sec. 6).
"""
from __future__ import annotations

import math

import numpy as np


def uniform_coords(n: int, length: float = 1.0) -> np.ndarray:
    """n+1 equally spaced nodes on [0, length]."""
    return np.linspace(0.0, length, n + 1)


def wall_coords(n: int, c: float, length: float = 1.0) -> np.ndarray:
    """Near-wall clustering, Eq. (tanh): x_i = L/2 {1 + tanh[c(2i/n - 1)]/tanh c}."""
    if c == 0.0:
        return uniform_coords(n, length)
    i = np.arange(n + 1, dtype=np.float64)
    x = 0.5 * length * (1.0 + np.tanh(c * (2.0 * i / n - 1.0)) / math.tanh(c))
    x[0], x[-1] = 0.0, length
    return x


def centre_coords(n: int, c: float, length: float = 1.0) -> np.ndarray:
    """Near-centre clustering, Eq. (tanh_inv) (n even)."""
    if n % 2:
        raise ValueError("centre clustering needs an even number of intervals")
    if c == 0.0:
        return uniform_coords(n, length)
    i = np.arange(n + 1, dtype=np.float64)
    lo = 0.5 * length * np.tanh(2.0 * c * i / n) / math.tanh(c)
    hi = 0.5 * length * (2.0 - np.tanh(c * (2.0 - 2.0 * i / n)) / math.tanh(c))
    x = np.where(i <= n // 2, lo, hi)
    x[0], x[-1], x[n // 2] = 0.0, length, 0.5 * length
    return x


def spacing_ratio(x: np.ndarray) -> float:
    """max / min of the interval lengths."""
    d = np.diff(x)
    return float(d.max() / d.min())


def c_for_ratio(n: int, ratio: float, kind: str = "wall") -> float:
    """Stretching parameter c giving max/min spacing = ratio (bisection)."""
    f = wall_coords if kind == "wall" else centre_coords
    lo, hi = 1e-6, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if spacing_ratio(f(n, mid)) < ratio:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def coords(n: int, kind: str = "wall", c: float | None = None, ratio: float | None = None) -> np.ndarray:
    """Coordinates of one axis: kind in {'uniform', 'wall', 'centre'}."""
    if kind == "uniform":
        return uniform_coords(n)
    if c is None:
        c = c_for_ratio(n, ratio, kind)
    return wall_coords(n, c) if kind == "wall" else centre_coords(n, c)


def rhs_gaussian(ny1: int, nx1: int, seed: int) -> np.ndarray:
    """f ~ N(0,1) at every node (boundary entries are never read)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((ny1, nx1))


def rhs_uniform(ny1: int, nx1: int, seed: int) -> np.ndarray:
    """f ~ U(-1,1), the paper's random right-hand side (Sec. 6)."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, (ny1, nx1))


def manufactured(x: np.ndarray, y: np.ndarray, noise: float = 0.0, seed: int = 0):
    """u* = sin(pi x) sin(pi y) (zero on the unit-square boundary) and the
    right-hand side f = -2 pi^2 u* of div(grad u) = f, plus noise * max|f| *
    U(-1,1).  Returns (u_exact, f)."""
    X, Y = np.meshgrid(x, y)
    ue = np.sin(math.pi * X) * np.sin(math.pi * Y)
    f = -2.0 * math.pi ** 2 * ue
    if noise:
        g = np.random.Generator(np.random.PCG64(seed))
        f = f + noise * np.abs(f).max() * g.uniform(-1.0, 1.0, f.shape)
    return ue, f


def random_field(ny1: int, nx1: int, seed: int) -> np.ndarray:
    """Zero-boundary random field (an initial error / guess)."""
    a = np.random.Generator(np.random.PCG64(seed)).standard_normal((ny1, nx1))
    a[0, :] = a[-1, :] = 0.0
    a[:, 0] = a[:, -1] = 0.0
    return a
