"""Seeded synthetic inputs shared by the GPU tests, the oracle tests and the benchmark.

This module only draws random numbers and arranges them in the layouts the rest of the
code expects; it holds none of the method's arithmetic (no fluxes, no growth factors, no
Philox, no spectra). Every array is float64 numpy; callers cast to what they need.

Layouts: gas state [5, n, n, n] (rho, m_x, m_y, m_z, eps), C order [z][y][x];
particle arrays [3, n^3] in Lagrangian order (x, y, z components).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def gas_state(n: int, seed: int, rho_mean: float = 0.16, rho_rel: float = 0.3,
              vel: float = 0.05, pressure: float = 1e-4, gamma: float = 5.0 / 3.0,
              shape=None):
    """A smooth-ish random gas state: density rho_mean (1 + rho_rel * r), velocities of
    rms `vel`, positive pressure around `pressure`. Energy eps = P / (gamma - 1) +
    |m|^2 / (2 rho). Values are drawn per cell and lightly smoothed over neighbours so the
    limiter sees both smooth regions and sign changes."""
    g = rng(seed)
    shp = tuple(shape) if shape is not None else (n, n, n)

    def smooth(x):
        y = x.copy()
        for ax in range(x.ndim):
            if x.shape[ax] > 2:
                y = (np.roll(y, 1, ax) + 2 * y + np.roll(y, -1, ax)) / 4
        return y

    rho = rho_mean * (1 + rho_rel * np.tanh(smooth(g.normal(size=shp))))
    v = vel * smooth(g.normal(size=(3,) + shp))
    P = pressure * (1 + 0.5 * np.tanh(smooth(g.normal(size=shp))))
    m = rho * v
    eps = P / (gamma - 1) + (m * m).sum(0) / (2 * rho)
    return np.concatenate([rho[None], m, eps[None]])


def displacements(n: int, seed: int, scale: float):
    """Random particle displacements [3, n^3] of rms `scale` (same units as the box)."""
    return scale * rng(seed).normal(size=(3, n ** 3))


def momenta(n: int, seed: int, scale: float):
    return scale * rng(seed).normal(size=(3, n ** 3))


def field(n: int, seed: int, scale: float = 1.0, shape=None):
    """A white Gaussian field [n, n, n] (or `shape`)."""
    shp = tuple(shape) if shape is not None else (n, n, n)
    return scale * rng(seed).normal(size=shp)


def white_noise(n: int, seed: int):
    """Standard normal white noise for the initial conditions (numpy generator; the
    simulator's own Philox noise is a separate, method-defined stream)."""
    return rng(seed).normal(size=(n, n, n))


def uniform_params(seed: int, count: int, ranges: dict):
    """`count` parameter draws, each key uniform in its (lo, hi) range."""
    g = rng(seed)
    return [{k: float(g.uniform(lo, hi)) for k, (lo, hi) in ranges.items()} for _ in range(count)]
