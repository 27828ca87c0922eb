"""Seeded synthetic initial states.

This module is shared by the tests, ``bench.py`` and ``smoke()``. It holds only
random draws and the definitions of the initial fields: none of the time
advancing arithmetic. Every array it returns is host (numpy) memory, laid out
as the library expects: ``nv`` planes of ``ny x nx``, row-major, x fastest.

Generators (numpy ``default_rng``, PCG64):

* ``uniform``      -- i.i.d. U[0, 1) per point.
* ``fourier_mode`` -- sin(2 pi p x / nx) sin(2 pi q y / ny) on integer x, y.
* ``smooth_field`` -- a sum of ``nmodes`` plane waves; integer wave vectors
  (kx, ky) uniform in [-kmax, kmax]^2 without (0, 0), amplitude N(0,1)/|k|^2,
  phase U[0, 2 pi).
* ``euler_pulse``  -- rho = 1 + 0.1 phi, u = v = 0, p = 1 + 0.1 phi (or p = 1
  with ``literal=True``), phi a 16-mode smooth field scaled to max |phi| = 1;
  returned as the conserved variables (rho, rho u, rho v, E) with
  E = p / (gamma - 1).
* ``random_words`` -- i.i.d. 64-bit words.
* ``wave_source``  -- a Gaussian bump of width ``sigma`` grid points at the
  centre of the grid (the wave equation's initial source), at rest.
"""
from __future__ import annotations

import numpy as np


def uniform(nx: int, ny: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random((ny, nx))


def fourier_mode(nx: int, ny: int, p: int, q: int) -> np.ndarray:
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    return np.outer(np.sin(2.0 * np.pi * q * y / ny), np.sin(2.0 * np.pi * p * x / nx))


def smooth_field(nx: int, ny: int, seed: int, nmodes: int = 32, kmax: int = 8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    out = np.zeros((ny, nx))
    made = 0
    while made < nmodes:
        kx, ky = (int(v) for v in rng.integers(-kmax, kmax + 1, size=2))
        if kx == 0 and ky == 0:
            continue
        k2 = float(kx * kx + ky * ky)
        amp = rng.standard_normal() / k2
        phase = rng.uniform(0.0, 2.0 * np.pi)
        out += amp * np.cos(2.0 * np.pi * (kx * x / nx + ky * y / ny) + phase)
        made += 1
    return out


def euler_pulse(nx: int, ny: int, seed: int, gamma: float = 1.4, literal: bool = False,
                nmodes: int = 16) -> np.ndarray:
    phi = smooth_field(nx, ny, seed, nmodes=nmodes)
    phi = phi / np.max(np.abs(phi))
    rho = 1.0 + 0.1 * phi
    p = np.ones_like(rho) if literal else 1.0 + 0.1 * phi
    U = np.zeros((4, ny, nx))
    U[0] = rho
    U[3] = p / (gamma - 1.0)
    return U


def random_words(nx: int, ny: int, seed: int, nv: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**64, size=(nv, ny, nx), dtype=np.uint64)


def wave_source(nx: int, ny: int, sigma: float = 4.0) -> np.ndarray:
    """(u^0, u^{-1}) of a source at rest at the grid centre, shape (2, ny, nx)."""
    x = np.arange(nx, dtype=np.float64)[None, :] - nx / 2
    y = np.arange(ny, dtype=np.float64)[:, None] - ny / 2
    u = np.exp(-(x * x + y * y) / (sigma * sigma))
    return np.stack([u, u.copy()])
