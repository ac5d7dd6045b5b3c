"""Seeded synthetic inputs shaped like the paper's workloads.

This module only generates distributions on the velocity grid; it holds none of the
collision-operator arithmetic and imports neither the CUDA library nor the oracle, so
both sides of a parity test can draw the same inputs from it.

Workloads (paper arxiv 1608.08009):
  * two_maxwellians -- per cell, f = sum of two Maxwellians with density U[0.5, 2],
    bulk velocity per component N(0, 0.3^2), temperature U[0.5, 1.5] (the mixed states
    a transport substep leaves in a cell, Sec. 3.1; Maxwellian of Sec. 2).
  * two_gaussians_test13 -- the hard-sphere relaxation datum of Test 1.3 (Sec. 5):
    two Gaussians of variance 0.2 centred at +-(-1, -1, -0.25), total mass 1.
  * bkw -- the 3D BKW datum for Maxwell molecules at shape parameter K (rho = 1, T = 1).
  * two_maxwellians_2d -- the two-Maxwellian cells in two velocity dimensions (the 2D
    Maxwell-molecule grids of Sec. 3.3).
  * sod_states -- the two equilibrium states of the Sod-like Riemann problem of Part 2 of
    the numerics (rho = 1, u = 0, T = 2.5 left of the middle; 0.125, 0, 0.25 right).
"""

from __future__ import annotations

import math

import numpy as np


def velocity_axis(N: int, L: float) -> np.ndarray:
    """v_j = -L + j * 2L/N, j = 0..N-1 (grid placement reading: v = 0 is a node)."""
    return -L + (2.0 * L / N) * np.arange(N)


def _maxwellian(v, rho, u, T):
    vx = v[:, None, None]
    vy = v[None, :, None]
    vz = v[None, None, :]
    d2 = (vx - u[0]) ** 2 + (vy - u[1]) ** 2 + (vz - u[2]) ** 2
    return rho * (2.0 * math.pi * T) ** -1.5 * np.exp(-d2 / (2.0 * T))


def sod_states(N: int, L: float):
    """(left, right) Maxwellians [N, N, N] of the Sod-like data of Part 2: rho = 1, u = 0,
    T = 2.5 for x <= length / 2 and rho = 0.125, u = 0, T = 0.25 beyond."""
    v = velocity_axis(N, L)
    zero = (0.0, 0.0, 0.0)
    return _maxwellian(v, 1.0, zero, 2.5), _maxwellian(v, 0.125, zero, 0.25)


def two_maxwellian_params(n_cells: int, seed: int):
    """Per-cell (rho[2], u[2,3], T[2]) drawn from a numpy PCG64 stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = rng.uniform(0.5, 2.0, size=(n_cells, 2))
    u = rng.normal(0.0, 0.3, size=(n_cells, 2, 3))
    T = rng.uniform(0.5, 1.5, size=(n_cells, 2))
    return rho, u, T


def two_maxwellians(n_cells: int, N: int, L: float, seed: int, cells=None, dtype=np.float64) -> np.ndarray:
    """f[c, x, y, z] for the requested cells (default all) of a seeded batch.

    The parameters of cell c depend only on (seed, c), so any subset of cells can be
    regenerated exactly (used for sampled checks on large batches).
    """
    rho, u, T = two_maxwellian_params(n_cells, seed)
    v = velocity_axis(N, L)
    idx = range(n_cells) if cells is None else cells
    idx = list(idx)
    out = np.empty((len(idx), N, N, N), dtype=dtype)
    for o, c in enumerate(idx):
        out[o] = _maxwellian(v, rho[c, 0], u[c, 0], T[c, 0]) + _maxwellian(v, rho[c, 1], u[c, 1], T[c, 1])
    return out


def two_maxwellians_2d(n_cells: int, N: int, L: float, seed: int, cells=None, dtype=np.float64) -> np.ndarray:
    """2D cells f[c, x, y]: the sum of two 2D Maxwellians per cell with the parameters of
    two_maxwellians (density U[0.5, 2], drift N(0, 0.3^2) per component, temperature
    U[0.5, 1.5]; the third drift component is unused)."""
    rho, u, T = two_maxwellian_params(n_cells, seed)
    v = velocity_axis(N, L)
    VX, VY = v[:, None], v[None, :]
    idx = list(range(n_cells) if cells is None else cells)
    out = np.empty((len(idx), N, N), dtype=dtype)
    for o, c in enumerate(idx):
        f = 0.0
        for i in range(2):
            f = f + rho[c, i] / (2.0 * math.pi * T[c, i]) * np.exp(
                -((VX - u[c, i, 0]) ** 2 + (VY - u[c, i, 1]) ** 2) / (2.0 * T[c, i]))
        out[o] = f
    return out


def two_gaussians_test13(N: int, L: float, sigma2: float = 0.2, v1=(-1.0, -1.0, -0.25)) -> np.ndarray:
    """Test 1.3 initial datum: (1/2)[G(v - v1) + G(v + v1)], G of variance sigma2."""
    v = velocity_axis(N, L)
    u = np.asarray(v1, dtype=np.float64)
    return 0.5 * (_maxwellian(v, 1.0, u, sigma2) + _maxwellian(v, 1.0, -u, sigma2))


def bkw(N: int, L: float, K: float) -> np.ndarray:
    """3D BKW profile (2 pi K)^{-3/2} e^{-v^2/2K} [(5K-3)/(2K) + (1-K) v^2/(2K^2)]."""
    v = velocity_axis(N, L)
    v2 = v[:, None, None] ** 2 + v[None, :, None] ** 2 + v[None, None, :] ** 2
    return (2.0 * math.pi * K) ** -1.5 * np.exp(-v2 / (2.0 * K)) * ((5.0 * K - 3.0) / (2.0 * K) + (1.0 - K) * v2 / (2.0 * K * K))


def bkw_L_for_support(S: float) -> float:
    """Half-width L of the grid for support radius S: L = (3 + sqrt 2) S / 2 (Sec. 3.3)."""
    return (3.0 + math.sqrt(2.0)) * S / 2.0
