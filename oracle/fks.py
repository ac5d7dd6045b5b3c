"""Fast Kinetic Scheme in one space dimension: transport of the piecewise-constant
distribution coupled to the collision step (arxiv 1608.08009, Sec. 3.1).

TEST INFRASTRUCTURE ONLY (part of the oracle package; see its docstring).

What it computes, for cells j = 0 .. n_x - 1 of width dx along x (centres at
(j + 1/2) dx), velocities v_k of the 3D grid and time steps t^{n+1} = t^n + dt:

* Transport stage (Eq. transport, Eq. f_bar).  The piecewise-constant function
  fbar_k(x), constant on the intervals of the initial mesh, is advected exactly:
  fbar_k(x, t) = fbar_k(x - v_{k,x} t, 0).  Its intervals move as a whole, so after a
  time t the interval that started as cell i covers [i dx + s, (i + 1) dx + s) with
  s = v_x t, and the centre of cell j lies in the interval of index
  i = j - shift(v_x, t, dx), shift = ceil(s / dx - 1/2) (half-open intervals).  Sampling
  at the centres (the collision stage's input f*_{j,k}) therefore moves each x-velocity's
  values by the change of that shift over the step; values that enter the domain come
  from outside it: the fixed states left of x = 0 and right of x = n_x dx (the Dirichlet
  boundary conditions of Part 2 of the numerics).
* Collision stage (Eq. relax with the rescaled operator Q / tau of Part 2, forward Euler
  Eq. f_coll): f^{n+1}_j = Pi(f*_j + (dt / tau) Q(f*_j)), Pi the projection of Sec. 3.2
  onto the moments of f*_j (collisions conserve them).  By Eq. expdt the update belongs
  to the interval that covers the centre, so the new centre values are the masses of the
  moved intervals: no further reconstruction is needed.

The time t accumulates as t += dt once per step (the same floating-point sequence any
implementation of the scheme with this interface produces), and shift is evaluated from
it in float64.
"""

from __future__ import annotations

import math

import numpy as np

from .grid import VelocityGrid
from .operator import collide, moments, project_f


def shift(vx: float, t: float, dx: float) -> int:
    """Index shift of the interval covering a cell centre after the intervals moved by
    s = vx t: the centre of cell j lies in the interval that started as cell j - shift."""
    return int(math.ceil(vx * t / dx - 0.5))


def transport(f: np.ndarray, grid: VelocityGrid, t0: float, t1: float, dx: float, left: np.ndarray,
              right: np.ndarray) -> np.ndarray:
    """Centre values after the transport stage from t0 to t1 (Eq. f_bar).

    f: [n_x, N, N, N] centre values at t0 (x-velocity index on axis 1); left, right:
    [N, N, N] the states outside the domain.  Each x-velocity's column of cells moves by
    d = shift(t1) - shift(t0) cells; cells uncovered at the inflow side take the
    boundary state."""
    nx = f.shape[0]
    out = np.empty_like(f)
    for kx in range(grid.N):
        vx = float(grid.v[kx])
        d = shift(vx, t1, dx) - shift(vx, t0, dx)
        for j in range(nx):
            src = j - d
            if src < 0:
                out[j, kx] = left[kx]
            elif src >= nx:
                out[j, kx] = right[kx]
            else:
                out[j, kx] = f[src, kx]
    return out


def step(f: np.ndarray, grid: VelocityGrid, t: float, dt: float, dx: float, tau: float, left: np.ndarray,
         right: np.ndarray) -> np.ndarray:
    """One FKS step from time t: transport stage, then the collision stage
    f^{n+1}_j = Pi(f*_j + (dt / tau) Q(f*_j)) (Eq. f_coll, rescaled by 1 / tau)."""
    fs = transport(f, grid, t, t + dt, dx, left, right)
    U = moments(fs, grid)
    Q = collide(fs, grid, project=False)
    return project_f(fs + (dt / tau) * Q, U, grid)


def run(f0: np.ndarray, grid: VelocityGrid, dt: float, steps: int, dx: float, tau: float, left: np.ndarray,
        right: np.ndarray, collisions: bool = True) -> np.ndarray:
    """`steps` FKS steps from t = 0 (collisions = False: the transport stage alone)."""
    f = np.array(f0, dtype=np.float64)
    t = 0.0
    for _ in range(steps):
        if collisions:
            f = step(f, grid, t, dt, dx, tau, left, right)
        else:
            f = transport(f, grid, t, t + dt, dx, left, right)
        t += dt
    return f


def maxwellian(grid: VelocityGrid, rho: float, u: float, T: float) -> np.ndarray:
    """rho (2 pi T)^(-3/2) exp(-|v - (u, 0, 0)|^2 / (2 T)) on the grid (the local
    equilibrium of the Sod-like initial data of Part 2)."""
    vx, vy, vz = grid.velocities()
    return rho * (2.0 * np.pi * T) ** -1.5 * np.exp(-((vx - u) ** 2 + vy ** 2 + vz ** 2) / (2.0 * T))


def sod(grid: VelocityGrid, nx: int, length: float = 2.0):
    """Sod-like Riemann data of Part 2 on [0, length]: rho = 1, u = 0, T = 2.5 for
    x <= length / 2 and rho = 0.125, u = 0, T = 0.25 beyond, at local equilibrium.
    Returns (f0 [nx, N, N, N], left state, right state, dx)."""
    dx = length / nx
    fl = maxwellian(grid, 1.0, 0.0, 2.5)
    fr = maxwellian(grid, 0.125, 0.0, 0.25)
    xc = (np.arange(nx) + 0.5) * dx
    f0 = np.where((xc <= 0.5 * length)[:, None, None, None], fl[None], fr[None])
    return f0, fl, fr, dx
