"""Spectral transforms, the fast collision operator, projection, moments, time step (FP64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Paper references (arxiv 1608.08009):
  * Sec. 3.3, Eqs. (FU)/(FC): f_N(v) = sum_k fhat_k e^{i xi_k . v},
    fhat_k = (2 pi)^-3 int f e^{-i xi_k . v} dv  -> on the grid (rectangle rule, which
    is exact for trigonometric polynomials) fhat_k = n^-1 sum_j f(v_j) e^{-i xi_k . v_j}.
  * Sec. 3.3, Eq. (ode) with the separated approximation of beta_F: Q-hat_k =
    sum_{l+m=k} [K(l,m) - K(m,m)] fhat_l fhat_m, K(l,m) = sum_i w_i alpha_i(l) alpha'_i(m).
    In physical space (Sec. 4.2: one forward transform, then per direction the
    coefficients and inverse transforms, then the gather into Q):
        Q+(v) = sum_i w_i [sum_l alpha_i(l) fhat_l e^{i xi_l v}] [sum_m alpha'_i(m) fhat_m e^{i xi_m v}]
        L(v)  = sum_m D(m) fhat_m e^{i xi_m v},   D(m) = K(m, m)
        Q(v)  = Q+(v) - f(v) L(v).
    Readings: the sum over l + m = k is the circular one (mod N) that the product of
    two trigonometric polynomials takes on the grid; every mode with a component equal
    to -N/2 is removed from fhat before the products so that each inverse transform is
    exactly real; the loss multiplies the grid values f(v) themselves.
  * Sec. 3.2, Eq. (minim1): f = f~ + C^T (C C^T)^-1 (U - C f~) with the rows of C the
    discrete collision invariants (1, v, |v|^2/2) dv^3 (the paper writes |v|^2; the
    factor 1/2 only rescales a row and leaves the projection unchanged).
  * Sec. 3.1, Eq. (f_coll): forward Euler f^{n+1} = f^n + dt Q(f^n), projected after
    every collision step (Sec. 3.2).  Reading for second order: Heun's method with the
    same projection after each stage.
  * Eq. (i5) / (DM): moments U = (rho, rho u, E) = sum_k (1, v_k, |v_k|^2 / 2) f_k dv^3.
"""

from __future__ import annotations

import numpy as np

from .grid import VelocityGrid

_AX = (-3, -2, -1)


def _phase(grid: VelocityGrid, sign: float) -> np.ndarray:
    """exp(sign * i * L * (xi_x + xi_y + xi_z)) on the mode grid.

    Since v_j = -L + j dv and xi_k j dv = 2 pi k j / N, the kernel of Eq. (FC) on the
    grid is e^{-i xi_k . v_j} = e^{+i L sum(xi_k)} e^{-2 pi i k . j / N}.
    """
    px = np.exp(sign * 1j * grid.L * grid.xi)
    return px[:, None, None] * px[None, :, None] * px[None, None, :]


def nyquist_mask(grid: VelocityGrid) -> np.ndarray:
    """True at every mode with some component k_d = -N/2."""
    nyq = grid.k == -(grid.N // 2)
    return nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :]


def forward(f: np.ndarray, grid: VelocityGrid, zero_nyquist: bool = True) -> np.ndarray:
    """fhat_k = n^-1 sum_j f(v_j) e^{-i xi_k . v_j} over the last three axes (Eq. FC)."""
    fh = np.fft.fftn(f, axes=_AX) / grid.n * _phase(grid, +1.0)
    if zero_nyquist:
        fh = np.where(nyquist_mask(grid), 0.0, fh)
    return fh


def inverse(gh: np.ndarray, grid: VelocityGrid) -> np.ndarray:
    """g(v_j) = sum_k ghat_k e^{i xi_k . v_j} over the last three axes (Eq. FU)."""
    return np.fft.ifftn(gh * _phase(grid, -1.0), axes=_AX) * grid.n


def gain_loss(f: np.ndarray, grid: VelocityGrid):
    """Return (Q+, L) of the fast method for f of shape [..., N, N, N]."""
    fh = forward(f, grid)
    Qp = np.zeros(f.shape)
    for i in range(grid.M_eff):
        g1 = inverse(grid.alpha[i] * fh, grid).real
        g2 = inverse(grid.alphap[i] * fh, grid).real
        Qp += grid.w[i] * g1 * g2
    Lo = inverse(grid.D * fh, grid).real
    return Qp, Lo


def collide(f: np.ndarray, grid: VelocityGrid, project: bool = True) -> np.ndarray:
    """Fast spectral Q(f, f) on the grid (Sec. 3.3 and Sec. 4.2), optionally projected.

    f has shape [..., N, N, N] (cells first), values f(v_x, v_y, v_z) with v_z fastest.
    """
    f = np.asarray(f, dtype=np.float64)
    Qp, Lo = gain_loss(f, grid)
    Q = Qp - f * Lo
    if project:
        Q = project_Q(Q, grid)
    return Q


def _shift_index(grid: VelocityGrid) -> np.ndarray:
    """idx[k, l] = flat index of the mode k - l (mod N per component)."""
    N = grid.N
    a = np.arange(N)
    kx, ky, kz = np.meshgrid(a, a, a, indexing="ij")
    kx, ky, kz = kx.ravel(), ky.ravel(), kz.ravel()
    mx = (kx[:, None] - kx[None, :]) % N
    my = (ky[:, None] - ky[None, :]) % N
    mz = (kz[:, None] - kz[None, :]) % N
    return (mx * N + my) * N + mz


def collide_brute_force(f: np.ndarray, grid: VelocityGrid, project: bool = False) -> np.ndarray:
    """Q from the O(n^2) wrapped spectral sum (Eq. ode with the separated kernel).

    Q-hat_k = sum_l fhat_l fhat_{k-l} K(l, k-l) - fhat^u_l D(k-l) fhat_{k-l}, with
    K(l, m) = sum_i w_i alpha_i(l) alpha'_i(m), fhat Nyquist-free and fhat^u the
    transform of f itself (the loss multiplies the grid values of f).  Small N only.
    """
    f = np.asarray(f, dtype=np.float64)
    n = grid.n
    A = grid.alpha.reshape(grid.M_eff, n)
    Ap = grid.alphap.reshape(grid.M_eff, n)
    K = (A * grid.w[:, None]).T @ Ap           # [l, m]
    Dm = grid.D.reshape(n)
    idx = _shift_index(grid)                     # [k, l] -> m
    lidx = np.arange(n)[None, :]
    Kkl = K[lidx, idx]                           # K(l, k - l)
    single = f.ndim == 3
    fb = f[None] if single else f
    out = np.empty(fb.shape)
    for c in range(fb.shape[0]):
        fh = forward(fb[c], grid).reshape(n)
        fhu = forward(fb[c], grid, zero_nyquist=False).reshape(n)
        fm = fh[idx]                             # fhat_{k-l}
        Qh = np.sum(fh[None, :] * fm * Kkl - fhu[None, :] * fm * Dm[idx], axis=1)
        out[c] = inverse(Qh.reshape(grid.N, grid.N, grid.N), grid).real
    if project:
        out = project_Q(out, grid)
    return out[0] if single else out


def constraint_matrix(grid: VelocityGrid) -> np.ndarray:
    """C [5, n]: rows (1, v_x, v_y, v_z, |v|^2 / 2) dv^3 in (x, y, z) C order (Sec. 3.2)."""
    vx, vy, vz = np.meshgrid(grid.v, grid.v, grid.v, indexing="ij")
    rows = [np.ones_like(vx), vx, vy, vz, 0.5 * (vx * vx + vy * vy + vz * vz)]
    return np.stack([r.ravel() for r in rows]) * grid.dv ** 3


def _projector(grid: VelocityGrid) -> tuple[np.ndarray, np.ndarray]:
    C = constraint_matrix(grid)
    P = np.linalg.solve(C @ C.T, C).T            # C^T (C C^T)^-1, shape [n, 5]
    return C, P


def moments(f: np.ndarray, grid: VelocityGrid) -> np.ndarray:
    """U = (rho, rho u_x, rho u_y, rho u_z, E) for f [..., N, N, N] (Eq. DM)."""
    C = constraint_matrix(grid)
    fl = np.asarray(f, dtype=np.float64).reshape(*np.shape(f)[:-3], grid.n)
    return fl @ C.T


def project_f(ft: np.ndarray, U: np.ndarray, grid: VelocityGrid) -> np.ndarray:
    """f = f~ + C^T (C C^T)^-1 (U - C f~) (Eq. minim1)."""
    C, P = _projector(grid)
    shp = ft.shape
    fl = ft.reshape(*shp[:-3], grid.n)
    r = np.asarray(U) - fl @ C.T
    return (fl + r @ P.T).reshape(shp)


def project_Q(Q: np.ndarray, grid: VelocityGrid) -> np.ndarray:
    """Q - C^T (C C^T)^-1 C Q: Eq. (minim1) applied to f~ = f + dt Q with U = C f."""
    return project_f(Q, np.zeros(Q.shape[:-3] + (5,)), grid)


def relax(f: np.ndarray, grid: VelocityGrid, dt: float, steps: int, rk_order: int = 1) -> np.ndarray:
    """Homogeneous relaxation df/dt = Q(f) (Eq. relax), projected onto U0 = moments(f0).

    rk_order 1: f <- Pi(f + dt Q(f))                       (Eq. f_coll + Eq. minim1)
    rk_order 2: f1 = Pi(f + dt Q(f)); f <- Pi(f/2 + (f1 + dt Q(f1))/2)   (Heun; reading)
    Pi(g) = g + C^T (C C^T)^-1 (U0 - C g).
    """
    f = np.array(f, dtype=np.float64)
    U0 = moments(f, grid)
    for _ in range(steps):
        if rk_order == 1:
            f = project_f(f + dt * collide(f, grid, project=False), U0, grid)
        elif rk_order == 2:
            f1 = project_f(f + dt * collide(f, grid, project=False), U0, grid)
            f = project_f(0.5 * f + 0.5 * (f1 + dt * collide(f1, grid, project=False)), U0, grid)
        else:
            raise ValueError("rk_order must be 1 or 2")
    return f
