"""Two-dimensional fast spectral operator for Maxwell molecules (FP64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Paper references (arxiv 1608.08009):
  * Sec. 3.3, dimension two.  For Maxwell molecules in 2D the Carleman kernel Btilde is
    a constant, so the decoupling assumption (Eq. decoup) holds exactly.  With
    x = rho e, y = rho' e' (rho, rho' in [-R, R], e, e' on the unit circle) the kernel
    becomes B_F(l, m) = Btilde int_0^pi phi2(xi_l . e_theta) phi2(xi_m . e_{theta+pi/2})
    d theta, where phi2(s) = int_{-R}^{R} e^{i rho s} d rho = 2 R Sinc(R s).
  * Eq. (dfor0): the theta integral is periodic, so A equally spaced angles
    theta_p = pi p / A with weight pi / A are spectrally accurate:
    alpha_p(l) = Btilde phi2(xi_l . e_p), alpha'_p(m) = phi2(xi_m . e_p-perp).
  * The rest is the 3D algorithm of the operator module in two dimensions: the grid
    v_j = -L + j dv, modes k in {-N/2 .. N/2-1}^2 with xi_k = pi k / L, every mode with a
    component -N/2 removed, Q = Q+ - f L with L = inverse(D fhat), D = sum_p w_p
    alpha_p alpha'_p, the projection of Sec. 3.2 (Eq. minim1) on the invariants
    (1, v_x, v_y, |v|^2/2) dv^2, forward Euler (Eq. f_coll) or Heun.
  * Sec. 3.3 truncation rule, as in 3D: support radius S = 2 L / (3 + sqrt 2), Carleman
    radius R = 2 S.
  * Sec. 5, Test 1.1: the 2D BKW solution
    f(v, t) = exp(-v^2 / (2 K)) [2 K - 1 + (1 - K) v^2 / (2 K)] / (2 pi K^2),
    K(t) = 1 - exp(-t / 8) / 2 (the paper calls K "S"); f(v, 0) = v^2 exp(-v^2) / pi.
    Reading of the normalisation: the closed form holds for the collision kernel
    B = 1 / (2 pi) on the unit circle, i.e. Btilde = 2 B = 1 / pi (Eq. Btilde with
    d_v = 2); the residual pin in tests/test_oracle_plane.py checks it.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

_AX = (-2, -1)


def sinc(x):
    """Sinc(x) = sin(x) / x with Sinc(0) = 1."""
    return np.sinc(np.asarray(x) / np.pi)


def phi2(s, R):
    """phi2(s) = int_{-R}^{R} e^{i rho s} d rho = 2 R Sinc(R s) (Sec. 3.3, dimension two)."""
    return 2.0 * R * sinc(R * np.asarray(s, dtype=np.float64))


@dataclasses.dataclass
class PlaneGrid:
    N: int
    L: float
    A: int                   # number of angles
    Btilde: float
    S: float
    R: float
    dv: float
    v: np.ndarray            # [N]
    k: np.ndarray            # [N] signed mode numbers (FFT order)
    xi: np.ndarray           # [N]
    theta: np.ndarray        # [A]
    w: np.ndarray            # [A]
    alpha: np.ndarray        # [A, N, N]
    alphap: np.ndarray       # [A, N, N]
    D: np.ndarray            # [N, N]

    @property
    def n(self) -> int:
        return self.N * self.N


def make_plane_grid(N: int, L: float, A: int = 8, Btilde: float = 1.0 / math.pi, R: float | None = None) -> PlaneGrid:
    """Grid, angles and separated tables of the 2D Maxwell-molecule operator."""
    if N % 2 or N < 4:
        raise ValueError("N must be even and >= 4")
    S = 2.0 * L / (3.0 + math.sqrt(2.0))
    if R is None or R <= 0:
        R = 2.0 * S
    dv = 2.0 * L / N
    v = -L + dv * np.arange(N)
    k = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    xi = np.pi * k / L
    theta = np.pi * np.arange(A) / A
    w = np.full(A, np.pi / A)
    XI, ETA = np.meshgrid(xi, xi, indexing="ij")
    alpha = np.empty((A, N, N))
    alphap = np.empty((A, N, N))
    for p, th in enumerate(theta):
        c, s = math.cos(th), math.sin(th)
        alpha[p] = Btilde * phi2(XI * c + ETA * s, R)      # xi . e_p
        alphap[p] = phi2(-XI * s + ETA * c, R)             # xi . e_p-perp
    D = np.einsum("p,pij,pij->ij", w, alpha, alphap)
    return PlaneGrid(N, L, A, Btilde, S, R, dv, v, k, xi, theta, w, alpha, alphap, D)


def _phase(g: PlaneGrid, sign: float) -> np.ndarray:
    p = np.exp(sign * 1j * g.L * g.xi)
    return p[:, None] * p[None, :]


def _nyquist(g: PlaneGrid) -> np.ndarray:
    nyq = g.k == -(g.N // 2)
    return nyq[:, None] | nyq[None, :]


def forward(f: np.ndarray, g: PlaneGrid, zero_nyquist: bool = True) -> np.ndarray:
    """fhat_k = n^-1 sum_j f(v_j) e^{-i xi_k . v_j}, Nyquist modes removed unless asked."""
    fh = np.fft.fft2(f, axes=_AX) / g.n * _phase(g, +1.0)
    return np.where(_nyquist(g), 0.0, fh) if zero_nyquist else fh


def inverse(h: np.ndarray, g: PlaneGrid) -> np.ndarray:
    """sum_k h_k e^{i xi_k . v_j} on the grid."""
    return np.fft.ifft2(h * _phase(g, -1.0), axes=_AX) * g.n


def gain_loss(f: np.ndarray, g: PlaneGrid):
    """(Q+, L) of the fast method for f of shape [..., N, N]."""
    fh = forward(f, g)
    Qp = np.zeros(f.shape)
    for p in range(g.A):
        Qp += g.w[p] * inverse(g.alpha[p] * fh, g).real * inverse(g.alphap[p] * fh, g).real
    return Qp, inverse(g.D * fh, g).real


def constraint_matrix(g: PlaneGrid) -> np.ndarray:
    """Rows (1, v_x, v_y, |v|^2/2) dv^2 at every grid point (x fastest-last order)."""
    VX, VY = np.meshgrid(g.v, g.v, indexing="ij")
    rows = [np.ones_like(VX), VX, VY, 0.5 * (VX * VX + VY * VY)]
    return np.stack([r.ravel() for r in rows]) * g.dv ** 2


def moments(f: np.ndarray, g: PlaneGrid) -> np.ndarray:
    """(rho, rho u_x, rho u_y, E) of f [..., N, N]."""
    C = constraint_matrix(g)
    return f.reshape(f.shape[:-2] + (-1,)) @ C.T


def project_f(ft: np.ndarray, U: np.ndarray, g: PlaneGrid) -> np.ndarray:
    """f = f~ + C^T (C C^T)^-1 (U - C f~) (Sec. 3.2, Eq. minim1)."""
    C = constraint_matrix(g)
    flat = ft.reshape(ft.shape[:-2] + (-1,))
    lam = np.linalg.solve(C @ C.T, (U - flat @ C.T)[..., None])[..., 0]
    return (flat + lam @ C).reshape(ft.shape)


def collide(f: np.ndarray, g: PlaneGrid, project: bool = True) -> np.ndarray:
    """Q = Q+ - f L, optionally projected so that its moments vanish."""
    Qp, Lo = gain_loss(f, g)
    Q = Qp - f * Lo
    if project:
        Q = project_f(Q, np.zeros(Q.shape[:-2] + (4,)), g)
    return Q


def collide_brute_force(f: np.ndarray, g: PlaneGrid) -> np.ndarray:
    """Wrapped O(n^2) spectral sum (Eq. ode with the separated kernel), unprojected:
    Q-hat_k = sum_{l+m = k mod N} [K(l, m) fhat_l - D(m) fhat^u_l] fhat_m with
    K(l, m) = sum_p w_p alpha_p(l) alpha'_p(m), fhat Nyquist-free and fhat^u the
    transform of f itself (the loss multiplies the grid values of f)."""
    N = g.N
    fh = forward(f, g)
    fhu = forward(f, g, zero_nyquist=False)
    Qh = np.zeros(f.shape[:-2] + (N, N), dtype=complex)
    # FFT-order indices add like the mode numbers mod N, so shifting the m-array by l
    # places the term of (l, m) at k = l + m (mod N)
    for l0 in range(N):
        for l1 in range(N):
            K = np.einsum("p,p,pij->ij", g.w, g.alpha[:, l0, l1], g.alphap)  # K(l, m) over m
            term = (K * fh[..., l0, l1][..., None, None] - g.D * fhu[..., l0, l1][..., None, None]) * fh
            Qh += np.roll(np.roll(term, l0, axis=-2), l1, axis=-1)
    return inverse(Qh, g).real


def relax(f: np.ndarray, g: PlaneGrid, dt: float, steps: int, rk_order: int = 1) -> np.ndarray:
    """Forward Euler (Eq. f_coll) or Heun, projected onto the initial moments each stage."""
    U0 = moments(f, g)
    for _ in range(steps):
        Q = collide(f, g, project=False)
        f1 = project_f(f + dt * Q, U0, g)
        if rk_order == 1:
            f = f1
        else:
            Q1 = collide(f1, g, project=False)
            f = project_f(0.5 * f + 0.5 * (f1 + dt * Q1), U0, g)
    return f


def bkw(g: PlaneGrid, t: float) -> np.ndarray:
    """2D BKW solution of Test 1.1 (Sec. 5) on the grid, K(t) = 1 - exp(-t/8)/2."""
    K = 1.0 - 0.5 * math.exp(-t / 8.0)
    VX, VY = np.meshgrid(g.v, g.v, indexing="ij")
    v2 = VX * VX + VY * VY
    return np.exp(-v2 / (2.0 * K)) * (2.0 * K - 1.0 + (1.0 - K) * v2 / (2.0 * K)) / (2.0 * math.pi * K * K)


def bkw_dt(g: PlaneGrid, t: float, h: float = 1e-4) -> np.ndarray:
    """Central difference of bkw in t."""
    return (bkw(g, t + h) - bkw(g, t - h)) / (2.0 * h)
