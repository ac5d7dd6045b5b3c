"""Velocity grid, half-sphere direction sets and separated kernel tables (FP64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Paper references (arxiv 1608.08009):
  * Sec. 3.1, Eq. (DM): uniform velocity grid with step dv, f_k ~ f(v_k).
  * Sec. 3.3, truncation paragraph: f supported in a ball of radius S, periodised on
    [-T, T]^3 with T = (3 + sqrt 2) S / 2; here T is the half-width L of the grid, so
    S = 2 L / (3 + sqrt 2).  The Carleman balls have radius R; reading: R = 2 S (the
    classical kernel, Eq. KM, integrates |q| <= 2 lambda pi = 2 S, and for v, v* in
    B(S) the Carleman variables x = v' - v, y = v'* - v satisfy |x|, |y| <= |q| <= 2 S).
  * Sec. 3.3, Eqs. (FU)/(FC): Fourier modes k in {-N/2 .. N/2-1}^3; in physical units
    the wave vector of mode k is xi_k = (pi / L) k.
  * Sec. 3.3, Eq. (Btilde) with the VHS kernel B = C_gamma |q|^gamma gives
    Btilde(x, y) = 4 C_gamma (|x|^2 + |y|^2)^((gamma - 1) / 2) in 3D; constant for
    hard spheres (gamma = 1).
  * Sec. 3.3, 3D decoupling formula: B_F(l, m) = Btilde * int_{S^2_+} phi(xi_l . e)
    psi(|Pi_{e-perp} xi_m|) de with phi(s) = int_{-R}^{R} |rho| e^{i rho s} d rho =
    R^2 [2 Sinc(R s) - Sinc^2(R s / 2)] (the printed hard-sphere phi) and psi the
    Fourier transform of the disk of radius R in the plane e-perp,
    psi(s) = 2 pi R J1(R s) / s.  (Reading: the printed psi carries a sin(theta)
    factor that belongs to the area element of the outer half-sphere integral; with
    it inside psi the formula contradicts Eq. (FKM).  The pin
    tests/test_oracle_pins.py::test_kernel_l0_closed_form shows the difference.)
  * Sec. 3.3, quadrature on the half sphere: product grid in (theta, varphi), uniform
    in both angles.  Reading: midpoints theta_p = (p + 1/2) pi / A1,
    varphi_q = (q + 1/2) pi / A2 and weights (pi / A1)(pi / A2) sin(theta_p).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import special


def wave_numbers(N: int) -> np.ndarray:
    """Signed Fourier mode numbers k in FFT storage order (Sec. 3.3, Eq. FU).

    Index i holds k = i for i < N/2 and k = i - N otherwise, so the Nyquist mode
    k = -N/2 sits at index N/2.
    """
    i = np.arange(N)
    return np.where(i < N // 2, i, i - N)


def product_factors(M: int, a1: int | None = None) -> tuple[int, int]:
    """Split M directions into an A1 x A2 product grid (Sec. 3.3 quadrature formula).

    Reading: A1 (polar angles) is the smallest divisor of M with A1 >= sqrt(M); A2 =
    M / A1.  M = 64 gives 8 x 8, the paper's "eight angles" per loop (Sec. 4.2).
    """
    if a1 is not None:
        if a1 <= 0 or M % a1:
            raise ValueError("a1 must divide M")
        return a1, M // a1
    for a in range(1, M + 1):
        if M % a == 0 and a * a >= M:
            return a, M // a
    raise ValueError("bad M")


def directions(M: int, kind: int = 0, a1: int | None = None):
    """Unit vectors e_j on the half sphere S^2_+ and quadrature weights w_j.

    kind 0 -- the paper's product grid in (theta, varphi) (Sec. 3.3), midpoint reading,
              weight (pi/A1)(pi/A2) sin(theta_p) (the area element of S^2).
    kind 1 -- spherical-Fibonacci points on the upper half sphere, equal weights
              2 pi / M (a direction set the paper does not use; offered for the
              quasi-uniform configurations).
    kind 2 -- Gauss product rule: Gauss-Legendre in cos(theta) on [-1, 1] (A1 nodes) x
              midpoints in varphi on [0, pi) (A2 nodes), weight u_p pi / A2.  Uniform in
              varphi as the paper asks, but exact for spherical harmonics of degree
              < min(2 A1, 2 A2); the midpoint rule in theta of kind 0 is only second
              order because |sin(theta)| has a kink at the poles.
    Returns (e [M, 3], w [M]).  Weights sum to ~2 pi, the area of S^2_+.
    """
    if kind == 0:
        A1, A2 = product_factors(M, a1)
        theta = (np.arange(A1) + 0.5) * np.pi / A1
        varphi = (np.arange(A2) + 0.5) * np.pi / A2
        th, vp = np.meshgrid(theta, varphi, indexing="ij")
        e = np.stack([np.sin(th) * np.cos(vp), np.sin(th) * np.sin(vp), np.cos(th)], axis=-1).reshape(M, 3)
        w = ((np.pi / A1) * (np.pi / A2) * np.sin(th)).reshape(M)
        return e, w
    if kind == 1:
        j = np.arange(M)
        z = 1.0 - (j + 0.5) / M
        r = np.sqrt(1.0 - z * z)
        ang = j * (np.pi * (3.0 - math.sqrt(5.0)))
        e = np.stack([r * np.cos(ang), r * np.sin(ang), z], axis=-1)
        w = np.full(M, 2.0 * np.pi / M)
        return e, w
    if kind == 2:
        A1, A2 = product_factors(M, a1)
        ct, ut = np.polynomial.legendre.leggauss(A1)
        varphi = (np.arange(A2) + 0.5) * np.pi / A2
        c, vp = np.meshgrid(ct, varphi, indexing="ij")
        st = np.sqrt(1.0 - c * c)
        e = np.stack([st * np.cos(vp), st * np.sin(vp), c], axis=-1).reshape(M, 3)
        w = (ut[:, None] * (np.pi / A2) * np.ones_like(vp)).reshape(M)
        return e, w
    raise ValueError("unknown direction kind")


def sinc(x):
    """Sinc(x) = sin(x) / x with Sinc(0) = 1 (the paper's Sinc, Sec. 3.3)."""
    return np.sinc(np.asarray(x) / np.pi)


def phi_hs(s, R):
    """phi(s) = int_{-R}^{R} |rho| e^{i rho s} d rho = R^2 [2 Sinc(R s) - Sinc^2(R s/2)].

    The hard-sphere closed form printed in Sec. 3.3.
    """
    s = np.asarray(s, dtype=np.float64)
    return R * R * (2.0 * sinc(R * s) - sinc(0.5 * R * s) ** 2)


def psi_hs(s, R):
    """psi(s) = int over the disk of radius R in a plane of e^{i s y_1} d^2y = 2 pi R J1(R s) / s.

    psi(0) = pi R^2.  (Reading of the Sec. 3.3 decoupling formula; see module docstring.)
    """
    x = R * np.asarray(s, dtype=np.float64)
    small = np.abs(x) < 1e-6
    xs = np.where(small, 1.0, x)
    ratio = np.where(small, 0.5 - x * x / 16.0, special.j1(xs) / xs)  # J1(x)/x
    return 2.0 * np.pi * R * R * ratio


def psi_printed(s, R):
    """The psi printed in Sec. 3.3 for hard spheres, 2 R^2 Sinc^2(R s / 2).

    Kept only so the pins can show that it does not reproduce Eq. (FKM).
    """
    return 2.0 * R * R * sinc(0.5 * R * np.asarray(s, dtype=np.float64)) ** 2


def gauss_legendre(n: int, a: float, b: float):
    """Gauss-Legendre nodes and weights on [a, b] (numpy's leggauss, mapped)."""
    x, u = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * u


@dataclasses.dataclass
class VelocityGrid:
    N: int
    L: float
    gamma: float
    C_gamma: float
    S: float                 # support radius of f
    R: float                 # Carleman ball radius
    dv: float
    v: np.ndarray            # [N] grid coordinates per axis
    k: np.ndarray            # [N] signed mode numbers (FFT order)
    xi: np.ndarray           # [N] wave numbers pi k / L
    e: np.ndarray            # [M, 3] directions
    w_dir: np.ndarray        # [M] direction weights
    rank: int                # radial rank (1 = closed-form hard spheres)
    w: np.ndarray            # [M * rank] weights of the separated terms
    alpha: np.ndarray        # [M * rank, N, N, N]
    alphap: np.ndarray       # [M * rank, N, N, N]
    D: np.ndarray            # [N, N, N] loss multiplier sum_i w_i alpha_i alphap_i

    @property
    def n(self) -> int:
        return self.N ** 3

    @property
    def M_eff(self) -> int:
        return self.w.shape[0]

    def velocities(self):
        """Broadcastable (vx, vy, vz) arrays of shape [N,1,1], [1,N,1], [1,1,N]."""
        return self.v[:, None, None], self.v[None, :, None], self.v[None, None, :]

    def wave_vectors(self):
        return self.xi[:, None, None], self.xi[None, :, None], self.xi[None, None, :]


def btilde(gamma: float, C_gamma: float, r1, r2):
    """Btilde(|x|, |y|) = 4 C_gamma (|x|^2 + |y|^2)^((gamma-1)/2), Eq. (Btilde), 3D VHS."""
    return 4.0 * C_gamma * (np.asarray(r1) ** 2 + np.asarray(r2) ** 2) ** (0.5 * (gamma - 1.0))


def _perp_norm(KX, KY, KZ, e):
    """|Pi_{e-perp} xi| = |xi x e| for a unit vector e (Sec. 3.3, argument of psi).

    The cross product is used instead of sqrt(|xi|^2 - (xi . e)^2), which loses all
    accuracy when xi is nearly parallel to e.
    """
    cx = KY * e[2] - KZ * e[1]
    cy = KZ * e[0] - KX * e[2]
    cz = KX * e[1] - KY * e[0]
    return np.sqrt(cx * cx + cy * cy + cz * cz)


def kernel_tables(N, L, e, w_dir, gamma=1.0, C_gamma=1.0, R=None, rank=None, inner_nodes=None):
    """alpha_i(k), alpha'_i(k), weights w_i and D(k) on the full N^3 mode set.

    rank == 1 (hard spheres, gamma = 1, Btilde constant; Sec. 3.3):
        alpha_j = Btilde phi(xi_k . e_j),  alpha'_j = psi(|xi_k - (xi_k . e_j) e_j|).
    rank > 1 (reading for gamma != 1, where Eq. (decoup) fails in 3D): Gauss-Legendre
        nodes rho_r, weights u_r on [0, R] for |x| give
        alpha_{j,r} = 2 u_r rho_r cos(rho_r xi_k . e_j),
        alpha'_{j,r} = 2 pi int_0^R rho' Btilde(rho_r, rho') J0(rho' |Pi xi_k|) d rho'
        (inner integral by Gauss-Legendre with `inner_nodes` nodes); w_{j,r} = w_j.
    D(k) = sum_i w_i alpha_i(k) alpha'_i(k) = K(k, k), the Carleman loss multiplier.
    """
    S = 2.0 * L / (3.0 + math.sqrt(2.0))
    if R is None or R <= 0:
        R = 2.0 * S
    if rank is None:
        rank = 1 if gamma == 1.0 else 16
    if inner_nodes is None:
        inner_nodes = 128
    xi = np.pi * wave_numbers(N) / L
    KX, KY, KZ = np.meshgrid(xi, xi, xi, indexing="ij")
    M = e.shape[0]
    Meff = M * rank
    alpha = np.empty((Meff, N, N, N))
    alphap = np.empty((Meff, N, N, N))
    w = np.repeat(w_dir, rank)
    if rank == 1:
        if gamma != 1.0:
            raise ValueError("rank 1 is exact only for hard spheres (gamma = 1)")
        bt = 4.0 * C_gamma
        for j in range(M):
            s = KX * e[j, 0] + KY * e[j, 1] + KZ * e[j, 2]
            perp = _perp_norm(KX, KY, KZ, e[j])
            alpha[j] = bt * phi_hs(s, R)
            alphap[j] = psi_hs(perp, R)
    else:
        rho, u = gauss_legendre(rank, 0.0, R)
        rq, uq = gauss_legendre(inner_nodes, 0.0, R)
        for j in range(M):
            s = KX * e[j, 0] + KY * e[j, 1] + KZ * e[j, 2]
            perp = _perp_norm(KX, KY, KZ, e[j])
            j0 = special.j0(rq[:, None] * perp.reshape(1, -1))  # [inner, n]
            for r in range(rank):
                alpha[j * rank + r] = 2.0 * u[r] * rho[r] * np.cos(rho[r] * s)
                g = uq * rq * btilde(gamma, C_gamma, rho[r], rq)  # [inner]
                alphap[j * rank + r] = (2.0 * np.pi * (g @ j0)).reshape(N, N, N)
    D = np.einsum("i,ixyz,ixyz->xyz", w, alpha, alphap)
    return S, R, rank, w, alpha, alphap, D


def make_grid(N: int, L: float, gamma: float = 1.0, M: int = 64, dirs_kind: int = 0,
              C_gamma: float = 1.0, R_trunc: float | None = None, rank: int | None = None,
              inner_nodes: int | None = None, a1: int | None = None) -> VelocityGrid:
    """Build the full grid description used by every oracle routine."""
    if N % 2 or N < 4:
        raise ValueError("N must be even and >= 4")
    e, w_dir = directions(M, dirs_kind, a1)
    S, R, rank, w, alpha, alphap, D = kernel_tables(N, L, e, w_dir, gamma, C_gamma, R_trunc, rank, inner_nodes)
    dv = 2.0 * L / N
    v = -L + dv * np.arange(N)
    k = wave_numbers(N)
    return VelocityGrid(N=N, L=L, gamma=gamma, C_gamma=C_gamma, S=S, R=R, dv=dv, v=v, k=k,
                        xi=np.pi * k / L, e=e, w_dir=w_dir, rank=rank, w=w, alpha=alpha,
                        alphap=alphap, D=D)
