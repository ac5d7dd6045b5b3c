"""Closed forms and independent quadratures that pin the oracle (FP64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  None of these routines shares
arithmetic with ``operator.collide``: they start again from the integral definitions.
"""

from __future__ import annotations

import math

import numpy as np
from scipy import special

from .grid import gauss_legendre, sinc


def carleman_kernel_l0(xi_norm, R: float, Btilde: float):
    """Exact B_F(0, m) = B_F(m, 0) of Eq. (FKM) for constant Btilde.

    int_{B_R} int_{B_R} delta(x . y) e^{i xi . y} dx dy: the x-integral over the plane
    y-perp inside B_R is pi R^2 / |y|, and int_{B_R} e^{i xi . y} / |y| dy =
    4 pi (1 - cos(R |xi|)) / |xi|^2.  At xi = 0 the value is 2 pi^2 R^4.
    """
    s = np.asarray(xi_norm, dtype=np.float64)
    small = np.abs(R * s) < 1e-4
    ss = np.where(small, 1.0, s)
    val = np.where(small, 2.0 * np.pi ** 2 * R ** 4 * (1.0 - (R * s) ** 2 / 12.0),
                   4.0 * np.pi ** 2 * R * R * (1.0 - np.cos(R * ss)) / (ss * ss))
    return Btilde * val


def phi_quadrature(s, R: float, nodes: int = 200):
    """phi(s) = int_{-R}^{R} |rho| e^{i rho s} d rho by Gauss-Legendre (no closed form)."""
    rho, u = gauss_legendre(nodes, 0.0, R)
    s = np.asarray(s, dtype=np.float64)
    return 2.0 * np.sum(u * rho * np.cos(rho * s[..., None]), axis=-1)


def psi_quadrature(s, R: float, nr: int = 120, nt: int = 256):
    """psi(s) = int over the disk |y| <= R in a plane of e^{i s y_1} d^2y, polar quadrature."""
    r, u = gauss_legendre(nr, 0.0, R)
    t = (np.arange(nt) + 0.5) * 2.0 * np.pi / nt
    s = np.asarray(s, dtype=np.float64)
    ph = np.cos(s[..., None, None] * r[:, None] * np.cos(t)[None, :])
    return np.sum(u[:, None] * r[:, None] * ph, axis=(-2, -1)) * (2.0 * np.pi / nt)


def classical_kernel(xl, xm, R_c: float, gamma: float, C_gamma: float, nodes: int = 160):
    """Classical B-hat(l, m) of Eq. (KM) for the VHS kernel |q| sigma = C |q|^gamma.

    l . q+ + m . q- = (l + m) . q / 2 + |q| (l - m) . omega / 2 and
    int_{S^2} e^{-i a . omega} d omega = 4 pi Sinc(|a|) reduce it to
    16 pi^2 C int_0^{R_c} rho^{2+gamma} Sinc(rho |l+m| / 2) Sinc(rho |l-m| / 2) d rho.
    xl, xm: wave vectors [..., 3].
    """
    rho, u = gauss_legendre(nodes, 0.0, R_c)
    a = np.linalg.norm(np.asarray(xl) + np.asarray(xm), axis=-1)
    b = np.linalg.norm(np.asarray(xl) - np.asarray(xm), axis=-1)
    integrand = rho ** (2.0 + gamma) * sinc(0.5 * rho * a[..., None]) * sinc(0.5 * rho * b[..., None])
    return 16.0 * np.pi ** 2 * C_gamma * np.sum(u * integrand, axis=-1)


def collide_classical(f: np.ndarray, grid, R_c: float, nodes: int = 96, chunk: int = 256) -> np.ndarray:
    """Q from the classical spectral sum Eq. (CF1): sum_{l+m=k} [B(l,m) - B(m,m)] fhat_l fhat_m.

    Uses the truncation |q| <= R_c of Eq. (KM).  B-hat(l, m) depends on l, m only
    through the integer lattice norms |k_l + k_m|^2 and |k_l - k_m|^2, so it is
    tabulated once on that lattice and gathered; the sum itself is the plain O(n^2)
    double loop, vectorised over l and chunked over k.  The circular sum on the grid
    is used (as in the fast oracle), so the two differ only by the truncation model
    and the direction quadrature.
    """
    from .operator import forward, inverse

    N, n = grid.N, grid.n
    c = (math.pi / grid.L) ** 2
    kmax2 = 3 * N * N
    a2 = np.arange(kmax2 + 1, dtype=np.float64)
    rho, u = gauss_legendre(nodes, 0.0, R_c)
    s_a = sinc(0.5 * rho[None, :] * np.sqrt(c * a2)[:, None])          # [A, nodes]
    table = 16.0 * np.pi ** 2 * grid.C_gamma * ((s_a * (u * rho ** (2.0 + grid.gamma))) @ s_a.T)  # [A, B]
    kk = grid.k
    KX, KY, KZ = np.meshgrid(kk, kk, kk, indexing="ij")
    kv = np.stack([KX.ravel(), KY.ravel(), KZ.ravel()], axis=-1)        # [n, 3] signed modes
    Bmm = table[4 * np.sum(kv * kv, axis=1), 0]                        # B(m, m): |2m|^2, 0
    fh = forward(f, grid).reshape(n)
    a = np.arange(N)
    ix, iy, iz = [t.ravel() for t in np.meshgrid(a, a, a, indexing="ij")]
    Qh = np.empty(n, dtype=complex)
    for k0 in range(0, n, chunk):
        kidx = np.arange(k0, min(n, k0 + chunk))
        mx = (ix[kidx, None] - ix[None, :]) % N
        my = (iy[kidx, None] - iy[None, :]) % N
        mz = (iz[kidx, None] - iz[None, :]) % N
        midx = (mx * N + my) * N + mz                                   # [kc, l] -> m
        km = kv[midx]                                                   # signed m
        sp = kv[None, :, :] + km
        sm = kv[None, :, :] - km
        Bkl = table[np.sum(sp * sp, axis=-1), np.sum(sm * sm, axis=-1)]
        Qh[kidx] = np.sum(fh[None, :] * fh[midx] * (Bkl - Bmm[midx]), axis=1)
    return inverse(Qh.reshape(N, N, N), grid).real


def maxwellian(vx, vy, vz, rho, u, T):
    """rho (2 pi T)^{-3/2} exp(-|v - u|^2 / 2T) (Sec. 2, M[f])."""
    d2 = (vx - u[0]) ** 2 + (vy - u[1]) ** 2 + (vz - u[2]) ** 2
    return rho * (2.0 * np.pi * T) ** -1.5 * np.exp(-d2 / (2.0 * T))


def hs_collision_frequency(v, rho, u, T, C_gamma: float = 1.0):
    """int int_{S^2} C |v - w| M(w) d omega dw = 4 pi C rho E|Z|, Z ~ N(v - u, T I).

    E|Z| = sqrt(2T) [exp(-c^2)/sqrt(pi) + (c + 1/(2c)) erf(c)], c = |v - u| / sqrt(2T)
    (mean of a non-central chi distribution with three degrees of freedom).
    """
    v = np.asarray(v, dtype=np.float64)
    c = np.linalg.norm(v - np.asarray(u), axis=-1) / math.sqrt(2.0 * T)
    small = c < 1e-6
    cs = np.where(small, 1.0, c)
    mean = np.where(small, 2.0 / math.sqrt(math.pi) * (1.0 + c * c / 3.0),
                    np.exp(-cs * cs) / math.sqrt(math.pi) + (cs + 0.5 / cs) * special.erf(cs))
    return 4.0 * math.pi * C_gamma * rho * math.sqrt(2.0 * T) * mean


def vhs_collision_frequency(v, rho, u, T, gamma: float, C_gamma: float = 1.0):
    """int int_{S^2} C |v - w|^gamma M(w) d omega dw = 4 pi C rho E|Z|^gamma, Z ~ N(v - u, T I).

    The moments of the non-central chi distribution with three degrees of freedom:
    E|Z|^g = (2T)^{g/2} Gamma((3 + g)/2) / Gamma(3/2) 1F1(-g/2; 3/2; -c^2),
    c = |v - u| / sqrt(2T) (Kummer's function from scipy).  g = 0 gives 1, g = 1 the
    erf form of hs_collision_frequency.
    """
    v = np.asarray(v, dtype=np.float64)
    c2 = np.sum((v - np.asarray(u)) ** 2, axis=-1) / (2.0 * T)
    mean = ((2.0 * T) ** (0.5 * gamma) * special.gamma(0.5 * (3.0 + gamma)) / special.gamma(1.5)
            * special.hyp1f1(-0.5 * gamma, 1.5, -c2))
    return 4.0 * math.pi * C_gamma * rho * mean


def _sphere_rule(nt: int, npp: int):
    """Gauss-Legendre in cos(theta) x trapezoid in varphi on S^2: nodes [P, 3], weights [P]."""
    ct, ut = np.polynomial.legendre.leggauss(nt)
    ph = (np.arange(npp) + 0.5) * 2.0 * np.pi / npp
    st = np.sqrt(1.0 - ct * ct)
    x = (st[:, None] * np.cos(ph)[None, :]).ravel()
    y = (st[:, None] * np.sin(ph)[None, :]).ravel()
    z = np.repeat(ct, npp)
    w = np.repeat(ut, npp) * (2.0 * np.pi / npp)
    return np.stack([x, y, z], axis=-1), w


def boltzmann_direct(v, gaussians, gamma: float = 1.0, C_gamma: float = 1.0, r_max: float = 10.0,
                     nr: int = 48, nt: int = 16, npp: int = 32) -> float:
    """Q_B(f)(v) of Eq. (bolt) by direct quadrature, f a sum of Maxwellians.

    gaussians: list of (rho, u[3], T).  B = C |q|^gamma.  With q = v - v* = r q^,
    v' = v - r (q^ - omega) / 2 and v'* = v - r (q^ + omega) / 2 (reading of the
    post-collision velocities; Sec. 2 prints '+' in both).  Radial Gauss-Legendre on
    [0, r_max]; product rules on both spheres.
    """
    v = np.asarray(v, dtype=np.float64)

    def f(x):
        out = 0.0
        for rho, u, T in gaussians:
            out = out + maxwellian(x[..., 0], x[..., 1], x[..., 2], rho, np.asarray(u), T)
        return out

    r, ur = gauss_legendre(nr, 0.0, r_max)
    sq, wq = _sphere_rule(nt, npp)
    so, wo = _sphere_rule(nt, npp)
    gain = 0.0
    for ri, ui in zip(r, ur):
        vp = v - 0.5 * ri * (sq[:, None, :] - so[None, :, :])
        vps = v - 0.5 * ri * (sq[:, None, :] + so[None, :, :])
        val = f(vp) * f(vps)
        gain += ui * ri ** (2.0 + gamma) * np.sum(wq[:, None] * wo[None, :] * val)
    vs = v - r[:, None, None] * sq[None, :, :]                        # v* = v - q
    loss_int = np.sum(ur[:, None] * r[:, None] ** (2.0 + gamma) * wq[None, :] * f(vs)) * 4.0 * np.pi
    return C_gamma * (gain - f(v) * loss_int)


def bkw_3d(vx, vy, vz, t: float):
    """3D BKW solution for Maxwell molecules with B = 1/(4 pi), rho = 1, u = 0, T = 1.

    f = (2 pi K)^{-3/2} exp(-|v|^2 / 2K) [(5K - 3)/(2K) + (1 - K)|v|^2 / (2K^2)],
    K(t) = 1 - exp(-t/6); valid (non-negative) for K >= 3/5.  The paper prints only the
    2D solution (Sec. 5, Test 1.1); this 3D form is the standard one and is checked
    by the moment identities and the residual test in tests/test_oracle_pins.py.
    """
    K = 1.0 - math.exp(-t / 6.0)
    v2 = vx * vx + vy * vy + vz * vz
    return (2.0 * math.pi * K) ** -1.5 * np.exp(-v2 / (2.0 * K)) * ((5.0 * K - 3.0) / (2.0 * K) + (1.0 - K) * v2 / (2.0 * K * K))


def bkw_3d_dt(vx, vy, vz, t: float, h: float = 1e-4):
    """Central difference of bkw_3d in t (for the residual pin)."""
    return (bkw_3d(vx, vy, vz, t + h) - bkw_3d(vx, vy, vz, t - h)) / (2.0 * h)


def bkw_t0_for_K(K: float) -> float:
    """Time at which K(t) = 1 - exp(-t/6) equals K."""
    return -6.0 * math.log(1.0 - K)
