"""The decomposition of the one-CTA-per-cell 32^3 kernel, restated on the host in float64.

collide_solo_kernel (paper_1608_08009_gb300/csrc/collide_solo.cuh) evaluates the gain and
the loss of the fast spectral operator (arxiv 1608.08009, Sec. 3.3; Sec. 4.2 for the
per-cell loop) from half of the spectrum and in two halves of each inverse transform.
This test restates that bookkeeping with numpy transforms, independently of the CUDA
code, and checks it against the oracle (oracle/operator.py, itself pinned in
test_oracle_pins.py):

  * only the pencils (ky < N/2, kz) of fhat along kx are kept; the mirror pencil
    (-ky, -kz) is formed from them as conj fhat(-kx), with the coefficients of
    (ky, kz) reversed in kx (alpha and alpha' are even);
  * which thread writes which (ky', kz') of the half field: every entry off the removed
    row ky' = N/2 and column kz' = N/2 exactly once;
  * one radix-2 decimation-in-frequency step along kx: for x = 2m + h the output is the
    N/2-point transform of u_h(k) = w^{hk} (c(k) + (-1)^h c(k + N/2)), w = exp(2 pi i / N);
  * the kz and ky passes of each half, and the accumulation of w Re Im by rows
    x = 2m + h.

It runs without a GPU in well under a second per term.
"""

import numpy as np
import pytest

import oracle as O
from paper_1608_08009_gb300 import workloads as W


def half_field_roles(N):
    """doA, doB over (ky < N/2, kz) as the kernel assigns them, and the mirror indices."""
    H = N // 2
    ky = np.arange(H)[:, None] * np.ones((1, N), dtype=int)
    kz = np.ones((H, 1), dtype=int) * np.arange(N)[None, :]
    doA = (kz != H) & ~((ky == 0) & (kz > H))
    doB = doA & ~((ky == 0) & (kz == 0))
    kyB = (N - ky) % N
    kzB = (N - kz) % N
    return ky, kz, doA, doB, kyB, kzB


def solo_transform(fh_half, T, N):
    """Inverse transform of the coefficients T * fhat, the kernel's way.

    fh_half: [H][N][N] = fhat(kx) at (ky < H, kz) as [ky][kz][kx]; T: [N][N][N]
    coefficients in mode order (kx, ky, kz).  Returns g[x][y][z] (complex), the unscaled
    inverse transform sum_k c(k) e^{+2 pi i k . j / N}.
    """
    H = N // 2
    ky, kz, doA, doB, kyB, kzB = half_field_roles(N)
    k = np.arange(N)
    TA = np.transpose(T[:, :H, :], (1, 2, 0))  # [ky][kz][kx]
    cA = TA * fh_half
    # mirror (-ky, -kz): coefficient T(-kx) of the same (ky, kz), spectrum conj fhat(-kx)
    rev = (-k) % N
    cB = TA[:, :, rev] * np.conj(fh_half[:, :, rev])
    g = np.zeros((N, N, N), dtype=complex)
    for h in (0, 1):
        tw = np.exp(2j * np.pi * h * np.arange(H) / N)
        sgn = (-1.0) ** h
        outA = np.fft.ifft(tw * (cA[:, :, :H] + sgn * cA[:, :, H:]), axis=2) * H  # [ky][kz][m]
        outB = np.fft.ifft(tw * (cB[:, :, :H] + sgn * cB[:, :, H:]), axis=2) * H
        Wf = np.full((H, N, N), np.nan + 0j)  # [m][ky'][kz']; NaN marks an unwritten entry
        writes = np.zeros((N, N), dtype=int)
        Wf[:, H, :] = 0.0  # the removed row ky' = N/2
        Wf[:, :, H] = 0.0  # the removed column kz' = N/2
        for a, b in zip(*np.nonzero(doA)):
            Wf[:, ky[a, b], kz[a, b]] = outA[a, b]
            writes[ky[a, b], kz[a, b]] += 1
        for a, b in zip(*np.nonzero(doB)):
            Wf[:, kyB[a, b], kzB[a, b]] = outB[a, b]
            writes[kyB[a, b], kzB[a, b]] += 1
        off = np.ones((N, N), dtype=bool)
        off[H, :] = False
        off[:, H] = False
        assert (writes[off] == 1).all(), "every entry off the removed row and column once"
        assert (writes[~off] == 0).all()
        assert not np.isnan(Wf).any()
        Wf = np.fft.ifft(Wf, axis=2) * N  # kz pass
        Wf = np.fft.ifft(Wf, axis=1) * N  # ky pass: [m][y][z]
        g[h::2] = Wf
    return g


@pytest.mark.parametrize("M", [4])
def test_half_spectrum_and_two_halves_reproduce_the_operator(M):
    N, L = 32, 8.0
    og = O.make_grid(N, L, M=M)
    f = W.two_maxwellians(1, N, L, seed=181)[0]
    # the kernel's inputs: fhat = n^-1 FFT(f) without the oracle's phase (it cancels
    # between a forward and an inverse transform), Nyquist modes removed
    fh = np.fft.fftn(f) / og.n
    nyq = np.zeros((N, N, N), dtype=bool)
    nyq[N // 2, :, :] = nyq[:, N // 2, :] = nyq[:, :, N // 2] = True
    fh[nyq] = 0.0
    fh_half = np.transpose(fh[:, : N // 2, :], (1, 2, 0))
    gain = np.zeros((N, N, N))
    for i in range(og.M_eff):
        g = solo_transform(fh_half, og.alpha[i] + 1j * og.alphap[i], N)
        gain += og.w[i] * g.real * g.imag
    loss = solo_transform(fh_half, og.D.astype(complex), N)
    Qp, Lo = O.operator.gain_loss(f, og)
    assert np.linalg.norm(gain - Qp) <= 1e-12 * np.linalg.norm(Qp)
    assert np.linalg.norm(loss.real - Lo) <= 1e-12 * np.linalg.norm(Lo)
    assert np.abs(loss.imag).max() <= 1e-12 * np.abs(Lo).max()  # the loss transform is real


def test_roles_cover_the_half_field_once_at_every_even_size():
    for N in (8, 16, 32, 64):
        H = N // 2
        ky, kz, doA, doB, kyB, kzB = half_field_roles(N)
        writes = np.zeros((N, N), dtype=int)
        np.add.at(writes, (ky[doA], kz[doA]), 1)
        np.add.at(writes, (kyB[doB], kzB[doB]), 1)
        off = np.ones((N, N), dtype=bool)
        off[H, :] = False
        off[:, H] = False
        assert (writes[off] == 1).all() and (writes[~off] == 0).all()
        # the lanes kz = N/2 form no pencil (they zero the removed column again)
        assert not doA[:, H].any()
