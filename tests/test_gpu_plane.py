"""2D Maxwell-molecule grids (boltz_create_grid2d) against the 2D oracle, through the C ABI.

Tolerances as for 3D: float64 <= 1e-12 relative L2; float32 <= 1.25 eps32 log2(n) kappa
(n = N^2, kappa = ||Q+|| / ||Q|| of the input)."""

import json
import math
import os

import numpy as np
import pytest

from oracle import plane as P
from paper_1608_08009_gb300 import boltz as B

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
BT = 1.0 / (2.0 * math.pi)  # C_gamma of the 2D BKW normalisation (Btilde = 1/pi)


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def two_gaussians(cells, N, L, seed):
    """Seeded 2D cells: two Maxwellians with random density, drift and temperature."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = -L + (2.0 * L / N) * np.arange(N)
    VX, VY = np.meshgrid(v, v, indexing="ij")
    out = np.empty((cells, N, N))
    for c in range(cells):
        f = 0.0
        for _ in range(2):
            rho, T = rng.uniform(0.5, 2.0), rng.uniform(0.5, 1.5)
            ux, uy = rng.normal(0.0, 0.3, 2)
            f = f + rho / (2 * math.pi * T) * np.exp(-((VX - ux) ** 2 + (VY - uy) ** 2) / (2 * T))
        out[c] = f
    return out


def fp32_tol(f, g):
    Qp, Lo = P.gain_loss(f, g)
    return 1.25 * EPS32 * math.log2(g.n) * np.linalg.norm(Qp) / np.linalg.norm(Qp - f * Lo)


@pytest.mark.parametrize("N,L,A", [(8, 4.0, 8), (16, 6.0, 8), (32, 9.0, 16), (64, 12.0, 8)])
def test_collide2d_parity(N, L, A):
    f = two_gaussians(5, N, L, seed=N)
    og = P.make_plane_grid(N, L, A=A)
    Qref = P.collide(f, og)
    with B.Grid2D(N, L, A, C_gamma=BT) as g:
        tab = g.tables()
        assert np.max(np.abs(tab[2] - og.alpha)) <= 1e-13 * np.abs(og.alpha).max()
        assert np.max(np.abs(tab[4] - og.D)) <= 1e-13 * np.abs(og.D).max()
        precs = [(B.BOLTZ_FP32_FFT, torch.float32)] + ([(B.BOLTZ_FP64, torch.float64)] if N <= 32 else [])
        for prec, dt in precs:
            ft = torch.from_numpy(f).to(device="cuda", dtype=dt)
            Q = torch.empty_like(ft)
            B.boltz_collide(g.batch(5, prec, dt == torch.float64), ft, Q)
            B.boltz_stream_status()
            tol = 1e-12 if prec == B.BOLTZ_FP64 else fp32_tol(f, og)
            assert rel_l2(Q.double().cpu().numpy(), Qref) <= tol, (prec, rel_l2(Q.double().cpu().numpy(), Qref))
        if N == 64:
            with pytest.raises(B.BoltzError) as ei:
                B.boltz_collide(g.batch(1, B.BOLTZ_FP64, True), torch.zeros(1, N, N, dtype=torch.float64, device="cuda"),
                                torch.zeros(1, N, N, dtype=torch.float64, device="cuda"))
            assert ei.value.status == B.BOLTZ_EUNSUPPORTED


@pytest.mark.parametrize("rk", [1, 2])
def test_relax2d_and_moments(rk):
    N, L, A, cells = 16, 6.0, 8, 37  # 37 cells: a ragged last CTA
    f = two_gaussians(cells, N, L, seed=7)
    og = P.make_plane_grid(N, L, A=A)
    ref = P.relax(f, og, 0.02, 3, rk_order=rk)
    with B.Grid2D(N, L, A, C_gamma=BT) as g:
        ft = torch.from_numpy(f).cuda()
        B.boltz_relax(g.batch(cells), ft, 0.02, 3, rk)
        U = torch.empty(cells, 5, dtype=torch.float64, device="cuda")
        B.boltz_moments(g.batch(cells), ft, U)
        B.boltz_stream_status()
        out = ft.cpu().numpy()
        assert rel_l2(out - f, ref - f) <= 1e-11
        U = U.cpu().numpy()
        Uref = P.moments(f, og)
        assert np.abs(U[:, 3]).max() == 0.0
        assert np.max(np.abs(U[:, [0, 1, 2, 4]] - Uref) / np.abs(Uref).max(axis=1, keepdims=True)) < 1e-13


def test_bkw2d_table_test1_on_the_gpu():
    """Test 1.1 on the GPU (float64, 32^2 on [-9, 9]^2, eight angles, 500 Euler steps of
    0.02): the same errors as the oracle's run, within the band of the printed Table test1
    (tests/golden/bkw2d_table_test1.json)."""
    rows = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bkw2d_table_test1.json")))["rows"]
    row = rows[2]
    og = P.make_plane_grid(row["N"], row["L"], A=8)
    f0 = P.bkw(og, 0.0)[None]
    ref = P.relax(f0, og, 0.02, 500)[0]
    with B.Grid2D(row["N"], row["L"], 8, C_gamma=BT) as g:
        ft = torch.from_numpy(f0.copy()).cuda()
        B.boltz_relax(g.batch(1), ft, 0.02, 500, 1)
        B.boltz_stream_status()
        out = ft.cpu().numpy()[0]
    ex = P.bkw(og, 10.0)
    l1 = np.abs(out - ex).sum() / np.abs(ex).sum()
    l1_ref = np.abs(ref - ex).sum() / np.abs(ex).sum()
    assert abs(l1 - l1_ref) <= 1e-6 * l1_ref
    assert row["L1"] / 6 <= l1 <= 6 * row["L1"]


def test_indexed_2d_cells():
    N, L, pool = 8, 4.0, 6
    f = two_gaussians(pool, N, L, seed=11)
    with B.Grid2D(N, L, 8, C_gamma=BT) as g:
        fd = torch.from_numpy(f).cuda()
        Qall = torch.empty_like(fd)
        B.boltz_collide(g.batch(pool), fd, Qall)
        idx = torch.tensor([4, 1], dtype=torch.int64, device="cuda")
        Q = torch.zeros_like(fd)
        B.boltz_collide_indexed(g.batch(2), fd, Q, idx, pool)
        B.boltz_stream_status()
        assert torch.equal(Q[4], Qall[4]) and torch.equal(Q[1], Qall[1])
        assert torch.count_nonzero(Q[[0, 2, 3, 5]]).item() == 0
