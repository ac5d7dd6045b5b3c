"""Fast Kinetic Scheme in one space dimension (boltz_fks_*) against the oracle's FKS
(oracle/fks.py, Sec. 3.1): transport of the piecewise-constant distribution fused into the
collision launch, Sod-like data of Part 2 (1D x 3D as in Test 2.3), Dirichlet states at
both ends; and a domain split into two sub-domains with ghost cells (Sec. 4.2, fig.
mpi-decomp) equal to the whole domain bit for bit."""

import math

import numpy as np
import pytest

import oracle as O
from oracle import fks as K
from paper_1608_08009_gb300 import boltz as B

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


def _setup(N=16, L=8.0, M=16, nx=10, groups=1):
    og = O.make_grid(N, L, M=M)
    f0, left, right, dx = K.sod(og, nx, length=2.0)
    dt = 0.8 * dx / L  # Eq. Time with room: |v_x| <= L on the grid
    Lmax = float(np.abs(O.operator.gain_loss(f0, og)[1]).max())
    tau = 2.0 * dt * Lmax  # forward Euler on the collision stage: dt / tau max L = 1/2
    g = B.Grid(N, L, 1.0, M, term_groups=groups)
    return og, g, f0, left, right, dx, dt, tau, Lmax


def _run_gpu(g, fks, f0, left, right, dt, tau, steps, prec, f64=True, rows=1):
    dtype = torch.float64 if f64 else torch.float32
    a = torch.from_numpy(np.ascontiguousarray(f0)).to(device="cuda", dtype=dtype)
    b = torch.empty_like(a)
    lo = torch.from_numpy(np.ascontiguousarray(left)).to(device="cuda", dtype=dtype)
    hi = torch.from_numpy(np.ascontiguousarray(right)).to(device="cuda", dtype=dtype)
    batch = g.batch(a.shape[0], prec, f64)
    for _ in range(steps):
        fks.step(batch, a, b, lo, hi, dt, tau)
        a, b = b, a
    B.boltz_stream_status()
    return a.double().cpu().numpy()


@pytest.mark.parametrize("groups", [1, 3])
def test_fks_sod_matches_the_oracle(groups):
    og, g, f0, left, right, dx, dt, tau, Lmax = _setup(groups=groups)
    steps = 6
    ref = K.run(f0, og, dt, steps, dx, tau, left, right)
    free = K.run(f0, og, dt, steps, dx, tau, left, right, collisions=False)
    coll = np.linalg.norm(ref - free)  # what the collision stages changed
    with B.Fks(g, 10, dx) as fks:
        out = _run_gpu(g, fks, f0, left, right, dt, tau, steps, B.BOLTZ_FP64)
        assert math.isclose(fks.time, steps * dt, rel_tol=1e-15)
    assert np.linalg.norm(out - ref) <= 1e-11 * coll
    # float32 transforms (f stored in float64): each collision stage within the float32
    # bound of its own input, an earlier stage's error reaching later ones through the
    # linearised operator (norm ~ max L), so (1 + dt / tau max L) per further step
    Qp, Lo = O.operator.gain_loss(f0, og)
    tol32 = 1.25 * EPS32 * math.log2(og.n) * np.linalg.norm(Qp) / np.linalg.norm(Qp - f0 * Lo)
    with B.Fks(g, 10, dx) as fks:
        out32 = _run_gpu(g, fks, f0, left, right, dt, tau, steps, B.BOLTZ_FP32_FFT)
    assert np.linalg.norm(out32 - ref) <= tol32 * (1.0 + dt / tau * Lmax) ** steps * coll
    g.close()


def test_fks_shifts_and_rows():
    """The library's column moves equal the oracle's interval shifts step after step, and
    several rows (each with its own boundary states) advance in one launch as if alone."""
    og, g, f0, left, right, dx, dt, tau, _ = _setup(N=8, L=4.0, M=8, nx=6)
    rng = np.random.default_rng(3)
    f0b = f0 * rng.uniform(0.8, 1.2, f0.shape)  # a second, different row
    with B.Fks(g, 6, dx) as fks:
        t = 0.0
        for _ in range(5):
            d = fks.shifts(dt)
            assert d == [K.shift(og.v[k], t + dt, dx) - K.shift(og.v[k], t, dx) for k in range(8)]
            fks.time = t + dt
            t += dt
    rows = np.concatenate([f0, f0b])
    lo = np.stack([left, 0.5 * left])
    hi = np.stack([right, 2.0 * right])
    with B.Fks(g, 6, dx) as fks:
        out = _run_gpu(g, fks, rows, lo, hi, dt, tau, 3, B.BOLTZ_FP64)
    r0 = K.run(f0, og, dt, 3, dx, tau, left, right)
    r1 = K.run(f0b, og, dt, 3, dx, tau, 0.5 * left, 2.0 * right)
    for got, ref in ((out[:6], r0), (out[6:], r1)):
        assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    g.close()


def test_split_domain_with_ghost_cells_equals_the_whole_domain():
    """Two sub-domains of 5 cells each, advanced by their own FKS states with the other
    one's edge cells (from the start of the step) as boundary states, give the bits of the
    10-cell domain: the transport reads at most one cell across a boundary."""
    og, g, f0, left, right, dx, dt, tau, _ = _setup(N=8, L=4.0, M=8, nx=10)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    whole = dev(f0)
    tmp = torch.empty_like(whole)
    lo, hi = dev(left[None]), dev(right[None])
    parts = [dev(f0[:5]), dev(f0[5:])]
    ptmp = [torch.empty_like(p) for p in parts]
    with B.Fks(g, 10, dx) as fw, B.Fks(g, 5, dx) as fa, B.Fks(g, 5, dx) as fb:
        for _ in range(6):
            fw.step(g.batch(10), whole, tmp, lo, hi, dt, tau)
            whole, tmp = tmp, whole
            ghost_a = parts[1][:1].clone()   # right neighbour's first cell
            ghost_b = parts[0][-1:].clone()  # left neighbour's last cell
            fa.step(g.batch(5), parts[0], ptmp[0], lo, ghost_a, dt, tau)
            fb.step(g.batch(5), parts[1], ptmp[1], ghost_b, hi, dt, tau)
            parts, ptmp = ptmp, parts
        B.boltz_stream_status()
    assert torch.equal(torch.cat(parts), whole)
    g.close()


def test_fks_argument_errors():
    og, g, f0, left, right, dx, dt, tau, _ = _setup(N=8, L=4.0, M=8, nx=4)
    a = torch.from_numpy(f0).cuda()
    b = torch.empty_like(a)
    lo, hi = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    with B.Fks(g, 4, dx) as fks:
        with pytest.raises(B.BoltzError) as ei:  # transport condition
            fks.step(g.batch(4), a, b, lo, hi, 1.5 * dx / 4.0 * 2.0, tau)
        assert ei.value.status == B.BOLTZ_EINVAL and "Eq. Time" in str(ei.value)
        with pytest.raises(B.BoltzError) as ei:  # in place
            fks.step(g.batch(4), a, a, lo, hi, dt, tau)
        assert ei.value.status == B.BOLTZ_EINVAL
        with pytest.raises(B.BoltzError) as ei:  # not whole rows
            fks.step(g.batch(3), a, b, lo, hi, dt, tau)
        assert ei.value.status == B.BOLTZ_EINVAL
        assert fks.time == 0.0  # failed steps do not advance the time
    g.close()
