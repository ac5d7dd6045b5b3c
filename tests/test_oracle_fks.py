"""Pins of the oracle's Fast Kinetic Scheme in one space dimension (oracle/fks.py,
Sec. 3.1 of arxiv 1608.08009): the transport stage against the exact free-streaming
solution of the piecewise-constant data and a direct search of the covering interval;
the collision stage against the homogeneous relaxation; the boundary mass balance."""

import numpy as np
import pytest

import oracle as O
from oracle import fks as K


def test_shift_is_the_covering_interval():
    """shift(v, t, dx): the centre of cell j lies in the interval that started as cell
    j - shift, found here by scanning the moved half-open intervals [i dx + s, (i+1) dx + s)."""
    rng = np.random.default_rng(5)
    dx = 0.0625
    for _ in range(400):
        vx, t = rng.uniform(-16, 16), rng.uniform(0, 0.3)
        s = vx * t
        j = 7
        xc = (j + 0.5) * dx
        cover = [i for i in range(-200, 200) if i * dx + s <= xc < (i + 1) * dx + s]
        assert cover == [j - K.shift(vx, t, dx)]


def test_free_streaming_is_exact_transport_of_the_piecewise_constant_data():
    """Without collisions, K steps give fbar(x_j - v_x t) of the initial piecewise-constant
    function (the boundary states outside [0, n_x dx]) at every centre, exactly: the
    interval index floor((x_j - v_x t) / dx) evaluated directly at the final time."""
    g = O.make_grid(8, 4.0, M=4)
    nx, dx, dt, steps = 11, 0.1, 0.0173, 9
    rng = np.random.default_rng(1)
    f0 = rng.uniform(0.5, 1.5, (nx, 8, 8, 8))
    left, right = rng.uniform(2, 3, (8, 8, 8)), rng.uniform(4, 5, (8, 8, 8))
    f = K.run(f0, g, dt, steps, dx, 1.0, left, right, collisions=False)
    t = 0.0
    for _ in range(steps):
        t += dt
    for j in range(nx):
        for kx in range(8):
            i = int(np.floor(((j + 0.5) * dx - g.v[kx] * t) / dx))
            want = left[kx] if i < 0 else right[kx] if i >= nx else f0[i, kx]
            assert np.array_equal(f[j, kx], want), (j, kx, i)
    # fast velocities crossed several cells, slow ones none
    assert K.shift(g.v[0], t, dx) <= -5 and K.shift(g.v[4], t, dx) == 0


def test_uniform_state_reduces_to_the_homogeneous_relaxation():
    """A uniform state with equal boundary states is unchanged by transport, so one FKS
    step is one forward-Euler relaxation step of dt / tau in every cell (to the rounding
    of the batched moment sums)."""
    from paper_1608_08009_gb300 import workloads as W

    g = O.make_grid(8, 4.0, M=8)
    cell = W.two_maxwellians(1, 8, 4.0, seed=3)[0]
    nx, dt, tau = 3, 0.01, 0.5
    f0 = np.repeat(cell[None], nx, axis=0)
    out = K.step(f0, g, 0.0, dt, 0.05, tau, cell, cell)
    ref = O.relax(cell[None], g, dt / tau, 1)[0]
    for j in range(nx):
        assert np.abs(out[j] - ref).max() <= 1e-14 * np.abs(ref).max()


def test_mass_changes_only_through_the_boundaries():
    """Collisions conserve each cell's mass, so over one step the total mass changes by
    what the shifted columns bring in (boundary states) minus what they push out."""
    g = O.make_grid(8, 4.0, M=8)
    f0, left, right, dx = K.sod(g, 10, length=2.0)
    dt, tau, t = 0.02, 0.05, 0.013
    f1 = K.step(f0, g, t, dt, dx, tau, left, right)
    dv3 = g.dv ** 3
    flux = 0.0
    for kx in range(8):
        d = K.shift(g.v[kx], t + dt, dx) - K.shift(g.v[kx], t, dx)
        assert abs(d) <= 1
        if d == 1:
            flux += (left[kx].sum() - f0[-1, kx].sum()) * dv3
        elif d == -1:
            flux += (right[kx].sum() - f0[0, kx].sum()) * dv3
    m0, m1 = f0.sum() * dv3, f1.sum() * dv3
    assert abs((m1 - m0) - flux) <= 1e-13 * m0
    assert flux != 0.0  # the step moved columns across both boundaries


@pytest.mark.parametrize("nx", [8])
def test_sod_stays_positive_and_conservative_per_cell(nx):
    """Sod-like data of Part 2 (rho 1 / 0.125, T 2.5 / 0.25) over a few steps: density
    positive everywhere, and each cell's collision stage keeps the moments of its f*."""
    g = O.make_grid(8, 4.0, M=8)
    f0, left, right, dx = K.sod(g, nx, length=2.0)
    # dt <= min(dx / |v|max, tau / mu) (Test 2.3's condition, with room): forward Euler on
    # the collision stage stays stable while dt / tau times the largest loss rate is < 2
    dt, tau = 0.5 * dx / 4.0, 2.0
    Lmax = np.abs(O.operator.gain_loss(f0, g)[1]).max()
    assert dt / tau * Lmax < 1.0
    f, t = f0, 0.0
    for _ in range(4):
        fs = K.transport(f, g, t, t + dt, dx, left, right)
        f = K.step(f, g, t, dt, dx, tau, left, right)
        U0, U1 = O.moments(fs, g), O.moments(f, g)
        assert np.max(np.abs(U1 - U0) / np.abs(U0).max(axis=1, keepdims=True)) < 1e-12
        t += dt
    assert (O.moments(f, g)[:, 0] > 0).all()
