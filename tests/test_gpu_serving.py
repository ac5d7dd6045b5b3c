"""Serving loop (boltz_server_*): results alone vs in the mix, against the oracle, and
admission by HBM budget.

A job's result must not depend on which other jobs share the device: the server runs
every resident cell through the same per-cell arithmetic, so the comparison is exact.
Each step projects onto the moments the cell has at that step, i.e. the same as calling
boltz_relax with steps = 1 repeatedly, which the first test also checks.  Served jobs in
a mix are also held to the oracle's relaxation within the float32 bound.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1608_08009_gb300 import boltz as B
from paper_1608_08009_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DT = 0.004


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


def _cells(gi_f):
    """Cells of a job's f: a 3D array is one cell, a 4D array a batch."""
    return 1 if gi_f.ndim == 3 else gi_f.shape[0]


def _run(server, jobs, schedule):
    """jobs: list of (grid_index, f, steps), f one cell [N, N, N] or a batch [c, N, N, N];
    schedule: iteration at which each is submitted."""
    outs = [torch.empty(f.size, dtype=torch.float32).pin_memory() for _, f, _ in jobs]
    ins = [_pinned(f.ravel()) for _, f, _ in jobs]
    ids = [None] * len(jobs)
    it = 0
    while True:
        for k, (gi, f, steps) in enumerate(jobs):
            if ids[k] is None and schedule[k] <= it:
                ids[k] = server.submit(gi, ins[k], outs[k], steps, _cells(f))
        server.step()
        it += 1
        if all(i is not None for i in ids) and all(server.poll(i) for i in ids):
            break
        assert it < 10000
    return [o.numpy().reshape(f.shape) for o, (_, f, _) in zip(outs, jobs)]


def test_result_alone_equals_result_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g16 = B.Grid(16, 6.0, 1.0, 16)
    g32 = B.Grid(32, 8.0, 1.0, 16)
    f16 = W.two_maxwellians(4, 16, 6.0, seed=3)
    f32 = W.two_maxwellians(3, 32, 8.0, seed=4)
    target = (1, f32[0], 7)
    s1 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 26)
    alone = _run(s1, [target], [0])[0]
    s1.close()
    mix = [(0, f16[0], 12), (1, f32[1], 3), target, (0, f16[1], 5), (1, f32[2], 9), (0, f16[2], 1)]
    s2 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 26)
    res = _run(s2, mix, [0, 0, 2, 3, 3, 6])
    s2.close()
    assert np.array_equal(res[2], alone)
    # the same as stepping the cell with boltz_relax one step at a time
    ft = torch.from_numpy(f32[0].astype(np.float32)).cuda().reshape(1, 32, 32, 32)
    for _ in range(7):
        B.boltz_relax(g32.batch(1, B.BOLTZ_FP32_FFT, False), ft, DT, 1, 1)
    B.boltz_stream_status()
    assert np.array_equal(ft.cpu().numpy()[0], alone)
    assert not np.array_equal(alone, f32[0].astype(np.float32))


def test_admission_respects_the_hbm_budget():
    """The server holds exactly its budget on the device; admission counts each job's
    distributions and term-group scratch against it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g32 = B.Grid(32, 8.0, 1.0, 8)
    cell = 32 ** 3 * 4
    s = B.Server([g32], B.BOLTZ_FP32_FFT, DT, 2 * cell + 4096)  # two cells and the index lists
    f = W.two_maxwellians(4, 32, 8.0, seed=9)
    outs = [torch.empty(32 ** 3, dtype=torch.float32).pin_memory() for _ in range(4)]
    ids = [s.submit(0, _pinned(f[k].ravel()), outs[k], 3) for k in range(4)]
    resident, queued = s.step()
    assert (resident, queued) == (2, 2)
    st = s.stats()
    assert st["reserved_bytes"] == 2 * cell + 4096 and st["used_bytes"] <= st["reserved_bytes"]
    assert st["used_bytes"] >= 2 * cell
    for _ in range(20):
        s.step()
    torch.cuda.synchronize()
    assert all(s.poll(i) for i in ids)
    st = s.stats()
    assert st["peak_used_bytes"] <= st["reserved_bytes"] and st["resident_cells"] == 0
    B.boltz_stream_status()
    s.close()
    # with term groups the scratch ((G + 1) N^3 floats per cell) counts too: a budget of
    # two cells' distributions holds no cell of a 4-group grid
    g4 = B.Grid(32, 8.0, 1.0, 8, term_groups=4)
    with pytest.raises(B.BoltzError) as ei:
        B.Server([g4], B.BOLTZ_FP32_FFT, DT, 2 * cell + 4096)
    assert ei.value.status == B.BOLTZ_EINVAL
    s = B.Server([g4], B.BOLTZ_FP32_FFT, DT, 2 * 7 * cell + 8192)  # two cells with scratch and alignment
    ids = [s.submit(0, _pinned(f[k].ravel()), outs[k], 2) for k in range(3)]
    assert s.step() == (2, 1)
    assert s.stats()["used_bytes"] >= 2 * 6 * cell
    for _ in range(20):
        s.step()
    torch.cuda.synchronize()
    assert all(s.poll(i) for i in ids)
    # a job that can never fit is refused at submission
    big = torch.empty(3 * 32 ** 3, dtype=torch.float32).pin_memory()
    with pytest.raises(B.BoltzError) as ei:
        s.submit(0, big, big, 1, 3)
    assert ei.value.status == B.BOLTZ_EINVAL
    s.close()
    g4.close()
    g32.close()


def test_blocked_grid_does_not_hold_back_others():
    """A large batch job waiting for room on one grid does not stop jobs of another grid
    from being admitted (queues are per grid)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g32 = B.Grid(32, 8.0, 1.0, 8)
    g16 = B.Grid(16, 6.0, 1.0, 8)
    cell32 = 32 ** 3 * 4
    s = B.Server([g32, g16], B.BOLTZ_FP32_FFT, DT, 3 * cell32 + 8192)
    f32 = W.two_maxwellians(3, 32, 8.0, seed=21).astype(np.float32)
    f16 = W.two_maxwellians(2, 16, 6.0, seed=22).astype(np.float32)
    o = [torch.empty(x.size, dtype=torch.float32).pin_memory() for x in (f32[:2], f32, f16[0], f16[1])]
    j0 = s.submit(0, _pinned(f32[:2].ravel()), o[0], 6, 2)  # two of the three 32^3 slots
    j1 = s.submit(0, _pinned(f32.ravel()), o[1], 2, 3)      # waits: needs all three
    j2 = s.submit(1, _pinned(f16[0].ravel()), o[2], 2)
    j3 = s.submit(1, _pinned(f16[1].ravel()), o[3], 2)
    s.step()
    st = s.stats()
    assert st["resident_jobs"] == 3 and st["queued_jobs"] == 1  # the 16^3 jobs got in
    for _ in range(40):
        s.step()
    torch.cuda.synchronize()
    assert all(s.poll(j) for j in (j0, j1, j2, j3))
    B.boltz_stream_status()
    s.close()


def test_batch_job_alone_equals_in_the_mix():
    """A multi-cell job (term groups, so its scratch is carved from the arena) gives the
    same bits alone and among single-cell and batch jobs of two grids."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g16 = B.Grid(16, 6.0, 1.0, 16, term_groups=3)
    g32 = B.Grid(32, 8.0, 1.0, 16, term_groups=2)
    f16 = W.two_maxwellians(6, 16, 6.0, seed=23)
    f32 = W.two_maxwellians(5, 32, 8.0, seed=24)
    target = (1, f32[:3], 5)
    s1 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 28)
    alone = _run(s1, [target], [0])[0]
    s1.close()
    mix = [(0, f16[:4], 7), (1, f32[3], 2), target, (0, f16[4], 3), (1, f32[4], 6), (0, f16[5:], 1)]
    s2 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 28)
    res = _run(s2, mix, [0, 0, 1, 1, 3, 4])
    s2.close()
    assert np.array_equal(res[2], alone)
    # each cell of the batch equals the same cell served alone as a single-cell job
    s3 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 28)
    single = _run(s3, [(1, f32[1], 5)], [0])[0]
    s3.close()
    assert np.array_equal(alone[1], single)
    g16.close()
    g32.close()


def test_served_jobs_match_the_oracle():
    """Jobs served in a mix against the oracle's forward-Euler relaxation of the same
    float32-rounded cells: the increment f_k - f_0 within the float32 bound of one
    collision (1.25 eps32 log2(n) kappa) plus the float32 rounding of the stored state at
    every step (eps32 ||f|| per step, relative to the increment)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps32 = 2.0 ** -24
    grids = {16: (6.0, 3), 32: (8.0, 2)}
    gs = [B.Grid(N, L, 1.0, 16, term_groups=G) for N, (L, G) in grids.items()]
    f16 = W.two_maxwellians(3, 16, 6.0, seed=25).astype(np.float32)
    f32 = W.two_maxwellians(2, 32, 8.0, seed=26).astype(np.float32)
    jobs = [(0, f16[:2], 4), (1, f32[0], 3), (0, f16[2], 6), (1, f32[1:], 2)]
    s = B.Server(gs, B.BOLTZ_FP32_FFT, DT, 1 << 28)
    res = _run(s, jobs, [0, 0, 1, 2])
    s.close()
    for (gi, f, steps), out in zip(jobs, res):
        N = 16 if gi == 0 else 32
        og = O.make_grid(N, grids[N][0], M=16)
        fb = f.reshape((-1,) + (N,) * 3).astype(np.float64)
        ref = O.relax(fb, og, DT, steps)
        Qp, Lo = O.operator.gain_loss(fb, og)
        kappa = np.linalg.norm(Qp) / np.linalg.norm(Qp - fb * Lo)
        inc = np.linalg.norm(ref - fb)
        tol = 1.25 * eps32 * math.log2(og.n) * kappa + steps * eps32 * np.linalg.norm(fb) / inc
        err = np.linalg.norm(out.reshape(fb.shape) - ref) / inc
        assert err <= tol, (gi, steps, err, tol)
    for g in gs:
        g.close()


def test_pump_gives_the_same_results_as_step():
    """A serving loop driven by the non-blocking pump (grids advance at their own pace,
    two iterations in flight each) returns the same bits as the blocking step."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g16 = B.Grid(16, 6.0, 1.0, 16, term_groups=4)
    g32 = B.Grid(32, 8.0, 1.0, 16)
    f16 = W.two_maxwellians(3, 16, 6.0, seed=13)
    f32 = W.two_maxwellians(2, 32, 8.0, seed=14)
    jobs = [(0, f16[0], 9), (1, f32[0], 4), (0, f16[1], 2), (1, f32[1], 6), (0, f16[2], 11)]
    s1 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 26)
    ref = _run(s1, jobs, [0, 0, 1, 2, 2])
    s1.close()
    s2 = B.Server([g16, g32], B.BOLTZ_FP32_FFT, DT, 1 << 26)
    outs = [torch.empty(f.size, dtype=torch.float32).pin_memory() for _, f, _ in jobs]
    ins = [_pinned(f.ravel()) for _, f, _ in jobs]
    ids = [s2.submit(gi, ins[k], outs[k], st) for k, (gi, _, st) in enumerate(jobs)]
    for _ in range(200000):
        s2.pump()
        if all(s2.poll(i) for i in ids):
            break
    assert all(s2.poll(i) for i in ids)
    B.boltz_stream_status()
    s2.close()
    for o, r, (_, f, _) in zip(outs, ref, jobs):
        assert np.array_equal(o.numpy().reshape(f.shape), r)


def test_checkpoint_and_resume_on_another_server():
    """A job stopped after some iterations and resubmitted (its state and remaining steps)
    to a new server finishes with the same bits as the uninterrupted run."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g32 = B.Grid(32, 8.0, 1.0, 16)
    f = W.two_maxwellians(1, 32, 8.0, seed=17)[0]
    ref = _run(B.Server([g32], B.BOLTZ_FP32_FFT, DT, 1 << 26), [(0, f, 9)], [0])[0]
    s1 = B.Server([g32], B.BOLTZ_FP32_FFT, DT, 1 << 26)
    out = torch.empty(f.size, dtype=torch.float32).pin_memory()
    j = s1.submit(0, _pinned(f.ravel()), out, 9)
    for _ in range(4):
        s1.step()
    state = torch.empty(f.size, dtype=torch.float32).pin_memory()
    left = s1.checkpoint(j, state)
    assert left == 5
    s1.close()
    s2 = B.Server([g32], B.BOLTZ_FP32_FFT, DT, 1 << 26)
    res = _run(s2, [(0, state.numpy().reshape(f.shape), left)], [0])[0]
    s2.close()
    assert np.array_equal(res, ref)
    g32.close()


def test_server_allocation_failure_is_reported():
    """A pool that cannot be allocated (a 16 TiB budget) returns BOLTZ_ENOMEM, no crash."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g16 = B.Grid(16, 6.0, 1.0, 8)
    with pytest.raises(B.BoltzError) as ei:
        B.Server([g16], B.BOLTZ_FP32_FFT, DT, 16 << 40)
    assert ei.value.status == B.BOLTZ_ENOMEM
    g16.close()
