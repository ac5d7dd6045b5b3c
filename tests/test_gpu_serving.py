"""Serving loop (boltz_server_*): results alone vs in the mix, admission by HBM budget.

A job's result must not depend on which other jobs share the device: the server runs
every resident cell through the same per-cell arithmetic, so the comparison is exact.
Each step projects onto the moments the cell has at that step, i.e. the same as calling
boltz_relax with steps = 1 repeatedly, which the first test also checks.
"""

import numpy as np
import pytest

from paper_1608_08009_gb300 import boltz as B
from paper_1608_08009_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DT = 0.004


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


def _run(server, jobs, schedule):
    """jobs: list of (grid_index, f, steps); schedule: iteration at which each is submitted."""
    outs = [torch.empty(f.size, dtype=torch.float32).pin_memory() for _, f, _ in jobs]
    ins = [_pinned(f.ravel()) for _, f, _ in jobs]
    ids = [None] * len(jobs)
    it = 0
    while True:
        for k, (gi, f, steps) in enumerate(jobs):
            if ids[k] is None and schedule[k] <= it:
                ids[k] = server.submit(gi, ins[k], outs[k], steps)
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
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g32 = B.Grid(32, 8.0, 1.0, 8)
    cell = 32 ** 3 * 4
    s = B.Server([g32], B.BOLTZ_FP32_FFT, DT, 2 * cell)  # room for two resident cells
    f = W.two_maxwellians(4, 32, 8.0, seed=9)
    outs = [torch.empty(32 ** 3, dtype=torch.float32).pin_memory() for _ in range(4)]
    ids = [s.submit(0, _pinned(f[k].ravel()), outs[k], 3) for k in range(4)]
    resident, queued = s.step()
    assert (resident, queued) == (2, 2)
    for _ in range(20):
        s.step()
    torch.cuda.synchronize()
    assert all(s.poll(i) for i in ids)
    B.boltz_stream_status()
    s.close()


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
