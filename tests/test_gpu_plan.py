"""Ragged batches through boltz_plan_* (one CUDA graph per step loop, groups of cells on
different grids as concurrent branches), against boltz_relax and the oracle."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1608_08009_gb300 import boltz as B
from paper_1608_08009_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield


# (N, L, gamma, M, opts, prec, f dtype, cells)
GROUPS = [
    (8, 4.0, 1.0, 8, {}, B.BOLTZ_FP64, torch.float64, 3),
    (16, 6.0, 0.5, 8, {"radial_rank": 4, "dirs_kind": 2}, B.BOLTZ_FP32_FFT, torch.float32, 5),
    (24, 7.0, 1.0, 20, {"dirs_kind": 1}, B.BOLTZ_FP64, torch.float64, 2),
    (16, 6.0, 1.0, 16, {"term_groups": 4}, B.BOLTZ_FP32_FFT, torch.float32, 1),
    (32, 8.0, 1.0, 16, {}, B.BOLTZ_FP32_FFT, torch.float32, 2),
]


def _make(seed_base=300):
    grids, fs = [], []
    for i, (N, L, gamma, M, opts, prec, dt, cells) in enumerate(GROUPS):
        grids.append(B.Grid(N, L, gamma, M, **opts))
        f = W.two_maxwellians(cells, N, L, seed_base + i)
        f[1::2] = W.bkw(N, L, 0.75)  # ragged batches mix BKW-type cells in
        fs.append(torch.from_numpy(f).to(device="cuda", dtype=dt))
    return grids, fs


def _relax_each(grids, fs, dt, steps, rk, runs):
    out = []
    for (N, L, gamma, M, opts, prec, fdt, cells), g, f in zip(GROUPS, grids, fs):
        x = f.clone()
        for _ in range(runs):
            B.boltz_relax(g.batch(cells, prec, fdt == torch.float64), x, dt, steps, rk)
        out.append(x)
    B.boltz_stream_status()
    return out


@pytest.mark.parametrize("rk", [1, 2])
@pytest.mark.parametrize("flags", [0, B.BOLTZ_PLAN_SERIAL])
def test_plan_equals_per_group_relax(rk, flags):
    """Without autotuning every group runs boltz_relax's launches: bitwise equal, also
    when the plan is run twice (each run projects onto the moments it started from)."""
    grids, fs = _make()
    ref = _relax_each(grids, fs, 0.003, 2, rk, runs=2)
    work = [f.clone() for f in fs]
    groups = [(g, w, spec[5]) for g, w, spec in zip(grids, work, GROUPS)]
    with B.Plan(groups, 0.003, 2, rk, flags) as p:
        p.run()
        p.run()
        B.boltz_stream_status()
        for i in range(len(GROUPS)):
            info = p.info(i)
            assert info["tuned_us"] == 0.0
    for a, b in zip(work, ref):
        assert torch.equal(a, b)
    for g in grids:
        g.close()


def test_plan_autotuned_matches_oracle():
    """Autotuned plan: every group's choice is valid and the result agrees with the
    oracle (FP64 groups to 1e-11 of the increment, FP32 groups within the float32
    bound), the FP32 groups also with boltz_relax at the default configuration."""
    grids, fs = _make(400)
    work = [f.clone() for f in fs]
    groups = [(g, w, spec[5]) for g, w, spec in zip(grids, work, GROUPS)]
    with B.Plan(groups, 0.003, 2, 1, B.BOLTZ_PLAN_AUTOTUNE) as p:
        p.run()
        B.boltz_stream_status()
        infos = [p.info(i) for i in range(len(GROUPS))]
    for i, ((N, L, gamma, M, opts, prec, fdt, cells), f, w, info) in enumerate(zip(GROUPS, fs, work, infos)):
        assert info["tuned_us"] > 0.0 and info["term_groups"] >= 1 and info["cluster"] >= 1
        og = O.make_grid(N, L, gamma=gamma, M=M, dirs_kind=opts.get("dirs_kind", 0), rank=opts.get("radial_rank"))
        f0 = f.double().cpu().numpy()
        ref = O.relax(f0, og, 0.003, 2)
        d = w.double().cpu().numpy() - f0
        rel = np.linalg.norm(d - (ref - f0)) / np.linalg.norm(ref - f0)
        if prec == B.BOLTZ_FP64:
            assert rel <= 1e-11, (i, rel)
        else:
            Qp, Lo = O.operator.gain_loss(f0, og)
            kappa = np.linalg.norm(Qp) / np.linalg.norm(Qp - f0 * Lo)
            assert rel <= 1.25 * EPS32 * math.log2(og.n) * kappa * 2, (i, rel)
    for g in grids:
        g.close()


def test_plan_rejects_shared_grid_and_bad_args():
    with B.Grid(8, 4.0, 1.0, 8) as g:
        f = torch.zeros(1, 8, 8, 8, dtype=torch.float64, device="cuda")
        with pytest.raises(B.BoltzError) as ei:
            B.Plan([(g, f, B.BOLTZ_FP64), (g, f.clone(), B.BOLTZ_FP64)], 0.01, 1)
        assert ei.value.status == B.BOLTZ_EINVAL
        with pytest.raises(B.BoltzError):
            B.Plan([(g, f, B.BOLTZ_FP64)], -1.0, 1)


def test_plan_precision_tuning_is_opt_in_and_float32_class():
    """BOLTZ_PLAN_TUNE_PRECISION may move a float32 FFT group of N = 16 to the 3xTF32
    tensor-core transforms; either way the result stays within twice the float32 bound of
    the oracle (3xTF32 is float32-class), and without the flag the precision never
    changes."""
    N, L, M, cells, dt = 16, 6.0, 16, 64, 0.003
    from paper_1608_08009_gb300 import workloads as W

    f = torch.from_numpy(W.two_maxwellians(cells, N, L, seed=171)).float().cuda()
    og = O.make_grid(N, L, M=M)
    f0 = f.double().cpu().numpy()
    ref = O.relax(f0, og, dt, 1)
    Qp, Lo = O.operator.gain_loss(f0, og)
    tol = 2 * 1.25 * EPS32 * math.log2(og.n) * np.linalg.norm(Qp) / np.linalg.norm(Qp - f0 * Lo) + 4 * EPS32 * \
        np.linalg.norm(f0) / np.linalg.norm(ref - f0)
    for flags, may_switch in ((B.BOLTZ_PLAN_AUTOTUNE, False),
                              (B.BOLTZ_PLAN_AUTOTUNE | B.BOLTZ_PLAN_TUNE_PRECISION, True)):
        with B.Grid(N, L, 1.0, M) as g:
            w = f.clone()
            with B.Plan([(g, w, B.BOLTZ_FP32_FFT)], dt, 1, 1, flags) as p:
                p.run()
                B.boltz_stream_status()
                prec = p.info(0)["prec"]
            assert prec == B.BOLTZ_FP32_FFT or (may_switch and prec == B.BOLTZ_3XTF32_DFT)
            d = w.double().cpu().numpy() - f0
            assert np.linalg.norm(d - (ref - f0)) / np.linalg.norm(ref - f0) <= tol, prec
