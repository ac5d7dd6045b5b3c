"""boltz_relax_noalloc against boltz_relax (rk_order 1) through the C ABI.

The no-allocation entry point serves callers that cannot let the library call
cudaMalloc / cudaFree: its per-cell moment targets live in a fixed array in the
library's device image.  It must give the same result as the allocating entry point,
call after call, although every call reuses (and leaves behind) the same array.  This
file is collected last so a failure here does not hide the other GPU tests.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1608_08009_gb300 import boltz as B
from paper_1608_08009_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def fp32_tol(f, og):
    Qp, Lo = O.operator.gain_loss(f, og)
    kappa = np.linalg.norm(Qp) / np.linalg.norm(Qp - f * Lo)
    return 1.25 * 2.0 ** -24 * math.log2(og.n) * kappa


def test_relax_noalloc_matches_relax_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, L, M, dt, steps = 16, 6.0, 16, 0.004, 3
    og = O.make_grid(N, L, M=M)
    with B.Grid(N, L, 1.0, M) as g:
        # two calls in a row with different batches: the second reuses the array the
        # first one left behind
        for call, (cells, seed) in enumerate(((7, 101), (3, 202))):
            f = W.two_maxwellians(cells, N, L, seed=seed)
            for prec in (B.BOLTZ_FP64, B.BOLTZ_FP32_FFT):
                tol = 1e-12 if prec == B.BOLTZ_FP64 else fp32_tol(f, og)
                ref = torch.from_numpy(f).cuda()
                out = torch.from_numpy(f).cuda()
                B.boltz_relax(g.batch(cells, prec), ref, dt, steps, 1)
                B.boltz_relax_noalloc(g.batch(cells, prec), out, dt, steps)
                B.boltz_stream_status()
                d_ref = ref.cpu().numpy() - f
                d_out = out.cpu().numpy() - f
                assert rel_l2(d_out, d_ref) <= tol, (call, prec)


def test_relax_noalloc_rejects_oversize_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with B.Grid(16, 6.0, 1.0, 8) as g:
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_relax_noalloc(g.batch(65537), 1, 0.1, 1)
        assert ei.value.status == B.BOLTZ_EINVAL
        assert "65536" in str(ei.value)
