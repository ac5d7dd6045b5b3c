"""boltz_relax_noalloc against boltz_relax (rk_order 1) through the C ABI.

The no-allocation entry point serves callers that cannot let the library call
cudaMalloc / cudaFree: its per-cell moment targets live in a fixed array in the
library's device image.  It runs the same launches as the allocating entry point (one
term group, targets computed by the first launch), so on grids with one term group it
must give the same bits, call after call, although every call reuses (and leaves behind)
the same array.  This file is collected last so a failure here does not hide the other
GPU tests.
"""

import numpy as np
import pytest

from paper_1608_08009_gb300 import boltz as B
from paper_1608_08009_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _grid(kind):
    if kind == "3d16":
        return B.Grid(16, 6.0, 1.0, 16), (16, 16, 16), lambda c, s: W.two_maxwellians(c, 16, 6.0, seed=s)
    if kind == "3d32":
        return B.Grid(32, 8.0, 1.0, 8), (32, 32, 32), lambda c, s: W.two_maxwellians(c, 32, 8.0, seed=s)
    return (B.Grid2D(16, 6.0, 8, C_gamma=1.0 / (2.0 * np.pi)), (16, 16),
            lambda c, s: W.two_maxwellians_2d(c, 16, 6.0, seed=s))


CASES = [("3d16", B.BOLTZ_FP64, True), ("3d16", B.BOLTZ_FP32_FFT, True), ("3d16", B.BOLTZ_FP32_FFT, False),
         ("3d16", B.BOLTZ_TF32_DFT, False), ("3d32", B.BOLTZ_FP32_FFT, False), ("2d", B.BOLTZ_FP64, True),
         ("2d", B.BOLTZ_FP32_FFT, False)]


@pytest.mark.parametrize("kind,prec,fp64", CASES)
def test_relax_noalloc_matches_relax_on_consecutive_calls(kind, prec, fp64):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dt, steps = 0.004, 3
    g, shape, make = _grid(kind)
    dtype = torch.float64 if fp64 else torch.float32
    with g:
        # two calls in a row with different batches: the second reuses the array the
        # first one left behind (and the second batch is smaller, so stale rows remain)
        for call, (cells, seed) in enumerate(((7, 101), (3, 202))):
            f = torch.from_numpy(make(cells, seed)).to(dtype)
            ref = f.cuda()
            out = f.cuda()
            B.boltz_relax(g.batch(cells, prec, fp64), ref, dt, steps, 1)
            B.boltz_relax_noalloc(g.batch(cells, prec, fp64), out, dt, steps)
            B.boltz_stream_status()
            assert not torch.equal(out.cpu(), f), (call, kind, prec)  # the state moved
            assert torch.equal(out, ref), (call, kind, prec)


def test_relax_noalloc_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with B.Grid(16, 6.0, 1.0, 8) as g:
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_relax_noalloc(g.batch(65537), 1, 0.1, 1)
        assert ei.value.status == B.BOLTZ_EINVAL
        assert "65536" in str(ei.value)
        bad = g.batch(1)
        bad.prec = 17  # an unknown precision is an argument error, as in every entry point
        with pytest.raises(B.BoltzError) as ei:
            B.boltz_relax_noalloc(bad, 1, 0.1, 1)
        assert ei.value.status == B.BOLTZ_EINVAL
