"""The 2D kernel converts float <-> double on the integer pipes (GB300 issues the hardware
conversions to its narrow FP64 pipe, which binds that kernel).  These conversions must be
exact: the library's self-check compares them with the hardware conversions, float ->
double on every float bit pattern and double -> float on 2^32 pseudo-random doubles plus
the ties and near-ties between neighbouring floats."""

import pytest

from paper_1608_08009_gb300 import boltz as B

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_integer_pipe_conversions_match_the_hardware():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f2d, d2f = B.boltz_selftest_conversions()
    assert (f2d, d2f) == (0, 0)
