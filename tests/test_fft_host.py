"""The kernels' register FFT, built for the host and checked without a GPU.

Every pass of the collision kernels (the forward transform of f and the inverse
transforms of each term, arxiv 1608.08009 Sec. 3.3 and Sec. 4.2) runs the fully unrolled
radix-4/2 (and radix-3) transform of csrc/fft_regs.cuh.  tests/fft_host_check.cpp compiles
that header as plain C++ and compares every length the kernels use, both signs, in
float64 and float32, with a direct float64 DFT; it also checks the factored twiddles of
the radix-4 stages (w = lam i^e (1 + i mu), rho = lam(3m) / lam(m)) against
exp(2 pi i m / 192).
"""

import json
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1608_08009_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "fft_host_check.cpp")
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    inc = _cuda_include()
    if gxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_host_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-w", "-I", inc, "-I", CSRC, SRC, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True, timeout=120).stdout
    return json.loads(out)


def test_factored_twiddles(report):
    # lam * (turned u) reproduces w x for every m and both signs; rho pairs w with w^3
    assert report["factor_err"] <= 8 * EPS64
    assert report["rho_err"] <= 8 * EPS64


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 6, 12, 24, 48])
def test_float64_transform(report, n):
    fwd, inv = report["f64"][f"N{n}"]
    bound = 3 * EPS64 * (math.log2(n) + 1)
    assert fwd <= bound and inv <= bound, (n, fwd, inv, bound)


@pytest.mark.parametrize("n", [8, 16, 32, 64, 24, 48])
def test_float32_transform(report, n):
    fwd, inv = report["f32"][f"N{n}"]
    bound = 3 * EPS32 * (math.log2(n) + 1)
    assert fwd <= bound and inv <= bound, (n, fwd, inv, bound)
    # and not exact: the float32 path really rounds in float32
    assert fwd > EPS64 * 1e3
