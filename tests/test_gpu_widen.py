"""The integer float32 -> float64 widening used by the float64 kernels that read
float32 inputs (Jacobian apply on the mixed-precision Z, FGMRES update) is exact
for every class of input: zeros, subnormals, normals, infinities and NaNs."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1603_04570_gb300 import _build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("widen") / "widen_probe.so")
    cmd = [_build.nvcc(), *_build.ARCH, "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-shared", os.path.join(HERE, "cuda", "widen_probe.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.widen_probe.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return lib


def test_widening_is_exact_on_every_class(probe):
    rng = np.random.default_rng(3)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan,
                        np.finfo(np.float32).tiny, -np.finfo(np.float32).tiny,      # smallest normal
                        np.finfo(np.float32).max, -np.finfo(np.float32).max,
                        1.0, -1.0, 0.1, 3.0e-39], dtype=np.float32)                  # 3e-39: subnormal
    subn = np.array([1, 2, 3, 0x3fffff, 0x400000, 0x7fffff, 0x80000001, 0x807fffff], dtype=np.uint32).view(np.float32)
    rand_bits = rng.integers(0, 2**32, 4096, dtype=np.uint64).astype(np.uint32).view(np.float32)
    x = np.concatenate([special, subn, rand_bits]).astype(np.float32)
    out = np.empty(x.size, dtype=np.float64)
    assert probe.widen_probe(x.ctypes.data, out.ctypes.data, x.size) == 0
    with np.errstate(invalid="ignore"):                  # signalling NaNs among the random bit patterns
        ref = x.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(out), nan)
    assert np.array_equal(out[~nan].view(np.uint64), ref[~nan].view(np.uint64))   # bitwise, signs of zero too
