"""The library's fifth-generation tensor-core primitives (csrc/tc.cuh:
tensor-memory allocation, shared-memory and instruction descriptors, the
single-thread MMA issue, mbarrier completion and tcgen05.ld) against numpy: a
test-only kernel (tests/cuda/tcgen05_gemm.cu) computes C = A B^T for BF16 A
(128 x K) and B (N x K) in FP32 on the tensor cores.  BF16 products are exact
in FP32, so the only difference from the FP64 reference is the FP32
summation order."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def tc_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("tc") / "libtc_gemm.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "cuda", "tcgen05_gemm.cu"), "-o", out], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.tc_gemm.restype = ctypes.c_int
    lib.tc_gemm.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 3
    return lib


def bf16_bits(x):
    """Round-to-nearest-even FP32 -> BF16 bit patterns, and their values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r, (r.astype(np.uint32) << 16).view(np.float32)


def run(lib, n, k, swap, rng):
    a16, a = bf16_bits(rng.standard_normal((128, k)))
    b16, b = bf16_bits(rng.standard_normal((n, k)))
    c = np.empty((128, n), dtype=np.float32)
    rc = lib.tc_gemm(a16.ctypes.data, b16.ctypes.data, c.ctypes.data, n, k, swap)
    return rc, c, a.astype(np.float64) @ b.astype(np.float64).T


@pytest.mark.parametrize("n,k", [(16, 16), (32, 32), (64, 64), (48, 16)])
def test_tcgen05_bf16_gemm(tc_lib, n, k):
    rng = np.random.default_rng(n * 100 + k)
    rc, c, ref = run(tc_lib, n, k, 0, rng)
    assert rc == 0
    assert np.max(np.abs(c - ref)) <= 1e-5 * np.max(np.abs(ref)) + 1e-6
