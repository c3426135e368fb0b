"""Pin of the oracle's Philox4x32-10 against an independent implementation:
cuRAND's device generator (curandStatePhilox4_32_10_t, the same published
algorithm of Salmon et al., SC'11), run by a test-only kernel
(tests/cuda/philox_curand.cu) built here with nvcc.  The four output words
must agree bit for bit over random counters and keys, so a mistake shared by
the oracle and the library's own copy (a swapped multiplier, a misplaced key
increment) would fail.  Section 2.6's per-cell streams, the seeding and the
kill draws all rest on this generator.
"""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.philox import philox4x32_10, site_uniform
from paper_2105_00448_gb300 import hca

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("philox") / "libphilox_curand.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "cuda", "philox_curand.cu"), "-o", out], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.philox_curand.restype = ctypes.c_int
    lib.philox_curand.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    return lib


def curand_words(lib, ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty_like(ctr)
    assert lib.philox_curand(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0]) == 0
    return out


def test_oracle_philox_matches_curand_bit_for_bit(curand_lib):
    n = 200_000
    rng = np.random.default_rng(2105)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    ctr[:, 1] &= (1 << 30) - 1          # keeps cuRAND's offset 4 (c0 | c1 << 32) within 64 bits
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    # edge values: all-zero and all-one words
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF, (1 << 30) - 1, 0xFFFFFFFF, 0xFFFFFFFF], [1, 0, 0, 0], [0, 0, 0, 1]]
    key[:4] = [[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0, 0], [1, 0]]
    got = curand_words(curand_lib, ctr, key)
    ref = np.stack(philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], key[:, 0], key[:, 1]), axis=1)
    assert np.array_equal(got.astype(np.uint64), ref)


def test_site_uniforms_are_curand_words(curand_lib):
    """The 24-bit uniforms of the library and the oracle are cuRAND's first
    output word of counter (site lo, site hi, step, purpose), key = seed."""
    seed, step, purpose = (7 << 32) | 12345, 41, 3
    sites = np.arange(1 << 20, (1 << 20) + 65536, dtype=np.uint64)
    ctr = np.stack([sites & 0xFFFFFFFF, sites >> 32, np.full_like(sites, step), np.full_like(sites, purpose)], axis=1)
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64), (sites.size, 1))
    w0 = curand_words(curand_lib, ctr, key)[:, 0].astype(np.uint64)
    u_curand = (w0 >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    assert np.array_equal(site_uniform(seed, sites, step, purpose), u_curand)
    import torch

    dst = torch.empty(sites.size, dtype=torch.float32, device="cuda")
    hca.hca_philox_uniforms(seed, int(sites[0]), sites.size, step, purpose, dst)
    assert np.array_equal(dst.cpu().numpy().astype(np.float64), u_curand)
