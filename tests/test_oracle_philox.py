"""Pins for the oracle's Philox4x32-10 generator.

These CPU tests pin the generator by what a counter-based generator must do:
uniform, independent outputs across counters, keys and purposes, full
avalanche of a one-bit counter change, and the exact 24-bit uniform mapping.
Its output bits are pinned against an independent implementation, cuRAND's
Philox4_32_10 device generator, in tests/test_gpu_philox_curand.py (needs a
GPU); bit identity with the library's own copy is checked in the GPU parity
tests.
"""

import numpy as np
import pytest

from oracle.philox import philox4x32_10, site_uniform


def test_uniform_moments_and_chi2():
    u = site_uniform(seed=1, site=np.arange(1_000_000), step=7, purpose=3)
    assert u.min() >= 0.0 and u.max() < 1.0
    n = u.size
    # mean 1/2, variance 1/12 within 5 sigma
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    counts = np.bincount((u * 256).astype(int), minlength=256)
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    # chi2 with 255 dof: mean 255, sd ~22.6; 6 sigma band
    assert 255 - 6 * 22.6 < chi2 < 255 + 6 * 22.6


def test_streams_independent():
    sites = np.arange(200_000)
    a = site_uniform(5, sites, 0, 0)
    b = site_uniform(5, sites, 0, 1)          # other purpose
    c = site_uniform(5, sites, 1, 0)          # other step
    d = site_uniform(6, sites, 0, 0)          # other seed
    e = site_uniform(5, sites + 1, 0, 0)      # neighbouring site
    bound = 5 / np.sqrt(sites.size)
    for other in (b, c, d, e):
        assert abs(np.corrcoef(a, other)[0, 1]) < bound
    # lag-1 serial correlation along the site axis
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < bound


def test_avalanche():
    rng = np.random.default_rng(0)
    n = 4000
    c = [rng.integers(0, 2**32, n, dtype=np.uint64) for _ in range(4)]
    k = [rng.integers(0, 2**32, n, dtype=np.uint64) for _ in range(2)]
    base = philox4x32_10(*c, *k)
    for word in range(4):
        for bit in (0, 13, 31):
            cc = [x.copy() for x in c]
            cc[word] ^= np.uint64(1 << bit)
            flip = philox4x32_10(*cc, *k)
            changed = sum(np.unpackbits((b ^ f).astype(np.uint32).view(np.uint8)).sum()
                          for b, f in zip(base, flip))
            frac = changed / (n * 128)
            assert abs(frac - 0.5) < 0.01, (word, bit, frac)


def test_output_words_uniform_bits():
    out = philox4x32_10(np.arange(100_000), 0, 0, 0, 3, 4)
    for w in out:
        bits = np.unpackbits(w.astype(np.uint32).view(np.uint8)).reshape(-1, 32)
        p = bits.mean(axis=0)
        assert np.all(np.abs(p - 0.5) < 5 * np.sqrt(0.25 / bits.shape[0]))


def test_uniform_is_exact_24_bit():
    u = site_uniform(9, np.arange(10_000), 2, 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert np.all((u * 2**24) == np.floor(u * 2**24))


def test_counter_is_partition_independent():
    # The same (seed, site, step, purpose) gives the same number whatever set
    # of sites is drawn together (the paper's requirement in Section 2.6).
    sites = np.arange(1000)
    full = site_uniform(3, sites, 4, 2)
    part = np.concatenate([site_uniform(3, s, 4, 2) for s in np.array_split(sites[::-1], 7)])
    assert np.array_equal(full[::-1], part)


@pytest.mark.parametrize("seed", [0, 2**32 + 5, 2**63 + 11])
def test_seed_high_word_used(seed):
    a = site_uniform(seed, np.arange(64), 0, 0)
    b = site_uniform(seed ^ (1 << 40), np.arange(64), 0, 0)
    assert not np.array_equal(a, b)
