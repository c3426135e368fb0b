"""Philox4x32-10 counter-based random numbers (vectorised numpy).

The paper asks that each cell draw its own stream, independent of the process
count (Section 2.6, "Choosing a scalable parallel RNG"), and uses a PCG
generator.  This oracle keys a counter-based generator by (seed, site, step,
purpose) instead, which gives the same independence from any partition of the
lattice.

Philox4x32-10 follows the published definition of Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds; each
round multiplies counter words 0 and 2 by two fixed 32-bit multipliers, forms
the new counter from the high/low product halves xor-ed with the other two
counter words and the key, and adds the two Weyl constants to the key between
rounds.

Uniforms are 24-bit: u = (w >> 8) * 2**-24, exactly representable in float32
and float64, in [0, 1).
"""

from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (as uint64 arrays) for the counters."""
    c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & MASK32
                              for v in (c0, c1, c2, c3, k0, k1))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (a.copy() for a in (c0, c1, c2, c3))
    k0 = np.broadcast_to(k0, c0.shape).copy()
    k1 = np.broadcast_to(k1, c0.shape).copy()
    for _ in range(10):
        prod0 = PHILOX_M0 * c0          # < 2**64: exact in uint64
        prod1 = PHILOX_M1 * c2
        hi0, lo0 = prod0 >> np.uint64(32), prod0 & MASK32
        hi1, lo1 = prod1 >> np.uint64(32), prod1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & MASK32
        k1 = (k1 + PHILOX_W1) & MASK32
    return c0, c1, c2, c3


def site_uniform(seed: int, site, step: int, purpose: int) -> np.ndarray:
    """24-bit uniform for each site id, keyed by (seed, site, step, purpose).

    Counter = (site low word, site high word, step, purpose); key = (seed low
    word, seed high word); the first output word is used.
    """
    site = np.asarray(site, dtype=np.uint64)
    seed = int(seed)
    w0, _, _, _ = philox4x32_10(site & MASK32, site >> np.uint64(32),
                                np.uint64(step & 0xFFFFFFFF), np.uint64(purpose),
                                np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    return (w0 >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
