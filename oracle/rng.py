"""Counter-based uniform numbers for the stochastic hard-concrete gate (the
training-time sampling of the gate the paper adopts, Sec. 3.2.2).  Test
infrastructure only; shares no code with the CUDA path, which implements the
same generator on its own.

Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011): a 4 x 32-bit counter and a 2 x 32-bit key; a round
multiplies words 0 and 2 by M0 = 0xD2511F53 and M1 = 0xCD9E8D57 into 64-bit
products (hi, lo) and forms (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key
is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds; ten
rounds.

The gate noise of Gaussian i at step t under seed s: the first output word x
of the counter (i, t, 0, 0) and key (s mod 2^32, s >> 32), mapped to
u = ((x >> 9) + 1/2) / 2^23 in (0, 1) (24 significant bits: exactly
representable in FP32).
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """ctr [4][...] and key [2][...] uint32 arrays (broadcast); returns [4][...]."""
    c = [np.asarray(v, np.uint64) & MASK for v in ctr]
    k0 = np.asarray(key[0], np.uint64) & MASK
    k1 = np.asarray(key[1], np.uint64) & MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = c[0] * np.uint64(M0)
        p1 = c[2] * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [(hi1 ^ c[1] ^ k0) & MASK, lo1, (hi0 ^ c[3] ^ k1) & MASK, lo0]
    return [v.astype(np.uint32) for v in c]


def gate_uniform(n, seed, step):
    """u [n] float32 in (0, 1): the gate noise of Gaussians 0..n-1 at step."""
    i = np.arange(n, dtype=np.uint64)
    z = np.zeros(n, np.uint64)
    x = philox4x32_10([i, z + np.uint64(step & MASK), z, z], [np.uint64(seed & MASK), np.uint64((seed >> 32) & MASK)])[0]
    return (((x >> np.uint32(9)).astype(np.float64) + 0.5) / float(1 << 23)).astype(np.float32)
