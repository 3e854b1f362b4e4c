"""Oracle: the counter-based generator both sides implement (test infrastructure).

Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011): ten rounds of two 32x32 -> 64-bit multiplications
(multipliers 0xD2511F53 and 0xCD9E8D57) on a 4-word counter with a 2-word key
bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.  A
standard normal comes from the first two output words by the Box-Muller
transform with u = (x + 1/2) / 2^32.

The Langevin thermostat draws one normal per atom, Cartesian component, half
step (phase 0: before the first half-kick, phase 1: after the second) and MD
step, from counter (component index, phase, step low word, step high word)
and key (seed low word, seed high word).
"""
import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """ctr: 4 uint32 arrays (broadcastable), key: 2 uint32 values -> 4 uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) for x in ctr]
    k0, k1 = np.uint64(key[0] & MASK), np.uint64(key[1] & MASK)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return [x.astype(np.uint32) for x in c]


def normals(n, phase, step, seed):
    """n standard normals for components 0..n-1 at (phase, step) under seed."""
    idx = np.arange(n, dtype=np.uint64)
    ctr = [idx, np.full(n, phase, dtype=np.uint64), np.full(n, step & MASK, dtype=np.uint64),
           np.full(n, (step >> 32) & MASK, dtype=np.uint64)]
    x = philox4x32_10(ctr, (seed & MASK, (seed >> 32) & MASK))
    u1 = (x[0].astype(np.float64) + 0.5) / 4294967296.0
    u2 = (x[1].astype(np.float64) + 0.5) / 4294967296.0
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
