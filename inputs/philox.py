"""Counter-based random numbers: Philox4x32-10 and the normal deviates drawn
from it per global DoF id.

Philox4x32-10 is the generator of Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3" (SC'11): a 128-bit counter and a 64-bit
key go through ten rounds of two 32x32->64-bit multiplications, with the key
bumped by two Weyl constants between rounds.  It is written here from that
definition in plain numpy; the CUDA side implements the same definition on its
own (the two share no code).

The serving path draws the right-hand-side noise of a Poisson request from it:
the deviate of global DoF i under seed s is a Box-Muller transform of the
first two output words of Philox(counter = (i mod 2^32, i >> 32, 0, 0),
key = (s mod 2^32, s >> 32)):
    u1 = (w0 + 1) / 2^32 in (0, 1],  u2 = w1 / 2^32 in [0, 1),
    g  = sqrt(-2 ln u1) cos(2 pi u2).
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter: np.ndarray, key) -> np.ndarray:
    """counter: uint32 [n, 4]; key: two uint32 words.  Returns uint32 [n, 4]."""
    c = np.asarray(counter, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0  # exact: both factors < 2^32
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def philox_normal(ids: np.ndarray, seed: int) -> np.ndarray:
    """Standard normal deviates, one per non-negative integer id (float64)."""
    ids = np.asarray(ids, dtype=np.uint64).ravel()
    ctr = np.zeros((ids.size, 4), dtype=np.uint64)
    ctr[:, 0] = ids & _MASK
    ctr[:, 1] = ids >> np.uint64(32)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.float64)
    u1 = (w[:, 0] + 1.0) * 2.0**-32
    u2 = w[:, 1] * 2.0**-32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
