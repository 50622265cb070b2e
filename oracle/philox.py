"""Oracle Philox4x32-10 generator and Box-Muller normals.  TEST INFRASTRUCTURE ONLY.

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  One round maps
a 4x32-bit counter (c0, c1, c2, c3) and a 2x32-bit key (k0, k1) to

  (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

with multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is
bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.

Counter layout used for the gDC draws (the CUDA side implements the same
published generator independently):

  key     = (seed & 0xffffffff, seed >> 32)
  counter = (j, suspension, step, stream)   stream 0: W, stream 1: W-tilde

Output words (x0, x1, x2, x3) of counter j give two 53-bit uniforms
u = (x0 >> 5) * 2^-27 + (x1 >> 6) * 2^-53 and v from (x2, x3), and two
normals by Box-Muller: sqrt(-2 ln(1 - u)) * (cos 2 pi v, sin 2 pi v).
Normal k of a draw is component k % 2 of counter j = k // 2.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

STREAM_W = 0
STREAM_WTILDE = 1


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Vectorised Philox4x32-10.  ctr: (n, 4) uint32-valued; key: (k0, k1).  Returns (n, 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4) & _MASK
    c0, c1, c2, c3 = c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy()
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0)), lo1, (hi0 ^ c3 ^ np.uint64(k1)), lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def raw_words(seed: int, susp: int, step: int, stream: int, n_ctr: int) -> np.ndarray:
    j = np.arange(n_ctr, dtype=np.uint64)
    ctr = np.stack([j, np.full_like(j, susp), np.full_like(j, step & 0xFFFFFFFF),
                    np.full_like(j, stream)], axis=1)
    return philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))


def normals(seed: int, susp: int, step: int, stream: int, count: int) -> np.ndarray:
    """The first ``count`` N(0,1) draws of (seed, suspension, step, stream)."""
    n_ctr = (count + 1) // 2
    x = raw_words(seed, susp, step, stream, n_ctr).astype(np.float64)
    u = np.floor(x[:, 0] / 32.0) * 2.0 ** -27 + np.floor(x[:, 1] / 64.0) * 2.0 ** -53
    v = np.floor(x[:, 2] / 32.0) * 2.0 ** -27 + np.floor(x[:, 3] / 64.0) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log1p(-u))
    z = np.stack([rad * np.cos(2.0 * np.pi * v), rad * np.sin(2.0 * np.pi * v)], axis=1)
    return z.reshape(-1)[:count]
