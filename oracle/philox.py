"""Oracle: Philox4x32-10 and the Gaussian test-matrix entries.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper draws the blocks G_beta of the test matrices (eq. h1constraints,
eq. neartestmatrices) from the standard normal distribution and says no more.
Both implementations must draw the same numbers, so each one implements the
counter-based generator Philox4x32-10 from its published definition (Salmon,
Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
ten rounds of two 32x32->64-bit multiplications with multipliers 0xD2511F53 and
0xCD9E8D57, and a Weyl key schedule with increments 0x9E3779B9 and 0xBB67AE85.

Reading (paper silent): entry (i, j) of G_beta for side s (0 = Omega, 1 = Psi)
at cut level l is drawn with key = seed (64 bits) and counter
  (j, i, gid(beta), (s << 8) | l)
where i is the row within the box and gid the global box id.  The two 64-bit
halves of the output give uniforms u = ((x >> 12) + 1/2) * 2^-52 in (0, 1) (the sum
is exact, so u never rounds to 1), and
Box-Muller gives z = sqrt(-2 ln u1) cos(2 pi u2).  Keying by box (not by colour)
makes G_beta the same in every colour where beta is active.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.  ctr: 4 uint32 arrays; key: 2 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & MASK for k in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = c0 * np.uint64(M0)          # < 2^64: exact in uint64
        p1 = c2 * np.uint64(M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def uniform53(lo32, hi32):
    """Uniform in (0, 1) from 64 random bits: ((x >> 12) + 1/2) 2^-52, exact."""
    x = (np.asarray(hi32, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo32, dtype=np.uint64)
    return ((x >> np.uint64(12)).astype(np.float64) + 0.5) * (2.0 ** -52)


def gaussian_block(seed: int, side: int, level: int, gid: int, rows: int, cols: int) -> np.ndarray:
    """G (rows x cols) for one box: entry (i, j) from counter (j, i, gid, side<<8|level)."""
    i, j = np.meshgrid(np.arange(rows, dtype=np.uint64), np.arange(cols, dtype=np.uint64),
                       indexing="ij")
    i, j = i.ravel(), j.ravel()
    n = i.shape[0]
    ctr = (j, i, np.full(n, gid, dtype=np.uint64),
           np.full(n, (side << 8) | level, dtype=np.uint64))
    key = (np.full(n, seed & MASK, dtype=np.uint64), np.full(n, (seed >> 32) & MASK, dtype=np.uint64))
    x0, x1, x2, x3 = philox4x32_10(ctr, key)
    u1, u2 = uniform53(x0, x1), uniform53(x2, x3)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.reshape(rows, cols)
