"""Philox4x32-10 counter-based generator and Box-Muller normals (numpy, oracle side).

Written from the published definition (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter
and 2 x 32-bit key; each of 10 rounds multiplies words 0 and 2 by the
constants 0xD2511F53 / 0xCD9E8D57 (64-bit products split hi/lo), mixes the
high halves with the other words and the key, and the key is bumped by the
Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.

Stream layout used by this library (the CUDA path implements the same
definition independently):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (element, stream, sample & 0xffffffff, sample >> 32)
    stream  = 2 * system + 0 for the real-space z1 (one call per particle),
              2 * system + 1 for the wave-space dW2 (two calls per mode).
Uniforms use the top 23 bits, u = ((x >> 9) + 0.5) * 2^-23 = (2k + 1) 2^-24,
which needs 24 significant bits and so is exact in float32 as well, and pairs (u_a, u_b) map to normals by Box-Muller:
    z = sqrt(-2 ln u_a) * (cos 2 pi u_b, sin 2 pi u_b).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint32-valued arrays; returns 4 uint64 arrays < 2^32."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def uniform23(x):
    """((x >> 9) + 0.5) * 2^-23 in (0, 1), exactly representable in float32."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def normals4(element, stream, seed, sample):
    """Four N(0,1) per element index: Box-Muller on one Philox block."""
    element = np.asarray(element, dtype=np.uint64)
    seed = np.uint64(seed)
    sample = np.uint64(sample)
    x0, x1, x2, x3 = philox4x32_10(element, np.uint64(stream) + 0 * element,
                                   sample & MASK, sample >> np.uint64(32),
                                   seed & MASK, seed >> np.uint64(32))
    ua, ub, uc, ud = uniform23(x0), uniform23(x1), uniform23(x2), uniform23(x3)
    ra = np.sqrt(-2.0 * np.log(ua))
    rc = np.sqrt(-2.0 * np.log(uc))
    return np.stack([ra * np.cos(2 * np.pi * ub), ra * np.sin(2 * np.pi * ub),
                     rc * np.cos(2 * np.pi * ud), rc * np.sin(2 * np.pi * ud)], axis=-1)
