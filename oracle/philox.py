"""Philox4x64-10 and the Gaussian sketch Omega (oracle side).

The paper fills Omega with Gaussian random numbers (Sec. IV) without naming a
generator. Both sides implement one counter-based generator from its published
definition: Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), followed by the Box-Muller
transform. Pinned against ``numpy.random.Philox`` raw output (a known-answer
test) in the test suite.

Omega element (i, j) of a sketch uses
    counter = (i >> 1, j, site | stage << 16, row | env << 16)
    key     = (seed, layer)
and the word pair (x0, x1) for even i, (x2, x3) for odd i:
    u = ((x >> 11) + 0.5) * 2^-53,   z = sqrt(-2 ln u1) * cos(2 pi u2).
i is the C-order flat row index of the sketched space.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.ndarray, b: np.uint64):
    """Full 64x64 -> 128-bit product as (hi, lo), from 32-bit halves."""
    a0 = a & _MASK32
    a1 = a >> _S32
    b0 = b & _MASK32
    b1 = b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _MASK32) + (p10 & _MASK32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(ctr, key):
    """Apply 10 Philox4x64 rounds. ctr: 4 uint64 arrays (broadcastable), key: 2 uint64."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) for x in ctr)
        k0 = np.uint64(key[0])
        k1 = np.uint64(key[1])
        for rnd in range(10):
            hi0, lo0 = _mulhilo(c0, _M0)
            hi1, lo1 = _mulhilo(c2, _M1)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            if rnd < 9:
                k0 = k0 + _W0
                k1 = k1 + _W1
    return c0, c1, c2, c3


def uniform53(x: np.ndarray) -> np.ndarray:
    """Open-interval uniform (0,1) from the top 53 bits of a 64-bit word."""
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def gaussian_sketch(n: int, k: int, *, seed: int, layer: int, stage: int, site: int, row: int,
                    env: int = 0) -> np.ndarray:
    """Omega (n x k, float64) for one sketch; element (i, j) as in the module docstring."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(k, dtype=np.uint64)[None, :]
    w2 = np.uint64(site | (stage << 16))
    w3 = np.uint64(row | (env << 16))
    x0, x1, x2, x3 = philox4x64_10((i >> np.uint64(1), j, w2, w3), (seed, layer))
    odd = (i & np.uint64(1)).astype(bool)
    a = np.where(odd, x2, x0)
    b = np.where(odd, x3, x1)
    u1 = uniform53(a)
    u2 = uniform53(b)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
