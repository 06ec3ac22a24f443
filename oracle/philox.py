"""Counter-based Gaussian sketch cores for the random TT of Definition 2.1.

Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4x32-bit counter and a 2x32-bit key,
ten rounds; each round multiplies counter words 0 and 2 by the Philox
multipliers, mixes the high halves with the other two words and the round key,
and the key advances by the Weyl constants between rounds.

Sketch entry (this build's reading, the paper leaves the generator open):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (flat, core, pair, 0), flat the row-major index [lambda][i][gamma]
  u1 = ((x0 >> 6) * 2^26 + (x1 >> 6) + 1/2) * 2^-52   in (0, 1), exact in fp64
  u2 = ((x2 >> 6) * 2^26 + (x3 >> 6) + 1/2) * 2^-52
  g  = sqrt(-2 ln u1) * cos(2*pi*u2)                  (Box-Muller)
  R_k[lambda, i, gamma] = g / sqrt(l_{k-1} n_k l_k)   (variance of Definition 2.1)
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Philox4x32-10 block function.

    counter: uint32 array of shape (..., 4); key: pair of ints (k0, k1).
    Returns a uint32 array of shape (..., 4).
    """
    c = np.asarray(counter, dtype=np.uint32)
    x0 = c[..., 0].astype(np.uint64)
    x1 = c[..., 1].astype(np.uint64)
    x2 = c[..., 2].astype(np.uint64)
    x3 = c[..., 3].astype(np.uint64)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
        p0 = m0 * x0          # 32x32 -> 64-bit products, exact in uint64
        p1 = m1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def uniforms_from_words(xa, xb):
    """Map two 32-bit words to a uniform double in (0, 1) with 52 random bits.
    The value (k + 1/2) * 2^-52, k < 2^52, is exact in fp64, never 0 or 1."""
    hi = (np.asarray(xa, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    lo = (np.asarray(xb, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo + 0.5) * (2.0 ** -52)


def gaussian_from_words(words):
    """Box-Muller on one Philox output block (..., 4) -> one N(0,1) sample."""
    u1 = uniforms_from_words(words[..., 0], words[..., 1])
    u2 = uniforms_from_words(words[..., 2], words[..., 3])
    return np.sqrt(-2.0 * np.log(u1)) * np.cos((2.0 * np.pi) * u2)


def sketch_core(seed: int, core: int, shape, pair: int = 0):
    """One Gaussian sketch core R_k of shape (l_{k-1}, n_k, l_k), Definition 2.1."""
    a, n, b = (int(v) for v in shape)
    count = a * n * b
    ctr = np.zeros((count, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(count, dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] = np.uint32(core)
    ctr[:, 2] = np.uint32(pair)
    key = (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    g = gaussian_from_words(philox4x32_10(ctr, key))
    return (g / np.sqrt(float(a * n * b))).reshape(a, n, b)


def sketch_tt(seed: int, n, ell, pair: int = 0):
    """Random Gaussian TT R with ranks ell = [1, l_1, ..., l_{d-1}, 1] (Definition 2.1)."""
    return [sketch_core(seed, k, (ell[k], n[k], ell[k + 1]), pair) for k in range(len(n))]
