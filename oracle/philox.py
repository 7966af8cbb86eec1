"""Counter-based Gaussian test matrices for the oracle (test infrastructure).

The randomized method draws a standard Gaussian test matrix Omega (n x l) for
each side of the pair (Algorithm 1, "Let Omega_i be a Gaussian random matrix";
the fixed-rank variant of Theorem 3 uses one n x (k+p) block).  To let the CUDA
path and this oracle draw the *same* Omega without sharing code, both implement
the published Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller transform
(Box & Muller, Ann. Math. Stat. 1958) from their definitions.

Philox4x32-10 (SC'11, Section 3 "Philox"):
  state  : four 32-bit counter words (c0, c1, c2, c3), key (k0, k1)
  round  : (h0, l0) = hi/lo(0xD2511F53 * c0), (h1, l1) = hi/lo(0xCD9E8D57 * c2)
           (c0, c1, c2, c3) <- (h1 ^ c1 ^ k0, l1, h0 ^ c3 ^ k1, l0)
  key    : after every round k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32)
  output : the counter after 10 rounds.

Mapping of the generator onto Omega (the same definition is written out in
the C header of the library):
  element Omega[i, j] of the row-major n x l matrix has flat index e = i*l + j;
  t = e >> 1 and slot = e & 1.
  counter = (t mod 2^32, pair, side, stream), key = (seed mod 2^32, seed >> 32)
  words x0..x3 -> u1 = ((x0 >> 5) * 2^26 + (x1 >> 6) + 0.5) * 2^-53  in (0, 1)
                  u2 = ((x2 >> 5) * 2^26 + (x3 >> 6))       * 2^-53  in [0, 1)
  r = sqrt(-2 ln u1), theta = 2 pi u2;  slot 0 -> r cos(theta), slot 1 -> r sin(theta).
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counters (SC'11, Section 3).

    All arguments are broadcastable integer arrays holding values < 2^32.
    Returns four uint32 arrays.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & MASK32
            k1 = (k1 + _W1) & MASK32
        p0 = _M0 * c0  # exact: both factors < 2^32, product < 2^64
        p1 = _M1 * c2
        h0, l0 = p0 >> np.uint64(32), p0 & MASK32
        h1, l1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = h1 ^ c1 ^ k0, l1, h0 ^ c3 ^ k1, l0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def philox_words(num: int, seed: int, pair: int = 0, side: int = 0, stream: int = 0):
    """The raw 4 x num uint32 words for counters t = 0..num-1."""
    t = np.arange(num, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(t, pair, side, stream, seed & 0xFFFFFFFF, seed >> 32)


def gaussian(n: int, l: int, seed: int, pair: int = 0, side: int = 0, stream: int = 0) -> np.ndarray:
    """Omega in R^{n x l}, i.i.d. N(0,1), float64 (Box-Muller on Philox words)."""
    total = n * l
    npairs = (total + 1) // 2
    x0, x1, x2, x3 = philox_words(npairs, seed, pair, side, stream)
    a = (x0 >> 5).astype(np.float64)
    b = (x1 >> 6).astype(np.float64)
    c = (x2 >> 5).astype(np.float64)
    d = (x3 >> 6).astype(np.float64)
    u1 = (a * 67108864.0 + b + 0.5) * 2.0 ** -53
    u2 = (c * 67108864.0 + d) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    return z[:total].reshape(n, l)
