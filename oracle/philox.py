"""Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), written from the published round function.

The paper leaves the random source of its sampling steps unspecified
(Algorithm 2's iid proposals and Algorithm 3's uniform z).  Both this oracle and
the CUDA path draw them from Philox4x32-10 with the same counter layout:

  key     = (seed & 0xffffffff, seed >> 32)
  counter = (draw index j, round index i, stream, 0)
  stream 0: proposal uniforms of Algorithm 2, stream 1: the z of Algorithm 3
  u       = ((w0 >> 5) * 2^26 + (w1 >> 6)) / 2^53  in [0, 1)   (53-bit double)
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF

STREAM_PROPOSE = 0
STREAM_REJECT = 1


def philox4x32_10(ctr, key):
    """One Philox4x32 block with 10 rounds.  ctr: 4 ints, key: 2 ints (uint32 each)."""
    c0, c1, c2, c3 = (int(v) & MASK for v in ctr)
    k0, k1 = (int(v) & MASK for v in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform(seed, stream, rnd, j):
    """The 53-bit uniform double in [0, 1) for draw j of round rnd on a stream."""
    seed = int(seed)
    w = philox4x32_10((j, rnd, stream, 0), (seed & MASK, (seed >> 32) & MASK))
    return ((w[0] >> 5) * 67108864 + (w[1] >> 6)) / 9007199254740992.0


def uniforms(seed, stream, rnd, count):
    return np.array([uniform(seed, stream, rnd, j) for j in range(count)], dtype=np.float64)
