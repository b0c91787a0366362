"""Philox4x32-10 counter-based generator and the draws of Algorithm 1 (oracle side).

Philox4x32 is defined in Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11: a 4-word counter and a 2-word key; each of the 10 rounds multiplies
words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57, takes the 64-bit products
apart into hi/lo halves and permutes/xors them with words 1, 3 and the key; the key is
bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.

Pinned by tests/golden/philox4x32_10_kat.txt (the known-answer vectors published with
that paper's Random123 library).

Draws used by the solvers (the paper leaves the sampling scheme open; these are the
readings recorded in the design notes):
  counter = (k mod 2^32, k >> 32, job, tag), key = (seed mod 2^32, seed >> 32)
  word 0 -> subset index      i_k   = floor(u0 * N / 2^32)        (uniform, with replacement)
  word 1 -> skip coin         theta = [u1 < floor(p * 2^32)]        (p >= 1 means always 1)
  word 2 -> L-SVRG refresh    coin  = [u2 < floor(2^32 / N)]        (probability 1/N)
"""
from __future__ import annotations

import numpy as np

MASK32 = 0xFFFFFFFF
M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85

TAG_SCHEDULE = 0     # subset / coin draws of the outer iteration
TAG_POWER = 1        # start vector of the power iteration


def philox4x32_10(ctr, key):
    """One block: ctr = 4 uint32 ints, key = 2 uint32 ints -> tuple of 4 uint32 ints."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & MASK32, (p0 >> 32) ^ c3 ^ k1, p0 & MASK32)
    return c0, c1, c2, c3


def philox4x32_10_many(c0: np.ndarray, c1, c2, c3, key) -> np.ndarray:
    """Vectorised form over arrays of counters; returns uint64 array [len, 4] of 32-bit words."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    n = c0.shape[0]
    c1 = np.broadcast_to(np.asarray(c1, dtype=np.uint64), (n,)) & MASK32
    c2 = np.broadcast_to(np.asarray(c2, dtype=np.uint64), (n,)) & MASK32
    c3 = np.broadcast_to(np.asarray(c3, dtype=np.uint64), (n,)) & MASK32
    k0, k1 = int(key[0]) & MASK32, int(key[1]) & MASK32
    m32 = np.uint64(MASK32)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0), p1 & m32,
                          (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1), p0 & m32)
    return np.stack([c0, c1, c2, c3], axis=1)


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & MASK32, seed >> 32)


def words(seed: int, k0: int, count: int, job: int = 0, tag: int = TAG_SCHEDULE) -> np.ndarray:
    """Philox blocks for counters k = k0 .. k0+count-1: uint64 array [count, 4]."""
    k = np.arange(k0, k0 + count, dtype=np.uint64)
    return philox4x32_10_many(k & np.uint64(MASK32), k >> np.uint64(32), job, tag, seed_key(seed))


def skip_threshold(p: float) -> int:
    """floor(p * 2^32) taken in float64; p >= 1 gives 2^32 (the coin always shows 1)."""
    if p >= 1.0:
        return 1 << 32
    return int(np.floor(np.float64(p) * np.float64(4294967296.0)))


def schedule(seed: int, iters: int, n_subsets: int, p: float, job: int = 0):
    """(i_k, theta_k, lsvrg_coin_k) for k = 0..iters-1, exact integer arithmetic."""
    w = words(seed, 0, iters, job, TAG_SCHEDULE)
    i = ((w[:, 0] * np.uint64(n_subsets)) >> np.uint64(32)).astype(np.int64)
    theta = (w[:, 1] < np.uint64(skip_threshold(p)) if p < 1.0 else np.ones(iters, bool))
    coin = w[:, 2] < np.uint64((1 << 32) // n_subsets)
    return i, np.asarray(theta, dtype=bool), np.asarray(coin, dtype=bool)


def uniform01(seed: int, count: int, job: int = 0, tag: int = TAG_POWER) -> np.ndarray:
    """count numbers (u + 0.5) / 2^32 in (0, 1); element e uses word e % 4 of block e // 4."""
    nblk = (count + 3) // 4
    w = words(seed, 0, nblk, job, tag).reshape(-1)[:count]
    return (w.astype(np.float64) + 0.5) / 4294967296.0
