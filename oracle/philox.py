"""Philox4x32-10 counter-based generator and the draws built on it (oracle, numpy).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter and a 2x32-bit key, ten
rounds, each round two 32x32->64 multiplies by 0xD2511F53 and 0xCD9E8D57 whose high and low
halves are XOR-mixed with the other two counter words and the key; the key is bumped by the
Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.

The stochastic subgrid step (Sec. 2.4.2) treats its Gumbel draws as model inputs (Eq.
reparam). Making them a pure function of (seed, cell, step, instance) lets the forward
pass, the recomputation inside the adjoint and the CPU oracle see bit-identical draws.

Counter layout (shared definition, implemented independently on each side):
    key = (seed & 0xffffffff, seed >> 32)
    ctr = (linear cell index, step index, instance index, stream tag)
    stream tag 0: initial white noise, tag 1: subgrid Gumbel pair.
Uniform from a 32-bit word x: u = ((x >> 9) + 0.5) * 2^-23, an odd multiple of 2^-24 in
(0, 1), exactly representable in float32 and float64, so both sides start from the same u.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

TAG_IC_NOISE = 0
TAG_SUBGRID = 1


def philox4x32_10(ctr, key):
    """Ten Philox rounds. ctr: 4 arrays (broadcastable) of uint32 values; key: 2 ints.
    Returns 4 uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in ctr]
    c = list(np.broadcast_arrays(*c))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = np.uint64((int(k0) + W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + W1) & 0xFFFFFFFF)
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return [x.astype(np.uint32) for x in c]


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def uniform_from_word(x):
    """u = ((x >> 9) + 0.5) * 2^-23 in float64 (exact)."""
    x = np.asarray(x, dtype=np.uint32)
    return ((x >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def words(seed: int, n_cells: int, step: int, instance: int, tag: int):
    """Philox output words for cells 0..n_cells-1 at (step, instance, tag)."""
    idx = np.arange(n_cells, dtype=np.uint64)
    return philox4x32_10((idx, np.uint64(step), np.uint64(instance), np.uint64(tag)),
                         seed_key(seed))


def gumbel_pair(seed: int, n_cells: int, step: int, instance: int = 0):
    """(g0, g1) ~ Gumbel(0, 1) per cell: g = -ln(-ln u) (Sec. 2.4.2)."""
    w = words(seed, n_cells, step, instance, TAG_SUBGRID)
    u0, u1 = uniform_from_word(w[0]), uniform_from_word(w[1])
    return -np.log(-np.log(u0)), -np.log(-np.log(u1))


def uniform_pair(seed: int, n_cells: int, step: int, instance: int = 0):
    w = words(seed, n_cells, step, instance, TAG_SUBGRID)
    return uniform_from_word(w[0]), uniform_from_word(w[1])


def white_noise(seed: int, n: int, instance: int = 0):
    """N(0,1) white noise on an n^3 grid (C order [z][y][x]), Box-Muller on words 0, 1:
    z = sqrt(-2 ln u1) cos(2 pi u2)."""
    w = words(seed, n ** 3, 0, instance, TAG_IC_NOISE)
    u1, u2 = uniform_from_word(w[0]), uniform_from_word(w[1])
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(n, n, n)
