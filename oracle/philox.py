"""Philox counter-based generator for the oracle — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import anything
under oracle/. The CUDA library has its own, separately written Philox.

Philox4xW-R (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
SC'11, Section 3.2): a counter of four W-bit words and a key of two words; each of R rounds
multiplies counter words 0 and 2 by fixed constants, keeps the high and low halves of the
double-width products, and mixes them with words 1, 3 and the round key; between rounds the
key is advanced by two Weyl constants. The radiation step of the method (Fig. 1 C) draws its
random numbers from Philox4x32-10 keyed by the run seed, with counter (cell, step,
stream<<24 | sub, world).

The word-size generic form below is pinned in tests against numpy's Philox4x64-10 (a
library routine with the same round structure) and, for the 4x32 width used here, against the
known-answer vectors the generator's authors publish with their Random123 library.
"""
from __future__ import annotations

import numpy as np

_CONST = {
    32: (0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85),
    64: (0xD2E7470EE14C6C93, 0xCA5A826395121157, 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B),
}

# stream ids of the counter's third word (stream << 24 | sub)
STREAM_MUTATE = 0
STREAM_MERGE = 1
STREAM_GAUSS = 2


def philox_py(ctr, key, width=32, rounds=10):
    """Scalar Philox4xW-R on Python ints: ctr = 4 words, key = 2 words -> 4 words."""
    m0, m1, w0, w1 = _CONST[width]
    mask = (1 << width) - 1
    c = [int(v) & mask for v in ctr]
    k = [int(v) & mask for v in key]
    for r in range(rounds):
        if r:
            k = [(k[0] + w0) & mask, (k[1] + w1) & mask]
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        c = [(p1 >> width) ^ c[1] ^ k[0], p1 & mask, (p0 >> width) ^ c[3] ^ k[1], p0 & mask]
    return c


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=10):
    """Vectorised Philox4x32-R over numpy arrays of counters (uint32 results)."""
    m0, m1, w0, w1 = (np.uint64(v) for v in _CONST[32])
    lo = np.uint64(0xFFFFFFFF)
    sh = np.uint64(32)
    shape = np.broadcast(c0, c1, c2, c3).shape
    c = [np.broadcast_to(np.asarray(v, np.uint64) & lo, shape).copy() for v in (c0, c1, c2, c3)]
    k = [np.uint64(int(k0) & 0xFFFFFFFF), np.uint64(int(k1) & 0xFFFFFFFF)]
    for r in range(rounds):
        if r:
            k = [(k[0] + w0) & lo, (k[1] + w1) & lo]
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        c = [(p1 >> sh) ^ c[1] ^ k[0], p1 & lo, (p0 >> sh) ^ c[3] ^ k[1], p0 & lo]
    return [v.astype(np.uint32) for v in c]


def seed_key(seed: int):
    """The 64-bit run seed split into Philox key words (low, high)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def draw(cells, step, stream, sub, world, seed):
    """Four uint32 words for each cell: counter (cell, step, stream<<24|sub, world)."""
    k0, k1 = seed_key(seed)
    c2 = ((int(stream) & 0xFF) << 24) | (int(sub) & 0xFFFFFF)
    return philox4x32(np.asarray(cells, np.uint64), int(step) & 0xFFFFFFFF, c2,
                      int(world) & 0xFFFFFFFF, k0, k1)


def uniform01(u):
    """Open-interval uniform from a 32-bit word: ((u >> 8) + 0.5) * 2^-24, exact in FP64."""
    return ((np.asarray(u, np.uint64) >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def box_muller(u1, u2):
    """Two standard normals from two open-interval uniforms (Box & Muller, 1958)."""
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    return r * np.cos(theta), r * np.sin(theta)


def threshold(p: float) -> int:
    """Hit threshold for probability p: a hit is a raw 32-bit word below floor(p * 2^32)."""
    return min(int(np.floor(float(p) * 2.0 ** 32)), 0xFFFFFFFF)
