"""Philox4x32-10 counter-based generator, written from its published definition.

Reference: J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11, Section 3 (the Philox S-box: two 32x32->64-bit
multiplies per round, Weyl key schedule). The paper under study (Section
2.2.1) draws a random orthogonal matrix P and the k-means initial centroids
(Section 3.1.1, Phase 1) at random; both the oracle and the CUDA path derive
those draws from this generator so that they can be compared.

This oracle module is test infrastructure: only tests, the smoke check and
the benchmark's CPU-baseline leg may import it.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
SH32 = np.uint64(32)

# Stream ids (third counter word) of the method's random draws.
STREAM_ROTATION = 1      # Gaussian entries of the matrix orthogonalised into P
STREAM_KMEANS_INIT = 2   # ranks rows to pick the initial centroids
STREAM_TRAIN_SAMPLE = 3  # ranks rows to pick the k-means training subset


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Ten Philox rounds over counters ``ctr`` (n x 4 uint32) with ``key``.

    One round maps (c0, c1, c2, c3) to (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
    hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the key is bumped by the Weyl constants
    (W0, W1) between rounds.
    """
    ctr = np.asarray(ctr, dtype=np.uint32).reshape(-1, 4)
    c0, c1, c2, c3 = (ctr[:, i].astype(np.uint64) for i in range(4))
    key = np.asarray(key, dtype=np.uint64).reshape(-1, 2)
    k0 = key[:, 0].copy()
    k1 = key[:, 1].copy()
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> SH32, p0 & MASK32
        hi1, lo1 = p1 >> SH32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + W0) & MASK32
        k1 = (k1 + W1) & MASK32
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def seed_key(seed: int):
    """The 64-bit seed split into the two 32-bit key words."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def stream_block(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Philox output for counters (index_lo, index_hi, stream, 0)."""
    index = np.asarray(index, dtype=np.uint64)
    ctr = np.zeros((index.size, 4), np.uint32)
    ctr[:, 0] = (index & MASK32).astype(np.uint32)
    ctr[:, 1] = (index >> SH32).astype(np.uint32)
    ctr[:, 2] = stream
    return philox4x32_10(ctr, seed_key(seed))


def u64_words(w: np.ndarray):
    """Two 64-bit words (w0 | w1<<32, w2 | w3<<32) of a Philox block."""
    w = w.astype(np.uint64)
    return w[:, 0] | (w[:, 1] << SH32), w[:, 2] | (w[:, 3] << SH32)


def row_keys(seed: int, stream: int, n: int) -> np.ndarray:
    """Rank key of rows 0..n-1: (first output word << 32) | row, as uint64.

    Keys are unique, and their integer order is (random word, row id) order.
    """
    rows = np.arange(n, dtype=np.uint64)
    w0 = stream_block(seed, stream, rows)[:, 0].astype(np.uint64)
    return (w0 << SH32) | rows


def unit_open(a: np.ndarray) -> np.ndarray:
    """Map a uint64 to the open interval (0, 1): ((a >> 12) + 0.5) * 2^-52.

    Both steps are exact in binary64, so every implementation of this map
    yields the same double.
    """
    return ((a >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def gaussian(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform.

    Pair i (outputs 2i and 2i+1) uses block (i, stream): u1, u2 from the two
    64-bit words, radius sqrt(-2 ln u1), angle 2 pi u2 (Box and Muller, 1958).
    """
    npair = (n + 1) // 2
    a, b = u64_words(stream_block(seed, stream, np.arange(npair, dtype=np.uint64)))
    u1, u2 = unit_open(a), unit_open(b)
    rho = np.sqrt(-2.0 * np.log(u1))
    theta = 6.283185307179586 * u2
    g = np.empty(2 * npair)
    g[0::2] = rho * np.cos(theta)
    g[1::2] = rho * np.sin(theta)
    return g[:n]
