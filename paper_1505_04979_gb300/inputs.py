"""Seeded synthetic inputs: information bits, Gaussian noise and the BPSK/AWGN
channel the paper simulates (Sec. IV: AWGN channel, BPSK modulation).

This module is shared by the oracle-side tests and the GPU-side tests and
benchmark.  It holds none of the decoder's arithmetic: no encoder, no message
update, no freezing rule.  Callers pass the transmitted codeword x (computed by
whichever side they test) to :func:`channel_llr`.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), implemented here from its
published definition so that every codeword of every workload can be
regenerated independently from (seed, stream, codeword index).
"""
from __future__ import annotations

import math

import numpy as np

# Philox4x32 constants (Salmon et al., SC'11): multipliers and Weyl key increments.
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)

# stream identifiers
STREAM_INFO = 1
STREAM_NOISE = 2
STREAM_DRAW = 3

DEFAULT_SEED = 1505049790


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of uint32 counters and a uint32 key.

    Returns four uint32 arrays.  Each round maps counter (c0, c1, c2, c3) with
    key (k0, k1) to (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1,
    lo(M0*c0)); the key is bumped by (W0, W1) between rounds.
    """
    c0 = np.asarray(c0, np.uint64) & _MASK32
    c1 = np.asarray(c1, np.uint64) & _MASK32
    c2 = np.asarray(c2, np.uint64) & _MASK32
    c3 = np.asarray(c3, np.uint64) & _MASK32
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for r in range(10):
        if r:
            k0 = np.uint64((int(k0) + PHILOX_W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + PHILOX_W1) & 0xFFFFFFFF)
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32), c3.astype(np.uint32))


def random_words(seed: int, stream: int, cw_index: np.ndarray, n_words: int) -> np.ndarray:
    """[len(cw_index), n_words] uint32 words for the given codewords.

    Counter = (block, codeword index low 32 bits, codeword index high 32 bits,
    stream); key = (seed low 32 bits, seed high 32 bits).  Word w of a codeword
    is output lane w % 4 of counter block w // 4.
    """
    cw = np.asarray(cw_index, np.uint64).reshape(-1)
    nblk = (n_words + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64)
    c0 = np.broadcast_to(blk[None, :], (cw.size, nblk))
    c1 = np.broadcast_to((cw & _MASK32)[:, None], (cw.size, nblk))
    c2 = np.broadcast_to((cw >> np.uint64(32))[:, None], (cw.size, nblk))
    c3 = np.full((cw.size, nblk), stream, np.uint64)
    o = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.stack(o, axis=-1).reshape(cw.size, nblk * 4)
    return np.ascontiguousarray(out[:, :n_words])


def info_bits(seed: int, cw_index, frozen: np.ndarray) -> np.ndarray:
    """Uniform source words u ([len(cw_index), N] uint8) with u_i = 0 on frozen i."""
    frozen = np.asarray(frozen, np.uint8)
    N = frozen.shape[0]
    words = random_words(seed, STREAM_INFO, cw_index, (N + 31) // 32)
    bit = np.arange(N)
    u = (words[:, bit // 32] >> (bit % 32).astype(np.uint32)) & np.uint32(1)
    u = u.astype(np.uint8)
    u[:, frozen.astype(bool)] = 0
    return u


def gaussian(seed: int, cw_index, N: int) -> np.ndarray:
    """Standard normal samples ([len(cw_index), N] float64), Box-Muller on Philox words.

    Pair p of a codeword uses words 2p and 2p+1: u1 = (w0 + 1) / 2^32 in (0, 1],
    u2 = w1 / 2^32, giving sqrt(-2 ln u1) cos(2 pi u2) and sqrt(-2 ln u1) sin(2 pi u2).
    """
    npair = (N + 1) // 2
    w = random_words(seed, STREAM_NOISE, cw_index, 2 * npair).astype(np.float64)
    u1 = (w[:, 0::2] + 1.0) * (1.0 / 4294967296.0)
    u2 = w[:, 1::2] * (1.0 / 4294967296.0)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((w.shape[0], 2 * npair), np.float64)
    z[:, 0::2] = r * np.cos(2.0 * math.pi * u2)
    z[:, 1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:, :N]


def uniform(seed: int, cw_index, lo: float, hi: float, which: int = 0) -> np.ndarray:
    """One uniform draw in [lo, hi) per codeword (stream 3, word `which`), float64."""
    w = random_words(seed, STREAM_DRAW, cw_index, which + 1)[:, which].astype(np.float64)
    return lo + (hi - lo) * w * (1.0 / 4294967296.0)


def choice(seed: int, cw_index, n: int, which: int = 0) -> np.ndarray:
    """One index in [0, n) per codeword (stream 3, word `which`)."""
    w = random_words(seed, STREAM_DRAW, cw_index, which + 1)[:, which].astype(np.uint64)
    return (w % np.uint64(n)).astype(np.int64)


def sigma(ebn0_db, rate: float):
    """AWGN standard deviation for BPSK at Eb/N0 (dB, scalar or array) and code rate K/N."""
    return np.sqrt(1.0 / (2.0 * rate * 10.0 ** (np.asarray(ebn0_db, np.float64) / 10.0)))


def channel_llr(x: np.ndarray, z: np.ndarray, sig) -> np.ndarray:
    """BPSK (0 -> +1, 1 -> -1) plus noise sig*z; LLR = 2y/sig^2 rounded to binary32.
    ``sig`` is a scalar or one value per codeword (row)."""
    sig = np.asarray(sig, np.float64)
    if sig.ndim == 1:
        sig = sig[:, None]
    y = (1.0 - 2.0 * np.asarray(x, np.float64)) + sig * np.asarray(z, np.float64)
    return (2.0 * y / (sig * sig)).astype(np.float32)


def noiseless_llr(x: np.ndarray, c: float = 2.0) -> np.ndarray:
    """c (1 - 2x): the channel LLR of an error-free observation."""
    return (c * (1.0 - 2.0 * np.asarray(x, np.float64))).astype(np.float32)
