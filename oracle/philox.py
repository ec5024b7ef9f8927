"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle, test infrastructure).

Philox4x32 with 10 rounds as published by Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): each round multiplies
words 0 and 2 by 0xD2511F53 and 0xCD9E8D57, mixes the high halves with the key,
and the key is bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85.

Noise streams of the PSE method that are drawn in-kernel use this generator:
    counter = (index_lo, index_hi, step, stream), key = (seed_lo, seed_hi),
    u1 = (w0 + 0.5) 2^-32,  u2 = (w1 + 0.5) 2^-32,
    z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2).
Stream 1 is the Lanczos start vector (one z0 per entry), stream 2 the
wave-space noise (z0 -> real part, z1 -> imaginary part per entry), stream 3
the direction of the random finite difference (one z0 per entry).

Parity: pinned by the Random123 known-answer vectors (tests/test_oracle_philox.py).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: (..., 4) uint32, key: (..., 2) uint32 -> (..., 4) uint32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    with np.errstate(over='ignore'):
        for _ in range(10):
            p0 = M0 * c[0].astype(np.uint64)
            p1 = M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = k0 + W0
            k1 = k1 + W1
    return np.stack(c, axis=-1)


def normals(seed, step, stream, index):
    """(z0, z1) for integer indices (array) under (seed, step, stream)."""
    index = np.asarray(index, dtype=np.uint64)
    ctr = np.zeros(index.shape + (4,), dtype=np.uint32)
    ctr[..., 0] = (index & _MASK).astype(np.uint32)
    ctr[..., 1] = (index >> np.uint64(32)).astype(np.uint32)
    ctr[..., 2] = np.uint32(step & 0xFFFFFFFF)
    ctr[..., 3] = np.uint32(stream)
    key = np.zeros(index.shape + (2,), dtype=np.uint32)
    key[..., 0] = np.uint32(seed & 0xFFFFFFFF)
    key[..., 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)
    u1 = (w[..., 0].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (w[..., 1].astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)


def lanczos_noise(seed, step, N, index0=0):
    """w1: (N, 8) standard normals of stream 1 (indices index0 + 8 n + c)."""
    z0, _ = normals(seed, step, 1, index0 + np.arange(8 * N, dtype=np.uint64))
    return z0.reshape(N, 8)


def wave_noise(seed, step, Ng, index0=0):
    """w2: (3, Ng, Ng, Ng/2+1, 2) standard normals of stream 2 (indices index0 + flat position)."""
    n = 3 * Ng * Ng * (Ng // 2 + 1)
    z0, z1 = normals(seed, step, 2, index0 + np.arange(n, dtype=np.uint64))
    return np.stack([z0, z1], axis=-1).reshape(3, Ng, Ng, Ng // 2 + 1, 2)


def rfd_noise(seed, step, N, index0=0):
    """W: (N, 3) standard normals of stream 3 (indices index0 + 3 n + d), the RFD direction."""
    z0, _ = normals(seed, step, 3, index0 + np.arange(3 * N, dtype=np.uint64))
    return z0.reshape(N, 3)
