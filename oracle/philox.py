"""Philox4x32-10 counter-based generator and Box-Muller normals.

The paper draws its anchor fields from an i.i.d. Gaussian vector (Sec. 3.2,
Fig. 7; Sec. 3.4); the white noise here comes from Philox4x32-10 (Salmon,
Moraes, Dror & Shaw, SC'11), a published counter-based generator, so that
the CUDA path and this oracle can reproduce one stream independently.

Definition (per round, 10 rounds, key bumped after each round):
  (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2          (32x32 -> 64-bit products)
  c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  k0 <- k0 + W0,  k1 <- k1 + W1                          (mod 2^32)
with M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85.

Stream layout used by the simulator: frame seed s gives the key
(s mod 2^32, s >> 32); white-noise sample i of field l comes from the call with
counter (i // 4, l, 0, 0), word i % 4.  Uniforms are u = (k + 1/2) 2^-32, and
each word pair (u_a, u_b) = (w0, w1) or (w2, w3) gives two normals
  sqrt(-2 ln u_a) cos(2 pi u_b),  sqrt(-2 ln u_a) sin(2 pi u_b),
evaluated here in FP64.

Pins (tests/test_oracle_philox.py): bit-exact against cuRAND's host
Philox4_32_10 generator (run as a library, block i = counter (0, 0, i, 0)),
moments and cross-stream correlation of the normals.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs broadcast; returns four uint64 arrays of 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> S32, p0 & MASK
        hi1, lo1 = p1 >> S32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def key_of_seed(seed: int) -> tuple[int, int]:
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def words(seed: int, field: int, n: int) -> np.ndarray:
    """The first n 32-bit words of stream (seed, field), in sample order."""
    k0, k1 = key_of_seed(seed)
    q = np.arange((n + 3) // 4, dtype=np.uint64)
    w = philox4x32_10(q, field, 0, 0, k0, k1)
    return np.stack(w, axis=1).reshape(-1)[:n]


def uniforms(w: np.ndarray) -> np.ndarray:
    """u = (k + 1/2) 2^-32 in (0, 1), exact in FP64."""
    return (w.astype(np.float64) + 0.5) * 2.0**-32


def normals(seed: int, field: int, n: int) -> np.ndarray:
    """n standard normals of stream (seed, field) by Box-Muller in FP64."""
    m = (n + 3) // 4 * 4
    u = uniforms(words(seed, field, m)).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    t = 2.0 * np.pi * u[:, 1]
    z = np.stack([r * np.cos(t), r * np.sin(t)], axis=1).reshape(-1)
    return z[:n]
