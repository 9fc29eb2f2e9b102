"""Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), restated from its published definition, plus the
counter layout and transforms the device path uses for z (Algorithm 1, first
step) and for the Rademacher probes (Section 6).

Definition (per round, with key (k0, k1)):
    (hi0, lo0) = mulhilo(0xD2511F53, c0),  (hi1, lo1) = mulhilo(0xCD9E8D57, c2)
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
and between rounds the key advances by the Weyl constants
    (k0, k1) <- (k0 + 0x9E3779B9, k1 + 0xBB67AE85)   (mod 2^32); 10 rounds.

Counter layout used on both sides:
* Gaussian element e of vector s: one Philox call per group g = e // 4 with
  counter (g, s, 0, 0), key (seed mod 2^32, seed >> 32); words (w0, w1) give
  elements 4g, 4g+1 and (w2, w3) give 4g+2, 4g+3 by Box-Muller:
  u = ((w >> 8) + 1/2) 2^-24, r = sqrt(-2 log u_a), z = r cos(2 pi u_b),
  r sin(2 pi u_b).
* Rademacher element e of probe s: counter (e // 128, s, 1, 0); bit e % 32 of
  word (e // 32) % 4; +1 if set, -1 otherwise.

Parity: the raw 32-bit words are compared bit-exactly with the device; the
Gaussian values (device FP32 libm vs this FP64 transform) to ~1e-6.  The word
stream is pinned bit for bit to an independent implementation of the same
generator in a library of the image (Triton's tl.philox, run on the CPU by its
interpreter), and the transforms by statistical tests
(tests/test_oracle_philox.py).

This module is test infrastructure: only the tests, the smoke check and the
benchmark's CPU baseline use it.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox-4x32-10 on uint32 arrays; returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def gaussian_words(nvec, n, seed):
    """Raw words for the Gaussian stream: uint32 array [nvec][ceil(n/4)*4]."""
    k0, k1 = _key(seed)
    ng = (int(n) + 3) // 4
    g = np.tile(np.arange(ng, dtype=np.uint64), int(nvec))
    s = np.repeat(np.arange(int(nvec), dtype=np.uint64), ng)
    w = philox4x32_10(g, s, 0, 0, k0, k1)
    return np.stack(w, axis=-1).reshape(int(nvec), ng * 4)


def gaussian(nvec, n, seed):
    """z ~ N(0, I) in FP64, shape [nvec][n], from the Gaussian stream."""
    w = gaussian_words(nvec, n, seed).astype(np.float64)
    u = (np.floor(w / 256.0) + 0.5) * 2.0 ** -24
    ua, ub = u[:, 0::2], u[:, 1::2]
    r = np.sqrt(-2.0 * np.log(ua))
    out = np.empty_like(u)
    out[:, 0::2] = r * np.cos(2 * np.pi * ub)
    out[:, 1::2] = r * np.sin(2 * np.pi * ub)
    return out[:, : int(n)]


def rademacher(nvec, n, seed):
    """+-1 probes, shape [nvec][n], from the Rademacher stream."""
    k0, k1 = _key(seed)
    ng = (int(n) + 127) // 128
    g = np.tile(np.arange(ng, dtype=np.uint64), int(nvec))
    s = np.repeat(np.arange(int(nvec), dtype=np.uint64), ng)
    w = np.stack(philox4x32_10(g, s, 1, 0, k0, k1), axis=-1).reshape(int(nvec), ng * 4)
    e = np.arange(int(n))
    words = w[:, e // 32]
    bits = (words >> (e % 32).astype(np.uint32)) & np.uint32(1)
    return np.where(bits == 1, 1.0, -1.0)
