"""Philox4x32-10 counter-based generator (oracle; test infrastructure).

Written from the published description (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11, Sec. 3.3): a 4 x 32-bit counter and a 2 x 32-bit key; each of the ten
rounds multiplies counter words 0 and 2 by two fixed odd multipliers, swaps
the halves of the 64-bit products into place and XORs the high halves with
the other two counter words and the round key; the key is advanced between
rounds by the Weyl constants floor(2^32 (golden ratio - 1)) and
floor(2^32 (sqrt 3 - 1)).

Sampling convention of this project (one draw per nucleus k of sample s in
radical pair ``pair`` under ``seed``):
    counter = (k, s mod 2^32, s div 2^32, pair),  key = (seed mod 2^32, seed div 2^32)
    u1 = ((x0 >> 5) 2^26 + (x1 >> 6)) / 2^53,  u2 likewise from (x2, x3)
    cos(theta) = 1 - 2 u1,  phi = 2 pi u2         (uniform on the sphere, Eq. 17)
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9  # floor(2^32 * (golden ratio - 1))
PHILOX_W1 = 0xBB67AE85  # floor(2^32 * (sqrt(3) - 1))
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.

    ``ctr``: integer array (..., 4); ``key``: integer array (..., 2).
    Returns uint64 array (..., 4) holding 32-bit outputs.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK
    k = np.asarray(key, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    w0, w1 = np.uint64(PHILOX_W0), np.uint64(PHILOX_W1)
    for r in range(10):
        if r > 0:
            k0 = (k0 + w0) & _MASK
            k1 = (k1 + w1) & _MASK
        p0 = m0 * c0  # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def uniform53(hi, lo):
    """Map two 32-bit words to a double in [0, 1) with 53 random bits."""
    hi = np.asarray(hi, dtype=np.uint64) >> np.uint64(5)
    lo = np.asarray(lo, dtype=np.uint64) >> np.uint64(6)
    return (hi.astype(np.float64) * 67108864.0 + lo.astype(np.float64)) * (1.0 / 9007199254740992.0)


def draw_uniforms(seed: int, pair: int, samples, n_nuc: int):
    """(u1, u2) arrays of shape (len(samples), n_nuc) for the given sample indices."""
    s = np.asarray(samples, dtype=np.uint64).reshape(-1)
    n_s = s.size
    ctr = np.zeros((n_s, n_nuc, 4), dtype=np.uint64)
    ctr[..., 0] = np.arange(n_nuc, dtype=np.uint64)[None, :]
    ctr[..., 1] = (s & _MASK)[:, None]
    ctr[..., 2] = (s >> np.uint64(32))[:, None]
    ctr[..., 3] = np.uint64(pair)
    key = np.zeros((n_s, n_nuc, 2), dtype=np.uint64)
    seed = int(seed)
    key[..., 0] = np.uint64(seed & 0xFFFFFFFF)
    key[..., 1] = np.uint64((seed >> 32) & 0xFFFFFFFF)
    x = philox4x32_10(ctr, key)
    return uniform53(x[..., 0], x[..., 1]), uniform53(x[..., 2], x[..., 3])


def draw_angles(seed: int, pair: int, samples, n_nuc: int):
    """(theta, phi) of shape (len(samples), n_nuc): uniform directions on S^2."""
    u1, u2 = draw_uniforms(seed, pair, samples, n_nuc)
    theta = np.arccos(1.0 - 2.0 * u1)
    phi = 2.0 * np.pi * u2
    return theta, phi


def draw_basis_indices(seed: int, pair: int, samples, Z: int):
    """Nuclear basis index of each sample for basis-state sampling (Eq. 14
    sampled): counter (0xFFFFFFFF, s mod 2^32, s div 2^32, pair) -- word 0 is
    never a nucleus index -- and the u1 map above; index = min(floor(u Z), Z - 1)."""
    s = np.asarray(samples, dtype=np.uint64).reshape(-1)
    ctr = np.zeros((s.size, 4), dtype=np.uint64)
    ctr[:, 0] = np.uint64(0xFFFFFFFF)
    ctr[:, 1] = s & _MASK
    ctr[:, 2] = s >> np.uint64(32)
    ctr[:, 3] = np.uint64(pair)
    seed = int(seed)
    key = np.zeros((s.size, 2), dtype=np.uint64)
    key[:, 0] = np.uint64(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint64((seed >> 32) & 0xFFFFFFFF)
    x = philox4x32_10(ctr, key)
    u = uniform53(x[:, 0], x[:, 1])
    return np.minimum(np.floor(u * float(Z)).astype(np.int64), int(Z) - 1)
