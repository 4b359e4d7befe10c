"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

Written from the published definition: a 4x64-bit counter and a 2x64-bit key;
each of 10 rounds multiplies words 0 and 2 by the constants M0, M1 into
128-bit products, and permutes/xors the halves with the other words and the
round key; the key is bumped by the Weyl constants W0, W1 between rounds.

Counter layout used by the method (both sides implement the same layout):

    spin draw   site i of realization n, proposal t : ctr = (i >> 2, t, n, 0), word i & 3
    MH uniform  proposal t of realization n         : ctr = (0, t, n, 1),      word 0
    init spins  site i of realization n             : ctr = (i >> 2, 0, n, 2), word i & 3
    key = (seed, 0)

A 64-bit word w becomes the uniform u = (2 * (w >> 12) + 1) * 2**-53, which is
exact in float64 and lies strictly inside (0, 1).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)

TAG_SPIN, TAG_MH, TAG_INIT = 0, 1, 2

_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.ndarray, b: np.uint64):
    """128-bit product of uint64 arrays a and scalar b -> (hi, lo)."""
    a = a.astype(np.uint64)
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _LO32) + (hl & _LO32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    lo = a * b  # wraps modulo 2**64
    return hi, lo


def philox4x64_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x64-10 of counters ctr (..., 4) uint64 under key (k0, k1) -> (..., 4) uint64."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    x0, x1, x2, x3 = (ctr[..., j].copy() for j in range(4))
    k0 = np.uint64(key[0])
    k1 = np.uint64(key[1])
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint64((int(k0) + int(W0)) & 0xFFFFFFFFFFFFFFFF)
                k1 = np.uint64((int(k1) + int(W1)) & 0xFFFFFFFFFFFFFFFF)
            hi0, lo0 = _mulhilo(x0, M0)
            hi1, lo1 = _mulhilo(x2, M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=-1)


def to_uniform(w: np.ndarray) -> np.ndarray:
    """64-bit words -> float64 uniforms (2k+1) 2^-53 in (0, 1), k = w >> 12."""
    k = (np.asarray(w, dtype=np.uint64) >> np.uint64(12)).astype(np.float64)
    return (2.0 * k + 1.0) * 2.0 ** -53


def site_words(n_sites: int, t: np.ndarray, n: int, tag: int, seed: int) -> np.ndarray:
    """Word for every (proposal t, site i): array (len(t), n_sites) uint64."""
    t = np.asarray(t, dtype=np.uint64).reshape(-1)
    groups = (n_sites + 3) // 4
    ctr = np.zeros((t.size, groups, 4), np.uint64)
    ctr[..., 0] = np.arange(groups, dtype=np.uint64)[None, :]
    ctr[..., 1] = t[:, None]
    ctr[..., 2] = np.uint64(n)
    ctr[..., 3] = np.uint64(tag)
    out = philox4x64_10(ctr, (seed, 0)).reshape(t.size, groups * 4)
    return out[:, :n_sites]


def spin_uniforms(L: int, t: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Uniforms of the spin draws: (len(t), L*L), raster site order."""
    return to_uniform(site_words(L * L, t, n, TAG_SPIN, seed))


def mh_uniforms(t: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Uniform of the accept test of proposal t in realization n."""
    t = np.asarray(t, dtype=np.uint64).reshape(-1)
    ctr = np.zeros((t.size, 4), np.uint64)
    ctr[:, 1] = t
    ctr[:, 2] = np.uint64(n)
    ctr[:, 3] = np.uint64(TAG_MH)
    return to_uniform(philox4x64_10(ctr, (seed, 0))[:, 0])


def init_spins(L: int, n: int, seed: int) -> np.ndarray:
    """Random initial configuration (bits, 1 = spin +1): top bit of each site's word."""
    w = site_words(L * L, np.zeros(1, np.uint64), n, TAG_INIT, seed)[0]
    return (w >> np.uint64(63)).astype(np.uint8).reshape(L, L)
