"""Exact references for pinning the oracle (Eq. 2-4, Eq. 6).

* Brute force (L <= 4, 2^16 states): Z, P and the exact conditionals of Eq. 4
  along given configurations.
* Row transfer matrix (L up to about 14): the exact boundary functions F_r as
  dense 2^L vectors, hence the exact log Z (Eq. 6) and the exact conditionals
  of Eq. 4-5 at any site of any configuration.

Row configurations are integers y with bit c = spin bit of column c.
"""
from __future__ import annotations

import numpy as np

from .ising import boltzmann_matrix, energy, spin


def all_configs(L: int) -> np.ndarray:
    """Every configuration of L*L spins as bits (2^N, L, L); site 0 is the most significant bit."""
    N = L * L
    x = np.arange(2 ** N, dtype=np.int64)
    bits = (x[:, None] >> np.arange(N - 1, -1, -1)[None, :]) & 1
    return bits.astype(np.uint8).reshape(-1, L, L)


def _logsumexp(a, axis=None):
    m = np.max(a, axis=axis, keepdims=True)
    out = m + np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True))
    return np.squeeze(out, axis=axis) if axis is not None else out.item()


def brute_force(Jh, Jv, beta):
    """(configs, E, log P, log Z) over all 2^(L^2) configurations."""
    L = Jh.shape[0]
    cfg = all_configs(L)
    E = energy(Jh, Jv, cfg)
    lw = -beta * E
    lz = _logsumexp(lw)
    return cfg, E, lw - lz, lz


def brute_conditional_logits(Jh, Jv, beta, sigma):
    """Exact log P(s_i=+1 | s_<i) - log P(s_i=-1 | s_<i) along each configuration (S, L*L)."""
    L = Jh.shape[0]
    N = L * L
    _, _, logp, _ = brute_force(Jh, Jv, beta)
    sigma = np.asarray(sigma).reshape(-1, N).astype(np.int64)
    S = sigma.shape[0]
    out = np.zeros((S, N))
    for i in range(N):
        # log marginal of every prefix of length i+1
        lm = _logsumexp(logp.reshape(2 ** (i + 1), 2 ** (N - i - 1)), axis=1)
        prefix = np.zeros(S, np.int64)
        for j in range(i):
            prefix = prefix * 2 + sigma[:, j]
        out[:, i] = lm[prefix * 2 + 1] - lm[prefix * 2]
    return out


def _row_bits(L):
    y = np.arange(2 ** L, dtype=np.int64)
    return ((y[:, None] >> np.arange(L)[None, :]) & 1).astype(np.uint8)   # (2^L, L), column c = bit c


def _row_field(Jh_row, beta, bits):
    """log of exp(beta sum_c Jh[c] s_c s_{c+1}) for every row configuration."""
    s = spin(bits)
    if Jh_row.size == 0:
        return np.zeros(bits.shape[0])
    return beta * np.sum(np.asarray(Jh_row, np.float64)[None, :] * s[:, :-1] * s[:, 1:], axis=1)


def _apply_vertical(logv, Jv_row, beta, L):
    """out(y') = sum_y v(y) prod_c B(Jv[c])[y_c, y'_c], in the log domain with one shift."""
    m = np.max(logv)
    v = np.exp(logv - m).reshape((2,) * L)
    for c in range(L):
        B = boltzmann_matrix(beta, Jv_row[c])
        ax = L - 1 - c
        v = np.moveaxis(np.tensordot(B.T, v, axes=([1], [ax])), 0, ax)
    with np.errstate(divide="ignore"):
        return np.log(v.reshape(-1)) + m


def transfer_log_z(Jh, Jv, beta):
    """Exact log Z by the row transfer matrix, top to bottom (Eq. 6)."""
    L = Jh.shape[0]
    bits = _row_bits(L)
    logv = _row_field(Jh[0], beta, bits)
    for r in range(1, L):
        logv = _apply_vertical(logv, Jv[r - 1], beta, L) + _row_field(Jh[r], beta, bits)
    return _logsumexp(logv)


def boundary_functions(Jh, Jv, beta):
    """Exact log F_r(y) for r = 0..L-1 (bottom-up), F_r over rows r..L-1 as in the bMPS cache."""
    L = Jh.shape[0]
    bits = _row_bits(L)
    F = [None] * L
    F[L - 1] = _row_field(Jh[L - 1], beta, bits)
    for r in range(L - 2, -1, -1):
        # sum over the row below: v(y) = sum_{y'} prod_c B(Jv[r,c])[y_c, y'_c] F_{r+1}(y')
        F[r] = _apply_vertical(F[r + 1], Jv[r], beta, L) + _row_field(Jh[r], beta, bits)
    return F


def transfer_conditional_logits(Jh, Jv, beta, sigma):
    """Exact logits of Eq. 5 along configurations sigma (S, L, L), from the exact F_r."""
    L = Jh.shape[0]
    F = boundary_functions(Jh, Jv, beta)
    bits = _row_bits(L)
    s_bits = spin(bits)
    sigma = np.asarray(sigma)
    S = sigma.shape[0]
    out = np.zeros((S, L * L))
    for k in range(S):
        for r in range(L):
            lw = F[r].copy()
            if r > 0:
                s_up = spin(sigma[k, r - 1])
                lw = lw + beta * np.sum(np.asarray(Jv[r - 1], np.float64)[None, :] * s_up[None, :] * s_bits, axis=1)
            alive = np.ones(2 ** L, bool)
            for c in range(L):
                lp = _logsumexp(np.where(alive & (bits[:, c] == 1), lw, -np.inf))
                lm = _logsumexp(np.where(alive & (bits[:, c] == 0), lw, -np.inf))
                out[k, r * L + c] = lp - lm
                alive &= bits[:, c] == sigma[k, r, c]
    return out
