"""Importance-sampling observables of one realization from S proposals.

Test infrastructure: only the tests use it; the CUDA path never imports it.

The proposals s_k are drawn from q; with weights w_k = exp(-beta E(s_k)) / q(s_k)
(Eq. 1, Eq. 9), Z = E_q[w] (Sec. 2.3: the proposals' log q makes importance
sampling of the Boltzmann distribution possible, Eq. 10 uses the same ratio),
and a Boltzmann average is <O> = sum_k w_k O(s_k) / sum_k w_k. Replica
observables use the pairs (s_0, s_1), (s_2, s_3), ... of independent proposals
with pair weights w_a w_b:

    overlap q_ab = (1/N) sum_i s_i^a s_i^b        (N = L^2 spins)
    <q^2>, <q^4>, Binder ratio g = (3 - <q^4> / <q^2>^2) / 2.

Returned per realization, in this order:
    log Z estimate = log mean_k w_k, effective sample size (sum w)^2 / sum w^2,
    energy per spin <E> / N, <q^2>, <q^4>, g.
Weights are formed in the log domain, shifted by their maximum; float64 throughout.
"""
from __future__ import annotations

import numpy as np

N_OBS = 6


def observables(sigma, log_q, E, beta):
    """sigma (S, L, L) bits (1 = +1), log_q (S,), E (S,) -> array of the 6 values above."""
    sigma = np.asarray(sigma)
    S = sigma.shape[0]
    N = sigma[0].size
    lw = -beta * np.asarray(E, dtype=np.float64) - np.asarray(log_q, dtype=np.float64)
    m = lw.max()
    w = np.exp(lw - m)
    sw = w.sum()
    log_z = m + np.log(sw / S)
    ess = sw * sw / np.sum(w * w)
    e_mean = np.sum(w * E) / sw / N
    s = 2.0 * sigma.reshape(S, N).astype(np.float64) - 1.0
    P = S // 2
    if P == 0:
        return np.array([log_z, ess, e_mean, np.nan, np.nan, np.nan])
    q = np.sum(s[0:2 * P:2] * s[1:2 * P:2], axis=1) / N
    wp = w[0:2 * P:2] * w[1:2 * P:2]
    q2 = np.sum(wp * q * q) / wp.sum()
    q4 = np.sum(wp * q ** 4) / wp.sum()
    g = 0.5 * (3.0 - q4 / (q2 * q2))
    return np.array([log_z, ess, e_mean, q2, q4, g])


def nishimori_beta(p: float) -> float:
    """Inverse temperature of the Nishimori line of the +-J model with antiferromagnetic
    bond probability p: exp(-2 beta) = p / (1 - p)."""
    return 0.5 * np.log((1.0 - p) / p)
