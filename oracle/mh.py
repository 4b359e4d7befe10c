"""Independence Metropolis-Hastings over TNMC proposals (Sec. 2.3, Eq. 10).

A proposal s' drawn from q is accepted with probability
min(1, q(s) P(s') / (q(s') P(s))) = min(1, exp(log r)) with

    log r = (-beta E(s') - log q(s')) - (-beta E(s) - log q(s)).

Readings of the paper: one chain per realization; proposals are consumed in
their id order; the accept test is u < exp(log r) taken as log u < log r in
float64, u the Philox uniform of the proposal (stream 1). The initial state is
a uniformly random configuration (stream 2) scored by the proposal's own q.
"""
from __future__ import annotations

import numpy as np

from . import philox


def chain(state, proposals, beta, seed, prop_base, n):
    """Run the chain of realization n through S proposals.

    state     : (sigma (L, L), log_q, E) of the current configuration
    proposals : (sigma (S, L, L), log_q (S,), E (S,))
    Returns (new_state, accept (S,) uint8, log_r (S,), u (S,)).
    """
    sig, lq, E = state
    sig = np.array(sig, copy=True)
    P_sig, P_lq, P_E = proposals
    S = P_lq.shape[0]
    t = np.arange(S, dtype=np.uint64) + np.uint64(prop_base)
    u = philox.mh_uniforms(t, n, seed)
    acc = np.zeros(S, np.uint8)
    log_r = np.zeros(S)
    for k in range(S):
        log_r[k] = (-beta * P_E[k] - P_lq[k]) - (-beta * E - lq)
        if np.log(u[k]) < log_r[k]:
            acc[k] = 1
            sig, lq, E = P_sig[k].copy(), float(P_lq[k]), float(P_E[k])
    return (sig, lq, E), acc, log_r, u
