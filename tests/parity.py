"""Helpers shared by the GPU parity tests: run the oracle on the same seeded
inputs and compare element by element (CPU side only; imports no CUDA code)."""
from __future__ import annotations

import numpy as np

from oracle import bmps, mh, philox, sampler
from workloads import draw_bonds, to_paper_layout

# A draw whose uniform lies this close to the oracle's probability of +1 may
# legitimately go the other way on the GPU (float64 rounding of the contraction
# and of exp/log differs between the two sides); such draws are counted.
BAND_FP64 = 1e-9


def realizations(Ls, kind, base_seed=1000, p=0.5):
    return [draw_bonds(L, base_seed + n, kind, p) for n, L in enumerate(Ls)]


def packed_J(reals):
    return np.ascontiguousarray(np.concatenate([to_paper_layout(Jh, Jv).reshape(-1, 4) for Jh, Jv in reals]))


def split_spins(flat, Ls, S):
    out, o = [], 0
    for L in Ls:
        out.append(flat[o:o + S * L * L].reshape(S, L, L))
        o += S * L * L
    return out


def oracle_envs(reals, beta, chi, cutoff=bmps.DEFAULT_CUTOFF):
    return [bmps.build_envs(Jh, Jv, beta, chi, cutoff) for Jh, Jv in reals]


def compare_proposals(rows, Jh, Jv, beta, seed, prop_base, n, g_sig, g_lq, g_E, band=BAND_FP64,
                      lq_atol=1e-9):
    """Free-running parity of one realization's proposals.

    Returns (n_equal, n_boundary). Raises AssertionError when a configuration
    differs at a draw that was not within ``band`` of the decision boundary, or
    when log q / E of an identical configuration disagree.
    """
    S, L, _ = g_sig.shape
    o_sig, o_lq, o_E, o_lg = sampler.propose(rows, Jh, Jv, beta, S, seed, prop_base, n)
    t = np.arange(S, dtype=np.uint64) + np.uint64(prop_base)
    u = philox.spin_uniforms(L, t, n, seed)
    n_eq, n_bd = 0, 0
    for k in range(S):
        a, b = g_sig[k].reshape(-1), o_sig[k].reshape(-1)
        if np.array_equal(a, b):
            n_eq += 1
            assert g_E[k] == o_E[k], (k, g_E[k], o_E[k])
            assert abs(g_lq[k] - o_lq[k]) <= lq_atol * max(1.0, abs(o_lq[k])), (k, g_lq[k], o_lq[k])
        else:
            i = int(np.argmax(a != b))
            p = sampler.sigmoid(o_lg[k, i])
            assert abs(u[k, i] - p) < band, f"sample {k} differs at site {i}: u={u[k, i]!r} p={p!r}"
            n_bd += 1
    return n_eq, n_bd


def oracle_chain(state, props, beta, seed, prop_base, n):
    return mh.chain(state, props, beta, seed, prop_base, n)
