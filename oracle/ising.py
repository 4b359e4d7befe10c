"""Edwards-Anderson model on an open L x L lattice (Sec. 2.1, Eq. 1-2, Eq. 7).

Spin bit sigma in {0, 1} stands for s = 2 sigma - 1 (bit 1 is spin +1, the
listing's ``2 * cfg - 1`` in Sec. 3.3). Sites are numbered in raster order
i = r * L + c (Eq. 3, Fig. 1a), r = 0 the top row.
"""
from __future__ import annotations

import numpy as np


def spin(sigma):
    """Bit -> spin value: 0 -> -1, 1 -> +1."""
    return 2.0 * np.asarray(sigma, dtype=np.float64) - 1.0


def boltzmann_matrix(beta: float, J: float) -> np.ndarray:
    """Eq. 7: B[sigma, sigma'] = exp(beta J s s'), rows/columns ordered s = -1, +1."""
    s = np.array([-1.0, 1.0])
    return np.exp(beta * float(J) * np.outer(s, s))


def boltzmann_matrix_normalised(beta: float, J: float):
    """Eq. 7 divided by exp(beta |J|): entries {1, exp(-2 beta |J|)}; returns (B_hat, beta |J|).

    The scale is carried as a log so that beta = 3 does not overflow; the
    product of the two is Eq. 7 exactly.
    """
    scale = beta * abs(float(J))
    s = np.array([-1.0, 1.0])
    return np.exp(beta * float(J) * np.outer(s, s) - scale), scale


def energy(Jh: np.ndarray, Jv: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """Eq. 1: E(s) = - sum_<ij> J_ij s_i s_j for bit arrays sigma (..., L, L).

    Summed in float64 in raster order of sites; at each site the bond to the
    left neighbour first, then the bond to the upper neighbour. For +-J bonds
    the result is an exact integer.
    """
    sigma = np.asarray(sigma)
    L = sigma.shape[-1]
    s = spin(sigma)
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    E = np.zeros(sigma.shape[:-2], np.float64)
    for r in range(L):
        for c in range(L):
            if c > 0:
                E = E - Jh[r, c - 1] * s[..., r, c] * s[..., r, c - 1]
            if r > 0:
                E = E - Jv[r - 1, c] * s[..., r, c] * s[..., r - 1, c]
    return E
