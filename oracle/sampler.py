"""Row-by-row ancestral proposals from the cached environments (Sec. 3.3, Eq. 4-5, Eq. 9).

For row r, given the rows above (``s_up`` = row r-1):

* right environments (computed right to left): R_{L-1} = 1 and
  R_c = T_{c+1}[s_up(c+1)] R_{c+1}, divided by its 2-norm, where
  T_c[u] = sum_s B(Jv[r-1, c])[u, s] M_c[:, s, :] folds the vertical bond to
  the sampled spin above into the cache tensor M_c of row r;
* left sweep (left to right): rho_s = | l M_c[:, s, :] R_c | for s in {0, 1};
  logit = log(rho_1 / rho_0) + 2 beta Jv[r-1, c] s_up(c) (Eq. 5); the spin is
  +1 with probability sigmoid(logit); log q gains log sigmoid(+-logit) (Eq. 9);
  l <- l M_c[:, s, :] divided by its 2-norm.

Reading of the paper: for row 0 there is no row above; the fold uses the all-ones
matrix (J = 0) and the up-field is 0. The draw is: spin +1 iff u < sigmoid(logit)
with u the Philox uniform of that site (``philox.py``). If rho_0 = rho_1 = 0
the conditional is undefined and the call raises.

Everything is float64; loops run over rows and columns, numpy vectorises over
samples.
"""
from __future__ import annotations

import numpy as np

from . import philox
from .bmps import RowEnv
from .ising import boltzmann_matrix, energy


def log_sigmoid(x):
    """log(1 / (1 + exp(-x))), stable for either sign."""
    x = np.asarray(x, dtype=np.float64)
    return -(np.maximum(-x, 0.0) + np.log1p(np.exp(-np.abs(x))))


def sigmoid(x):
    x = np.asarray(x, dtype=np.float64)
    return np.exp(log_sigmoid(x))


def _fold_up(M: np.ndarray, beta: float, Jv: float | None) -> np.ndarray:
    """T[i, u, k] = sum_s B(Jv)[u, s] M[i, s, k]; the all-ones matrix when there is no bond above."""
    B = np.ones((2, 2)) if Jv is None else boltzmann_matrix(beta, Jv)
    return np.einsum("isk,us->iuk", M, B)


def run_rows(rows, Jh, Jv, beta, u=None, forced=None, correction=None):
    """Propose (u given) or score (forced spins given) S configurations of one realization.

    rows       : list of RowEnv, the cache indexed by row
    u          : (S, L*L) uniforms for the draws, raster order (propose mode)
    forced     : (S, L, L) spin bits to score (teacher-forced mode)
    correction : optional callable (sigma so far, r, c, logit) -> Delta added to
                 the logit before the draw and before log q (``learned.Correction``)
    Returns (sigma (S, L, L) uint8, log_q (S,), logits (S, L*L)), the logits
    being the ones drawn from (corrected when a correction is given).
    """
    L = len(rows)
    S = (u if u is not None else forced).shape[0]
    sigma = np.zeros((S, L, L), np.uint8)
    log_q = np.zeros(S)
    logits = np.zeros((S, L * L))
    for r in range(L):
        M = rows[r].tensors
        up = sigma[:, r - 1, :] if r > 0 else None
        # right environments
        R = [None] * L
        R[L - 1] = np.ones((S, M[L - 1].shape[2]))
        for c in range(L - 2, -1, -1):
            T = _fold_up(M[c + 1], beta, Jv[r - 1, c + 1] if r > 0 else None)
            sel = up[:, c + 1] if r > 0 else np.zeros(S, np.intp)
            Tsel = T[:, sel, :]                              # (D_l, S, D_r)
            Rc = np.einsum("isk,sk->si", Tsel, R[c + 1])
            R[c] = Rc / np.linalg.norm(Rc, axis=1, keepdims=True)
        # left sweep
        left = np.ones((S, 1))
        for c in range(L):
            v = np.einsum("si,ijk->sjk", left, M[c])         # (S, 2, D_r)
            rho = np.abs(np.einsum("sjk,sk->sj", v, R[c]))   # (S, 2)
            if np.any((rho[:, 0] == 0) & (rho[:, 1] == 0)):
                raise FloatingPointError(f"both conditionals vanish at row {r} col {c}")
            with np.errstate(divide="ignore"):
                logit = np.log(rho[:, 1]) - np.log(rho[:, 0])
            if r > 0:
                s_up = 2.0 * up[:, c] - 1.0
                logit = logit + 2.0 * beta * float(Jv[r - 1, c]) * s_up
            if correction is not None:
                logit = logit + correction(sigma, r, c, logit)
            i = r * L + c
            if forced is not None:
                bit = forced[:, r, c].astype(np.uint8)
            else:
                bit = (u[:, i] < sigmoid(logit)).astype(np.uint8)
            sigma[:, r, c] = bit
            logits[:, i] = logit
            log_q += np.where(bit == 1, log_sigmoid(logit), log_sigmoid(-logit))
            left = v[np.arange(S), bit, :]
            left = left / np.linalg.norm(left, axis=1, keepdims=True)
    return sigma, log_q, logits


def propose(rows, Jh, Jv, beta, S, seed, prop_base, n, correction=None):
    """S proposals of realization n with ids prop_base .. prop_base+S-1: (sigma, log_q, E, logits)."""
    L = len(rows)
    t = np.arange(S, dtype=np.uint64) + np.uint64(prop_base)
    u = philox.spin_uniforms(L, t, n, seed)
    sigma, log_q, logits = run_rows(rows, Jh, Jv, beta, u=u, correction=correction)
    return sigma, log_q, energy(Jh, Jv, sigma), logits


def score(rows, Jh, Jv, beta, sigma, correction=None):
    """Teacher-forced log q and energy of given configurations: (log_q, E, logits)."""
    _, log_q, logits = run_rows(rows, Jh, Jv, beta, forced=np.asarray(sigma), correction=correction)
    return log_q, energy(Jh, Jv, sigma), logits
