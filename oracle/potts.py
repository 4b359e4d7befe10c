"""q-state Potts extension of the method (Sec. 5: the approach carries over to Potts
models; the physical index of every tensor then runs over q states instead of 2).

Model: states s_i in {0, ..., q-1} on the L x L lattice, bonds as in Sec. 3.1,

    E(s) = - sum_<ij> J_ij delta(s_i, s_j),      P(s) = exp(-beta E(s)) / Z.

For q = 2, delta(s, s') = (1 + s s') / 2 in spin language, so the q = 2 Potts model at
(beta, J) is the Ising model of Eq. 1 at (beta / 2, J) up to the factor exp(beta sum J / 2)
in Z: the pin that ties this module to the (independently pinned) Ising oracle.

Everything follows the Ising oracle with d = q:
* Boltzmann matrices (Eq. 7 with delta in place of s s') are used normalised,
  B(J)[a, b] = exp(beta J delta(a, b) - beta max(J, 0)), entries in (0, 1]; the removed
  exp(beta max(J, 0)) goes into the log scale;
* the bottom row is the MPS A_0[0, s, b] = B(Jh)[s, b], A_c[a, s, b] = delta(a, s) B(Jh)[s, b],
  A_{L-1}[a, s, 0] = delta(a, s) (bond q); each higher row applies the copy-tensor MPO
  W[a, s, b, n] = delta(a, s) B(Jh)[s, b] B(Jv)[s, n] and compresses with bmps.compress;
* proposals are drawn row by row and site by site from
      p(s) = rho_s B(Jv[r-1, c])[s_up, s] / sum_s' (...),  rho_s = | l M_c[:, s, :] R_c |,
  with the right environments folding the vertical bonds to the row above as in the
  Ising sampler (all-ones for row 0). The draw with the site's Philox uniform u
  (philox.spin_uniforms) takes the first state k with u < p_0 + ... + p_k, the partial
  sums formed in float64 in the order k = 0, 1, ...; log q adds log p_s (Eq. 9).
States are stored as uint8 values 0 .. q-1.
"""
from __future__ import annotations

import itertools
from typing import List

import numpy as np

from . import bmps, philox


def energy(Jh: np.ndarray, Jv: np.ndarray, states: np.ndarray) -> np.ndarray:
    """E(s) = -sum J delta(s_i, s_j) for states (..., L, L), summed in float64 in raster
    order of sites: at each site the bond to the left neighbour first, then the bond to
    the upper neighbour. Exact integers for +-J bonds."""
    st = np.asarray(states).astype(np.int64)
    L = st.shape[-1]
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    E = np.zeros(st.shape[:-2], np.float64)
    for r in range(L):
        for c in range(L):
            if c > 0:
                E = E - Jh[r, c - 1] * (st[..., r, c] == st[..., r, c - 1])
            if r > 0:
                E = E - Jv[r - 1, c] * (st[..., r, c] == st[..., r - 1, c])
    return E


def boltzmann_normalised(beta: float, J: float, q: int):
    """(B, log scale): B[a, b] = exp(beta J delta(a, b) - beta max(J, 0)); scale = beta max(J, 0)."""
    scale = beta * max(float(J), 0.0)
    B = np.exp(beta * float(J) * np.eye(q) - scale)
    return B, scale


def bottom_row_mps(Jh_row: np.ndarray, beta: float, q: int):
    """Bottom-row MPS of bond q (module docstring); returns (tensors, log_scale)."""
    L = Jh_row.size + 1
    if L == 1:
        return [np.ones((1, q, 1))], 0.0
    tensors, log_scale = [], 0.0
    for c in range(L):
        if c < L - 1:
            B, sc = boltzmann_normalised(beta, Jh_row[c], q)
            log_scale += sc
        if c == 0:
            A = B.reshape(1, q, q).copy()
        elif c < L - 1:
            A = np.zeros((q, q, q))
            for s in range(q):
                A[s, s, :] = B[s, :]
        else:
            A = np.zeros((q, q, 1))
            for s in range(q):
                A[s, s, 0] = 1.0
        tensors.append(A)
    return tensors, log_scale


def row_mpo(Jh_row: np.ndarray, Jv_row: np.ndarray, beta: float, q: int):
    """Transfer MPO of row r, tensors W[left, up, right, down]: copy tensors of q states
    with B(Jh) on the right leg and B(Jv) on the down leg; returns (tensors, log_scale)."""
    L = Jv_row.size
    tensors, log_scale = [], 0.0
    for c in range(L):
        Bd, sd = boltzmann_normalised(beta, Jv_row[c], q)
        log_scale += sd
        if c < L - 1:
            Br, sr = boltzmann_normalised(beta, Jh_row[c], q)
            log_scale += sr
        else:
            Br = np.ones((q, 1))
        Dl = 1 if c == 0 else q
        W = np.zeros((Dl, q, Br.shape[1], q))
        for s in range(q):
            W[0 if c == 0 else s, s, :, :] = np.outer(Br[s, :], Bd[s, :])
        tensors.append(W)
    return tensors, log_scale


def build_envs(Jh: np.ndarray, Jv: np.ndarray, beta: float, q: int, chi: int,
               cutoff: float = bmps.DEFAULT_CUTOFF) -> List[bmps.RowEnv]:
    """The cache rows L-1 .. 0 (indexed by row), as bmps.build_envs with q states."""
    L = Jh.shape[0]
    rows: List[bmps.RowEnv] = [None] * L
    mps, lam = bottom_row_mps(Jh[L - 1], beta, q)
    for r in range(L - 1, -1, -1):
        if r < L - 1:
            mpo, sc = row_mpo(Jh[r], Jv[r], beta, q)
            mps = bmps.multiply(mpo, mps)
            lam += sc
        if L > 1:
            mps, sc, spec, gaps, disc = bmps.compress(mps, chi, cutoff)
        else:
            spec, gaps, disc, sc = [], [], [], 0.0
        lam += sc
        rows[r] = bmps.RowEnv([A.copy() for A in mps], lam, spec, gaps, disc)
    return rows


def log_z(rows: List[bmps.RowEnv]) -> float:
    """Eq. 6: the top row's MPS summed over every physical index (as for Ising)."""
    return bmps.log_z(rows)


def _fold_up(M: np.ndarray, beta: float, Jv, q: int) -> np.ndarray:
    """T[i, u, k] = sum_s B(Jv)[u, s] M[i, s, k] (normalised B; all-ones without a bond above)."""
    B = np.ones((q, q)) if Jv is None else boltzmann_normalised(beta, Jv, q)[0]
    return np.einsum("isk,us->iuk", M, B)


def run_rows(rows, Jh, Jv, beta, q, u=None, forced=None):
    """Propose (uniforms u (S, L*L)) or score (forced states (S, L, L)) one realization:
    returns (states (S, L, L) uint8, log_q (S,), probabilities drawn from (S, L*L, q))."""
    L = len(rows)
    S = (u if u is not None else forced).shape[0]
    st = np.zeros((S, L, L), np.uint8)
    log_q = np.zeros(S)
    probs = np.zeros((S, L * L, q))
    for r in range(L):
        M = rows[r].tensors
        up = st[:, r - 1, :].astype(np.intp) if r > 0 else None
        R = [None] * L
        R[L - 1] = np.ones((S, M[L - 1].shape[2]))
        for c in range(L - 2, -1, -1):
            T = _fold_up(M[c + 1], beta, Jv[r - 1, c + 1] if r > 0 else None, q)
            sel = up[:, c + 1] if r > 0 else np.zeros(S, np.intp)
            Rc = np.einsum("isk,sk->si", T[:, sel, :], R[c + 1])
            R[c] = Rc / np.linalg.norm(Rc, axis=1, keepdims=True)
        left = np.ones((S, 1))
        for c in range(L):
            v = np.einsum("si,ijk->sjk", left, M[c])          # (S, q, D_r)
            w = np.abs(np.einsum("sjk,sk->sj", v, R[c]))      # (S, q)
            if r > 0:
                Bup = boltzmann_normalised(beta, Jv[r - 1, c], q)[0]
                w = w * Bup[up[:, c], :]
            tot = w.sum(axis=1)
            if np.any(tot == 0):
                raise FloatingPointError(f"every conditional vanishes at row {r} col {c}")
            p = w / tot[:, None]
            i = r * L + c
            if forced is not None:
                k = forced[:, r, c].astype(np.intp)
            else:
                cum = np.zeros(S)
                k = np.full(S, q - 1, np.intp)
                found = np.zeros(S, bool)
                for j in range(q - 1):
                    cum = cum + p[:, j]
                    hit = (~found) & (u[:, i] < cum)
                    k[hit] = j
                    found |= hit
            st[:, r, c] = k.astype(np.uint8)
            probs[:, i, :] = p
            with np.errstate(divide="ignore"):
                log_q += np.log(p[np.arange(S), k])
            left = v[np.arange(S), k, :]
            left = left / np.linalg.norm(left, axis=1, keepdims=True)
    return st, log_q, probs


def propose(rows, Jh, Jv, beta, q, S, seed, prop_base, n):
    """S proposals of realization n (ids prop_base ..): (states, log_q, E, probs)."""
    L = len(rows)
    t = np.arange(S, dtype=np.uint64) + np.uint64(prop_base)
    u = philox.spin_uniforms(L, t, n, seed)
    st, log_q, probs = run_rows(rows, Jh, Jv, beta, q, u=u)
    return st, log_q, energy(Jh, Jv, st), probs


def score(rows, Jh, Jv, beta, q, states):
    """Teacher-forced log q and energy of given states: (log_q, E, probs)."""
    _, log_q, probs = run_rows(rows, Jh, Jv, beta, q, forced=np.asarray(states))
    return log_q, energy(Jh, Jv, states), probs


# ------------------------------------------------------------------ exact references
def all_states(L: int, q: int) -> np.ndarray:
    """Every configuration of L*L sites (q^N, L, L); site 0 varies slowest."""
    N = L * L
    return np.array(list(itertools.product(range(q), repeat=N)), dtype=np.uint8).reshape(-1, L, L)


def brute_force(Jh, Jv, beta, q):
    """(states, E, log P, log Z) over all q^(L^2) configurations."""
    L = Jh.shape[0]
    st = all_states(L, q)
    E = energy(Jh, Jv, st)
    lw = -beta * E
    m = lw.max()
    lz = m + np.log(np.exp(lw - m).sum())
    return st, E, lw - lz, lz


def transfer_log_z(Jh, Jv, beta, q):
    """Exact log Z by the row transfer matrix over the q^L configurations of a row."""
    L = Jh.shape[0]
    rows = np.array(list(itertools.product(range(q), repeat=L)), dtype=np.int64)   # (q^L, L)

    def row_weight(r):
        e = np.zeros(rows.shape[0])
        for c in range(L - 1):
            e += Jh[r, c] * (rows[:, c] == rows[:, c + 1])
        return beta * e

    def vert(r):
        same = (rows[:, None, :] == rows[None, :, :]).astype(np.float64)   # (q^L, q^L, L)
        return beta * (same * Jv[r][None, None, :]).sum(axis=2)

    logf = row_weight(L - 1)
    for r in range(L - 2, -1, -1):
        a = vert(r) + logf[None, :]
        m = a.max(axis=1, keepdims=True)
        logf = row_weight(r) + (m[:, 0] + np.log(np.exp(a - m).sum(axis=1)))
    m = logf.max()
    return float(m + np.log(np.exp(logf - m).sum()))
