"""Boundary-MPS environments of the L x L Boltzmann network (Sec. 2.2, Sec. 3.2).

The network of Eq. 6 is contracted from the bottom boundary upward (Fig. 2):
row L-1 is an MPS whose physical legs are the bottom-row spins; each higher row
r is a transfer MPO whose site tensors are copy tensors (Eq. 8) with the
horizontal Boltzmann matrix on the right leg and the vertical one on the down
leg (Eq. 7). MPO x MPS doubles the bond; ``compress`` brings it back to chi.
After row r the MPS represents, as a function of the row-r spins,

    F_r(s_r) = sum over rows below r of exp(-beta E) restricted to the bonds
               inside rows r..L-1 (horizontal bonds of rows r..L-1 and the
               vertical bonds between them),

which is what the sampler needs for the conditionals of Eq. 4-5.

Site tensors are float64 arrays (D_left, 2, D_right), index order
[left, physical, right] as in Sec. 3.2; the physical index is the spin bit
(0: s = -1, 1: s = +1).

Readings of points the paper leaves open:
* compress = a left-to-right QR sweep (left-canonical form), then a
  right-to-left SVD sweep keeping, at each bond, the singular values that are
  among the chi largest AND above cutoff * (largest) -- the "truncation
  threshold" of Sec. 1. The threshold is not optional in practice: keeping
  numerically-zero singular values lets their noise directions grow under the
  next rows' transfer MPOs (at beta = 3, L = 32, log Z then drifts by ~10 as
  chi grows while the discarded weight is 1e-19); the default 1e-12 is far
  above float64 rounding and far below any physical weight.
* Boltzmann matrices are used normalised (entries {1, exp(-2 beta |J|)}), the
  removed factor exp(beta |J|) and every renormalisation go into a float64 log
  scale lambda_r, so F_r = exp(lambda_r) * contraction(tensors).
* combined bond index after MPO x MPS: (MPO leg major, MPS leg minor).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from .ising import boltzmann_matrix_normalised


@dataclasses.dataclass
class RowEnv:
    """Row r of the cache: site tensors, log scale and per-bond diagnostics."""
    tensors: List[np.ndarray]
    log_scale: float
    spectra: List[np.ndarray]      # singular values kept at bond c (c = 1..L-1), divided by the largest
    cut_gap: List[float]           # s_k / s_{k+1} - 1 at each bond where values were dropped (inf if none)
    discarded: List[float]         # sum of dropped s^2 / sum of all s^2 at each bond


def bottom_row_mps(Jh_row: np.ndarray, beta: float):
    """Sec. 3.2: MPS of the bottom row, bond 2; returns (tensors, log_scale).

    Site 0: A[0, s, b] = B(Jh[0])[s, b]; middle sites: A[a, s, b] = delta(a, s) B(Jh[c])[s, b];
    last site: A[a, s, 0] = delta(a, s).
    """
    L = Jh_row.size + 1
    if L == 1:
        return [np.ones((1, 2, 1))], 0.0
    tensors, log_scale = [], 0.0
    for c in range(L):
        if c < L - 1:
            B, sc = boltzmann_matrix_normalised(beta, Jh_row[c])
            log_scale += sc
        if c == 0:
            A = B.reshape(1, 2, 2).copy()
        elif c < L - 1:
            A = np.zeros((2, 2, 2))
            for s in range(2):
                A[s, s, :] = B[s, :]
        else:
            A = np.zeros((2, 2, 1))
            for s in range(2):
                A[s, s, 0] = 1.0
        tensors.append(A)
    return tensors, log_scale


def row_mpo(Jh_row: np.ndarray, Jv_row: np.ndarray, beta: float):
    """Sec. 3.2: the transfer MPO of row r, tensors W[left, up, right, down]; returns (tensors, log_scale).

    Every site is a copy tensor: the up (new physical) index equals the left
    index, and the right and down legs carry B(Jh[c]) and B(Jv[c]) from that
    spin. Site 0 has no left leg and site L-1 no right leg.
    """
    L = Jv_row.size
    tensors, log_scale = [], 0.0
    for c in range(L):
        Bd, sd = boltzmann_matrix_normalised(beta, Jv_row[c])
        log_scale += sd
        if c < L - 1:
            Br, sr = boltzmann_matrix_normalised(beta, Jh_row[c])
            log_scale += sr
        else:
            Br = np.ones((2, 1))  # no right neighbour: a trivial right leg
        Dl = 1 if c == 0 else 2
        Dr = Br.shape[1]
        W = np.zeros((Dl, 2, Dr, 2))
        for s in range(2):
            a = 0 if c == 0 else s
            W[a, s, :, :] = np.outer(Br[s, :], Bd[s, :])
        tensors.append(W)
    return tensors, log_scale


def multiply(mpo: List[np.ndarray], mps: List[np.ndarray]) -> List[np.ndarray]:
    """Fig. 2: MPO x MPS; new[(a, a'), s, (b, b')] = sum_n W[a, s, b, n] A[a', n, b'].

    The physical dimension d is read from the tensors (2 for Ising spins, q for Potts)."""
    out = []
    for W, A in zip(mpo, mps):
        T = np.einsum("asbn,xny->axsby", W, A)
        Dl = W.shape[0] * A.shape[0]
        Dr = W.shape[2] * A.shape[2]
        out.append(T.reshape(Dl, W.shape[1], Dr))
    return out


DEFAULT_CUTOFF = 1e-12


def compress(mps: List[np.ndarray], chi: int, cutoff: float = DEFAULT_CUTOFF):
    """Bring every bond to at most chi (Sec. 2.2, Sec. 3.2 ``compress``).

    1. Left-to-right QR sweep: A_c = Q R, A_c <- Q, A_{c+1} <- R A_{c+1}.
    2. Right-to-left SVD sweep: A_c (as D_l x (d D_r), d the physical dimension) = U S V^T, keep the k
       largest singular values (k <= chi, S[k-1] > cutoff * S[0], k >= 1),
       A_c <- V^T[:k], A_{c-1} <- A_{c-1} U[:, :k] S[:k].
    3. Site 0 is divided by its Frobenius norm.
    Every division by a norm is added to the returned log scale. Returns
    (tensors, log_scale, spectra, cut_gap, discarded); the diagnostics are
    indexed by bond c = 1 .. L-1 (bond c joins sites c-1 and c).
    """
    mps = [A.copy() for A in mps]
    L = len(mps)
    log_scale = 0.0
    for c in range(L - 1):
        Dl, d, Dr = mps[c].shape
        Q, R = np.linalg.qr(mps[c].reshape(Dl * d, Dr), mode="reduced")
        nrm = np.linalg.norm(R)
        if nrm > 0:
            R = R / nrm
            log_scale += np.log(nrm)
        mps[c] = Q.reshape(Dl, d, Q.shape[1])
        mps[c + 1] = np.einsum("ka,asb->ksb", R, mps[c + 1])
    spectra, gaps, disc = [None] * L, [np.inf] * L, [0.0] * L
    for c in range(L - 1, 0, -1):
        Dl, d, Dr = mps[c].shape
        U, S, Vh = np.linalg.svd(mps[c].reshape(Dl, d * Dr), full_matrices=False)
        k = min(chi, S.size, max(1, int(np.sum(S > cutoff * S[0]))))
        total = float(np.sum(S ** 2))
        if k < S.size:
            gaps[c] = (S[k - 1] / S[k] - 1.0) if S[k] > 0 else np.inf
            disc[c] = float(np.sum(S[k:] ** 2)) / total if total > 0 else 0.0
        spectra[c] = S[:k] / S[0] if S[0] > 0 else S[:k]
        s_max = S[0] if S[0] > 0 else 1.0
        log_scale += np.log(s_max)
        mps[c] = Vh[:k].reshape(k, d, Dr)
        mps[c - 1] = np.einsum("asb,bk->ask", mps[c - 1], U[:, :k] * (S[:k] / s_max))
    nrm = np.linalg.norm(mps[0])
    mps[0] = mps[0] / nrm
    log_scale += np.log(nrm)
    return mps, log_scale, spectra[1:], gaps[1:], disc[1:]


def build_envs(Jh: np.ndarray, Jv: np.ndarray, beta: float, chi: int,
               cutoff: float = DEFAULT_CUTOFF) -> List[RowEnv]:
    """Sec. 3.2 ``create_cache_ising``: the cache rows L-1 .. 0, returned indexed by row.

    Row L-1 is the bottom-row MPS (compressed like every other row so that all
    rows share one canonical form); for r = L-2 .. 0 the row MPO is applied to
    the row below and the result compressed to chi. lambda_r accumulates all
    log scales from the bottom up.
    """
    L = Jh.shape[0]
    rows: List[RowEnv] = [None] * L
    mps, lam = bottom_row_mps(Jh[L - 1], beta)
    for r in range(L - 1, -1, -1):
        if r < L - 1:
            mpo, sc = row_mpo(Jh[r], Jv[r], beta)
            mps = multiply(mpo, mps)
            lam += sc
        if L > 1:
            mps, sc, spec, gaps, disc = compress(mps, chi, cutoff)
        else:
            spec, gaps, disc, sc = [], [], [], 0.0
        lam += sc
        rows[r] = RowEnv([A.copy() for A in mps], lam, spec, gaps, disc)
    return rows


def log_z(rows: List[RowEnv]) -> float:
    """Eq. 6 from the top row: Z = exp(lambda_0) * sum_s F_0(s), summing every physical leg."""
    top = rows[0]
    v = np.ones(1)
    log_acc = 0.0
    for A in top.tensors:
        v = v @ A.sum(axis=1)
        nrm = np.linalg.norm(v)
        v = v / nrm
        log_acc += np.log(nrm)
    return top.log_scale + log_acc + np.log(abs(v.item()))


def contract_row(row: RowEnv, sigma_row: np.ndarray) -> float:
    """log F_r(sigma_row) for one configuration of row r (a test helper)."""
    v = np.ones(1)
    log_acc = 0.0
    for c, A in enumerate(row.tensors):
        v = v @ A[:, int(sigma_row[c]), :]
        nrm = np.linalg.norm(v)
        if nrm == 0:
            return -np.inf
        v = v / nrm
        log_acc += np.log(nrm)
    return row.log_scale + log_acc + np.log(abs(v.item()))
