"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no arithmetic of the method: it only draws disorder
realizations and lays them out. Both the CUDA path and the CPU oracle take
their inputs from here, so the two never feed each other.

Coupling layout (Sec. 3.1): a realization of side L is an (L, L, 4) float32
array ``J_mat`` whose last axis holds the couplings of site (r, c) to its
(left, up, right, down) neighbour, 0 where the open boundary has none.
Row r = 0 is the top row, column c = 0 the left column.

Workloads follow the paper's Edwards-Anderson experiments (Sec. 4): +-J bonds
with p = 1/2 (Sec. 3.1), or N(0, 1) bonds for the Gaussian model. Disorder of
realization n is drawn from ``numpy.random.default_rng(1000 + n)``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

SAMPLING_SEED = 42


def draw_bonds(L: int, seed: int, kind: str = "pmj", p: float = 0.5):
    """Return (Jh, Jv): Jh[r, c] joins (r, c)-(r, c+1); Jv[r, c] joins (r, c)-(r+1, c).

    kind "pmj": each bond is -1 with probability p, else +1 (p = 1/2 is EA).
    kind "gauss": each bond is N(0, 1), rounded to float32.
    """
    rng = np.random.default_rng(seed)
    nh, nv = L * (L - 1), (L - 1) * L
    if kind == "pmj":
        neg = rng.random(nh + nv) < p
        vals = np.where(neg, -1.0, 1.0)
    elif kind == "gauss":
        vals = rng.standard_normal(nh + nv)
    else:
        raise ValueError(f"unknown coupling kind {kind!r}")
    vals = vals.astype(np.float32)
    Jh = vals[:nh].reshape(L, L - 1) if L > 1 else np.zeros((L, 0), np.float32)
    Jv = vals[nh:].reshape(L - 1, L) if L > 1 else np.zeros((0, L), np.float32)
    return Jh, Jv


def to_paper_layout(Jh: np.ndarray, Jv: np.ndarray) -> np.ndarray:
    """(Jh, Jv) -> (L, L, 4) float32 with (left, up, right, down) per site."""
    L = Jh.shape[0]
    J = np.zeros((L, L, 4), np.float32)
    J[:, 1:, 0] = Jh
    J[1:, :, 1] = Jv
    J[:, :-1, 2] = Jh
    J[:-1, :, 3] = Jv
    return J


def from_paper_layout(J: np.ndarray):
    """(L, L, 4) -> (Jh, Jv); the inverse of :func:`to_paper_layout`."""
    return J[:, :-1, 2].copy(), J[:-1, :, 3].copy()


@dataclasses.dataclass
class Workload:
    """A batch of disorder realizations and the sampling parameters."""
    name: str
    Ls: List[int]
    beta: float
    chi: int
    S: int
    kind: str = "pmj"
    base_seed: int = 1000
    p: float = 0.5            # antiferromagnetic bond probability of the +-J model
    q: int = 2                # 2: Ising; 3 or 4: the q-state Potts extension

    @property
    def n_real(self) -> int:
        return len(self.Ls)

    def realization(self, n: int):
        return draw_bonds(self.Ls[n], self.base_seed + n, self.kind, self.p)

    def packed_J(self, idx: Sequence[int] | None = None) -> np.ndarray:
        """All realizations' paper-layout couplings, concatenated: (sum L^2, 4)."""
        idx = range(self.n_real) if idx is None else idx
        parts = [to_paper_layout(*self.realization(n)).reshape(-1, 4) for n in idx]
        return np.ascontiguousarray(np.concatenate(parts, axis=0))


def config(name: str) -> Workload:
    """The named workloads, shaped like the paper's EA runs (Sec. 4)."""
    if name == "L16":        # one +-J realization, L=16, beta=1, chi=16, 1000 MH proposals
        return Workload("L16_chi16_beta1_fp64", [16], 1.0, 16, 1000)
    if name == "uneven":     # 200 +-J realizations, L in {32..128}, beta=2, chi=32, S=256
        rng = np.random.default_rng(7)
        Ls = [int(x) for x in rng.choice([32, 48, 64, 96, 128], size=200)]
        return Workload("uneven200_L32-128_chi32_beta2", Ls, 2.0, 32, 256)
    if name == "L256":       # 64 +-J realizations, L=256, beta=3, chi=64, S=256
        return Workload("L256_chi64_beta3_n64_S256", [256] * 64, 3.0, 64, 256)
    if name == "gauss128":   # 128 Gaussian realizations, L=128, beta=2, chi=8
        return Workload("gauss_L128_chi8_beta2_n128", [128] * 128, 2.0, 8, 256, kind="gauss")
    if name == "L1024":      # 64 +-J realizations, L=1024, beta=3, chi=32, S=128
        return Workload("L1024_chi32_beta3_n64_S128", [1024] * 64, 3.0, 32, 128)
    if name == "paper":      # the paper's own configuration (Sec. 4): L=1024, beta=1, chi=8
        return Workload("paper_L1024_chi8_beta1_n64_S256", [1024] * 64, 1.0, 8, 256)
    if name == "L128b1x8":   # 8 realizations at L=128, beta=1, chi=32 (captures of the TF32 / BF16 builds)
        return Workload("L128_chi32_beta1_n8_S64", [128] * 8, 1.0, 32, 64)
    if name == "potts":      # the q-state Potts extension: 64 +-J realizations, q = 3, L=64, beta=1, chi=16
        return Workload("potts3_L64_chi16_beta1_n64_S256", [64] * 64, 1.0, 16, 256, q=3)
    if name == "potts_x4":   # 4 realizations of the Potts workload (profiler captures)
        return Workload("potts3_L64_chi16_beta1_n4_S64", [64] * 4, 1.0, 16, 64, q=3)
    # small cases of the L=256 workload's kernels (same beta, chi), for profiler captures
    if name == "L128x8":
        return Workload("L128_chi64_beta3_n8_S256", [128] * 8, 3.0, 64, 256)
    if name == "L64x64":    # the L=256 workload's sampler launch shape (64 x 256 chains) at L=64
        return Workload("L64_chi64_beta3_n64_S256", [64] * 64, 3.0, 64, 256)
    if name == "L64x2":     # two realizations at L=64 (same beta, chi): one build launch for captures
        return Workload("L64_chi64_beta3_n2_S64", [64] * 2, 3.0, 64, 64)
    if name == "L40x1":
        return Workload("L40_chi64_beta3_n1_S64", [40], 3.0, 64, 64)
    if name == "gauss128x8":   # 8 realizations of the Gaussian workload (profiler captures)
        return Workload("gauss_L128_chi8_beta2_n8", [128] * 8, 2.0, 8, 256, kind="gauss")
    raise KeyError(name)
