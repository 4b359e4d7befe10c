"""Pins of the q-state Potts oracle (oracle/potts.py) to things other than itself.

* a hand-computed energy on a 2 x 2 lattice, and the invariance of E under a global
  permutation of the q states;
* q = 2 is the Ising model at beta / 2 (delta(s, s') = (1 + s s') / 2): log Z against the
  Ising oracle's exact row transfer matrix, and the teacher-forced log q of the q = 2
  Potts sampler against the Ising sampler's at beta / 2;
* q = 3: log Z of the boundary MPS, exact at chi = 3^floor(L/2), against brute-force
  enumeration (L = 3, 3^9 states) and against the exact Potts row transfer matrix (L = 5);
* the forest closed form Z = q^(components) prod_e (exp(beta J_e) + q - 1) at L = 12 and
  beta = 2 (independent rows: Jv = 0);
* proposals with exact environments are draws from P: chi-squared of 60 000 proposals
  of an L = 2, q = 3 lattice against the brute-force distribution;
* q is invariant under a global permutation of the states (truncated by the cutoff, L = 6).
"""
import numpy as np
import pytest

from oracle import bmps, exact, philox, potts, sampler
from workloads import draw_bonds


def test_energy_hand_example():
    Jh = np.array([[1.0], [-1.0]])      # (0,0)-(0,1), (1,0)-(1,1)
    Jv = np.array([[-1.0, 1.0]])        # (0,0)-(1,0), (0,1)-(1,1)
    s = np.array([[2, 2], [2, 0]], np.uint8)
    # equal pairs: (0,0)-(0,1) J=+1, (0,0)-(1,0) J=-1; others differ
    assert potts.energy(Jh, Jv, s) == -(1.0) - (-1.0)
    s2 = np.array([[1, 1], [1, 1]], np.uint8)
    assert potts.energy(Jh, Jv, s2) == -(1.0 - 1.0 - 1.0 + 1.0)


def test_energy_permutation_invariant():
    Jh, Jv = draw_bonds(5, 11, "gauss")
    rng = np.random.default_rng(0)
    s = rng.integers(0, 4, size=(20, 5, 5)).astype(np.uint8)
    perm = np.array([2, 0, 3, 1], np.uint8)
    np.testing.assert_allclose(potts.energy(Jh, Jv, perm[s]), potts.energy(Jh, Jv, s), rtol=0, atol=1e-12)


@pytest.mark.parametrize("beta", [0.6, 2.0])
def test_q2_log_z_is_ising_at_half_beta(beta):
    L = 6
    Jh, Jv = draw_bonds(L, 1003, "gauss")
    rows = potts.build_envs(Jh, Jv, beta, 2, 8, cutoff=0.0)      # chi = 2^3: exact
    shift = beta * (float(Jh.astype(np.float64).sum()) + float(Jv.astype(np.float64).sum())) / 2.0
    ref = shift + exact.transfer_log_z(Jh, Jv, beta / 2.0)
    assert abs(potts.log_z(rows) - ref) < 1e-10 * abs(ref)


def test_q2_scores_are_the_ising_scores_at_half_beta():
    L, beta, S = 5, 1.3, 16
    Jh, Jv = draw_bonds(L, 1007, "pmj")
    rng = np.random.default_rng(3)
    states = rng.integers(0, 2, size=(S, L, L)).astype(np.uint8)
    p_rows = potts.build_envs(Jh, Jv, beta, 2, 4)
    i_rows = bmps.build_envs(Jh, Jv, beta / 2.0, 4)
    p_lq, p_E, _ = potts.score(p_rows, Jh, Jv, beta, 2, states)
    i_lq, i_E, _ = sampler.score(i_rows, Jh, Jv, beta / 2.0, states)
    np.testing.assert_allclose(p_lq, i_lq, rtol=1e-10, atol=1e-10)
    shift = (float(Jh.sum()) + float(Jv.sum())) / 2.0
    np.testing.assert_allclose(2.0 * p_E, i_E - 2.0 * shift, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind,beta", [("pmj", 0.8), ("gauss", 1.5)])
def test_q3_log_z_brute_force(kind, beta):
    L, q = 3, 3
    Jh, Jv = draw_bonds(L, 1011, kind)
    rows = potts.build_envs(Jh, Jv, beta, q, 3, cutoff=0.0)
    _, _, _, lz = potts.brute_force(Jh, Jv, beta, q)
    assert abs(potts.log_z(rows) - lz) < 1e-11 * abs(lz)


def test_q3_log_z_transfer_matrix():
    L, q, beta = 5, 3, 1.1
    Jh, Jv = draw_bonds(L, 1013, "pmj")
    rows = potts.build_envs(Jh, Jv, beta, q, 9, cutoff=0.0)
    ref = potts.transfer_log_z(Jh, Jv, beta, q)
    assert abs(potts.log_z(rows) - ref) < 1e-11 * abs(ref)
    # the transfer matrix itself against brute force on a smaller lattice
    Jh3, Jv3 = draw_bonds(3, 1015, "gauss")
    assert abs(potts.transfer_log_z(Jh3, Jv3, 0.9, q) - potts.brute_force(Jh3, Jv3, 0.9, q)[3]) < 1e-11


@pytest.mark.parametrize("q", [3, 4])
def test_forest_closed_form(q):
    L, beta = 12, 2.0
    Jh, _ = draw_bonds(L, 1017, "pmj")
    Jv = np.zeros((L - 1, L), np.float32)
    rows = potts.build_envs(Jh, Jv, beta, q, q)
    Jd = Jh.astype(np.float64)
    ref = L * np.log(q) + float(np.sum(np.log(np.exp(beta * Jd) + q - 1.0)))
    assert abs(potts.log_z(rows) - ref) < 1e-11 * abs(ref)


def test_exact_proposals_are_boltzmann_draws():
    L, q, beta, S = 2, 3, 0.9, 60000
    Jh, Jv = draw_bonds(L, 1019, "pmj")
    rows = potts.build_envs(Jh, Jv, beta, q, 3, cutoff=0.0)
    st, lq, E, _ = potts.propose(rows, Jh, Jv, beta, q, S, 5, 0, 0)
    codes = (st.reshape(S, -1).astype(np.int64) * (q ** np.arange(L * L - 1, -1, -1))).sum(axis=1)
    counts = np.bincount(codes, minlength=q ** (L * L))
    allst, _, logp, lz = potts.brute_force(Jh, Jv, beta, q)
    p = np.exp(logp)
    chi2 = float(((counts - S * p) ** 2 / (S * p)).sum())
    dof = q ** (L * L) - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof), chi2
    # exact environments: q = P, so log q + beta E = -log Z for every proposal
    np.testing.assert_allclose(lq + beta * E, -lz, atol=1e-10)


def test_proposal_probability_is_permutation_invariant():
    L, q, beta, S = 6, 3, 1.2, 24
    Jh, Jv = draw_bonds(L, 1021, "pmj")
    # truncated by the cutoff only: a global permutation maps degenerate multiplets of
    # singular values onto themselves, so a cutoff keeps or drops whole multiplets (a rank
    # cap inside a multiplet would break the symmetry)
    rows = potts.build_envs(Jh, Jv, beta, q, 27, cutoff=1e-3)
    assert max(A.shape[2] for A in rows[0].tensors) < 27
    st, lq, _, _ = potts.propose(rows, Jh, Jv, beta, q, S, 7, 0, 0)
    perm = np.array([1, 2, 0], np.uint8)
    lq2, _, _ = potts.score(rows, Jh, Jv, beta, q, perm[st])
    np.testing.assert_allclose(lq2, lq, rtol=1e-9, atol=1e-9)


def test_draw_rule_is_the_first_partial_sum_above_u():
    # one site (L = 1): p is uniform over q states, the state is floor(u q)
    q = 4
    rows = potts.build_envs(np.zeros((1, 0)), np.zeros((0, 1)), 1.0, q, 4)
    S = 4000
    st, lq, _, _ = potts.propose(rows, np.zeros((1, 0)), np.zeros((0, 1)), 1.0, q, S, 9, 0, 0)
    u = philox.spin_uniforms(1, np.arange(S, dtype=np.uint64), 0, 9)[:, 0]
    assert np.array_equal(st[:, 0, 0], np.floor(u * q).astype(np.uint8))
    np.testing.assert_allclose(lq, -np.log(q), atol=1e-15)


def test_mh_with_a_poor_potts_proposal_samples_boltzmann():
    """A chi = 1 Potts proposal (far from P), corrected by Eq. 10 with the Potts energy, samples
    P: chi-squared of the chain's states over the 81 states of an L = 2, q = 3 lattice."""
    from oracle import mh
    L, q, beta, S = 2, 3, 0.8, 60000
    Jh, Jv = draw_bonds(L, 1023, "pmj")
    rows = potts.build_envs(Jh, Jv, beta, q, 1)
    props = potts.propose(rows, Jh, Jv, beta, q, S, 11, 0, 0)[:3]
    start = (np.zeros((L, L), np.uint8), np.inf, 0.0)     # an empty chain: the first proposal is taken
    _, acc, _, _ = mh.chain(start, props, beta, 11, 0, 0)
    assert acc[0] == 1 and 0.05 < acc.mean() < 0.99
    codes = props[0].reshape(S, -1).astype(np.int64) @ (q ** np.arange(L * L - 1, -1, -1))
    states = np.empty(S, np.int64)
    cur = codes[0]
    for k in range(S):
        if acc[k]:
            cur = codes[k]
        states[k] = cur
    cnt = np.bincount(states, minlength=q ** (L * L))
    _, _, logp, _ = potts.brute_force(Jh, Jv, beta, q)
    exp_cnt = S * np.exp(logp)
    keep = exp_cnt > 10
    tau = 1.0 / acc.mean()          # successive states are correlated
    chi2 = float(((cnt[keep] - exp_cnt[keep]) ** 2 / exp_cnt[keep]).sum()) / tau
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)
