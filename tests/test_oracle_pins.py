"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one part of the oracle to a fact the paper or the mathematics
fixes: numpy's own Philox4x64-10, brute-force enumeration of Eq. 2-4, the
exact row transfer matrix, closed forms on forests, gauge invariance, and the
exactness of ancestral sampling when chi reaches the full Schmidt rank.
"""
import numpy as np
import pytest

from oracle import bmps, exact, mh, philox, sampler
from oracle.ising import boltzmann_matrix, energy
from workloads import draw_bonds, from_paper_layout, to_paper_layout


# ---------------------------------------------------------------- Philox
def test_philox_matches_numpy_bit_generator():
    """Philox4x64-10 words equal numpy.random.Philox (a library routine) on the same counter/key.

    numpy increments the counter before producing a block, so its state
    counter is the block's counter minus one.
    """
    rng = np.random.default_rng(0)
    for trial in range(20):
        ctr = rng.integers(1, 2 ** 63, size=4, dtype=np.uint64)
        ctr[3] = rng.integers(0, 4)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        prev = ctr.copy()
        prev[0] -= np.uint64(1)
        ref = np.random.Philox(counter=prev, key=key).random_raw(4)
        got = philox.philox4x64_10(ctr[None, :], key)[0]
        np.testing.assert_array_equal(got, ref)
    # carry from word 0 into word 1
    prev = np.array([2 ** 64 - 1, 5, 7, 1], dtype=np.uint64)
    ref = np.random.Philox(counter=prev, key=np.array([42, 0], np.uint64)).random_raw(4)
    got = philox.philox4x64_10(np.array([[0, 6, 7, 1]], np.uint64), (42, 0))[0]
    np.testing.assert_array_equal(got, ref)


def _numpy_philox_block(ctr, key):
    """The Philox4x64-10 block of a 256-bit counter from numpy.random.Philox, which
    increments its state counter (with carry) before producing a block."""
    v = sum(int(x) << (64 * k) for k, x in enumerate(ctr))
    v = (v - 1) % (1 << 256)
    prev = np.array([(v >> (64 * k)) & (2 ** 64 - 1) for k in range(4)], np.uint64)
    return np.random.Philox(counter=prev, key=np.array(key, np.uint64)).random_raw(4)


def _uniform_of(w):
    return (2 * (int(w) >> 12) + 1) * 2.0 ** -53       # exact in float64


def test_draw_counters_follow_the_published_layout():
    """The three streams against numpy's Philox on the counters the C ABI publishes: site i
    of proposal t in realization g, key (seed, 0): spin draw (i >> 2, t, g, 0) word i & 3;
    accept test (0, t, g, 1) word 0; random initial state (i >> 2, 0, g, 2) word i & 3,
    its top bit. Proposal ids from 0 to 2^40 + 3."""
    seed, g, L = 42, 5, 6
    ts = np.array([0, 1, 7, 123_456_789, 2 ** 40 + 3], np.uint64)
    u = philox.spin_uniforms(L, ts, g, seed)
    for a, t in enumerate(ts):
        for i in (0, 1, 3, 4, 17, L * L - 1):
            w = _numpy_philox_block([i >> 2, t, g, 0], (seed, 0))[i & 3]
            assert u[a, i] == _uniform_of(w), (t, i)
    um = philox.mh_uniforms(ts, g, seed)
    for a, t in enumerate(ts):
        assert um[a] == _uniform_of(_numpy_philox_block([0, t, g, 1], (seed, 0))[0]), t
    s = philox.init_spins(L, g, seed).reshape(-1)
    for i in range(L * L):
        w = _numpy_philox_block([i >> 2, 0, g, 2], (seed, 0))[i & 3]
        assert s[i] == int(w) >> 63, i


def test_uniform_map_open_interval_and_exact():
    w = np.array([0, 2 ** 64 - 1, 2 ** 63, 4095, 4096], dtype=np.uint64)
    u = philox.to_uniform(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == 2.0 ** -53 and u[1] == 1 - 2.0 ** -53
    assert u[2] == 0.5 + 2.0 ** -53 and u[3] == u[0] and u[4] == 3 * 2.0 ** -53


def test_uniforms_are_uniform():
    u = philox.spin_uniforms(64, np.arange(64), 3, 42).reshape(-1)   # 262144 draws
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = np.sum((hist - u.size / 64) ** 2 / (u.size / 64))
    assert chi2 < 120            # 63 dof: p ~ 1e-5 at 120
    assert abs(u.mean() - 0.5) < 5 / np.sqrt(12 * u.size)


# ---------------------------------------------------------------- layout and energy
def test_paper_layout_roundtrip_and_symmetry():
    Jh, Jv = draw_bonds(7, 11, "gauss")
    J = to_paper_layout(Jh, Jv)
    assert np.all(J[:, 0, 0] == 0) and np.all(J[0, :, 1] == 0)
    assert np.all(J[:, -1, 2] == 0) and np.all(J[-1, :, 3] == 0)
    np.testing.assert_array_equal(J[:, :-1, 2], J[:, 1:, 0])   # right of (r,c) = left of (r,c+1)
    np.testing.assert_array_equal(J[:-1, :, 3], J[1:, :, 1])   # down of (r,c) = up of (r+1,c)
    h2, v2 = from_paper_layout(J)
    np.testing.assert_array_equal(h2, Jh)
    np.testing.assert_array_equal(v2, Jv)


def test_energy_hand_example_2x2():
    Jh = np.array([[1.0], [-1.0]])           # (0,0)-(0,1) = 1, (1,0)-(1,1) = -1
    Jv = np.array([[-1.0, 1.0]])             # (0,0)-(1,0) = -1, (0,1)-(1,1) = 1
    sigma = np.array([[1, 0], [1, 1]])        # s = [[+1, -1], [+1, +1]]
    # E = -(1*(+1)(-1) + (-1)(+1)(+1) + (-1)(+1)(+1) + 1*(-1)(+1)) = -(-1 -1 -1 -1) = 4
    assert energy(Jh, Jv, sigma) == 4.0


def test_energy_ferromagnet_ground_state_and_symmetries():
    L = 9
    Jh, Jv = np.ones((L, L - 1)), np.ones((L - 1, L))
    up = np.ones((L, L), np.uint8)
    assert energy(Jh, Jv, up) == -2 * L * (L - 1)
    Jh, Jv = draw_bonds(L, 3, "pmj")
    rng = np.random.default_rng(1)
    s = rng.integers(0, 2, size=(20, L, L)).astype(np.uint8)
    E = energy(Jh, Jv, s)
    np.testing.assert_array_equal(E, energy(Jh, Jv, 1 - s))                # global flip
    assert np.all(E == np.round(E))                                         # +-J: integers
    # gauge: flip spin k and negate the four bonds at k
    r, c = 4, 5
    Jh2, Jv2 = Jh.copy(), Jv.copy()
    Jh2[r, c - 1] *= -1; Jh2[r, c] *= -1; Jv2[r - 1, c] *= -1; Jv2[r, c] *= -1
    s2 = s.copy(); s2[:, r, c] ^= 1
    np.testing.assert_array_equal(E, energy(Jh2, Jv2, s2))


def test_boltzmann_matrix_eq7():
    B = boltzmann_matrix(0.5, 2.0)
    np.testing.assert_allclose(B, [[np.e, 1 / np.e], [1 / np.e, np.e]])


# ---------------------------------------------------------------- log Z
@pytest.mark.parametrize("L,kind,beta", [(2, "pmj", 1.0), (3, "pmj", 1.0), (4, "pmj", 1.5), (4, "gauss", 0.8)])
def test_log_z_equals_brute_force_when_chi_is_exact(L, kind, beta):
    Jh, Jv = draw_bonds(L, 100 + L, kind)
    rows = bmps.build_envs(Jh, Jv, beta, chi=2 ** (L // 2))
    _, _, _, lz = exact.brute_force(Jh, Jv, beta)
    assert abs(bmps.log_z(rows) - lz) < 1e-12 * max(1.0, abs(lz))


@pytest.mark.parametrize("L,beta", [(6, 1.0), (8, 3.0)])
def test_log_z_equals_transfer_matrix(L, beta):
    Jh, Jv = draw_bonds(L, 7, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi=2 ** (L // 2))
    lz = exact.transfer_log_z(Jh, Jv, beta)
    assert abs(bmps.log_z(rows) - lz) < 1e-11 * abs(lz)


def test_transfer_matrix_equals_brute_force():
    Jh, Jv = draw_bonds(4, 9, "gauss")
    assert abs(exact.transfer_log_z(Jh, Jv, 1.3) - exact.brute_force(Jh, Jv, 1.3)[3]) < 1e-12


def _forest_log_z(Jh, Jv, beta):
    """Z = 2^N prod_e cosh(beta J_e) whenever the nonzero bonds form a forest."""
    L = Jh.shape[0]
    J = np.concatenate([Jh.ravel(), Jv.ravel()]).astype(np.float64)
    return L * L * np.log(2.0) + np.sum(np.log(np.cosh(beta * J)))


def test_log_z_forest_independent_rows():
    L = 12
    Jh, _ = draw_bonds(L, 21, "gauss")
    Jv = np.zeros((L - 1, L), np.float32)
    rows = bmps.build_envs(Jh, Jv, 2.0, chi=2)
    assert abs(bmps.log_z(rows) - _forest_log_z(Jh, Jv, 2.0)) < 1e-11 * L * L


def test_log_z_forest_comb_large():
    """Comb = all vertical bonds + the top row: a spanning tree; chi = 2 is exact at any L."""
    L = 40
    Jh, Jv = draw_bonds(L, 22, "pmj")
    Jh = Jh.copy(); Jh[1:, :] = 0
    rows = bmps.build_envs(Jh, Jv, 3.0, chi=2)
    assert abs(bmps.log_z(rows) - _forest_log_z(Jh, Jv, 3.0)) < 1e-10 * L * L


def test_log_z_gauge_invariant_under_truncation():
    """Flipping a spin and its four bonds acts unitarily on the MPS legs: truncated log Z is unchanged."""
    L, beta, chi = 8, 1.0, 4
    Jh, Jv = draw_bonds(L, 23, "pmj")
    base = bmps.log_z(bmps.build_envs(Jh, Jv, beta, chi))
    for (r, c) in [(0, 0), (3, 4), (7, 7), (5, 0)]:
        Jh2, Jv2 = Jh.copy(), Jv.copy()
        if c > 0: Jh2[r, c - 1] *= -1
        if c < L - 1: Jh2[r, c] *= -1
        if r > 0: Jv2[r - 1, c] *= -1
        if r < L - 1: Jv2[r, c] *= -1
        assert abs(bmps.log_z(bmps.build_envs(Jh2, Jv2, beta, chi)) - base) < 1e-11 * abs(base)


def test_log_z_converges_with_chi():
    L, beta = 10, 1.0
    Jh, Jv = draw_bonds(L, 24, "pmj")
    lz = exact.transfer_log_z(Jh, Jv, beta)
    errs = [abs(bmps.log_z(bmps.build_envs(Jh, Jv, beta, chi)) - lz) for chi in (2, 4, 8, 32)]
    assert errs[-1] < 1e-11 * abs(lz)
    assert errs[0] > errs[1] > errs[2]


def test_cache_rows_equal_exact_boundary_functions():
    L, beta = 6, 1.2
    Jh, Jv = draw_bonds(L, 25, "gauss")
    rows = bmps.build_envs(Jh, Jv, beta, chi=8)
    F = exact.boundary_functions(Jh, Jv, beta)
    ys = np.arange(2 ** L)
    bits = ((ys[:, None] >> np.arange(L)[None, :]) & 1)
    for r in range(L):
        got = np.array([bmps.contract_row(rows[r], b) for b in bits])
        top = F[r].max()
        # F_r itself to 1e-10 of its largest value (the 1e-12 singular-value cutoff
        # leaves configurations far below the largest one unresolved)
        np.testing.assert_allclose(np.exp(got - top), np.exp(F[r] - top), rtol=0, atol=1e-10)
        big = F[r] > top - 10.0
        np.testing.assert_allclose(got[big], F[r][big], rtol=0, atol=1e-9)


# ---------------------------------------------------------------- conditionals / q
@pytest.mark.parametrize("L", [3, 4])
def test_logits_equal_brute_force_conditionals(L):
    Jh, Jv = draw_bonds(L, 30 + L, "pmj")
    beta = 1.0
    rows = bmps.build_envs(Jh, Jv, beta, chi=2 ** (L // 2))
    sig, lq, E, lg = sampler.propose(rows, Jh, Jv, beta, 16, 42, 0, 0)
    ex = exact.brute_conditional_logits(Jh, Jv, beta, sig)
    np.testing.assert_allclose(lg, ex, atol=1e-10)
    _, _, logp, _ = exact.brute_force(Jh, Jv, beta)
    idx = [int("".join(map(str, s.reshape(-1))), 2) for s in sig]
    np.testing.assert_allclose(lq, logp[idx], atol=1e-10)


def test_logits_equal_transfer_conditionals_L6():
    L, beta = 6, 2.0
    Jh, Jv = draw_bonds(L, 36, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi=8)
    sig, lq, E, lg = sampler.propose(rows, Jh, Jv, beta, 6, 42, 100, 0)
    ex = exact.transfer_conditional_logits(Jh, Jv, beta, sig)
    np.testing.assert_allclose(lg, ex, atol=1e-9)


def test_score_equals_propose():
    L, beta = 6, 1.0
    Jh, Jv = draw_bonds(L, 37, "gauss")
    rows = bmps.build_envs(Jh, Jv, beta, chi=3)
    sig, lq, E, lg = sampler.propose(rows, Jh, Jv, beta, 8, 42, 0, 0)
    lq2, E2, lg2 = sampler.score(rows, Jh, Jv, beta, sig)
    np.testing.assert_array_equal(lq, lq2)
    np.testing.assert_array_equal(E, E2)


def test_forest_q_equals_p():
    """On a forest bMPS is exact at chi = 2, so log q = -beta E - log Z for every proposal."""
    L, beta = 10, 1.5
    Jh, Jv = draw_bonds(L, 38, "gauss")
    Jh = Jh.copy(); Jh[1:, :] = 0
    rows = bmps.build_envs(Jh, Jv, beta, chi=2)
    sig, lq, E, _ = sampler.propose(rows, Jh, Jv, beta, 32, 42, 0, 0)
    np.testing.assert_allclose(lq, -beta * E - _forest_log_z(Jh, Jv, beta), atol=1e-9)


def test_global_flip_symmetry_of_q():
    L, beta, chi = 6, 0.6, 4
    Jh, Jv = draw_bonds(L, 39, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi)
    gaps = [g for r in rows for g in r.cut_gap]
    assert min(gaps) > 1e-6          # no near-tie at a cut, so the truncation keeps the Z2 symmetry
    sig, lq, E, _ = sampler.propose(rows, Jh, Jv, beta, 16, 42, 0, 0)
    lq_f, E_f, _ = sampler.score(rows, Jh, Jv, beta, 1 - sig)
    np.testing.assert_allclose(lq_f, lq, atol=1e-10)
    np.testing.assert_array_equal(E_f, E)


def test_exact_proposals_follow_boltzmann_histogram():
    """With chi exact, ancestral draws are samples of P: chi-squared over the 512 states of L=3."""
    L, beta = 3, 0.7
    Jh, Jv = draw_bonds(L, 40, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi=2)
    S = 40000
    sig, lq, E, _ = sampler.propose(rows, Jh, Jv, beta, S, 42, 0, 0)
    _, _, logp, _ = exact.brute_force(Jh, Jv, beta)
    idx = sig.reshape(S, -1) @ (2 ** np.arange(8, -1, -1))
    cnt = np.bincount(idx, minlength=512)
    exp_cnt = S * np.exp(logp)
    keep = exp_cnt > 5
    chi2 = np.sum((cnt[keep] - exp_cnt[keep]) ** 2 / exp_cnt[keep])
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_importance_sampling_log_z_matches_bmps():
    """log E_q[exp(-beta E) / q] = log Z; with a truncated q the bMPS log Z is within the IS error."""
    L, beta = 6, 1.0
    Jh, Jv = draw_bonds(L, 41, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi=2)
    sig, lq, E, _ = sampler.propose(rows, Jh, Jv, beta, 4000, 42, 0, 0)
    lw = -beta * E - lq
    m = lw.max()
    w = np.exp(lw - m)
    is_lz = m + np.log(w.mean())
    err = w.std() / (w.mean() * np.sqrt(w.size))
    lz_exact = exact.transfer_log_z(Jh, Jv, beta)
    assert abs(is_lz - lz_exact) < 5 * err + 1e-12
    assert abs(bmps.log_z(rows) - lz_exact) < 0.5       # the truncated bMPS estimate is close


# ---------------------------------------------------------------- MH
def _mh_run(L, beta, chi, S, seed=42):
    Jh, Jv = draw_bonds(L, 50 + L, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi)
    s0 = philox.init_spins(L, 0, seed)
    lq0, E0, _ = sampler.score(rows, Jh, Jv, beta, s0[None])
    props = sampler.propose(rows, Jh, Jv, beta, S, seed, 0, 0)[:3]
    state, acc, _, _ = mh.chain((s0, lq0[0], E0[0]), props, beta, seed, 0, 0)
    return Jh, Jv, props, acc


def test_mh_exact_q_accepts_everything():
    _, _, _, acc = _mh_run(3, 1.0, 2, 500)
    assert acc.all()


def test_mh_chain_histogram_matches_boltzmann():
    """A poor chi = 1 proposal, corrected by Eq. 10, samples P: chi-squared over the 512 states."""
    L, beta, S = 3, 0.8, 60000
    Jh, Jv, (P_sig, P_lq, P_E), acc = _mh_run(L, beta, 1, S)
    assert 0.05 < acc.mean() < 0.99
    # rebuild the chain states from the accept bits
    s0 = philox.init_spins(L, 0, 42)
    idx_p = P_sig.reshape(S, -1) @ (2 ** np.arange(8, -1, -1))
    cur = int(s0.reshape(-1) @ (2 ** np.arange(8, -1, -1)))
    states = np.empty(S, np.int64)
    for k in range(S):
        if acc[k]:
            cur = idx_p[k]
        states[k] = cur
    cnt = np.bincount(states, minlength=512)
    _, _, logp, _ = exact.brute_force(Jh, Jv, beta)
    exp_cnt = S * np.exp(logp)
    keep = exp_cnt > 10
    # successive states are correlated; inflate the bound by the rejection run length
    tau = 1.0 / acc.mean()
    chi2 = np.sum((cnt[keep] - exp_cnt[keep]) ** 2 / exp_cnt[keep]) / tau
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_mh_accept_rule_matches_definition():
    L, beta = 4, 1.0
    Jh, Jv = draw_bonds(L, 60, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, 2)
    s0 = philox.init_spins(L, 2, 7)
    lq0, E0, _ = sampler.score(rows, Jh, Jv, beta, s0[None])
    P_sig, P_lq, P_E, _ = sampler.propose(rows, Jh, Jv, beta, 200, 7, 1000, 2)
    (_, lq_end, E_end), acc, log_r, u = mh.chain((s0, lq0[0], E0[0]), (P_sig, P_lq, P_E), beta, 7, 1000, 2)
    lq, E = lq0[0], E0[0]
    for k in range(200):
        ratio = np.exp(-beta * P_E[k] - P_lq[k]) / np.exp(-beta * E - lq)
        assert acc[k] == (u[k] < min(1.0, ratio)) or abs(u[k] - min(1.0, ratio)) < 1e-12
        if acc[k]:
            lq, E = P_lq[k], P_E[k]
    assert lq == lq_end and E == E_end


def test_truncation_threshold_is_needed_and_exact_against_transfer_matrix():
    """Reading of Sec. 1's truncation threshold, pinned to the exact row transfer matrix.

    L = 18, beta = 3: with the relative cutoff the bMPS log Z equals the exact
    one to 1e-7; keeping numerically-zero singular values (cutoff 0) lets noise
    grow and misses it by > 1e-4 although no physical weight was discarded.
    """
    L, beta = 18, 3.0
    Jh, Jv = draw_bonds(L, 1000, "pmj")
    lz = exact.transfer_log_z(Jh, Jv, beta)
    assert abs(bmps.log_z(bmps.build_envs(Jh, Jv, beta, 32, 1e-12)) - lz) < 1e-7
    assert abs(bmps.log_z(bmps.build_envs(Jh, Jv, beta, 32, 0.0)) - lz) > 1e-4
