"""Pins of the learned proposal correction in the oracle (CPU only).

Each pin checks the oracle against something other than itself: a brute-force
search over all bfloat16 values, central finite differences, closed forms of
the activation, of the loss's stationary point and of Adam's first step, the
normalisation of q over all 512 states of L = 3, the Boltzmann histogram of an
MH chain driven by a corrected proposal, and a hand-worked feature example.
"""
import numpy as np
import pytest

from oracle import bmps, exact, learned, mh, philox, sampler
from workloads import draw_bonds


# ---------------------------------------------------------------- bfloat16
def _all_bf16_values():
    bits = np.arange(1 << 16, dtype=np.uint32) << np.uint32(16)
    f = bits.view(np.float32)
    ok = np.isfinite(f)
    return f[ok].astype(np.float64), bits[ok]


def test_bf16_rounding_is_nearest_by_brute_force():
    vals, bits = _all_bf16_values()
    order = np.argsort(vals, kind="stable")
    vals, bits = vals[order], bits[order]
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-6, 6, 3000),
                        # exact midpoints between neighbours (ties)
                        0.5 * (vals[1000:1400] + vals[1001:1401])])
    x = x.astype(np.float32).astype(np.float64)
    got = learned.to_bf16(x)
    for xi, gi in zip(x, got):
        d = np.abs(vals - xi)
        near = np.flatnonzero(d == d.min())
        if near.size == 1:
            assert gi == vals[near[0]], (xi, gi)
        else:   # tie: the candidate whose last kept mantissa bit is 0
            even = [k for k in near if ((bits[k] >> 16) & 1) == 0 and vals[k] != 0.0 or vals[k] == 0.0]
            assert gi in vals[even], (xi, gi, vals[near])


def test_bf16_known_values():
    assert learned.to_bf16(1.0) == 1.0
    assert learned.to_bf16(1.0 + 2.0 ** -8) == 1.0               # tie, rounds to even
    assert learned.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, rounds to even (up)
    assert learned.to_bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    assert learned.to_bf16(-3.0) == -3.0


# ---------------------------------------------------------------- activation
def test_smooth_relu_closed_form():
    z = np.array([-5.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    np.testing.assert_array_equal(learned.act(z), [0.0, 0.0, 0.0625, 0.25, 0.5625, 1.0, 3.0])
    np.testing.assert_array_equal(learned.act_grad(z), [0.0, 0.0, 0.25, 0.5, 0.75, 1.0, 1.0])
    # value and slope continuous at the joins
    for k in (-1.0, 1.0):
        for h in (1e-7, -1e-7):
            assert abs(learned.act(k + h) - learned.act(k)) < 2e-7
            assert abs(learned.act_grad(k + h) - learned.act_grad(k)) < 1e-6


# ---------------------------------------------------------------- gradient
def _random_problem(seed, n=40):
    rng = np.random.default_rng(seed)
    theta = learned.init_params(seed).astype(np.float64)
    W1, b1, W2, b2, w3, b3 = learned.unpack(theta)
    theta = learned.pack(W1, rng.standard_normal(64) * 0.5, W2, rng.standard_normal(64) * 0.5,
                         rng.standard_normal(64) * 0.3, 0.2)
    X = rng.standard_normal((n, 7)) * np.array([3.0, 2.0, 2.0, 1.0, 1.0, 1.0, 0.5])
    p = rng.random(n)
    return theta, X, p


def test_gradient_matches_central_finite_differences():
    theta, X, p = _random_problem(1)
    _, g = learned.grad(theta, X, p, rounding=False)
    rng = np.random.default_rng(2)
    blocks = [(learned.OFF_W1, 64 * 16), (learned.OFF_B1, 64), (learned.OFF_W2, 4096),
              (learned.OFF_B2, 64), (learned.OFF_W3, 64), (learned.OFF_B3, 1)]
    h = 1e-6
    for off, size in blocks:
        idx = off + rng.choice(size, size=min(size, 12), replace=False)
        if off == learned.OFF_W1:   # only the 7 used input columns carry a gradient
            idx = np.array([off + 16 * k + j for k, j in zip(rng.integers(0, 64, 12), rng.integers(0, 7, 12))])
        for k in idx:
            tp, tm = theta.copy(), theta.copy()
            tp[k] += h
            tm[k] -= h
            fd = (learned.loss(tp, X, p, False) - learned.loss(tm, X, p, False)) / (2 * h)
            assert abs(fd - g[k]) < 1e-7 + 1e-5 * abs(fd), (off, k, fd, g[k])
    # padded input columns of W1 and the tail are inert
    W1g = g[learned.OFF_W1:learned.OFF_B1].reshape(64, 16)
    assert not W1g[:, 7:].any() and not g[learned.OFF_B3 + 1:].any()


def test_loss_stationary_where_corrected_logit_hits_target():
    """With w3 = 0 the output is b3; the loss gradient in b3 vanishes at b3 = logit(p) - x0."""
    theta, X, p = _random_problem(3, n=1)
    W1, b1, W2, b2, w3, b3 = learned.unpack(theta)
    b3 = np.log(p[0] / (1 - p[0])) - X[0, 0]
    t = learned.pack(W1, b1, W2, b2, np.zeros(64), b3)
    _, g = learned.grad(t, X, p, rounding=False)
    assert abs(g[learned.OFF_B3]) < 1e-12
    # and the loss there is the entropy of p
    H = -(p[0] * np.log(p[0]) + (1 - p[0]) * np.log(1 - p[0]))
    assert abs(learned.loss(t, X, p, False) - H) < 1e-12


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = learned.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(th, [-0.01, 0.01, -0.01, 0.0], rtol=1e-8)


def test_adam_two_steps_hand_computed():
    """Two Adam steps worked by hand with b1 = 1/2, b2 = 3/4, lr = 1/10, eps = 0.

    Coordinate A, gradients 1 then 3: m = 1/2, v = 1/4 after step 1 (update -lr);
    after step 2 m = 1/4 + 3/2 = 7/4, v = 3/16 + 9/4 = 39/16, bias-corrected
    m^ = (7/4)/(3/4) = 7/3 and v^ = (39/16)/(7/16) = 39/7.
    Coordinate B, gradients -2 then 1/2: m = -1, v = 1 after step 1 (update +lr);
    then m = -1/2 + 1/4 = -1/4, v = 3/4 + 1/16 = 13/16, m^ = -1/3, v^ = 13/7.
    Step 1 alone cannot tell b1 from b2 (the bias correction cancels both); step 2
    can: with the two swapped the same formulas give other numbers.
    """
    lr, b1, b2 = 0.1, 0.5, 0.75
    g1, g2 = np.array([1.0, -2.0]), np.array([3.0, 0.5])
    th, m, v = learned.adam(np.zeros(2), g1, np.zeros(2), np.zeros(2), 1, lr, b1, b2, eps=0.0)
    np.testing.assert_allclose(th, [-0.1, 0.1], rtol=1e-15)
    th, m, v = learned.adam(th, g2, m, v, 2, lr, b1, b2, eps=0.0)
    want = [-0.1 - 0.1 * (7 / 3) / np.sqrt(39 / 7), 0.1 + 0.1 * (1 / 3) / np.sqrt(13 / 7)]
    np.testing.assert_allclose(th, want, rtol=1e-14)
    np.testing.assert_allclose(m, [7 / 4, -1 / 4], rtol=1e-15)
    np.testing.assert_allclose(v, [39 / 16, 13 / 16], rtol=1e-15)
    th_s, m_s, v_s = learned.adam(np.zeros(2), g1, np.zeros(2), np.zeros(2), 1, lr, b2, b1, eps=0.0)
    th_s, _, _ = learned.adam(th_s, g2, m_s, v_s, 2, lr, b2, b1, eps=0.0)
    assert np.abs(th_s - np.array(want)).max() > 1e-3


def test_training_reaches_teacher_entropy_floor():
    """Targets drawn from a teacher network of the same form: Adam drives the loss to its floor."""
    rng = np.random.default_rng(4)
    teacher, X, _ = _random_problem(5, n=600)
    d, _ = learned.forward(teacher, X, rounding=False)
    z = X[:, 0] + d
    p = 1.0 / (1.0 + np.exp(-z))
    floor = float(np.mean(-(p * np.log(p) + (1 - p) * np.log(1 - p))))
    theta = learned.init_params(6).astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    first = learned.loss(theta, X, p, False)
    for step in range(1, 401):
        idx = rng.integers(0, X.shape[0], 128)
        _, g = learned.grad(theta, X[idx], p[idx], rounding=False)
        theta, m, v = learned.adam(theta, g, m, v, step, lr=3e-3)
    last = learned.loss(theta, X, p, False)
    assert last - floor < 0.2 * (first - floor), (first, last, floor)


# ---------------------------------------------------------------- features
def test_features_hand_example():
    L, beta = 3, 0.5
    Jh = np.array([[1, -1], [-1, 1], [1, 1]], np.float32)
    Jv = np.array([[1, 1, -1], [-1, 1, 1]], np.float32)
    sigma = np.array([[[1, 0, 1], [0, 1, 1], [1, 1, 0]]], np.uint8)   # s = +1 where 1
    logits = np.arange(9, dtype=np.float64)[None] * 0.1
    X = learned.features(Jh, Jv, beta, sigma, logits)[0].reshape(3, 3, 7)
    # site (1, 1): above s(0,1) = -1 with Jv[0,1] = 1; left s(1,0) = -1 with Jh[1,0] = -1;
    # right coupling Jh[1,1] = 1; below Jv[1,1] = 1; above-right s(0,2) = +1
    np.testing.assert_allclose(X[1, 1], [0.4, 2 * 0.5 * 1 * -1, 0.5 * -1 * -1, 1, 1, 1, 0.5])
    # site (0, 0): no neighbour above or left; right Jh[0,0] = 1; below Jv[0,0] = 1
    np.testing.assert_allclose(X[0, 0], [0.0, 0, 0, 1, 1, 0, 0.5])
    # site (2, 2): above s(1,2) = +1 with Jv[1,2] = 1; left s(2,1) = +1 with Jh[2,1] = 1; no right/below
    np.testing.assert_allclose(X[2, 2], [0.8, 1.0, 0.5, 0, 0, 0, 0.5])
    # an infinite logit (a vanished conditional) enters the network clamped to +-32
    lg_inf = logits.copy()
    lg_inf[0, 4] = np.inf
    lg_inf[0, 5] = -np.inf
    Xi = learned.features(Jh, Jv, beta, sigma, lg_inf)[0]
    assert Xi[4, 0] == 32.0 and Xi[5, 0] == -32.0
    # the oracle sampler's per-site features equal the batch features
    corr = learned.Correction(np.zeros(learned.N_PARAM), Jh, Jv, beta)
    for r in range(3):
        for c in range(3):
            x = corr.site_features(sigma, r, c, logits[:, r * 3 + c])
            np.testing.assert_allclose(x[0], X[r, c])


# ---------------------------------------------------------------- corrected sampler
def _strong_correction(seed):
    theta, _, _ = _random_problem(seed)
    W1, b1, W2, b2, w3, b3 = learned.unpack(theta)
    return learned.to_bf16(learned.pack(W1, b1, W2, b2, 2.0 * w3, 0.3))


def _all_configs(L):
    k = np.arange(2 ** (L * L))
    return ((k[:, None] >> np.arange(L * L - 1, -1, -1)) & 1).astype(np.uint8).reshape(-1, L, L)


def test_zero_network_is_plain_sampler():
    L, beta = 4, 1.0
    Jh, Jv = draw_bonds(L, 70, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, 2)
    corr = learned.Correction(np.zeros(learned.N_PARAM), Jh, Jv, beta)
    a = sampler.propose(rows, Jh, Jv, beta, 50, 3, 0, 0)
    b = sampler.propose(rows, Jh, Jv, beta, 50, 3, 0, 0, correction=corr)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_corrected_q_is_normalised_over_all_states():
    """sum_s q(s) = 1 over the 512 states of L = 3: the correction only reads spins already drawn."""
    L, beta = 3, 0.9
    Jh, Jv = draw_bonds(L, 71, "gauss")
    rows = bmps.build_envs(Jh, Jv, beta, 1)         # a poor chi, so q differs from P
    corr = learned.Correction(_strong_correction(7), Jh, Jv, beta)
    cfg = _all_configs(L)
    lq, _, lg = sampler.score(rows, Jh, Jv, beta, cfg, correction=corr)
    lq0, _, lg0 = sampler.score(rows, Jh, Jv, beta, cfg)
    assert abs(np.exp(lq).sum() - 1.0) < 1e-12
    assert np.abs(lg - lg0).max() > 0.1            # the correction does change q


def test_corrected_propose_equals_score_and_follows_q():
    L, beta, S = 3, 0.9, 30000
    Jh, Jv = draw_bonds(L, 72, "gauss")
    rows = bmps.build_envs(Jh, Jv, beta, 1)
    corr = learned.Correction(_strong_correction(8), Jh, Jv, beta)
    sig, lq, E, lg = sampler.propose(rows, Jh, Jv, beta, S, 42, 0, 0, correction=corr)
    lq2, E2, lg2 = sampler.score(rows, Jh, Jv, beta, sig[:500], correction=corr)
    np.testing.assert_allclose(lq[:500], lq2, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(E[:500], E2)
    # histogram of the draws against q over the 512 states
    cfg = _all_configs(L)
    q = np.exp(sampler.score(rows, Jh, Jv, beta, cfg, correction=corr)[0])
    idx = sig.reshape(S, -1) @ (2 ** np.arange(8, -1, -1))
    cnt = np.bincount(idx, minlength=512)
    exp_cnt = S * q
    keep = exp_cnt > 5
    chi2 = np.sum((cnt[keep] - exp_cnt[keep]) ** 2 / exp_cnt[keep])
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_mh_with_corrected_proposal_samples_boltzmann():
    """Eq. 10 with a corrected proposal samples P: final states of independent chains, chi-squared.

    For an independence sampler the distance to P after T steps is at most
    (1 - 1/M)^T with M = max_s P(s)/q(s), so with M <= 5 and T = 40 every chain
    has mixed; 3000 chains give 3000 independent draws of P.
    """
    L, beta, seed = 3, 0.8, 42
    n_chain, T = 3000, 40
    Jh, Jv = draw_bonds(L, 73, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, 2)          # exact environments; the correction alone bends q
    theta = _strong_correction(9)
    W1, b1, W2, b2, w3, b3 = learned.unpack(theta)
    corr = learned.Correction(learned.to_bf16(learned.pack(W1, b1, W2, b2, 0.15 * w3, 0.2)), Jh, Jv, beta)
    cfg = _all_configs(L)
    lq_all = sampler.score(rows, Jh, Jv, beta, cfg, correction=corr)[0]
    _, _, logp, _ = exact.brute_force(Jh, Jv, beta)
    M = np.exp(np.max(logp - lq_all))
    assert 1.2 < M <= 5.0, M
    P_sig, P_lq, P_E, _ = sampler.propose(rows, Jh, Jv, beta, n_chain * T, seed, 0, 0, correction=corr)
    finals = np.empty(n_chain, np.int64)
    w = 2 ** np.arange(8, -1, -1)
    n_acc = 0
    for k in range(n_chain):
        s0 = philox.init_spins(L, k, seed)
        lq0, E0, _ = sampler.score(rows, Jh, Jv, beta, s0[None], correction=corr)
        sl = slice(k * T, (k + 1) * T)
        (sig, _, _), acc, _, _ = mh.chain((s0, lq0[0], E0[0]), (P_sig[sl], P_lq[sl], P_E[sl]),
                                           beta, seed, k * T, 0)
        finals[k] = int(sig.reshape(-1) @ w)
        n_acc += int(acc.sum())
    assert 0.2 < n_acc / (n_chain * T) < 0.99
    cnt = np.bincount(finals, minlength=512)
    exp_cnt = n_chain * np.exp(logp)
    keep = exp_cnt > 5
    # pool the rare states into one bin
    obs = np.append(cnt[keep], cnt[~keep].sum())
    exp_ = np.append(exp_cnt[keep], exp_cnt[~keep].sum())
    chi2 = np.sum((obs - exp_) ** 2 / exp_)
    dof = obs.size - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)


# ---------------------------------------------------------------- importance-sampling observables
def test_observables_exact_proposal_gives_exact_log_z_and_unit_weights():
    """On a forest q = P exactly, so every weight equals Z: the IS log Z is the closed form."""
    from oracle import observables as ob
    L, beta = 5, 0.9
    Jh, Jv = draw_bonds(L, 80, "pmj")
    Jv = np.zeros_like(Jv)                      # independent rows: a forest
    rows = bmps.build_envs(Jh, Jv, beta, 2)
    sig, lq, E, _ = sampler.propose(rows, Jh, Jv, beta, 64, 42, 0, 0)
    v = ob.observables(sig, lq, E, beta)
    lz_exact = L * L * np.log(2.0) + np.sum(np.log(np.cosh(beta * Jh.astype(np.float64))))
    assert abs(v[0] - lz_exact) < 1e-10 and abs(v[1] - 64) < 1e-9


def test_observables_match_brute_force_averages():
    """With chi exact (L=3), the IS averages of E/N and q^2 converge to the enumerated ones."""
    from oracle import observables as ob
    L, beta, S = 3, 0.7, 20000
    Jh, Jv = draw_bonds(L, 81, "gauss")
    rows = bmps.build_envs(Jh, Jv, beta, 1)     # a poor chi: the weights do the correcting
    sig, lq, E, _ = sampler.propose(rows, Jh, Jv, beta, S, 42, 0, 0)
    v = ob.observables(sig, lq, E, beta)
    cfgs, E_all, logp, lz = exact.brute_force(Jh, Jv, beta)
    p = np.exp(logp)
    cfg = np.asarray(cfgs).reshape(len(p), -1).astype(np.float64) * 2 - 1
    qab = cfg @ cfg.T / 9.0
    q2_exact = p @ (qab ** 2) @ p
    assert abs(v[2] - p @ E_all / 9.0) < 0.02
    assert abs(v[3] - q2_exact) < 0.02
    # the IS log Z within five of its standard errors: var(w)/mean(w)^2 = S/ESS - 1
    err = np.sqrt((S / v[1] - 1.0) / S)
    assert abs(v[0] - lz) < 5 * err, (v[0], lz, err)


def test_binder_ratio_of_a_fully_ordered_sample_is_one():
    from oracle import observables as ob
    sig = np.ones((8, 4, 4), np.uint8)
    v = ob.observables(sig, np.zeros(8), np.zeros(8), 1.0)
    assert v[3] == 1.0 and v[4] == 1.0 and v[5] == 1.0
    assert abs(ob.nishimori_beta(0.1) - 0.5 * np.log(9.0)) < 1e-15


def test_nishimori_line_energy_identity_by_enumeration():
    """On the Nishimori line exp(-2 beta) = p / (1 - p) of the +-J model, the disorder average of
    the thermal energy is exactly -N_B (1 - 2p) (N_B bonds): enumerate all 2^12 bond
    configurations of a 3 x 3 lattice, weight each by p^(#antiferro) (1-p)^(#ferro), and
    average the brute-force <E>."""
    from oracle import observables as ob
    L, p = 3, 0.2
    beta = ob.nishimori_beta(p)
    nb = 2 * L * (L - 1)
    avg = 0.0
    for k in range(1 << nb):
        bits = (k >> np.arange(nb)) & 1          # 1 = antiferromagnetic
        J = np.where(bits == 1, -1.0, 1.0).astype(np.float32)
        Jh, Jv = J[:L * (L - 1)].reshape(L, L - 1), J[L * (L - 1):].reshape(L - 1, L)
        _, E, logp, _ = exact.brute_force(Jh, Jv, beta)
        avg += p ** bits.sum() * (1 - p) ** (nb - bits.sum()) * float(np.exp(logp) @ E)
    assert abs(avg - (-nb * (1 - 2 * p))) < 1e-10, avg
