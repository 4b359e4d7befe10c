"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

float64 mode: log Z and bond spectra to ~1e-10, proposals (spins, energies)
bit-exact, log q to 1e-9, MH accepts bit-exact; a configuration may differ only
at a draw whose uniform lies within 1e-9 of the oracle's probability (counted).
float32 mode: log Z per site to 1e-6 and a teacher-forced audit of every draw.
A configuration whose draws land near a tie at a truncation cut is not compared
bit for bit (the kept subspace is then decided by rounding); the cases below
have wide cut gaps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bmps, mh, philox, sampler  # noqa: E402
from oracle.ising import energy  # noqa: E402
import parity  # noqa: E402


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


def _run(P, Ls, chi, beta, prec, kind, S, seed=42, prop_base=0, diag=False):
    reals = parity.realizations(Ls, kind)
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, prec, max_samples=max(S, 1))
    d = t.set_diagnostics(S=S, logits=True, spectra=True, rowinfo=True) if diag else None
    t.build_envs(J)
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, seed, prop_base)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    return t, reals, lz, props, d, st, flags


CASES_FP64 = [
    ([2], 2, 1.0, "pmj"),
    ([3], 2, 0.7, "pmj"),
    ([4], 4, 1.5, "gauss"),
    ([5], 3, 1.0, "pmj"),       # truncated, odd chi
    ([8], 4, 2.0, "pmj"),       # truncated
    ([6, 3, 7], 8, 1.0, "gauss"),   # uneven batch, exact chi
    ([16], 16, 1.0, "pmj"),     # the L=16, chi=16, beta=1 workload
    ([1, 2], 1, 0.5, "pmj"),    # degenerate: L=1 and chi=1
]


@pytest.mark.parametrize("Ls,chi,beta,kind", CASES_FP64)
def test_fp64_log_z_spectra_and_proposals(P, Ls, chi, beta, kind):
    S = 70  # two CTAs of chains, the second one ragged
    t, reals, lz, props, (lg, sp, ri), st, flags = _run(P, Ls, chi, beta, "fp64", kind, S, diag=True)
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi)
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    lq = props.logq.cpu().numpy()
    E = props.E.cpu().numpy()
    sp = sp.cpu().numpy()
    ri = ri.cpu().numpy().reshape(-1, 14)
    bo = ro = 0
    total_bd = 0
    for n, (L, (Jh, Jv), rows) in enumerate(zip(Ls, reals, envs)):
        o_lz = bmps.log_z(rows)
        assert abs(lz[n] - o_lz) < 1e-10 * max(1.0, abs(o_lz)), (n, lz[n], o_lz)
        # per-row log scale is a gauge-dependent quantity; compare the spectra instead
        for r in range(L):
            for c in range(1, L):
                o_s = rows[r].spectra[c - 1]
                g_s = sp[(bo + r * (L + 1) + c) * chi:(bo + r * (L + 1) + c + 1) * chi]
                gap = rows[r].cut_gap[c - 1]
                keep = o_s > 1e-7
                if gap > 1e-6:
                    np.testing.assert_allclose(g_s[:keep.sum()], o_s[keep], rtol=1e-8, atol=1e-12)
        n_eq, n_bd = parity.compare_proposals(rows, Jh, Jv, beta, 42, 0, n, spins[n], lq[n], E[n])
        total_bd += n_bd
        bo += L * (L + 1)
        ro += L
    assert total_bd <= 1


@pytest.mark.parametrize("prec", ["fp64", "dfloat"])
def test_single_chain_at_a_far_proposal_base(P, prec):
    # S = 1: one chain in a CTA laid out for 64, and a proposal id far from 0 (the Philox
    # counter of the draw, Sec. 3.3); the oracle draws the same proposal from its own stream
    Ls, chi, beta, base = [7, 5, 1], 8, 1.1, 123_456_789
    t, reals, lz, props, _, st, flags = _run(P, Ls, chi, beta, prec, "pmj", 1, prop_base=base)
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi)
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, 1)
    lq, E = props.logq.cpu().numpy(), props.E.cpu().numpy()
    band, atol = (parity.BAND_FP64, 1e-9) if prec == "fp64" else (1e-7, 1e-8)
    n_bd = 0
    for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs)):
        assert abs(lz[n] - bmps.log_z(rows)) < 1e-9 * max(1.0, abs(lz[n]))
        n_bd += parity.compare_proposals(rows, Jh, Jv, beta, 42, base, n, spins[n], lq[n], E[n],
                                         band=band, lq_atol=atol)[1]
    assert n_bd == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_score_matches_propose(P, prec):
    Ls, chi, beta = [9, 6], 4, 1.3
    S = 64
    t, reals, lz, props, _, st, _ = _run(P, Ls, chi, beta, prec, "gauss", S)
    lq2, E2 = t.score(props.spins, S)
    tol = 1e-12 if prec == "fp64" else 1e-5
    np.testing.assert_allclose(lq2.cpu().numpy(), props.logq.cpu().numpy(), rtol=0, atol=tol * 100)
    np.testing.assert_array_equal(E2.cpu().numpy(), props.E.cpu().numpy())


def test_fp64_energies_exact_and_oracle_scoring(P):
    """The GPU scores the oracle's proposals: exact energies, log q to 1e-9."""
    Ls, chi, beta, S = [12], 6, 2.0, 128
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    t.build_envs(J)
    (Jh, Jv), = reals
    rows = bmps.build_envs(Jh, Jv, beta, chi)
    o_sig, o_lq, o_E, _ = sampler.propose(rows, Jh, Jv, beta, S, 42, 12345, 0)
    np.testing.assert_array_equal(o_E, energy(Jh, Jv, o_sig))
    g_lq, g_E = t.score(torch.from_numpy(o_sig.reshape(-1)).cuda(), S)
    np.testing.assert_array_equal(g_E.cpu().numpy()[0], o_E)
    np.testing.assert_allclose(g_lq.cpu().numpy()[0], o_lq, rtol=0, atol=1e-9)


def _oracle_proposals_on_gpu(P, t, Ls, reals, envs, beta, S, seed, base):
    """The oracle's proposals of every realization, and the same arrays as GPU inputs."""
    out = [sampler.propose(rows, Jh, Jv, beta, S, seed, base, n)[:3]
           for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs))]
    spins = torch.from_numpy(np.concatenate([o[0].reshape(-1) for o in out])).cuda()
    logq = torch.from_numpy(np.stack([o[1] for o in out])).cuda()
    E = torch.from_numpy(np.stack([o[2] for o in out])).cuda()
    return out, P.Proposals(spins, logq, E, S, base)


def test_fp64_mh_chain_bit_exact(P):
    """The GPU chain on the oracle's proposals takes the oracle chain's decisions.

    The initial state is the GPU's (its spins and score checked against the
    oracle first); the proposals fed to both chains are the oracle's own.
    """
    Ls, chi, beta, S = [8, 5], 4, 1.0, 200
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    t.build_envs(J)
    state = t.mh_init(seed=7)
    envs = parity.oracle_envs(reals, beta, chi)
    o_state = []
    g0 = parity.split_spins(state.spins.cpu().numpy(), Ls, 1)
    g_lq, g_E = state.logq.cpu().numpy(), state.E.cpu().numpy()
    for n, (L, (Jh, Jv), rows) in enumerate(zip(Ls, reals, envs)):
        s0 = philox.init_spins(L, n, 7)
        np.testing.assert_array_equal(g0[n][0], s0)
        o_lq, o_E, _ = sampler.score(rows, Jh, Jv, beta, s0[None])
        assert g_E[n] == o_E[0]
        assert abs(g_lq[n] - o_lq[0]) < 1e-9
        o_state.append((s0, float(o_lq[0]), float(o_E[0])))
    # both chains continue from the oracle's state value (equal to the GPU's to 1e-9)
    state.logq.copy_(torch.tensor([o[1] for o in o_state], dtype=torch.float64))
    total_acc = 0
    for step in range(2):
        base = 1000 * step
        o_props, g_props = _oracle_proposals_on_gpu(P, t, Ls, reals, envs, beta, S, 7, base)
        acc = t.mh_step(g_props, state, seed=7).cpu().numpy()
        for n in range(len(Ls)):
            (o_sig, o_lq, o_E), o_acc, o_lr, o_u = mh.chain(o_state[n], o_props[n], beta, 7, base, n)
            near = np.abs(np.log(o_u) - o_lr) < 1e-12
            assert np.array_equal(acc[n][~near], o_acc[~near])
            total_acc += int(acc[n].sum())
            o_state[n] = (o_sig, o_lq, o_E)
        torch.cuda.synchronize()
        g_sig = parity.split_spins(state.spins.cpu().numpy(), Ls, 1)
        for n in range(len(Ls)):
            np.testing.assert_array_equal(g_sig[n][0], o_state[n][0])
            assert state.E.cpu().numpy()[n] == o_state[n][2]
            assert state.logq.cpu().numpy()[n] == o_state[n][1]
    assert state.n_accept.cpu().numpy().sum() == total_acc
    assert total_acc > 0


def test_mh_from_empty_state_starts_at_first_proposal(P):
    Ls, chi, beta, S = [7, 4], 4, 1.2, 50
    reals = parity.realizations(Ls, "gauss")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    t.build_envs(J)
    envs = parity.oracle_envs(reals, beta, chi)
    state = t.mh_init_empty()
    o_props, g_props = _oracle_proposals_on_gpu(P, t, Ls, reals, envs, beta, S, 3, 0)
    acc = t.mh_step(g_props, state, seed=3).cpu().numpy()
    assert acc[:, 0].all()
    for n, L in enumerate(Ls):
        start = (np.zeros((L, L), np.uint8), np.inf, 0.0)
        (o_sig, o_lq, o_E), o_acc, o_lr, o_u = mh.chain(start, o_props[n], beta, 3, 0, n)
        assert o_acc[0] == 1
        near = np.abs(np.log(o_u) - o_lr) < 1e-12
        assert np.array_equal(acc[n][~near], o_acc[~near])
        assert state.logq.cpu().numpy()[n] == o_lq


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("Ls,chi,beta,kind", [([10, 7], 8, 2.0, "pmj"), ([8, 6], 16, 2.0, "pmj"),
                                             ([12], 8, 1.0, "gauss"), ([10], 32, 2.0, "pmj")])
def test_fp32_log_z_and_draw_audit(P, Ls, chi, beta, kind, prec):
    """float32 mode against the float64 oracle.

    |d log Z| / L^2 <= 1e-6 (cases whose cut gaps are wide); energies exact;
    teacher-forced audit on the oracle's proposals: at every site the GPU's
    float32 conditional takes the oracle's decision under the same uniform
    unless the uniform lies within 2e-3 of the oracle's probability; the free
    running GPU proposals equal the oracle's up to such a draw.
    log q: float32 rounding of the cache alone already moves log q by ~1e-3
    at beta = 2 (test_fp32_storage_bound in test_precision_model.py), so the
    bound here is 1e-2, not the float64 1e-9.
    """
    S = 64
    t, reals, lz, props, _, st, flags = _run(P, Ls, chi, beta, prec, kind, S)
    assert st == 0
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)   # the same truncation rule
    o_props = [sampler.propose(rows, Jh, Jv, beta, S, 42, 0, n)
               for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs))]
    spins_in = torch.from_numpy(np.concatenate([o[0].reshape(-1) for o in o_props])).cuda()
    g_lq, g_E, g_lg = t.score_logits(spins_in, S)
    g_lq, g_E, g_lg = g_lq.cpu().numpy(), g_E.cpu().numpy(), g_lg.cpu().numpy()
    g_sig = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    off = 0
    for n, (L, (Jh, Jv), rows) in enumerate(zip(Ls, reals, envs)):
        o_sig, o_lq, o_E, o_lg = o_props[n]
        assert min(g for r in rows for g in r.cut_gap) > 1e-2
        assert abs(lz[n] - bmps.log_z(rows)) / (L * L) < 1e-6
        np.testing.assert_array_equal(g_E[n], o_E)
        assert np.abs(g_lq[n] - o_lq).max() < 1e-2
        u = philox.spin_uniforms(L, np.arange(S, dtype=np.uint64), n, 42)
        p = sampler.sigmoid(o_lg)
        lg = g_lg[off:off + S * L * L].reshape(S, L * L)
        off += S * L * L
        gpu_decision = (u < sampler.sigmoid(lg)).astype(np.uint8)
        band = np.abs(u - p) < 2e-3
        assert np.array_equal(gpu_decision[~band], o_sig.reshape(S, -1)[~band])
        # free running: equal until a draw inside the band
        for k in range(S):
            a, b = g_sig[n][k].reshape(-1), o_sig[k].reshape(-1)
            if not np.array_equal(a, b):
                i = int(np.argmax(a != b))
                assert band[k, i], (n, k, i)


def test_bad_couplings_flagged(P):
    Ls = [4, 5]
    reals = parity.realizations(Ls, "pmj")
    Jnp = parity.packed_J(reals)
    Jnp[16 + 3, 2] = 7.0           # realization 1, site (0, 3): right != left of (0, 4)
    t = P.TNMC(Ls, 4, 1.0, "fp32", max_samples=8)
    t.build_envs(torch.from_numpy(Jnp).cuda())
    st, flags = t.device_status()
    assert flags[0] == 0 and flags[1] & P.FLAG_BAD_COUPLINGS
    assert st == 1   # TNMC_ERR_ARG


def test_argument_errors(P):
    with pytest.raises(P.TnmcError):
        P.TNMC([8], 65, 1.0, "fp32", max_samples=4)           # chi > 64
    t = P.TNMC([8], 4, 1.0, "fp32", max_samples=4)
    with pytest.raises(P.TnmcError) as e:
        t.propose(2, 1)                                       # before build
    assert e.value.status == 6
    reals = parity.realizations([8], "pmj")
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    with pytest.raises(P.TnmcError):
        t.propose(5, 1)                                       # S > max_samples


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_beta3_float64_truncation_matches_oracle(P, prec):
    """beta = 3: the float64 build (plain and mixed) follows the oracle row by row.

    Per-row log ||F_r|| and log Z agree to 1e-9 relative; the proposals come
    from an essentially exact q at this size (IS weights constant to 1e-6).

    The bond spectra of this instance are ill-conditioned: relative noise of
    1e-16 in the oracle's own SVD inputs already moves the normalised spectra
    by up to 5e-9 (4e-5 relative on the smallest kept values), and noise of
    1e-14, the orthogonality the Jacobi sweeps stop at (8 sqrt(n) eps), by up
    to 6e-8 on the rows checked here. The bound is therefore absolute, 2e-7 on
    spectra normalised to s_0 = 1, and every value the oracle keeps well above
    the cutoff must be kept.
    """
    Ls, chi, beta, S = [24], 32, 3.0, 64
    t, reals, lz, props, (lg, sp, ri), st, flags = _run(P, Ls, chi, beta, prec, "pmj", S, diag=True)
    assert st == 0
    (Jh, Jv), = reals
    rows = bmps.build_envs(Jh, Jv, beta, chi, t.cutoff)
    ri = ri.cpu().numpy().reshape(-1, 14)
    L = Ls[0]
    for r in range(L):
        # oracle lambda_r is log ||F_r|| (its MPS has unit norm)
        assert abs(ri[r, 0] - rows[r].log_scale) < 1e-9 * abs(rows[r].log_scale), r
    assert abs(lz[0] - bmps.log_z(rows)) < 1e-9 * abs(lz[0])
    sp = sp.cpu().numpy().reshape(L, L + 1, chi)
    for r in range(0, L, 5):
        for c in range(1, L):
            o_s = rows[r].spectra[c - 1]
            np.testing.assert_allclose(sp[r, c, :o_s.size], o_s, rtol=0, atol=2e-7)
            if o_s[-1] > 10 * t.cutoff:
                assert np.count_nonzero(sp[r, c]) >= o_s.size, (r, c)
    if prec == "fp64":
        # float32 sampling contractions lose the conditionals at beta = 3 (cancellation in
        # rho_s = |l M R|, see test_precision_model.py); float64 keeps them
        w = -(props.logq.cpu().numpy()[0] + beta * props.E.cpu().numpy()[0])
        assert w.std() < 1e-6


def test_fp64_single_cta_build_with_many_realizations(P):
    """More realizations than CTA pairs fit on the GPU: the float64 build runs one CTA per
    realization (both parity sectors on one SM). log Z of every realization and the
    proposals of a few match the oracle as in the paired build."""
    rng = np.random.default_rng(3)
    Ls = [int(x) for x in rng.integers(2, 7, size=160)]
    chi, beta, S = 4, 1.2, 24
    reals = parity.realizations(Ls, "gauss")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    t.build_envs(J)
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, 42, 0)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi)
    for n in range(len(Ls)):
        assert abs(lz[n] - bmps.log_z(envs[n])) < 1e-10 * max(1.0, abs(lz[n])), n
    sig = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    lq, E = props.logq.cpu().numpy(), props.E.cpu().numpy()
    for n in (0, 1, 77, 159):
        Jh, Jv = reals[n]
        n_eq, n_bd = parity.compare_proposals(envs[n], Jh, Jv, beta, 42, 0, n, sig[n], lq[n], E[n])
        assert n_eq + n_bd == S and n_bd <= 1


def test_observables_match_oracle(P):
    """tnmc_observables on the oracle's proposals (odd S, odd and even L) = the oracle's values."""
    from oracle import observables as ob
    Ls, chi, beta, S = [7, 6, 5], 4, 1.1, 51
    reals = parity.realizations(Ls, "pmj", p=0.3)
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    t.build_envs(J)
    envs = parity.oracle_envs(reals, beta, chi)
    o_props, g_props = _oracle_proposals_on_gpu(P, t, Ls, reals, envs, beta, S, 42, 0)
    got = t.observables(g_props).cpu().numpy()
    for n in range(len(Ls)):
        want = ob.observables(o_props[n][0], o_props[n][1], o_props[n][2], beta)
        np.testing.assert_allclose(got[n], want, rtol=1e-12, atol=1e-13)


def test_nishimori_line_energy_from_gpu_samples(P):
    """Exact at any size: on the Nishimori line the disorder average of the thermal energy is
    -N_B (1 - 2p). The GPU's importance-sampling energies of 64 realizations at L = 12 agree
    within four standard errors of the disorder average."""
    from oracle import observables as ob
    p, L, n_real, chi, S = 0.1, 12, 64, 8, 256
    beta = ob.nishimori_beta(p)
    Ls = [L] * n_real
    reals = parity.realizations(Ls, "pmj", base_seed=7000, p=p)
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    t.build_envs(J)
    obs = t.observables(t.propose(S, 42, 0)).cpu().numpy()
    e = obs[:, 2] * L * L                      # <E> per realization
    nb = 2 * L * (L - 1)
    assert obs[:, 1].min() > 0.5 * S           # the weights are nearly flat (a good q)
    assert abs(e.mean() + nb * (1 - 2 * p)) < 4 * e.std() / np.sqrt(n_real), (e.mean(), -nb * (1 - 2 * p))
