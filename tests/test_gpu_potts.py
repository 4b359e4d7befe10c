"""GPU parity of the q-state Potts extension (Sec. 5) against the FP64 oracle (oracle/potts.py).

Same bar as the float64 Ising path: log Z to 1e-10 relative; free-running proposals equal
state by state, except where the site's uniform lies within 1e-9 of a partial sum of the
oracle's conditional (float64 rounding of the contractions may move the draw there; such
draws are counted); energies exact (+-J) and log q to 1e-9 on equal proposals; scores of
the oracle's proposals; the MH kernel takes the oracle chain's decisions on them. Sizes
span one site, uneven batches, exact and truncated bonds, q = 3 and 4, +-J and Gaussian.

The global permutation symmetry of the Potts model makes singular values come in exactly
degenerate multiplets; a rank cap (chi) inside one leaves the kept subspace to rounding,
on the GPU and in the oracle alike. The truncating cases are therefore chosen where the
cutoff decides and every cut gap of the oracle is wide (checked below).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mh, philox, potts  # noqa: E402
import parity  # noqa: E402

BAND = 1e-9
CASES = [  # Ls, q, chi, beta, kind, cutoff
    ([4, 3], 3, 9, 0.8, "pmj", 1e-12),
    ([7], 3, 9, 1.2, "gauss", 1e-12),
    ([10, 6, 8], 3, 16, 0.7, "pmj", 1e-6),
    ([16, 9], 3, 16, 1.0, "pmj", 1e-5),
    ([6, 5], 4, 9, 1.0, "pmj", 1e-3),
    ([6, 5], 4, 9, 1.0, "gauss", 1e-4),
    ([1, 2], 3, 4, 1.0, "pmj", 1e-12),
]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


def _run(P, Ls, q, chi, beta, kind, S, seed=42, cutoff=1e-12, prec="fp64"):
    reals = parity.realizations(Ls, kind)
    t = P.TNMC(Ls, chi, beta, prec, max_samples=S, q=q, cutoff=cutoff)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, seed, 0)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    assert st == 0, flags
    envs = [potts.build_envs(Jh, Jv, beta, q, chi, t.cutoff) for Jh, Jv in reals]
    return t, reals, envs, lz, props


def _compare(rows, Jh, Jv, beta, q, S, seed, n, g_st, g_lq, g_E, band=BAND, lq_rtol=1e-9):
    L = len(rows)
    o_st, o_lq, o_E, o_p = potts.propose(rows, Jh, Jv, beta, q, S, seed, 0, n)
    u = philox.spin_uniforms(L, np.arange(S, dtype=np.uint64), n, seed)
    n_eq, n_bd = 0, 0
    for k in range(S):
        a, b = g_st[k].reshape(-1), o_st[k].reshape(-1)
        if np.array_equal(a, b):
            n_eq += 1
            assert g_E[k] == o_E[k], (k, g_E[k], o_E[k])
            assert abs(g_lq[k] - o_lq[k]) <= lq_rtol * max(1.0, abs(o_lq[k])), (k, g_lq[k], o_lq[k])
        else:
            i = int(np.argmax(a != b))
            cum = np.cumsum(o_p[k, i])[:-1]
            assert np.min(np.abs(u[k, i] - cum)) < band, (k, i, u[k, i], cum)
            n_bd += 1
    return n_eq, n_bd, (o_st, o_lq, o_E)


@pytest.mark.parametrize("Ls,q,chi,beta,kind,cutoff", CASES)
def test_potts_log_z_and_proposals(P, Ls, q, chi, beta, kind, cutoff):
    S = 40
    t, reals, envs, lz, props = _run(P, Ls, q, chi, beta, kind, S, cutoff=cutoff)
    assert min((g for rows in envs for r in rows for g in r.cut_gap), default=np.inf) > 1e-2
    g_st = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    assert max(int(x.max()) for x in g_st) <= q - 1
    bd = 0
    for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs)):
        o = potts.log_z(rows)
        assert abs(lz[n] - o) < 1e-10 * max(1.0, abs(o)), (n, lz[n], o)
        _, nb, _ = _compare(rows, Jh, Jv, beta, q, S, 42, n, g_st[n], props.logq.cpu().numpy()[n],
                            props.E.cpu().numpy()[n])
        bd += nb
    assert bd <= 2


def test_potts_exact_log_z_and_scores_and_mh(P):
    Ls, q, chi, beta, S = [3, 3], 3, 9, 0.9, 64
    t, reals, envs, lz, props = _run(P, Ls, q, chi, beta, "pmj", S)
    o_props = [potts.propose(rows, Jh, Jv, beta, q, S, 42, 0, n)
               for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs))]
    for n, (Jh, Jv) in enumerate(reals):
        assert abs(lz[n] - potts.brute_force(Jh, Jv, beta, q)[3]) < 1e-10 * abs(lz[n])
    # scores of the oracle's proposals
    spins_in = torch.from_numpy(np.concatenate([o[0].reshape(-1) for o in o_props])).cuda()
    g_lq, g_E = t.score(spins_in, S)
    g_lq, g_E = g_lq.cpu().numpy(), g_E.cpu().numpy()
    for n in range(len(Ls)):
        np.testing.assert_array_equal(g_E[n], o_props[n][2])
        np.testing.assert_allclose(g_lq[n], o_props[n][1], rtol=1e-10, atol=1e-10)
    # the MH kernel on the oracle's proposals, from an empty chain (first proposal accepted)
    state = t.mh_init_empty()
    op = P.Proposals(spins_in, torch.from_numpy(np.stack([o[1] for o in o_props])).cuda(),
                     torch.from_numpy(np.stack([o[2] for o in o_props])).cuda(), S, 0)
    acc = t.mh_step(op, state, 3).cpu().numpy()
    for n in range(len(Ls)):
        L = Ls[n]
        start = (np.zeros((L, L), np.uint8), np.inf, 0.0)
        (o_st, o_lq, o_E), o_acc, o_lr, o_u = mh.chain(start, o_props[n][:3], beta, 3, 0, n)
        near = np.abs(np.log(o_u) - o_lr) < 1e-12
        assert o_acc[0] == 1 and acc[n][0] == 1
        assert np.array_equal(acc[n][~near], o_acc[~near])


def test_potts_argument_and_mode_errors(P):
    with pytest.raises(P.TnmcError) as e:
        P.TNMC([4], 4, 1.0, "dfloat", max_samples=4, q=3)     # float64 and float32 only
    assert e.value.status == 7
    with pytest.raises(P.TnmcError) as e:
        P.TNMC([4], 4, 1.0, "fp64", max_samples=4, q=5)       # beyond the kernels' panels
    assert e.value.status == 7
    with pytest.raises(P.TnmcError) as e:
        P.TNMC([4], 4, 1.0, "fp64", max_samples=4, q=1)
    assert e.value.status == 1
    t = P.TNMC([4], 4, 1.0, "fp64", max_samples=4, q=3)
    reals = parity.realizations([4], "pmj")
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    with pytest.raises(P.TnmcError) as e:
        t.mh_init(1)                                          # random starts draw Ising bits
    assert e.value.status == 7


def test_potts_row_records_match_the_oracle_bonds(P):
    Ls, q, chi, beta = [10, 6, 8], 3, 16, 0.7
    reals = parity.realizations(Ls, "pmj")
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=8, q=q, cutoff=1e-6)
    _, _, ri = t.set_diagnostics(rowinfo=True)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    torch.cuda.synchronize()
    rec = ri.cpu().numpy().reshape(-1, 14)
    off = 0
    for (Jh, Jv), L in zip(reals, Ls):
        rows = potts.build_envs(Jh, Jv, beta, q, chi, 1e-6)
        for r in range(L):
            mean_bond = np.mean([A.shape[0] for A in rows[r].tensors[1:]])
            assert rec[off + r, 5] == mean_bond, (L, r)
            assert rec[off + r, 13] > 0 and rec[off + r, 7] >= 1
        off += L


@pytest.mark.parametrize("Ls,q,chi,beta,kind,cutoff", [
    ([10, 6, 8], 3, 16, 0.7, "pmj", 1e-6),
    ([16, 9], 3, 16, 1.0, "pmj", 1e-5),
    ([6, 5], 4, 9, 1.0, "gauss", 1e-4),
])
def test_potts_float32_against_the_oracle(P, Ls, q, chi, beta, kind, cutoff):
    """The float32 build, cache and sampling contractions (TNMC_FP32 with q_states): |d log Z| /
    L^2 <= 1e-6, energies exact, free-running proposals equal the oracle's up to a draw within
    2e-3 of a partial sum of the oracle's conditional (float32 rounding of the contractions),
    log q of equal proposals to 1e-2 relative (the float32 mode's bounds for Ising)."""
    S = 40
    t, reals, envs, lz, props = _run(P, Ls, q, chi, beta, kind, S, cutoff=cutoff, prec="fp32")
    assert min((g for rows in envs for r in rows for g in r.cut_gap), default=np.inf) > 1e-2
    g_st = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    n_eq = 0
    for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs)):
        L = Ls[n]
        assert abs(lz[n] - potts.log_z(rows)) / (L * L) < 1e-6, (n, lz[n], potts.log_z(rows))
        ne, _, _ = _compare(rows, Jh, Jv, beta, q, S, 42, n, g_st[n], props.logq.cpu().numpy()[n],
                            props.E.cpu().numpy()[n], band=2e-3, lq_rtol=1e-2)
        n_eq += ne
    assert n_eq >= 0.9 * S * len(Ls)
