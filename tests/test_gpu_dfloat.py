"""GPU parity of the double-float mode (TNMC_DFLOAT) against the FP64 oracle.

Double-float values carry 48 significant bits: unit roundoff 2^-48, 32 times
float64's 2^-53. Where a float64 bound is set by rounding it is scaled by that
factor (rounded up to a power of ten):
  * log Z: 1e-9 relative (float64: 1e-10);
  * bond spectra: 1e-7 relative plus 3.2e-11 absolute where the cut gap exceeds 1e-5
    (float64: 1e-8 and 1e-12 where it exceeds 1e-6);
  * free-running proposals equal to the oracle's up to draws whose uniform lies within
    1e-7 of the oracle's probability (float64: 1e-9), with log q of equal
    configurations to 1e-8 (float64: 1e-9) and energies exact;
  * beta = 3 (the benchmark regime, ill-conditioned spectra): per-row log ||F_r|| and
    log Z to 3.2e-8 relative (float64: 1e-9), spectra normalised to the largest value
    99 % within 2e-6 and all within 3.2e-4, log q to 3.2e-5 relative (float64: 98 %
    within 2e-7, all within 1e-5, log q 1e-6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bmps  # noqa: E402
import parity  # noqa: E402


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


def _run(P, Ls, chi, beta, kind, S, diag=True):
    reals = parity.realizations(Ls, kind)
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "dfloat", max_samples=S)
    d = t.set_diagnostics(S=S, spectra=True, rowinfo=True) if diag else None
    t.build_envs(J)
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, 42, 0)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    return t, reals, lz, props, d, st, flags


CASES = [
    ([2], 2, 1.0, "pmj"),
    ([5], 3, 1.0, "pmj"),           # truncated, odd chi
    ([8], 4, 2.0, "pmj"),           # truncated
    ([6, 3, 7], 8, 1.0, "gauss"),   # uneven batch, exact chi
    ([16], 16, 1.0, "pmj"),
    ([1, 2], 1, 0.5, "pmj"),        # degenerate: L=1 and chi=1
    ([12, 13], 64, 2.0, "pmj"),     # chi = 64 instantiation, exact at this size
    ([48], 64, 1.0, "pmj"),         # chi = 64, bonds cut at chi
]


@pytest.mark.parametrize("Ls,chi,beta,kind", CASES)
def test_dfloat_log_z_spectra_and_proposals(P, Ls, chi, beta, kind):
    S = 70  # two CTAs of chains, the second one ragged
    t, reals, lz, props, (_, sp, _), st, flags = _run(P, Ls, chi, beta, kind, S)
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    lq, E = props.logq.cpu().numpy(), props.E.cpu().numpy()
    sp = sp.cpu().numpy()
    bo, nbd = 0, 0
    for n, (L, (Jh, Jv), rows) in enumerate(zip(Ls, reals, envs)):
        o_lz = bmps.log_z(rows)
        assert abs(lz[n] - o_lz) < 1e-9 * max(1.0, abs(o_lz)), (n, lz[n], o_lz)
        for r in range(L):
            for c in range(1, L):
                o_s, gap = rows[r].spectra[c - 1], rows[r].cut_gap[c - 1]
                g_s = sp[(bo + r * (L + 1) + c) * chi:(bo + r * (L + 1) + c + 1) * chi]
                keep = o_s > 1e-7
                if gap > 1e-5:
                    np.testing.assert_allclose(g_s[:keep.sum()], o_s[keep], rtol=1e-7, atol=3.2e-11)
        _, b = parity.compare_proposals(rows, Jh, Jv, beta, 42, 0, n, spins[n], lq[n], E[n],
                                        band=1e-7, lq_atol=1e-8)
        nbd += b
        bo += L * (L + 1)
    assert nbd <= 2


@pytest.mark.parametrize("Ls", [(24,), (64,)])
def test_dfloat_beta3_follows_the_oracle(P, Ls):
    """beta = 3, chi = 64 (L = 24: bonds up to 20; L = 64: up to 56)."""
    Ls, beta, chi, S = list(Ls), 3.0, 64, 64
    t, reals, lz, props, (_, sp, ri), st, flags = _run(P, Ls, chi, beta, "pmj", S)
    assert st == 0 and not flags.any()
    (Jh, Jv), L = reals[0], Ls[0]
    rows = bmps.build_envs(Jh, Jv, beta, chi, t.cutoff)
    ri = ri.cpu().numpy().reshape(-1, 14)
    for r in range(L):
        assert abs(ri[r, 0] - rows[r].log_scale) < 3.2e-8 * abs(rows[r].log_scale), r
    assert abs(lz[0] - bmps.log_z(rows)) < 3.2e-8 * abs(lz[0])
    sp = sp.cpu().numpy().reshape(L, L + 1, chi)
    dev = np.concatenate([np.abs(sp[r, c, :rows[r].spectra[c - 1].size] - rows[r].spectra[c - 1])
                          for r in range(0, L, 4) for c in range(1, L)])
    assert dev.max() < 3.2e-4 and np.mean(dev < 2e-6) > 0.99, (dev.max(), np.mean(dev < 2e-6))
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    _, nbd = parity.compare_proposals(rows, Jh, Jv, beta, 42, 0, 0, spins[0],
                                      props.logq.cpu().numpy()[0], props.E.cpu().numpy()[0],
                                      band=1e-6, lq_atol=3.2e-5)
    assert nbd <= 1
    # an essentially exact q at L = 24: importance weights constant to 1e-5 (float64: 1e-6)
    if L == 24:
        w = -(props.logq.cpu().numpy()[0] + beta * props.E.cpu().numpy()[0])
        assert w.std() < 1e-5


def test_dfloat_scores_oracle_proposals_and_mh(P):
    """The double-float sampler scores the oracle's proposals (exact energies, log q to
    1e-8), and its MH chain on them takes the oracle's decisions."""
    from oracle import mh, sampler
    Ls, chi, beta, S = [9, 7], 8, 2.0, 96
    reals = parity.realizations(Ls, "gauss")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "dfloat", max_samples=S)
    t.build_envs(J)
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)
    outs = [sampler.propose(rows, Jh, Jv, beta, S, 5, 0, n)[:3]
            for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs))]
    spins = torch.from_numpy(np.concatenate([o[0].reshape(-1) for o in outs])).cuda()
    g_lq, g_E = t.score(spins, S)
    g_lq, g_E = g_lq.cpu().numpy(), g_E.cpu().numpy()
    for n, o in enumerate(outs):
        np.testing.assert_array_equal(g_E[n], o[2])
        np.testing.assert_allclose(g_lq[n], o[1], rtol=0, atol=1e-8 * max(1.0, np.abs(o[1]).max()))
    logq = torch.from_numpy(np.stack([o[1] for o in outs])).cuda()
    E = torch.from_numpy(np.stack([o[2] for o in outs])).cuda()
    state = t.mh_init_empty()
    acc = t.mh_step(P.Proposals(spins, logq, E, S, 0), state, seed=5).cpu().numpy()
    for n, L in enumerate(Ls):
        start = (np.zeros((L, L), np.uint8), np.inf, 0.0)
        _, o_acc, o_lr, o_u = mh.chain(start, outs[n], beta, 5, 0, n)
        near = np.abs(np.log(o_u) - o_lr) < 1e-12
        assert np.array_equal(acc[n][~near], o_acc[~near])
