"""Checkpointed environments (every K-th row cached, segments rebuilt before sampling)
give the same bits as the fully cached environments, through the C ABI, and meet the
oracle directly (Sec. 3.5: environments recomputed per segment)."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed", "dfloat"])
@pytest.mark.parametrize("K", [2, 3, 5])
def test_checkpointed_equals_full_cache(P, prec, K):
    Ls, chi, beta, S = [9, 6, 12], 4, 1.5, 70
    reals = parity.realizations(Ls, "gauss")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    full = P.TNMC(Ls, chi, beta, prec, max_samples=S)
    ck = P.TNMC(Ls, chi, beta, prec, max_samples=S, ckpt_every=K)
    # (MIXED also keeps float64 checkpoint rows, which outweigh the saving at these tiny sizes)
    assert ck.ws_bytes < full.ws_bytes or K >= 5 or prec == "mixed"
    for t in (full, ck):
        t.build_envs(J)
    assert torch.equal(full.log_z(), ck.log_z())
    a, b = full.propose(S, 42, 100), ck.propose(S, 42, 100)
    assert torch.equal(a.spins, b.spins) and torch.equal(a.logq, b.logq) and torch.equal(a.E, b.E)
    la, Ea = full.score(a.spins, S)
    lb, Eb = ck.score(a.spins, S)
    assert torch.equal(la, lb) and torch.equal(Ea, Eb)
    sa, sb = full.mh_init(5), ck.mh_init(5)
    assert torch.equal(sa.spins, sb.spins) and torch.equal(sa.logq, sb.logq)
    acc_a, acc_b = full.mh_step(a, sa, 5), ck.mh_step(b, sb, 5)
    assert torch.equal(acc_a, acc_b) and torch.equal(sa.n_accept, sb.n_accept)
    c, d = full.propose_static(S, 43, 7), ck.propose_static(S, 43, 7)
    assert torch.equal(c.spins, d.spins) and torch.equal(c.logq, d.logq)
    # with the learned correction on
    net = P.MLP(seed=1)
    net.params[5248:5312] = 0.2
    net.pack()
    full.set_correction(net.bf16)
    ck.set_correction(net.bf16)
    e, f = full.propose(S, 44, 0), ck.propose(S, 44, 0)
    assert torch.equal(e.spins, f.spins) and torch.equal(e.logq, f.logq)
    for t in (full, ck):
        st, flags = t.device_status()
        assert st == 0 and not flags.any()


def test_checkpoint_argument_checks(P):
    with pytest.raises(P.TnmcError):
        P.TNMC([8], 4, 1.0, "fp32", max_samples=4, ckpt_every=1)


def test_cluster_wait_that_runs_out_reports_timeout(P):
    """The float64 build hands parity sector 1 to a partner CTA; with a tiny wait budget the
    hand-offs run out: the call returns, the status is TNMC_ERR_TIMEOUT, the owner did the
    work itself, and at the default budget the same handle builds correctly again."""
    Ls, chi, beta = [10, 8], 8, 1.5
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    ref = P.TNMC(Ls, chi, beta, "fp64", max_samples=4)
    ref.build_envs(J)
    lz_ref = ref.log_z().cpu().numpy()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=4)
    t.set_wait_budget(1)
    t.build_envs(J)
    t.log_z()
    st, flags = t.device_status()
    assert st == 5 and (flags & 4).any(), (st, flags)      # TNMC_ERR_TIMEOUT, TNMC_FLAG_TIMEOUT
    t.set_wait_budget(0)
    t.build_envs(J)
    lz = t.log_z().cpu().numpy()
    st, flags = t.device_status()
    assert st == 0 and not flags.any()
    np.testing.assert_allclose(lz, lz_ref, rtol=1e-12)


@pytest.mark.parametrize("prec,K", [("fp64", 3), ("dfloat", 4)])
def test_checkpointed_handle_meets_the_oracle(P, prec, K):
    # direct parity of a checkpointed handle (not only through the full cache): log Z and the
    # free-running proposals, whose rows come from segments rebuilt from their checkpoints
    Ls, chi, beta, S = [13, 10], 8, 1.2, 48
    reals = parity.realizations(Ls, "pmj")
    t = P.TNMC(Ls, chi, beta, prec, max_samples=S, ckpt_every=K)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, 42, 0)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    rel, band, lq_atol = (1e-10, 1e-9, 1e-9) if prec == "fp64" else (1e-9, 1e-7, 1e-8)
    bd = 0
    for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs)):
        o = bmps.log_z(rows)
        assert abs(lz[n] - o) < rel * abs(o), (n, lz[n], o)
        _, nb = parity.compare_proposals(rows, Jh, Jv, beta, 42, 0, n, spins[n], props.logq.cpu().numpy()[n],
                                         props.E.cpu().numpy()[n], band=band, lq_atol=lq_atol)
        bd += nb
    assert bd <= 2
