"""The benchmark workload at full size, in the launch configuration bench.py times.

64 +-J realizations at L=256, beta=3, chi=64, 256 proposals each, float32 (bench.py's
default; about half a minute). The oracle cannot build L=256 environments in a test's
time, so the checks are on outputs it computes one by one and on properties that hold
at any size:

* configurations drawn from the oracle's own Philox stream (one per realization, every
  fourth checked) get the oracle's exact energies (Eq. 1) from the scoring kernel;
* the MH kernel (Eq. 10), fed proposals made on the host (seeded spins, energies and
  log q, none from the GPU), takes the oracle chain's decisions and ends in its states;
* the scoring kernel, run on the benchmark's own proposals, reproduces their energies
  exactly and their log q to float32 accumulation level (two kernel instantiations);
* every log Z is finite, spins are bits, every finite log q is <= 0, and the only
  device flag float32 may raise at beta=3 is a vanished conditional (NUMERIC).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mh, philox  # noqa: E402
from oracle.ising import energy  # noqa: E402
from workloads import config  # noqa: E402


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


@pytest.fixture(scope="module")
def bench_run(P):
    """Environments and one round of proposals, as bench.py runs them."""
    wl = config("L256")
    J = torch.from_numpy(wl.packed_J()).cuda()
    t = P.TNMC(wl.Ls, wl.chi, wl.beta, "fp32", max_samples=wl.S)
    t.build_envs(J)
    lz = t.log_z().cpu().numpy()
    props = t.propose(wl.S, 42, 10_000_000)
    torch.cuda.synchronize()
    return wl, t, lz, props


def test_full_size_outputs_are_well_formed(P, bench_run):
    wl, t, lz, props = bench_run
    assert np.isfinite(lz).all()
    status, flags = t.device_status(clear=False)
    assert status in (0, 4), P.status_string(status)   # TNMC_OK or TNMC_ERR_NUMERIC
    assert set(np.unique(flags)) <= {0, P.FLAG_NUMERIC}
    assert int(props.spins.max().item()) <= 1
    lq = props.logq.cpu().numpy()
    fin = np.isfinite(lq)
    assert (lq[fin] <= 0).all()
    # chains of unflagged realizations never lose a conditional
    assert fin[flags == 0].all()


def test_full_size_score_reproduces_proposals(bench_run):
    wl, t, _, props = bench_run
    lq2, E2 = t.score(props.spins, wl.S)
    np.testing.assert_array_equal(E2.cpu().numpy(), props.E.cpu().numpy())
    a, b = lq2.cpu().numpy(), props.logq.cpu().numpy()
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    d = np.abs(a[fin] - b[fin])
    assert (d <= 1e-6 * np.maximum(1.0, np.abs(b[fin]))).all(), float(d.max())


def test_full_size_energies_of_oracle_configurations(bench_run):
    wl, t, _, _ = bench_run
    L, seed = wl.Ls[0], 5
    sig = np.stack([philox.init_spins(L, n, seed) for n in range(wl.n_real)])   # (n, L, L)
    _, E = t.score(torch.from_numpy(sig.reshape(-1)).cuda(), 1)
    E = E.cpu().numpy()[:, 0]
    for n in range(0, wl.n_real, 4):     # a sample of the realizations (0.2 s each here)
        Jh, Jv = wl.realization(n)
        assert E[n] == energy(Jh, Jv, sig[n]), n


def test_full_size_mh_takes_the_oracle_decisions(P, bench_run):
    wl, t, _, _ = bench_run
    L, S, beta, seed, base = wl.Ls[0], wl.S, wl.beta, 42, 7_000
    rng = np.random.default_rng(2024)
    sites = np.arange(L * L)
    # proposal k of realization n: a cheap seeded bit pattern; its energy an integer
    # and its log q = -beta E + N(0, 1), so that about half the proposals are accepted
    spins = np.empty((wl.n_real, S, L * L), np.uint8)
    for n in range(wl.n_real):
        mult = rng.integers(1, 1 << 20, size=S)
        spins[n] = ((sites[None, :] * mult[:, None] + n) >> 7) & 1
    E = rng.integers(-2 * L * L, 2 * L * L, size=(wl.n_real, S)).astype(np.float64)
    lq = -beta * E + rng.standard_normal((wl.n_real, S))
    props = P.Proposals(torch.from_numpy(spins.reshape(-1)).cuda(), torch.from_numpy(lq).cuda(),
                        torch.from_numpy(E).cuda(), S, base)
    state = t.mh_init_empty()
    acc = t.mh_step(props, state, seed).cpu().numpy()
    torch.cuda.synchronize()
    g_sig = state.spins.cpu().numpy().reshape(wl.n_real, L * L)
    g_lq, g_E = state.logq.cpu().numpy(), state.E.cpu().numpy()
    g_nacc = state.n_accept.cpu().numpy()
    n_near = 0
    for n in range(wl.n_real):
        start = (np.zeros(L * L, np.uint8), np.inf, 0.0)
        (o_sig, o_lq, o_E), o_acc, o_lr, o_u = mh.chain(start, (spins[n], lq[n], E[n]), beta, seed, base, n)
        near = np.abs(np.log(o_u) - o_lr) < 1e-12
        n_near += int(near.sum())
        assert np.array_equal(acc[n][~near], o_acc[~near]), n
        if not near.any():
            assert g_nacc[n] == o_acc.sum()
            assert g_E[n] == o_E and g_lq[n] == o_lq
            np.testing.assert_array_equal(g_sig[n], o_sig)
    assert 0.2 < acc.mean() < 0.8 and n_near <= 2
