"""The TF32 and BF16 contraction modes (tensor-core products in the float32 build).

TNMC_TF32 / TNMC_BF16 run the build's two dense products per site (the previous
row's site times the carried triangular factor, and the SVD input Q x blockdiag(U S))
on the tensor cores from TF32 (10 mantissa bits) or BF16 (7 bits) operands with
float32 accumulation (Sec. 3.2's contractions, in parity form); the QR and Jacobi
steps, the cache and the sampling contractions are float32, as in TNMC_FP32. Against
the FP64 oracle (same seeded couplings, same cutoff):

* the log Z error per site orders with the operands' precision, FP32 < TF32 < BF16,
  and stays within the bounds each mode is documented to meet at beta = 1
  (TF32 1e-4, BF16 2e-3: about 4x the errors measured over these instances; the
  unit roundoffs are 2^-11 and 2^-8);
* the TF32 build is not the FP32 build (the tensor-core path ran and rounded);
* energies of the proposals are exact (Eq. 1 on the drawn spins), and scoring the
  proposals reproduces their log q (the sampler's probabilities are those drawn).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bmps, ising  # noqa: E402
import parity  # noqa: E402

LS, CHI, BETA, S = [24, 20, 17, 24], 16, 1.0, 48
BOUND = {"fp32": 1e-6, "tf32": 1e-4, "bf16": 2e-3}


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


@pytest.fixture(scope="module")
def oracle_log_z():
    reals = parity.realizations(LS, "pmj")
    envs = parity.oracle_envs(reals, BETA, CHI, 1e-6)
    return reals, np.array([bmps.log_z(e) for e in envs])


def _run(P, reals, prec):
    t = P.TNMC(LS, CHI, BETA, prec, max_samples=S)
    assert t.cutoff == 1e-6
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, 42, 0)
    torch.cuda.synchronize()
    return t, lz, props


def test_log_z_error_orders_with_operand_precision(P, oracle_log_z):
    reals, o_lz = oracle_log_z
    err, lzs = {}, {}
    for prec in ("fp32", "tf32", "bf16"):
        t, lz, _ = _run(P, reals, prec)
        st, flags = t.device_status()
        assert st == 0, (prec, flags)
        lzs[prec] = lz
        err[prec] = max(abs(lz[n] - o_lz[n]) / (L * L) for n, L in enumerate(LS))
        assert err[prec] <= BOUND[prec], (prec, err)
    assert not np.array_equal(lzs["tf32"], lzs["fp32"])   # the tensor-core products ran
    assert err["fp32"] < err["tf32"] < err["bf16"], err


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_energies_exact_and_scores_reproduce_log_q(P, oracle_log_z, prec):
    reals, _ = oracle_log_z
    t, _, props = _run(P, reals, prec)
    spins = parity.split_spins(props.spins.cpu().numpy(), LS, S)
    E = props.E.cpu().numpy()
    for n, (Jh, Jv) in enumerate(reals):
        assert np.array_equal(E[n], ising.energy(Jh, Jv, spins[n])), n
    lq, E2 = t.score(props.spins, S)
    assert np.array_equal(E2.cpu().numpy(), E)
    np.testing.assert_allclose(lq.cpu().numpy(), props.logq.cpu().numpy(), rtol=1e-12, atol=1e-12)
    assert np.all(props.logq.cpu().numpy() <= 0.0)


@pytest.mark.parametrize("prec,bound", [("tf32", 1e-4), ("bf16", 2e-3)])
def test_tensor_modes_at_chi64(P, prec, bound):
    # the chi = 64 instantiation (the benchmark's) with the tensor-core products: L = 12, 13 at
    # beta = 1, where chi = 64 is exact, against the oracle's log Z at the mode's cutoff
    Ls, chi, beta = [12, 13], 64, 1.0
    reals = parity.realizations(Ls, "pmj")
    t = P.TNMC(Ls, chi, beta, prec, max_samples=8)
    assert t.plan_ch == 64
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    torch.cuda.synchronize()
    assert t.device_status()[0] == 0
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)
    for n, L in enumerate(Ls):
        assert abs(lz[n] - bmps.log_z(envs[n])) / (L * L) <= bound, (n, lz[n], bmps.log_z(envs[n]))
