"""tnmc_propose_static: proposals for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they want proposals: a runtime that
owns every allocation and handed the library only its workspace at setup, a
pool that is already fully reserved, or code in a region where the allocator
must not be entered. This entry point takes the chains' right-environment
scratch from a fixed device array inside the library instead of the
workspace. Its outputs must equal tnmc_propose's, here checked bit for bit on
two calls in a row through the C ABI. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import parity  # noqa: E402


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("prec,ckpt,learned", [("fp64", 0, False), ("fp32", 0, False),
                                               ("fp64", 4, False), ("fp32", 0, True)])
def test_static_scratch_matches_workspace_scratch(P, prec, ckpt, learned):
    Ls, chi, beta, S = [9, 6, 12], 8, 1.5, 40
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, prec, max_samples=S, ckpt_every=ckpt)
    t.build_envs(J)
    if learned:
        net = P.MLP(seed=3)
        theta = net.params.cpu().numpy()
        theta[P.MLP_OFF["w3"]:P.MLP_OFF["b3"]] = 0.3 * np.random.default_rng(1).standard_normal(64)
        net.load(theta)
        t.set_correction(net.bf16)
    lib = t.lib
    for call, base in enumerate([0, 5000]):
        ref = t.propose(S, 42, base)
        got = t.alloc_proposals(S, base)
        st = lib.tnmc_propose_static(t.h, S, 42, base, _ptr(got.spins), _ptr(got.logq), _ptr(got.E))
        assert st == 0, (call, P.status_string(st))
        torch.cuda.synchronize()
        assert torch.equal(got.spins, ref.spins), call
        np.testing.assert_array_equal(got.E.cpu().numpy(), ref.E.cpu().numpy())
        np.testing.assert_allclose(got.logq.cpu().numpy(), ref.logq.cpu().numpy(), rtol=0, atol=1e-12)
    status, flags = t.device_status()
    assert status == 0 and not flags.any()


def test_static_scratch_allocates_nothing_and_keeps_chain_order(P):
    """No device memory changes hands during a call (free bytes seen by the driver are
    unchanged across it), and S above max_samples only appends chains: the first 4
    chains of a 64-chain call are those of a 4-chain tnmc_propose call."""
    Ls, chi = [10, 7], 8
    reals = parity.realizations(Ls, "gauss")
    t = P.TNMC(Ls, chi, 1.1, "fp64", max_samples=4)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    big = t.alloc_proposals(64, 0)
    t.propose_static(64, 9, 0, out=big)           # first call: looks up the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = t.lib.tnmc_propose_static(t.h, 64, 9, 0, _ptr(big.spins), _ptr(big.logq), _ptr(big.E))
    torch.cuda.synchronize()
    assert st == 0 and torch.cuda.mem_get_info()[0] == free0
    small = t.propose(4, 9, 0)
    torch.cuda.synchronize()
    sb = parity.split_spins(big.spins.cpu().numpy(), Ls, 64)
    ss = parity.split_spins(small.spins.cpu().numpy(), Ls, 4)
    for n in range(len(Ls)):
        np.testing.assert_array_equal(sb[n][:4], ss[n])
    np.testing.assert_array_equal(big.logq.cpu().numpy()[:, :4], small.logq.cpu().numpy())
    np.testing.assert_array_equal(big.E.cpu().numpy()[:, :4], small.E.cpu().numpy())


def test_static_scratch_limits(P):
    limit = P.load_library().tnmc_propose_static_limit()
    assert limit == 32 << 20
    Ls, chi = [8], 4
    reals = parity.realizations(Ls, "pmj")
    t = P.TNMC(Ls, chi, 1.0, "fp64", max_samples=4)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    # S above max_samples is fine while the scratch fits (8 x 64 x 8 x 8 B = 32 KiB)
    out = t.propose_static(64, 7, 0)
    torch.cuda.synchronize()
    assert out.spins.numel() == 64 * 64
    # a request whose scratch exceeds the array is refused, nothing is launched
    S_big = limit // (8 * 8 * 8) + 1          # S x sum L x chi(8) x 8 B > limit
    big = t.alloc_proposals(S_big)
    st = t.lib.tnmc_propose_static(t.h, S_big, 7, 0, _ptr(big.spins), _ptr(big.logq), _ptr(big.E))
    assert st == 1
