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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_matches_workspace_scratch(P, prec):
    Ls, chi, beta, S = [9, 6, 12], 8, 1.5, 40
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, prec, max_samples=S)
    t.build_envs(J)
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
