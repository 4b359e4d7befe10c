"""A whole step (coupling ingest, environments, log Z, proposals, MH) captured in one
CUDA graph and replayed gives the same bits as the same calls made eagerly: every call
of the step only enqueues work on the handle's stream (no host synchronisation, no
allocation), including the float64 build's CTA-pair launch."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "dfloat"])
def test_step_captured_in_a_cuda_graph(P, prec):
    Ls, chi, beta, S = [9, 6, 12], 8, 1.5, 64
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()

    def make():
        stream = torch.cuda.Stream()
        t = P.TNMC(Ls, chi, beta, prec, max_samples=S, stream=stream)
        props = t.alloc_proposals(S, 0)
        logz = torch.empty(len(Ls), dtype=torch.float64, device="cuda")
        acc = torch.empty((len(Ls), S), dtype=torch.uint8, device="cuda")
        return t, stream, props, logz, acc

    # eager
    t, stream, props, logz, acc = make()
    with torch.cuda.stream(stream):
        state = t.mh_init_empty()
        for step in range(2):
            t.build_envs(J)
            t.log_z(out=logz)
            t.propose(S, 42, 1000 * step, out=props)
            t.mh_step(props, state, 42, accept=acc)
    torch.cuda.synchronize()
    ref = (logz.clone(), props.spins.clone(), props.logq.clone(), acc.clone(), state.n_accept.clone(),
           state.spins.clone())

    # captured: one step per replay, the proposal ids advanced between replays
    t, stream, props, logz, acc = make()
    with torch.cuda.stream(stream):
        state = t.mh_init_empty()
    torch.cuda.synchronize()
    graphs = []
    for step in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            t.build_envs(J)
            t.log_z(out=logz)
            t.propose(S, 42, 1000 * step, out=props)
            t.mh_step(props, state, 42, accept=acc)
        graphs.append(g)
    # capture runs nothing: reset the chain and replay in order
    with torch.cuda.stream(stream):
        fresh = t.mh_init_empty()
        state.spins.copy_(fresh.spins)
        state.logq.copy_(fresh.logq)
        state.E.copy_(fresh.E)
        state.n_accept.zero_()
    torch.cuda.synchronize()
    for g in graphs:
        g.replay()
    torch.cuda.synchronize()
    got = (logz, props.spins, props.logq, acc, state.n_accept, state.spins)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    status, flags = t.device_status()
    assert status == 0 and not flags.any()


def test_handle_on_side_stream_orders_with_the_callers_stream(P):
    """A handle on its own stream, called from the default stream without a stream
    context: the couplings written on the default stream (after a long kernel) are
    complete before the build reads them, and the outputs are complete before the
    default stream reads them."""
    Ls, chi, beta, S = [12, 9], 8, 1.3, 48
    reals = parity.realizations(Ls, "pmj")
    Jh = torch.from_numpy(parity.packed_J(reals))
    ref = P.TNMC(Ls, chi, beta, "fp64", max_samples=S)
    ref.build_envs(Jh.cuda())
    want_lz = ref.log_z().cpu()
    want = ref.propose(S, 42, 0)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    t = P.TNMC(Ls, chi, beta, "fp64", max_samples=S, stream=side)
    for k in range(3):
        J = torch.zeros_like(Jh, device="cuda")
        big = torch.randn(4096, 4096, device="cuda")
        for _ in range(8):
            big = big @ big / 64.0            # keep the default stream busy
        J.copy_(Jh, non_blocking=False)
        J += big[0, 0] * 0.0                  # the couplings depend on the long kernel chain
        t.build_envs(J)
        lz = t.log_z()
        props = t.propose(S, 42, 0)
        got_lz = lz.clone()                   # default-stream reads of the outputs
        got_spins = props.spins.clone()
        torch.cuda.synchronize()
        assert torch.equal(got_lz.cpu(), want_lz), k
        assert torch.equal(got_spins, want.spins), k
