"""Build layouts and their autotuner (tnmc_set_build_variant, tnmc_autotune_build).

Every layout computes the same method (they differ in how the CTA's threads share the
Jacobi rounds and whether a realization gets one CTA or a pair), so each one is held
to the oracle with the precision's own bounds; the autotuner keeps the layout that
was fastest in its own timing, and that layout is also (within timing noise) the
fastest on full builds of the same realizations.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bmps  # noqa: E402
import parity  # noqa: E402

CANDIDATES = [0, 1, 2, 4, 12]
CANDIDATES_FP32 = [0, 8, 16, 17, 18, 32, 40]   # one CTA (4 or 8 lanes), pairs (bit 4), QR preconditioning (bit 5)
# valid layouts the autotuner does not time: preconditioned CTA pairs (bits 4 and 5; won 6 middle
# rows of the L = 256 float32 workload by 2.5 % but lost the full build by 11 %)
LAYOUTS_FP32 = CANDIDATES_FP32 + [48, 49, 50]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


@pytest.mark.parametrize("prec", ["fp64", "dfloat"])
@pytest.mark.parametrize("variant", CANDIDATES)
def test_every_layout_matches_the_oracle(P, prec, variant):
    Ls, chi, beta, S = [9, 6, 12], 8, 1.5, 40
    reals = parity.realizations(Ls, "pmj")
    t = P.TNMC(Ls, chi, beta, prec, max_samples=S)
    t.set_build_variant(variant)
    assert t.build_variant == variant
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, 42, 0)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    rel, band, lq_atol = (1e-10, 1e-9, 1e-9) if prec == "fp64" else (1e-9, 1e-7, 1e-8)
    for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs)):
        o = bmps.log_z(rows)
        assert abs(lz[n] - o) < rel * abs(o), (n, lz[n], o)
        _, nbd = parity.compare_proposals(rows, Jh, Jv, beta, 42, 0, n, spins[n], props.logq.cpu().numpy()[n],
                                          props.E.cpu().numpy()[n], band=band, lq_atol=lq_atol)
        assert nbd <= 1


@pytest.mark.parametrize("variant", LAYOUTS_FP32)
def test_every_float32_layout_matches_the_oracle(P, variant):
    # float32: |d log Z| / L^2 <= 1e-6 (where cut gaps are wide, beta = 1) and every draw the
    # oracle's outside the float32 band; the pair layouts move sector 1's Jacobi to a second SM,
    # bit 5 preconditions the Jacobi with a pivoted QR
    Ls, chi, beta, S = [9, 6, 12, 16], 8, 1.0, 40
    reals = parity.realizations(Ls, "pmj")
    t = P.TNMC(Ls, chi, beta, "fp32", max_samples=S)
    t.set_build_variant(variant)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    props = t.propose(S, 42, 0)
    torch.cuda.synchronize()
    st, flags = t.device_status()
    assert st == 0 and not flags.any()
    envs = parity.oracle_envs(reals, beta, chi, t.cutoff)
    spins = parity.split_spins(props.spins.cpu().numpy(), Ls, S)
    for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs)):
        L = Ls[n]
        assert abs(lz[n] - bmps.log_z(rows)) / (L * L) <= 1e-6, (n, variant)
        parity.compare_proposals(rows, Jh, Jv, beta, 42, 0, n, spins[n], props.logq.cpu().numpy()[n],
                                 props.E.cpu().numpy()[n], band=2e-3, lq_atol=1e-2)


def test_bad_layout_refused(P):
    t = P.TNMC([4], 4, 1.0, "fp64", max_samples=4)
    for bad in (3, -1, 64, 19):
        with pytest.raises(P.TnmcError):
            t.set_build_variant(bad)


def test_autotuner_keeps_the_fastest_layout(P):
    Ls, chi, beta = [40] * 6, 32, 2.0
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "dfloat", max_samples=8)
    times = t.autotune(J, rows=8)
    assert sorted(times) == sorted(CANDIDATES)
    assert t.build_variant == min(times, key=times.get)
    with pytest.raises(P.TnmcError) as e:      # the timing launches invalidated the cache
        t.propose(2, 1)
    assert e.value.status == 6
    # full builds of each layout: the kept one is within timing noise of the fastest
    full = {}
    for v in CANDIDATES:
        t.set_build_variant(v)
        best = float("inf")
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(t.stream)
            t.build_envs(J)
            e1.record(t.stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        full[v] = best
    chosen = min(times, key=times.get)
    assert full[chosen] <= 1.25 * min(full.values()), (times, full)


def test_autotuner_on_a_built_handle_times_middle_rows(P):
    # after a full build the candidates are timed on rows from the middle of the lattice
    # (rebuilt from the cached row below them); the kept layout is within timing noise of
    # the fastest full build, and the handle rebuilt with it meets the oracle
    Ls, chi, beta = [48] * 6, 32, 1.0
    reals = parity.realizations(Ls, "pmj")
    J = torch.from_numpy(parity.packed_J(reals)).cuda()
    t = P.TNMC(Ls, chi, beta, "fp32", max_samples=8)
    t.build_envs(J)
    times = t.autotune(J, rows=6)
    assert sorted(times) == sorted(CANDIDATES_FP32)
    chosen = min(times, key=times.get)
    assert t.build_variant == chosen
    full = {}
    for v in CANDIDATES_FP32:
        t.set_build_variant(v)
        best = float("inf")
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(t.stream)
            t.build_envs(J)
            e1.record(t.stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        full[v] = best
    assert full[chosen] <= 1.25 * min(full.values()), (times, full)
    t.set_build_variant(chosen)
    t.build_envs(J)
    lz = t.log_z().cpu().numpy()
    envs = parity.oracle_envs(reals[:2], beta, chi, t.cutoff)
    for n in range(2):
        assert abs(lz[n] - bmps.log_z(envs[n])) / (Ls[n] ** 2) <= 1e-6
