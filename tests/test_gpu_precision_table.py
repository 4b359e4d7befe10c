"""Measured error of the reduced-precision modes against the FP64 oracle, per beta.

For each mode and beta in {1, 2, 3}: 4 +-J realizations at L = 32, chi = 32,
S = 64. Reported per case (and written as JSON lines to
$TNMC_PRECISION_TABLE when that variable names a file):
  * max |d log Z| / L^2 over the realizations (GPU build vs oracle build);
  * max |d log q| of the oracle's proposals scored by the GPU (teacher forced);
  * max |d logit| over the draws whose conditionals are finite on both sides;
  * the fraction of draws whose decision under the same uniform differs.
The asserted bounds are the ones the modes are documented to meet; beta = 3 in
float32 (cache and sampling) is documented to fail them and is only recorded.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bmps, philox, sampler  # noqa: E402
import parity  # noqa: E402

LS, CHI, S = [32] * 4, 32, 64
# (mode, beta) -> (bound on |d log Z| / L^2, bound on |d log q|); None: recorded only.
# The targets are |d log Z| / L^2 <= 1e-6 and |d log q| <= 1e-4 (TF32 and BF16 meet neither:
# their bounds below record the errors of the rounded products). float32 sampling
# contractions (FP32, MIXED) miss the log q target beyond beta = 1 and float32 builds
# miss the log Z one beyond beta = 1 on some instances (see test_gpu_chi64.py); the
# bounds below are the ones each mode meets.
BOUNDS = {
    ("fp32", 1.0): (1e-6, 1e-3), ("fp32", 2.0): None, ("fp32", 3.0): None,
    ("mixed", 1.0): (1e-6, 1e-4), ("mixed", 2.0): (1e-6, 1e-2), ("mixed", 3.0): (1e-6, None),
    ("dfloat", 1.0): (1e-6, 1e-4), ("dfloat", 2.0): (1e-6, 1e-4), ("dfloat", 3.0): (1e-6, 1e-4),
    # tensor-core products from TF32 / BF16 operands: about 4x the measured errors (log Z per
    # site 2.3e-5 / 5.0e-4 / 1.6e-2 in TF32, 3.9e-4 / 4.4e-3 / 6.9e-2 in BF16 at beta = 1 / 2 / 3);
    # their sampling loses the conditionals beyond beta = 1 (log q recorded only)
    ("tf32", 1.0): (1e-4, 1.0), ("tf32", 2.0): (2e-3, None), ("tf32", 3.0): (7e-2, None),
    ("bf16", 1.0): (2e-3, 10.0), ("bf16", 2.0): (2e-2, None), ("bf16", 3.0): (0.3, None),
}


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


_ORACLE = {}


def _oracle(beta, cutoff):
    key = (beta, cutoff)
    if key not in _ORACLE:
        reals = parity.realizations(LS, "pmj")
        envs = parity.oracle_envs(reals, beta, CHI, cutoff)
        props = [sampler.propose(rows, Jh, Jv, beta, S, 42, 0, n)
                 for n, ((Jh, Jv), rows) in enumerate(zip(reals, envs))]
        _ORACLE[key] = (reals, envs, props)
    return _ORACLE[key]


@pytest.mark.parametrize("mode,beta", sorted(BOUNDS))
def test_precision_against_oracle(P, mode, beta):
    reals = parity.realizations(LS, "pmj")
    t = P.TNMC(LS, CHI, beta, mode, max_samples=S)
    t.build_envs(torch.from_numpy(parity.packed_J(reals)).cuda())
    lz = t.log_z().cpu().numpy()
    # the oracle truncates with the mode's own cutoff: the table measures arithmetic, not the rule
    reals, envs, o_props = _oracle(beta, t.cutoff)
    spins_in = torch.from_numpy(np.concatenate([o[0].reshape(-1) for o in o_props])).cuda()
    g_lq, _, g_lg = t.score_logits(spins_in, S)
    g_lq, g_lg = g_lq.cpu().numpy(), g_lg.cpu().numpy()
    dz, dq, dl, flips, draws = 0.0, 0.0, 0.0, 0, 0
    for n, L in enumerate(LS):
        o_sig, o_lq, _, o_lg = o_props[n]
        dz = max(dz, abs(lz[n] - bmps.log_z(envs[n])) / (L * L))
        dq = max(dq, float(np.abs(g_lq[n] - o_lq).max()))
        lg = g_lg[n * S * L * L:(n + 1) * S * L * L].reshape(S, L * L)
        fin = np.isfinite(lg) & np.isfinite(o_lg)
        dl = max(dl, float(np.abs(lg - o_lg)[fin].max(initial=0.0)))
        u = philox.spin_uniforms(L, np.arange(S, dtype=np.uint64), n, 42)
        flips += int(((u < sampler.sigmoid(lg)) != (u < sampler.sigmoid(o_lg))).sum())
        draws += u.size
    row = {"mode": mode, "beta": beta, "L": LS[0], "chi": CHI, "realizations": len(LS), "S": S,
           "cutoff": t.cutoff, "max_dlogZ_per_site": dz, "max_dlogq": dq, "max_dlogit": dl,
           "decision_flip_fraction": flips / draws}
    print(json.dumps(row))
    out = os.environ.get("TNMC_PRECISION_TABLE")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps(row) + "\n")
    b = BOUNDS[(mode, beta)]
    if b is not None:
        assert np.isfinite(dz), row
        assert dz <= b[0], row
        if b[1] is not None:
            assert dq <= b[1], row
