"""Why float32 mode cannot meet a 1e-4 bound on log q at beta >= 2 (CPU only).

Rounding the float64 oracle's own cache tensors to float32, and contracting
them in float64, already moves log q by more than 1e-4: the conditional
weights rho_s = |l M_c[s] R_c| of strongly polarised spins are small
differences of O(1) terms, so a relative rounding of the tensors is amplified.
The GPU's float32 mode is therefore bounded by storage, not by its arithmetic.
"""
import numpy as np

from oracle import bmps, sampler
from workloads import draw_bonds


def _rounded(rows, dtype):
    return [bmps.RowEnv([A.astype(dtype).astype(np.float64) for A in r.tensors], r.log_scale,
                        r.spectra, r.cut_gap, r.discarded) for r in rows]


def test_fp32_storage_bound():
    L, chi, beta = 10, 8, 2.0
    Jh, Jv = draw_bonds(L, 1000, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi)
    sig, lq, _, lg = sampler.propose(rows, Jh, Jv, beta, 64, 42, 0, 0)
    lq32, _, lg32 = sampler.score(_rounded(rows, np.float32), Jh, Jv, beta, sig)
    lq16, _, _ = sampler.score(_rounded(rows, np.float16), Jh, Jv, beta, sig)
    d32 = np.abs(lq32 - lq).max()
    assert 1e-4 < d32 < 1e-2                  # float32 storage alone: ~1e-3
    assert np.abs(lq16 - lq).max() > 10 * d32  # the error scales with the storage precision
    # log Z is insensitive: rounding shifts it by far less than 1e-6 per site
    assert abs(bmps.log_z(_rounded(rows, np.float32)) - bmps.log_z(rows)) / L ** 2 < 1e-8
