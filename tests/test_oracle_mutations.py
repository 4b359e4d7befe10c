"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one plausible slip into a copy of an oracle function and
checks that the matching exact reference disagrees with it.
"""
import numpy as np

from oracle import bmps, exact, sampler
from workloads import draw_bonds


def test_dropped_up_field_is_caught(monkeypatch):
    L, beta = 3, 1.0
    Jh, Jv = draw_bonds(L, 33, "pmj")
    rows = bmps.build_envs(Jh, Jv, beta, chi=2)
    orig = sampler.run_rows

    def no_field(rows_, Jh_, Jv_, beta_, u=None, forced=None, correction=None):
        return orig(rows_, Jh_, np.zeros_like(Jv_), beta_, u=u, forced=forced, correction=correction)

    sig, _, _, good = sampler.propose(rows, Jh, Jv, beta, 8, 42, 0, 0)
    ex = exact.brute_conditional_logits(Jh, Jv, beta, sig)
    assert np.abs(good - ex).max() < 1e-10
    monkeypatch.setattr(sampler, "run_rows", no_field)
    _, _, bad = sampler.score(rows, Jh, Jv, beta, sig)
    assert np.abs(bad - ex).max() > 1e-3


def test_transposed_vertical_matrix_in_mpo_is_caught(monkeypatch):
    """Putting B(Jv) on the right leg and B(Jh) on the down leg changes log Z."""
    L, beta = 4, 1.0
    Jh, Jv = draw_bonds(L, 34, "gauss")
    lz = exact.brute_force(Jh, Jv, beta)[3]
    orig = bmps.row_mpo

    def swapped(Jh_row, Jv_row, beta_):
        Jv_sw = np.concatenate([Jh_row, Jv_row[-1:]])
        return orig(Jv_row[:-1], Jv_sw, beta_)

    monkeypatch.setattr(bmps, "row_mpo", swapped)
    bad = bmps.log_z(bmps.build_envs(Jh, Jv, beta, chi=4))
    assert abs(bad - lz) > 1e-3
