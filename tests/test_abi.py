"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/tnmc.h declares; host-only calls (sizes, argument checks) work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2509_19006_b300 import build
    build.build()
    import paper_2509_19006_b300 as P
    return P


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(tnmc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(P):
    lib = ctypes.CDLL(P.LIB_PATH)
    names = declared_functions()
    assert "tnmc_build_envs" in names and "tnmc_propose" in names and "tnmc_mh_step" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(P.EXPORTED) <= set(names)


def test_workspace_size_host_only(P):
    small = P.workspace_size([16], 16, 1.0, P.TNMC_FP64, 1000)
    assert small > 0
    cache, env, samp = P.layout_info([256] * 64, 64, 3.0, P.TNMC_FP32, 256)
    assert cache == 64 * 256 * 256 * 64 * 64 * 4          # one chi x chi float matrix per site
    assert samp == 256 * 64 * 256 * 64 * 4                # right environments of every chain
    # float64 doubles the cache
    c64, _, _ = P.layout_info([256] * 64, 64, 3.0, P.TNMC_FP64, 256)
    assert c64 == 2 * cache


@pytest.mark.parametrize("args", [
    ([16], 0, 1.0, 1, 4),        # chi < 1
    ([16], 65, 1.0, 1, 4),       # chi > 64
    ([0], 4, 1.0, 1, 4),         # L < 1
    ([16], 4, -1.0, 1, 4),       # beta < 0
    ([16], 4, float("nan"), 1, 4),
    ([16], 4, 1.0, 9, 4),        # unknown precision
    ([16], 4, 1.0, 1, 0),        # max_samples < 1
    ([], 4, 1.0, 1, 4),          # no realization
    ([16], 4, 1.0, 1, 4, 1.0),   # cutoff >= 1 keeps nothing
    ([16], 4, 1.0, 1, 4, 0.0, 1),        # a checkpoint every row is the full cache
    ([16], 4, 1.0, 1, 4, 0.0, 0, 1),     # one state per site
])
def test_argument_checks(P, args):
    with pytest.raises(P.TnmcError) as e:
        P.workspace_size(*args)
    assert e.value.status == 1


def test_potts_requests_beyond_the_kernels_are_unsupported(P):
    for args in (([16], 4, 1.0, P.TNMC_DFLOAT, 4, 0.0, 0, 3),    # double-float Potts
                 ([16], 4, 1.0, P.TNMC_FP64, 4, 0.0, 4, 3),      # checkpoints
                 ([16], 32, 1.0, P.TNMC_FP64, 4, 0.0, 0, 3),     # chi above the panels
                 ([16], 4, 1.0, P.TNMC_FP64, 4, 0.0, 0, 5)):     # q above the panels
        with pytest.raises(P.TnmcError) as e:
            P.workspace_size(*args)
        assert e.value.status == 7, args
    assert P.workspace_size([16], 16, 1.0, P.TNMC_FP32, 4, 0.0, 0, 3) > 0


def test_tensor_core_precisions_size_like_float32(P):
    # TF32 / BF16 round the build's products only: cache, scratch and workspace are float32's
    for prec in (P.TNMC_TF32, P.TNMC_BF16):
        assert P.workspace_size([16, 9], 8, 1.0, prec, 4) == P.workspace_size([16, 9], 8, 1.0, P.TNMC_FP32, 4)


def test_status_strings(P):
    for code in range(8):
        assert P.status_string(code)


def test_mlp_layout_constants_agree_with_oracle(P):
    """The header's parameter layout of the learned correction equals the oracle's, and the binding's."""
    from oracle import learned
    text = open(os.path.join(ROOT, "include", "tnmc.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define (TNMC_MLP_\w+) (\d+)", text)}
    assert defs["TNMC_MLP_FEATURES"] == learned.N_FEAT
    assert defs["TNMC_MLP_IN"] == learned.IN_PAD and defs["TNMC_MLP_HIDDEN"] == learned.HIDDEN
    for name in ("W1", "B1", "W2", "B2", "W3", "B3"):
        assert defs[f"TNMC_MLP_OFF_{name}"] == getattr(learned, f"OFF_{name}"), name
        key = {"W1": "W1", "B1": "b1", "W2": "W2", "B2": "b2", "W3": "w3", "B3": "b3"}[name]
        assert P.MLP_OFF[key] == defs[f"TNMC_MLP_OFF_{name}"], name
    assert defs["TNMC_MLP_PARAMS"] == learned.N_PARAM == P.MLP_PARAMS
    assert P.load_library().tnmc_mlp_scratch_floats() > 0


def test_checkpointing_fits_the_L1024_workload(P):
    """64 realizations at L = 1024, chi = 32, S = 128 in float32: the full cache alone is
    275 GB; with a checkpoint every 32 rows the whole workspace is about 20 GB."""
    Ls = [1024] * 64
    cache_full, _, _ = P.layout_info(Ls, 32, 3.0, P.TNMC_FP32, 128)
    assert cache_full == 64 * 1024 * 1024 * 32 * 32 * 4
    cache_ck, _, samp = P.layout_info(Ls, 32, 3.0, P.TNMC_FP32, 128, ckpt_every=32)
    assert cache_ck == 64 * (32 + 32) * 1024 * 32 * 32 * 4
    assert P.workspace_size(Ls, 32, 3.0, P.TNMC_FP32, 128, ckpt_every=32) < 21e9
    with pytest.raises(P.TnmcError):
        P.workspace_size(Ls, 32, 3.0, P.TNMC_FP32, 128, ckpt_every=1)
    # MIXED (float64 build, float32 cache) also keeps its checkpoint rows in float64
    ws_mixed = P.workspace_size(Ls, 32, 3.0, P.TNMC_MIXED, 128, ckpt_every=32)
    assert ws_mixed - P.workspace_size(Ls, 32, 3.0, P.TNMC_FP32, 128, ckpt_every=32) >= 64 * 32 * 1024 * 32 * 32 * 8


def test_every_declaration_cites_its_passage_and_errors():
    """Each call of include/tnmc.h is documented on its own: a passage of the paper (Sec.,
    Eq. or Fig.) or the statement that the paper has no counterpart, and its error
    behaviour (the errors it returns, that it cannot fail, or what it returns)."""
    import re
    src = open(os.path.join(ROOT, "include", "tnmc.h")).read()
    names = []
    for m in re.finditer(r"^\w[\w\s\*]*?\b(tnmc_\w+)\(", src, re.M):
        before = src[:m.start()]
        c0, c1 = before.rfind("/*"), before.rfind("*/")
        assert c0 >= 0 and c1 > c0 and before[c1 + 2:].strip() == "", m.group(1)
        comment = " ".join(before[c0:c1].split())       # one line: phrases may wrap
        assert re.search(r"Sec\.|Eq\.|Fig\.|no counterpart|does not state", comment), m.group(1)
        assert re.search(r"Errors?:|Cannot fail|Returns|-1 for a NULL", comment), m.group(1)
        names.append(m.group(1))
    assert len(names) >= 29
