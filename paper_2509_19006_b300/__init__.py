"""Python binding of ``libtnmc.so``, the batched TNMC hot path on one B300.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. torch supplies device memory (the workspace and the caller's
buffers) and the CUDA stream. There is no CPU fallback: if the library is
missing or no CUDA device is present the calls raise.

The names follow the C ABI in ``include/tnmc.h``.
"""
from __future__ import annotations

import ctypes
import functools
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtnmc.so")

TNMC_FP64, TNMC_FP32, TNMC_TF32, TNMC_BF16, TNMC_MIXED, TNMC_DFLOAT = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": TNMC_FP64, "fp32": TNMC_FP32, "tf32": TNMC_TF32, "bf16": TNMC_BF16,
              "mixed": TNMC_MIXED, "dfloat": TNMC_DFLOAT}
FLAG_BAD_COUPLINGS, FLAG_NUMERIC, FLAG_TIMEOUT = 1, 2, 4

EXPORTED = [
    "tnmc_status_string", "tnmc_workspace_size", "tnmc_create", "tnmc_destroy",
    "tnmc_build_envs", "tnmc_log_z", "tnmc_propose", "tnmc_score", "tnmc_mh_init",
    "tnmc_mh_step", "tnmc_set_diagnostics", "tnmc_get_device_status", "tnmc_layout_info",
    "tnmc_propose_static", "tnmc_propose_static_limit", "tnmc_set_correction",
    "tnmc_mlp_features", "tnmc_mlp_scratch_floats", "tnmc_mlp_grad", "tnmc_mlp_adam",
    "tnmc_mlp_pack", "tnmc_mlp_forward", "tnmc_mh_init_empty", "tnmc_set_wait_budget",
    "tnmc_observables", "tnmc_set_realization_ids", "tnmc_set_build_variant",
    "tnmc_get_build_variant", "tnmc_autotune_build",
]

# learned proposal correction: parameter vector layout (include/tnmc.h)
MLP_PARAMS = 5320
MLP_OFF = {"W1": 0, "b1": 1024, "W2": 1088, "b2": 5184, "w3": 5248, "b3": 5312}
MLP_FEAT_STRIDE = 8


class TnmcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [
        ("n_real", ctypes.c_int32),
        ("L", ctypes.POINTER(ctypes.c_int32)),
        ("chi", ctypes.c_int32),
        ("beta", ctypes.c_double),
        ("prec", ctypes.c_int32),
        ("max_samples", ctypes.c_int32),
        ("cutoff", ctypes.c_double),
        ("ckpt_every", ctypes.c_int32),
        ("q_states", ctypes.c_int32),
    ]


_lib = None


def load_library():
    """Load libtnmc.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtnmc.so not built (expected at {LIB_PATH}); run the package build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t
    cfgp = ctypes.POINTER(_Config)
    sig = {
        "tnmc_status_string": ([i32], ctypes.c_char_p),
        "tnmc_workspace_size": ([cfgp, ctypes.POINTER(sz)], i32),
        "tnmc_layout_info": ([cfgp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(sz)], i32),
        "tnmc_create": ([cfgp, vp, sz, vp, ctypes.POINTER(vp)], i32),
        "tnmc_destroy": ([vp], None),
        "tnmc_build_envs": ([vp, vp], i32),
        "tnmc_log_z": ([vp, vp], i32),
        "tnmc_propose": ([vp, i32, u64, u64, vp, vp, vp], i32),
        "tnmc_score": ([vp, i32, vp, vp, vp], i32),
        "tnmc_mh_init": ([vp, u64, vp, vp, vp], i32),
        "tnmc_mh_init_empty": ([vp, vp, vp, vp], i32),
        "tnmc_set_wait_budget": ([vp, ctypes.c_int64], i32),
        "tnmc_set_realization_ids": ([vp, vp], i32),
        "tnmc_set_build_variant": ([vp, i32], i32),
        "tnmc_get_build_variant": ([vp], i32),
        "tnmc_autotune_build": ([vp, vp, i32, vp, vp, vp], i32),
        "tnmc_observables": ([vp, i32, vp, vp, vp, vp], i32),
        "tnmc_mh_step": ([vp, i32, u64, u64, vp, vp, vp, vp, vp, vp, vp, vp], i32),
        "tnmc_set_diagnostics": ([vp, vp, vp, vp], i32),
        "tnmc_get_device_status": ([vp, vp, i32], i32),
        "tnmc_propose_static": ([vp, i32, u64, u64, vp, vp, vp], i32),
        "tnmc_propose_static_limit": ([], sz),
        "tnmc_set_correction": ([vp, vp, i32], i32),
        "tnmc_mlp_features": ([vp, i32, vp, vp, vp], i32),
        "tnmc_mlp_scratch_floats": ([], sz),
        "tnmc_mlp_grad": ([vp, vp, ctypes.c_int64, i32, u64, i32, vp, vp, vp, vp, vp], i32),
        "tnmc_mlp_adam": ([vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, vp, vp], i32),
        "tnmc_mlp_pack": ([vp, vp, vp], i32),
        "tnmc_mlp_forward": ([vp, ctypes.c_int64, vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load_library().tnmc_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != 0:
        raise TnmcError(status, what)


def _cfg(Ls: Sequence[int], chi: int, beta: float, prec: int, max_samples: int, cutoff: float = 0.0,
         ckpt_every: int = 0, q: int = 2):
    arr = (ctypes.c_int32 * len(Ls))(*[int(x) for x in Ls])
    cfg = _Config(len(Ls), ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)), int(chi),
                  float(beta), int(prec), int(max_samples), float(cutoff), int(ckpt_every), int(q))
    return cfg, arr


def workspace_size(Ls, chi, beta, prec, max_samples, cutoff=0.0, ckpt_every=0, q=2) -> int:
    lib = load_library()
    cfg, keep = _cfg(Ls, chi, beta, prec, max_samples, cutoff, ckpt_every, q)
    out = ctypes.c_size_t(0)
    _check(lib.tnmc_workspace_size(ctypes.byref(cfg), ctypes.byref(out)), "tnmc_workspace_size")
    return out.value


def layout_info(Ls, chi, beta, prec, max_samples, ckpt_every=0):
    lib = load_library()
    cfg, keep = _cfg(Ls, chi, beta, prec, max_samples, 0.0, ckpt_every)
    a, b, c = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib.tnmc_layout_info(ctypes.byref(cfg), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "tnmc_layout_info")
    return a.value, b.value, c.value


def _on_stream(fn):
    """Run a method with the object's stream current: the buffers it allocates or fills
    are then ordered with the library's launches on that stream, and the caching
    allocator reuses them only after the work queued there (stream-ordered reuse).

    When the caller's current stream is another one, the object's stream first waits
    for the work queued on the caller's stream (inputs made there are complete before
    the library reads them), and the caller's stream then waits for the library's work
    (outputs are complete before the caller reads or frees them). Under stream capture
    the caller orders its streams itself (cross-stream waits would join the capture)."""
    @functools.wraps(fn)
    def wrapped(self, *args, **kwargs):
        cuda = self.torch.cuda
        cur = cuda.current_stream(self.device)
        other = cur != self.stream and not cuda.is_current_stream_capturing()
        if other:
            self.stream.wait_stream(cur)
        with cuda.stream(self.stream):
            out = fn(self, *args, **kwargs)
        if other:
            cur.wait_stream(self.stream)
        return out
    return wrapped


def _ptr(t) -> int:
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Proposals:
    spins: "object"   # torch.uint8 [sum_n S L_n^2]
    logq: "object"    # torch.float64 [n_real, S]
    E: "object"       # torch.float64 [n_real, S]
    S: int
    prop_base: int


@dataclass
class ChainState:
    spins: "object"   # torch.uint8 [sum_n L_n^2]
    logq: "object"    # torch.float64 [n_real]
    E: "object"       # torch.float64 [n_real]
    n_accept: "object"  # torch.int64 [n_real]


class TNMC:
    """A handle on the library for one batch of realizations on one CUDA device."""

    DEFAULT_CUTOFF = {TNMC_FP64: 1e-12, TNMC_FP32: 1e-6, TNMC_MIXED: 1e-12, TNMC_DFLOAT: 1e-12,
                      TNMC_TF32: 1e-6, TNMC_BF16: 1e-6}

    def __init__(self, Ls: Sequence[int], chi: int, beta: float, prec: str | int = "fp32",
                 max_samples: int = 256, device="cuda:0", stream=None, cutoff: float = 0.0,
                 ckpt_every: int = 0, q: int = 2):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("TNMC needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.torch = torch
        self.Ls = [int(x) for x in Ls]
        self.chi, self.beta = int(chi), float(beta)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.max_samples = int(max_samples)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n_real = len(self.Ls)
        self.sum_L2 = sum(L * L for L in self.Ls)
        self.cutoff = float(cutoff) if cutoff > 0 else self.DEFAULT_CUTOFF.get(self.prec, 1e-6)
        self.ckpt_every = int(ckpt_every)
        self.q = int(q)   # 2: Ising; 3 or 4: the q-state Potts extension (states 0 .. q-1 per byte)
        self.plan_ch = next((c for c in (8, 16, 32, 64) if self.chi <= c), 0)   # kernel instantiation
        self._cfg, self._cfg_keep = _cfg(self.Ls, chi, beta, self.prec, max_samples, self.cutoff,
                                         self.ckpt_every, self.q)
        nbytes = ctypes.c_size_t(0)
        _check(self.lib.tnmc_workspace_size(ctypes.byref(self._cfg), ctypes.byref(nbytes)),
               "tnmc_workspace_size")
        self.ws_bytes = nbytes.value
        with torch.cuda.stream(self.stream):
            self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        h = ctypes.c_void_p(0)
        _check(self.lib.tnmc_create(ctypes.byref(self._cfg), ctypes.c_void_p(self._ws_ptr),
                                    self.ws_bytes, ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), "tnmc_create")
        self.h = h
        self._diag = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.tnmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    @_on_stream
    def build_envs(self, J):
        """J: float32 device tensor (sum L^2, 4) in the paper's (left, up, right, down) layout."""
        assert J.dtype == self.torch.float32 and J.is_cuda and J.is_contiguous()
        assert J.numel() == 4 * self.sum_L2
        self._J_keep = J
        _check(self.lib.tnmc_build_envs(self.h, _ptr(J)), "tnmc_build_envs")

    @_on_stream
    def log_z(self, out=None):
        out = out if out is not None else self.torch.empty(self.n_real, dtype=self.torch.float64, device=self.device)
        _check(self.lib.tnmc_log_z(self.h, _ptr(out)), "tnmc_log_z")
        return out

    @_on_stream
    def alloc_proposals(self, S: int, prop_base: int = 0) -> Proposals:
        t = self.torch
        return Proposals(t.empty(S * self.sum_L2, dtype=t.uint8, device=self.device),
                         t.empty((self.n_real, S), dtype=t.float64, device=self.device),
                         t.empty((self.n_real, S), dtype=t.float64, device=self.device), S, prop_base)

    @_on_stream
    def propose(self, S: int, seed: int, prop_base: int = 0, out: Optional[Proposals] = None) -> Proposals:
        out = out if out is not None else self.alloc_proposals(S, prop_base)
        out.S, out.prop_base = S, prop_base
        _check(self.lib.tnmc_propose(self.h, int(S), int(seed), int(prop_base), _ptr(out.spins),
                                     _ptr(out.logq), _ptr(out.E)), "tnmc_propose")
        return out

    @_on_stream
    def propose_static(self, S: int, seed: int, prop_base: int = 0, out: Optional[Proposals] = None) -> Proposals:
        """tnmc_propose with the library's fixed scratch array (no workspace scratch needed)."""
        out = out if out is not None else self.alloc_proposals(S, prop_base)
        out.S, out.prop_base = S, prop_base
        _check(self.lib.tnmc_propose_static(self.h, int(S), int(seed), int(prop_base), _ptr(out.spins),
                                            _ptr(out.logq), _ptr(out.E)), "tnmc_propose_static")
        return out

    @_on_stream
    def score(self, spins, S: int):
        t = self.torch
        lq = t.empty((self.n_real, S), dtype=t.float64, device=self.device)
        E = t.empty((self.n_real, S), dtype=t.float64, device=self.device)
        _check(self.lib.tnmc_score(self.h, int(S), _ptr(spins), _ptr(lq), _ptr(E)), "tnmc_score")
        return lq, E

    @_on_stream
    def mh_init(self, seed: int) -> ChainState:
        t = self.torch
        st = ChainState(t.empty(self.sum_L2, dtype=t.uint8, device=self.device),
                        t.empty(self.n_real, dtype=t.float64, device=self.device),
                        t.empty(self.n_real, dtype=t.float64, device=self.device),
                        t.zeros(self.n_real, dtype=t.int64, device=self.device))
        _check(self.lib.tnmc_mh_init(self.h, int(seed), _ptr(st.spins), _ptr(st.logq), _ptr(st.E)),
               "tnmc_mh_init")
        return st

    @_on_stream
    def mh_init_empty(self) -> ChainState:
        """A chain without a configuration: the first proposal of the next mh_step is accepted."""
        t = self.torch
        st = ChainState(t.empty(self.sum_L2, dtype=t.uint8, device=self.device),
                        t.empty(self.n_real, dtype=t.float64, device=self.device),
                        t.empty(self.n_real, dtype=t.float64, device=self.device),
                        t.zeros(self.n_real, dtype=t.int64, device=self.device))
        _check(self.lib.tnmc_mh_init_empty(self.h, _ptr(st.spins), _ptr(st.logq), _ptr(st.E)),
               "tnmc_mh_init_empty")
        return st

    @_on_stream
    def mh_step(self, props: Proposals, state: ChainState, seed: int, accept=None):
        t = self.torch
        acc = accept if accept is not None else t.empty((self.n_real, props.S), dtype=t.uint8, device=self.device)
        _check(self.lib.tnmc_mh_step(self.h, int(props.S), int(seed), int(props.prop_base),
                                     _ptr(props.spins), _ptr(props.logq), _ptr(props.E),
                                     _ptr(state.spins), _ptr(state.logq), _ptr(state.E), _ptr(acc),
                                     _ptr(state.n_accept)), "tnmc_mh_step")
        return acc

    @_on_stream
    def set_diagnostics(self, S: int = 0, logits: bool = False, spectra: bool = False, rowinfo: bool = False):
        """Allocate and register the optional diagnostic outputs (None disables)."""
        t = self.torch
        lg = t.zeros(S * self.sum_L2, dtype=t.float32, device=self.device) if logits else None
        sp = t.zeros(sum(L * (L + 1) for L in self.Ls) * self.chi, dtype=t.float64, device=self.device) if spectra else None
        ri = t.zeros(sum(self.Ls) * 14, dtype=t.float64, device=self.device) if rowinfo else None
        self._diag = (lg, sp, ri)
        z = ctypes.c_void_p(0)
        _check(self.lib.tnmc_set_diagnostics(self.h, _ptr(lg) if lg is not None else z,
                                             _ptr(sp) if sp is not None else z,
                                             _ptr(ri) if ri is not None else z), "tnmc_set_diagnostics")
        return self._diag

    @_on_stream
    def set_correction(self, params_bf16=None):
        """Use the learned correction (a bfloat16 parameter tensor, see MLP) or stop (None)."""
        if params_bf16 is None:
            _check(self.lib.tnmc_set_correction(self.h, ctypes.c_void_p(0), 0), "tnmc_set_correction")
            self._corr_keep = None
            return
        assert params_bf16.is_cuda and params_bf16.numel() == MLP_PARAMS and params_bf16.element_size() == 2
        self._corr_keep = params_bf16
        _check(self.lib.tnmc_set_correction(self.h, _ptr(params_bf16), 1), "tnmc_set_correction")

    @_on_stream
    def score_logits(self, spins, S: int):
        """Teacher-forced (log q, E, logits) of S configurations per realization."""
        t = self.torch
        saved = self._diag
        lg = t.empty(S * self.sum_L2, dtype=t.float32, device=self.device)
        z = ctypes.c_void_p(0)
        _check(self.lib.tnmc_set_diagnostics(self.h, _ptr(lg), z, z), "tnmc_set_diagnostics")
        try:
            lq, E = self.score(spins, S)
        finally:
            if saved is None:
                self.lib.tnmc_set_diagnostics(self.h, z, z, z)
            else:
                self.lib.tnmc_set_diagnostics(self.h, *[_ptr(x) if x is not None else z for x in saved])
        return lq, E, lg

    @_on_stream
    def mlp_features(self, spins, logits, S: int):
        """Training features (sum_n S L_n^2, 8) of S configurations per realization."""
        t = self.torch
        feat = t.empty((S * self.sum_L2, MLP_FEAT_STRIDE), dtype=t.float32, device=self.device)
        _check(self.lib.tnmc_mlp_features(self.h, int(S), _ptr(spins), _ptr(logits), _ptr(feat)),
               "tnmc_mlp_features")
        return feat

    @_on_stream
    def observables(self, props: Proposals):
        """Per realization (n_real, 6): IS log Z, ESS, E/N, <q^2>, <q^4>, Binder ratio."""
        t = self.torch
        out = t.empty((self.n_real, 6), dtype=t.float64, device=self.device)
        _check(self.lib.tnmc_observables(self.h, int(props.S), _ptr(props.spins), _ptr(props.logq),
                                         _ptr(props.E), _ptr(out)), "tnmc_observables")
        return out

    def set_realization_ids(self, ids=None):
        """Stream ids of the realizations (their indices in the whole set when this handle
        holds a shard of it); None restores 0 .. n_real-1."""
        import numpy as np
        if ids is None:
            _check(self.lib.tnmc_set_realization_ids(self.h, ctypes.c_void_p(0)), "tnmc_set_realization_ids")
            return
        arr = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
        assert arr.shape == (self.n_real,)
        _check(self.lib.tnmc_set_realization_ids(self.h, arr.ctypes.data_as(ctypes.c_void_p)),
               "tnmc_set_realization_ids")

    def set_build_variant(self, variant: int):
        """Kernel layout of the environment build (see include/tnmc.h)."""
        _check(self.lib.tnmc_set_build_variant(self.h, int(variant)), "tnmc_set_build_variant")

    @property
    def build_variant(self) -> int:
        return int(self.lib.tnmc_get_build_variant(self.h))

    @_on_stream
    def autotune(self, J, rows: int = 12):
        """Time the candidate build layouts on `rows` rows below the middle of these lattices
        (rebuilt from the cached row under them; the rows beneath are built first unless the
        handle is built) and keep the fastest; returns {variant: ms}. Build again before
        proposing."""
        import numpy as np
        assert J.dtype == self.torch.float32 and J.is_cuda and J.is_contiguous()
        cap = 16
        var = np.zeros(cap, np.int32)
        ms = np.zeros(cap, np.float32)
        n = ctypes.c_int32(cap)
        self._J_keep = J
        _check(self.lib.tnmc_autotune_build(self.h, _ptr(J), int(rows), var.ctypes.data_as(ctypes.c_void_p),
                                            ms.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)),
               "tnmc_autotune_build")
        return {int(v): float(t) for v, t in zip(var[:n.value], ms[:n.value])}

    def set_wait_budget(self, cycles: int):
        """Budget of the bounded device waits in SM cycles (0 = default, ~20 s)."""
        _check(self.lib.tnmc_set_wait_budget(self.h, int(cycles)), "tnmc_set_wait_budget")

    def device_status(self, clear: bool = True):
        """(status code, per-realization flags) after synchronising the stream."""
        import numpy as np
        flags = np.zeros(self.n_real, dtype=np.int32)
        st = self.lib.tnmc_get_device_status(self.h, flags.ctypes.data_as(ctypes.c_void_p), int(bool(clear)))
        return st, flags

    # ------------------------------------------------------------------ helpers
    def spin_offsets(self, S: int) -> List[int]:
        """Start of each realization's block in a spins array holding S configurations each."""
        offs, o = [], 0
        for L in self.Ls:
            offs.append(o)
            o += S * L * L
        return offs


class MLP:
    """Parameters, Adam state and buffers of the learned proposal correction on one device.

    ``params`` is the float32 master copy, ``bf16`` the bfloat16 copy the sampler reads.
    """

    def __init__(self, device="cuda:0", stream=None, seed: int = 0):
        import numpy as np
        import torch
        self.lib = load_library()
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        # W1, W2 ~ N(0, 1/fan_in); biases and the output layer zero, so Delta starts at 0
        rng = np.random.default_rng(seed)
        host = np.zeros(MLP_PARAMS, np.float32)
        W1 = np.zeros((64, 16), np.float32)
        W1[:, :7] = rng.standard_normal((64, 7)) / np.sqrt(7.0)
        host[0:1024] = W1.reshape(-1)
        host[1088:5184] = (rng.standard_normal((64, 64)) / 8.0).reshape(-1)
        with torch.cuda.stream(self.stream):
            self.params = torch.from_numpy(host).to(self.device)
            self.m = torch.zeros_like(self.params)
            self.v = torch.zeros_like(self.params)
            self.grad_buf = torch.zeros_like(self.params)
            self.loss_buf = torch.zeros(1, dtype=torch.float64, device=self.device)
            self.scratch = torch.empty(int(self.lib.tnmc_mlp_scratch_floats()), dtype=torch.float32,
                                       device=self.device)
            self.bf16 = torch.empty(MLP_PARAMS, dtype=torch.bfloat16, device=self.device)
        self.step = 0
        self.pack()

    def _s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    @_on_stream
    def load(self, params_f32):
        """Set the master copy (float32 tensor or array of MLP_PARAMS values) and its bfloat16 copy."""
        t = self.torch
        self.params.copy_(t.as_tensor(params_f32, dtype=t.float32))
        self.pack()

    @_on_stream
    def pack(self):
        _check(self.lib.tnmc_mlp_pack(_ptr(self.params), _ptr(self.bf16), self._s()), "tnmc_mlp_pack")

    @_on_stream
    def grad(self, feat, target_logit, batch: int = 0, seed: int = 0, step: int = 0):
        """(gradient, loss) tensors of the mean BCE; batch 0 = every row in order."""
        n = feat.shape[0]
        _check(self.lib.tnmc_mlp_grad(_ptr(feat), _ptr(target_logit), int(n), int(batch), int(seed),
                                      int(step), _ptr(self.bf16), _ptr(self.grad_buf),
                                      _ptr(self.loss_buf), _ptr(self.scratch), self._s()),
               "tnmc_mlp_grad")
        return self.grad_buf, self.loss_buf

    @_on_stream
    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.step += 1
        _check(self.lib.tnmc_mlp_adam(_ptr(self.params), _ptr(self.m), _ptr(self.v),
                                      _ptr(self.grad_buf), self.step, lr, beta1, beta2, eps,
                                      _ptr(self.bf16), self._s()), "tnmc_mlp_adam")

    @_on_stream
    def train(self, feat, target_logit, steps: int, batch: int, lr: float, seed: int = 0,
              lr_final: float | None = None):
        """Adam on minibatches drawn on the device; returns the loss of every step (tensor)."""
        t = self.torch
        losses = t.empty(steps, dtype=t.float64, device=self.device)
        for k in range(steps):
            rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, steps - 1))
            self.grad(feat, target_logit, batch, seed, self.step + 1)
            losses[k:k + 1].copy_(self.loss_buf)
            self.adam(rate)
        return losses

    @_on_stream
    def forward(self, feat):
        """Delta of every feature row by the tensor-core network the sampler uses."""
        t = self.torch
        out = t.empty(feat.shape[0], dtype=t.float32, device=self.device)
        _check(self.lib.tnmc_mlp_forward(_ptr(feat), int(feat.shape[0]), _ptr(self.bf16), _ptr(out),
                                         self._s()), "tnmc_mlp_forward")
        return out
