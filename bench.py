"""Benchmark of the batched TNMC hot path on B300 (one JSON line on stdout).

A step is one pass of the whole hot path over one batch: coupling ingest and
the boundary-MPS environments of every realization, S proposals per
realization with log q and energies, and the independence Metropolis-Hastings
scan (Sec. 3.2-3.4, Eq. 10). Default workload: 64 +-J realizations at L = 256,
beta = 3, chi = 64, S = 256 (the accepted-samples/s workload).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|fp32|mixed|dfloat|tf32|bf16]
                    [--impl ours|reference] [--workload L256|gauss128|L1024|...]
                    [--learned [--teacher-chi 32] [--train-steps 4000]] [--ckpt K]

--learned trains the learned proposal correction before the timed region (on
configurations of a chi = teacher-chi handle and both handles' conditionals)
and times steps whose proposals carry the correction; the line reports the
training time and the plain / corrected / teacher acceptance.

Under torchrun (N > 1) the realization set grows with N (weak scaling): N times
the workload's realizations, realization g drawn from seed 1000 + g, split over
the ranks by longest-processing-time-first on the build cost
(paper_2509_19006_b300.shard); each rank's handle names its realizations by g,
so their random numbers do not depend on N. No collective touches the data
path; the per-realization log Z and accepted counts are gathered at the end and
rank 0 prints the line with the whole-job throughput (the slowest rank's time).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import SAMPLING_SEED, config  # noqa: E402

def metric_name(wl) -> str:
    return (f"accepted samples/s at L={wl.Ls[0]},chi={wl.chi} "
            "(end to end: environments + proposals + MH)")
# Acceptance of the float64-accurate method at each workload, measured on the GPU (the
# oracle computes the same method; its own MH at these sizes would take hours). Both
# oracle legs (cpu_baseline and --impl reference) credit this value; a workload without
# an entry is credited acceptance 1 (an upper bound on the oracle's throughput).
REF_ACCEPTANCE = {
    "L256_chi64_beta3_n64_S256": 0.205,        # float64 and double-float: 0.202-0.206
    "uneven200_L32-128_chi32_beta2": 0.997,    # mixed 0.997, double-float 0.998
    "L1024_chi32_beta3_n64_S128": 0.034,       # double-float
}
# float32 instructions of one double-float multiply-add as the kernels implement it
# (TwoProd 2, two cross-term FMAs 2, two TwoSums 12, two FastTwoSums 6, two adds 2)
DF_FMA_OPS = 24


def measure_alu_peaks(dev):
    """Dense GEMM rates of this GPU in float64 and float32 (cuBLAS through torch, TF32
    off): the measured ALU ceilings the environment build is compared with, in GFLOP/s."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n, reps in (("fp64", torch.float64, 4096, 3), ("fp32", torch.float32, 8192, 5)):
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            torch.matmul(a, b)
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e9
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def workload_config(wl, world: int) -> dict:
    """The workload keys of the line's `config` object, the same in both arms' lines."""
    return {"workload": wl.name, "L": wl.Ls[0], "chi": wl.chi, "beta": wl.beta,
            "realizations_per_gpu": wl.n_real, "realizations": world * wl.n_real,
            "samples_per_realization": wl.S, "q_states": wl.q}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------- oracle arm
# Mean bond dimension over all rows of the oracle's own full build of realization 0 of
# the L = 256 workload (468 s on 8 threads): the bottom rows that a bounded sample can
# time have smaller bonds, so their per-row cost is scaled by (D_all / D_timed)^3 (the
# SVD cost). On that full build the model gives 345 s against the measured 468 s: the
# extrapolated oracle is still credited with 1.36x its real speed.
ORACLE_MEAN_BOND = {"L256_chi64_beta3_n64_S256": 43.31}


def oracle_sample(wl, seconds: float = 15.0):
    """Time the FP64 oracle on a bounded sample of the workload.

    One realization per distinct L (the first of that size), `seconds` shared evenly
    between them: its environment rows are built from the bottom up until its share
    has elapsed; the per-row cost of the last half of those rows is extrapolated to all
    L rows, scaled by (D_all / D_timed)^3 where the workload's all-row mean bond
    dimension D_all is known (ORACLE_MEAN_BOND). The sizes' times are averaged with the
    workload's count of each size. Proposals are not timed: the environment build
    dominates the oracle's time, so this is an upper bound on its throughput. Returns
    (mean seconds per realization, rows timed, wall s, mean bond of the timed rows of
    the first size).
    """
    t0 = time.perf_counter()
    sizes = sorted(set(wl.Ls), key=wl.Ls.index)
    total, rows, d0 = 0.0, 0, None
    for L in sizes:
        t_real, r, d = _oracle_realization(wl, wl.Ls.index(L), seconds / len(sizes))
        total += t_real * wl.Ls.count(L)
        rows += r
        d0 = d if d0 is None else d0
    return total / wl.n_real, rows, time.perf_counter() - t0, d0


def _oracle_realization(wl, n, seconds):
    from oracle import bmps, potts
    L, chi, beta = wl.Ls[n], wl.chi, wl.beta
    Jh, Jv = wl.realization(n)
    t0 = time.perf_counter()
    if wl.q > 2:
        bottom = lambda Jh_row: potts.bottom_row_mps(Jh_row, beta, wl.q)
        row_mpo = lambda Jh_row, Jv_row: potts.row_mpo(Jh_row, Jv_row, beta, wl.q)
    else:
        bottom = lambda Jh_row: bmps.bottom_row_mps(Jh_row, beta)
        row_mpo = lambda Jh_row, Jv_row: bmps.row_mpo(Jh_row, Jv_row, beta)
    mps, lam = bottom(Jh[L - 1])
    times, dims = [], []
    for r in range(L - 1, -1, -1):
        ts = time.perf_counter()
        if r < L - 1:
            mpo, sc = row_mpo(Jh[r], Jv[r])
            mps = bmps.multiply(mpo, mps)
        mps = bmps.compress(mps, chi)[0]
        times.append(time.perf_counter() - ts)
        dims.append(float(np.mean([A.shape[2] for A in mps[:-1]])) if L > 1 else 1.0)
        if time.perf_counter() - t0 > seconds and len(times) >= 4:
            break
    half = len(times) // 2
    per_row = sum(times[half:]) / len(times[half:])
    d_timed = float(np.mean(dims[half:]))
    d_all = ORACLE_MEAN_BOND.get(wl.name)
    if d_all:
        per_row *= (d_all / d_timed) ** 3
    return per_row * L, len(times), d_timed


def ref_acceptance(args, wl):
    if args.ref_acceptance is not None:
        return args.ref_acceptance
    return REF_ACCEPTANCE.get(wl.name, 1.0)


def oracle_sample_text(wl, rows_done, d_timed, acceptance):
    d_all = ORACLE_MEAN_BOND.get(wl.name)
    scale = (f", scaled by (D_all / D_timed)^3 = ({d_all} / {d_timed:.1f})^3 for the larger bonds of "
             f"the rows above (D_all: the oracle's own full build)" if d_all else "")
    sizes = sorted(set(wl.Ls))
    which = ("realization 0" if len(sizes) == 1 else
             f"one realization per size L in {sizes} (weighted by the count of each size)")
    acc = (f"acceptance {acceptance} (the float64-accurate method's at this workload, measured on "
           f"the GPU: the oracle cannot run its own MH at this size)" if wl.name in REF_ACCEPTANCE
           else f"acceptance {acceptance} assumed (an upper bound)")
    return (f"{which} of {wl.name}: bottom {rows_done} environment rows timed, per-row cost "
            f"extrapolated to all rows{scale}; proposals not timed; {acc}")


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        oracle_sample(wl, seconds=args.ref_seconds / 3)
    for _ in range(args.steps):
        t_real, rows_done, wall, d_timed = oracle_sample(wl, seconds=args.ref_seconds)
        # the oracle computes the same method; its acceptance is the method's (given)
        vals.append(wl.S * ref_acceptance(args, wl) / t_real)
    v = float(np.mean(vals))
    sample = oracle_sample_text(wl, rows_done, d_timed, ref_acceptance(args, wl))
    line = {"impl": "reference", "metric": metric_name(wl), "value": v, "unit": "accepted/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, world),
            "cpu_baseline": {"value": v, "unit": "accepted/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "accepted/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------- our arm
def train_correction(P, t, J, wl, args, dev):
    """Train the learned correction of handle t (setup, outside the timed region).

    Data: S configurations per realization drawn by a chi = args.teacher_chi
    handle, scored by both handles (their conditional logits); the network is
    trained on t's features against the teacher's logits, then installed in t.
    Returns the training summary, with plain / corrected / teacher acceptance
    of one extra MH pass each.
    """
    import torch
    S = wl.S
    t0 = time.perf_counter()
    teacher = P.TNMC(t.Ls, args.teacher_chi, wl.beta, args.prec, max_samples=S, device=dev,
                     cutoff=args.cutoff)
    t.build_envs(J)
    teacher.build_envs(J)
    props = teacher.propose(S, 7, 0)
    _, _, lg_s = t.score_logits(props.spins, S)
    _, _, lg_b = teacher.score_logits(props.spins, S)
    feat = t.mlp_features(props.spins, lg_s, S)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = P.MLP(device=dev, stream=t.stream, seed=3)
    t1 = time.perf_counter()
    net.train(feat, lg_b, steps=args.train_steps, batch=65536, lr=3e-3, lr_final=3e-4, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1

    def acceptance(h, corr):
        """Accept rate of a second round of S proposals per chain (the first round starts it)."""
        h.set_correction(corr)
        st = h.mh_init_empty()
        pr = h.propose(S, 11, 5_000_000)
        h.mh_step(pr, st, 11)
        n0 = st.n_accept.sum().item()
        pr = h.propose(S, 11, 5_000_000 + S)
        h.mh_step(pr, st, 11)
        torch.cuda.synchronize()
        return (st.n_accept.sum().item() - n0) / (S * h.n_real)

    a_plain = acceptance(t, None)
    a_teacher = acceptance(teacher, None)
    a_corr = acceptance(t, net.bf16)
    del feat, lg_s, lg_b, props, teacher
    torch.cuda.empty_cache()
    t.set_correction(net.bf16)
    t._net_keep = net
    return {"teacher_chi": args.teacher_chi, "train_steps": args.train_steps, "batch": 65536,
            "examples": S * sum(L * L for L in t.Ls),
            "data_s": t_data, "train_s": t_train,
            "acceptance_plain": a_plain, "acceptance_corrected": a_corr,
            "acceptance_teacher": a_teacher}


def run_arm(P, gw, ids, args, prec, steps, dev):
    """One precision timed on the same realizations (the headline comparison of the metric:
    plain float64 against the mixed-precision form): `steps` full steps (ingest,
    environments, log Z, S proposals, MH), each bracketed by CUDA events on the handle's
    stream after an L2 flush. Chains start at the first proposal of the first step; the
    acceptance counts only the MH decisions after that forced first acceptance."""
    import torch
    S = gw.S
    my_Ls = [gw.Ls[g] for g in ids]
    n = len(ids)
    J = torch.from_numpy(gw.packed_J(ids)).to(dev)
    t = P.TNMC(my_Ls, gw.chi, gw.beta, prec, max_samples=S, device=dev)
    t.set_realization_ids(ids)
    tune = t.autotune(J, rows=args.tune_rows) if args.tune_rows > 0 else {}
    props = t.alloc_proposals(S)
    acc = torch.empty((n, S), dtype=torch.uint8, device=dev)
    logz = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    _, _, rowinfo = t.set_diagnostics(rowinfo=True)
    state = t.mh_init_empty()
    stream = t.stream
    step_ms, env_ms, accepted, decided, by_step = [], [], 0, 0, []
    for k in range(steps):
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            t.build_envs(J)
            e1.record(stream)
            t.log_z(out=logz)
            t.propose(S, SAMPLING_SEED, 30_000_000 * (k + 1), out=props)
            t.mh_step(props, state, SAMPLING_SEED, accept=acc)
            e2.record(stream)
        torch.cuda.synchronize()
        a = int(acc.sum().item())
        if k == 0:
            a -= n                      # the forced first acceptance of every chain
            d = n * (S - 1)
        else:
            d = n * S
        accepted += a
        decided += d
        by_step.append(a / d)
        step_ms.append(e0.elapsed_time(e2))
        env_ms.append(e0.elapsed_time(e1))
        if k == 0:
            dmean = float(rowinfo.cpu().numpy().reshape(-1, 14)[:, 5].mean())
            t.set_diagnostics()
    st, _ = t.device_status()
    step_s = sum(step_ms) / len(step_ms) / 1e3
    acceptance = accepted / decided
    out = {"precision": prec, "steps": steps, "step_s": step_s,
           "env_build_s": sum(env_ms) / len(env_ms) / 1e3, "acceptance": acceptance,
           "acceptance_by_step": by_step,   # step k: the same proposal ids and seed in every arm
           "accepted_per_s": acceptance * n * S / step_s, "proposals_per_s": n * S / step_s,
           "cutoff": t.cutoff, "bond_dim_mean": dmean, "device_status": int(st),
           "build_variant": t.build_variant, "autotune_ms": tune}
    del t, J, props, acc, logz, flush, state, rowinfo
    torch.cuda.empty_cache()
    return out


def run_ours(args, wl):
    import torch
    import paper_2509_19006_b300 as P

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # weak scaling over one realization set: world x the workload's realizations,
    # split by LPT; realization g keeps its seed and random-number stream at any world size
    from paper_2509_19006_b300 import shard
    from workloads import Workload
    n_all = world * wl.n_real
    gw = Workload(wl.name, [wl.Ls[g % wl.n_real] for g in range(n_all)], wl.beta, wl.chi, wl.S,
                  kind=wl.kind, base_seed=wl.base_seed, p=wl.p, q=wl.q)
    ids = shard.lpt_partition(gw.Ls, gw.chi, world)[rank]
    my_Ls = [gw.Ls[g] for g in ids]
    peaks_alu = measure_alu_peaks(dev)
    Jhost = torch.from_numpy(gw.packed_J(ids)).pin_memory()
    J = Jhost.to(dev)
    S = wl.S
    if args.ckpt >= 0:
        ckpt = args.ckpt
    else:
        # checkpoints only where the full cache does not fit: its workspace against 60 % of the
        # device's free memory (the proposals, at L = 1024 17 GB of spins, need room beside it)
        full = P.workspace_size(my_Ls, wl.chi, wl.beta, P.PRECISIONS[args.prec], S,
                                cutoff=args.cutoff, q=wl.q)
        ckpt = 0 if full <= 0.6 * torch.cuda.mem_get_info(dev)[0] else 32
    t = P.TNMC(my_Ls, wl.chi, wl.beta, args.prec, max_samples=S, device=dev, cutoff=args.cutoff,
               ckpt_every=ckpt, q=wl.q)
    t.set_realization_ids(ids)
    n_mine = len(ids)
    # the build layout: the autotuner times the candidates on the bottom rows of these
    # realizations (setup, outside the timed region)
    # (the Potts build has one layout: nothing to tune)
    tune = t.autotune(J, rows=args.tune_rows) if args.tune_rows > 0 and wl.q == 2 else {}
    stream = t.stream
    learned = None
    if args.learned:
        learned = train_correction(P, t, J, wl, args, dev)
    props = t.alloc_proposals(S)
    state = None
    acc = torch.empty((n_mine, S), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (126 MB)
    logz = torch.empty(n_mine, dtype=torch.float64, device=dev)

    def step(base):
        nonlocal state
        t.build_envs(J)
        t.log_z(out=logz)
        t.propose(S, SAMPLING_SEED, base, out=props)
        if state is None:
            # the chain starts at its first proposal: a uniformly random start can have
            # q = 0 in float32 arithmetic (an unlikely forced spin's conditional cancels to 0)
            state = t.mh_init_empty()
        t.mh_step(props, state, SAMPLING_SEED, accept=acc)

    # warm-up (the first one also gathers the algorithmic flop count of the build)
    _, _, rowinfo = t.set_diagnostics(rowinfo=True)
    for w in range(args.warmup):
        step(1_000_000 * (w + 1))
        if w == 0:
            torch.cuda.synchronize()
            ri = rowinfo.cpu().numpy().reshape(-1, 14)
            flops_env = float(ri[:, 13].sum())
            dmean = float(ri[:, 5].mean())
            t.set_diagnostics()
    torch.cuda.synchronize()
    st, flags = t.device_status()
    if st != 0:
        print(f"warning: device status {st}, flags {np.unique(flags)}", file=sys.stderr)

    # ---------------- device-resident timed region
    ev = lambda: torch.cuda.Event(enable_timing=True)
    env_ms, step_ms, prop_ms, samp_ms, accepted = [], [], [], [], 0
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n_acc0 = state.n_accept.clone()
    t_all0 = ev(); t_all1 = ev()
    with torch.cuda.stream(stream):
        t_all0.record(stream)
        for k in range(args.steps):
            flush.zero_()
            e0, e1, e2, e3, e4 = ev(), ev(), ev(), ev(), ev()
            e0.record(stream)
            t.build_envs(J)
            e1.record(stream)
            t.log_z(out=logz)
            e4.record(stream)
            t.propose(S, SAMPLING_SEED, 10_000_000 * (k + 1), out=props)
            e3.record(stream)
            t.mh_step(props, state, SAMPLING_SEED, accept=acc)
            e2.record(stream)
            env_ms.append((e0, e1))
            step_ms.append((e0, e2))
            prop_ms.append((e1, e3))
            samp_ms.append((e4, e3))
        t_all1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    accepted = int((state.n_accept - n_acc0).sum().item())
    env_t = [a.elapsed_time(b) for a, b in env_ms]
    prop_t = [a.elapsed_time(b) for a, b in prop_ms]
    samp_t = [a.elapsed_time(b) for a, b in samp_ms]
    step_t = [a.elapsed_time(b) for a, b in step_ms]
    total_ms = t_all0.elapsed_time(t_all1)   # includes the L2 flushes between steps
    my_ms = sum(step_t)

    per_real = torch.stack([logz.double(), (state.n_accept - n_acc0).double()], dim=1)

    # ---------------- end to end through the public API with host buffers
    # (a bounded number of steps: the same metric, its wall time and proposal count stated)
    e2e_steps = min(args.steps, args.e2e_steps)
    h_acc = torch.empty((n_mine, S), dtype=torch.uint8).pin_memory()
    h_nacc = torch.empty(n_mine, dtype=torch.int64).pin_memory()
    h_logz = torch.empty(n_mine, dtype=torch.float64).pin_memory()
    e2e_acc = 0
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(e2e_steps):
            n0 = state.n_accept.clone()
            J.copy_(Jhost, non_blocking=True)
            t.build_envs(J)
            t.log_z(out=logz)
            t.propose(S, SAMPLING_SEED, 20_000_000 * (k + 1), out=props)
            t.mh_step(props, state, SAMPLING_SEED, accept=acc)
            h_acc.copy_(acc, non_blocking=True)
            h_nacc.copy_(state.n_accept - n0, non_blocking=True)
            h_logz.copy_(logz, non_blocking=True)
            stream.synchronize()
            e2e_acc += int(h_nacc.sum())
    e2e_s = time.perf_counter() - w0
    h2d = Jhost.numel() * 4
    d2h = h_acc.numel() + h_nacc.numel() * 8 + h_logz.numel() * 8

    # ---------------- gather over ranks (max time, summed work, per-realization results)
    vec = torch.tensor([my_ms, float(accepted), e2e_s, float(e2e_acc)], dtype=torch.float64, device=dev)
    full = shard.gather(dist if world > 1 else None, n_all, ids, per_real, device=dev)
    if world > 1:
        mx = vec.clone(); dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = vec.clone(); dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        my_ms_all, accepted_all, e2e_s_all, e2e_acc_all = mx[0].item(), sm[1].item(), mx[2].item(), sm[3].item()
    else:
        my_ms_all, accepted_all, e2e_s_all, e2e_acc_all = my_ms, accepted, e2e_s, e2e_acc
    assert int(full[:, 1].sum().item()) == int(accepted_all)

    # ---------------- the headline comparison arms (one GPU; the primary handle is released
    # first: the float64-sized caches of the arms do not fit beside it)
    arms = []
    cutoff_primary, plan_ch, variant_primary = t.cutoff, t.plan_ch, t.build_variant
    if world == 1 and args.arms:
        del t, props, state, acc, logz, flush
        torch.cuda.empty_cache()
        for spec in args.arms.split(","):
            prec_a, steps_a = spec.split(":")
            arms.append(run_arm(P, gw, ids, args, prec_a, int(steps_a), dev))

    if rank == 0:
        peaks = load_peaks()
        env_avg_s = sum(env_t) / len(env_t) / 1e3
        samp_avg_s = sum(samp_t) / len(samp_t) / 1e3
        achieved = flops_env / env_avg_s / 1e9
        if args.prec in ("fp32", "tf32", "bf16"):
            # TF32 / BF16 move only the dense products to the tensor cores: the QR and Jacobi
            # steps that bound the build stay on the float32 pipe
            peak, peak_src = peaks_alu["fp32"], "measured: cuBLAS float32 GEMM (TF32 off) on this GPU"
        elif args.prec == "dfloat":
            # a double-float multiply-add (2 flops) is DF_FMA_OPS float32 instructions on the
            # FP32 pipe, whose rate the float32 GEMM measures (2 flops per instruction)
            peak = peaks_alu["fp32"] / DF_FMA_OPS
            peak_src = (f"derived: measured cuBLAS float32 GEMM rate / {DF_FMA_OPS} (float32 "
                        "instructions per double-float multiply-add)")
        else:
            peak, peak_src = peaks_alu["fp64"], "measured: cuBLAS float64 GEMM on this GPU"
        proposals = n_mine * S * args.steps
        # DRAM bytes per launch of the float32, chi = 64 build in its preconditioned 8-lane
        # layout (variant 40): an ncu capture of 8 realizations at L = 128 (131072 site-rows)
        # read + wrote 2.178 GB; traffic grows with the site-rows written
        site_rows = sum(L * L for L in my_Ls)
        if args.prec == "fp32" and plan_ch == 64 and not ckpt and variant_primary == 40:
            traffic = 2.178e9 / 131072 * site_rows
            traffic_src = "ncu capture at L=128 x 8 realizations (layout 40), scaled by site-rows"
        else:
            traffic, traffic_src = None, "no capture of this instantiation"
        # sampler: algorithmic bytes per sample-site = the right environment spilled and read
        # back (2 D values: L D values per chain do not fit on chip), the cache read once per
        # pass per realization (2 D^2 values, shared by the S chains) and the spin written
        esz = 4 if args.prec in ("fp32", "tf32", "bf16") else 8
        samp_sites = S * site_rows
        # (a Potts site is q dense D x D matrices, an Ising site one parity-form matrix)
        site_mats = wl.q if wl.q > 2 else 1
        samp_bytes = samp_sites * (2.0 * dmean * esz + 2.0 * site_mats * dmean * dmean * esz / S + 1.0)
        hbm_peak = peaks.get("hbm_gbs") or 6484.6
        cpu = None
        if world == 1 and args.cpu_baseline:
            t_real, rows_done, _, d_timed = oracle_sample(wl, seconds=args.ref_seconds)
            acc_ref = ref_acceptance(args, wl)
            cpu = {"value": S * acc_ref / t_real, "unit": "accepted/s", "cores": cpu_cores(),
                   "kind": "oracle",
                   "sample": "FP64 oracle, " + oracle_sample_text(wl, rows_done, d_timed, acc_ref)}
        line = {
            "metric": metric_name(wl),
            "value": accepted_all / (my_ms_all / 1e3),
            "unit": "accepted/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": my_ms_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f64 build + f32 sampling",
                      "tf32": "f32 (tensor-core products from tf32 operands)",
                      "bf16": "f32 (tensor-core products from bf16 operands)",
                      "dfloat": "f32x2 (double-float)"}[args.prec],
            "data": ("synthetic Gaussian N(0,1) disorder, seeded" if wl.kind == "gauss"
                     else "synthetic +-J disorder (p = 1/2), seeded")
                    + (f", {wl.q}-state Potts" if wl.q > 2 else ""),
            "config": {**workload_config(wl, world),
                       "precision": args.prec, "cutoff": cutoff_primary, "ckpt_every": ckpt,
                       "build_variant": variant_primary, "autotune_ms": tune,
                       "learned_correction": bool(args.learned),
                       "l2": "flushed (256 MB write) before every timed step; environment cache >> L2"},
            "acceptance": accepted / proposals,
            "proposals_per_s": proposals * world / (my_ms_all / 1e3),
            "env_build_ms": env_avg_s * 1e3,
            "step_breakdown_ms": {"env_build": env_avg_s * 1e3,
                                  "log_z_and_proposals": sum(prop_t) / len(prop_t),
                                  "mh": my_ms / args.steps - env_avg_s * 1e3 - sum(prop_t) / len(prop_t)},
            "bond_dim_mean": dmean,
            "roofline": {"kernel": "env_build_kernel (boundary-MPS build)", "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": traffic,
                         "traffic_source": traffic_src,
                         "algorithmic_flops_per_launch": flops_env},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_acc_all / e2e_s_all, "unit": "accepted/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "wall_s": e2e_s_all, "accepted": int(e2e_acc_all),
                    "proposals": n_all * S * e2e_steps},
            "roofline_sampling": {"kernel": "sample_kernel (proposals)", "bound": "hbm",
                                  "achieved": samp_bytes / samp_avg_s / 1e9, "peak": hbm_peak,
                                  "unit": "GB/s", "frac": samp_bytes / samp_avg_s / 1e9 / hbm_peak,
                                  "algorithmic_bytes_per_launch": samp_bytes,
                                  "launch_ms": samp_avg_s * 1e3},
            "alu_peaks_measured_gflops": peaks_alu,
            "per_realization": {"log_z_mean": float(full[:, 0].mean().item()),
                                "accepted_min": int(full[:, 1].min().item()),
                                "accepted_max": int(full[:, 1].max().item())},
            "gpu_launches": args.steps * (2 + 1 + 1 + 1 + (2 * ((max(wl.Ls) + ckpt - 1) // ckpt) - 1
                                                          if ckpt else 0)),
            "clocks": clk,
            "hbm_gbs_measured": peaks.get("hbm_gbs"),
        }
        if learned is not None:
            line["learned"] = learned
        if arms:
            by = {a["precision"]: a for a in arms}
            line["headline"] = {
                "what": ("the metric's comparison at this workload, measured in this run on the same "
                         "realizations: plain float64 against the mixed-precision (double-float) form; "
                         "accepted/s = acceptance x proposals / step time"),
                "arms": arms,
                "dfloat_over_fp64_accepted_per_s": (by["dfloat"]["accepted_per_s"] / by["fp64"]["accepted_per_s"]
                                                    if "dfloat" in by and "fp64" in by else None)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sweep(args):
    """Acceptance against system size, and the time of the paper's L=1024 configuration.

    For each (beta, chi) the paper quotes (Sec. 4: P_acc ~ 0.37 at L = 1024, beta = 1,
    chi = 8; comparable at beta = 1.5, chi = 16), 16 +-J realizations per L: the
    environments, a first round of S proposals that starts the chains (tnmc_mh_init_empty),
    and a measured round; one JSON line per (beta, chi, L). Then 64 realizations at
    L = 1024, beta = 1, chi = 8: one step (environments, S proposals, MH) timed with CUDA
    events, and the time it implies for 10^3 accepted samples in each of 10^3 realizations
    (the paper's single-GPU figure is 3.3 h, on its own hardware).
    """
    import torch
    import paper_2509_19006_b300 as P
    from workloads import Workload
    S = 256
    sizes = [int(x) for x in args.sweep_sizes.split(",")]
    for beta, chi in [(0.66, 4), (1.0, 8), (1.5, 16)]:
        for L in sizes:
            wl = Workload(f"sweep_L{L}", [L] * 16, beta, chi, S)
            J = torch.from_numpy(wl.packed_J()).cuda()
            t = P.TNMC(wl.Ls, chi, beta, args.prec, max_samples=S)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            t.build_envs(J)
            ev[1].record()
            st = t.mh_init_empty()
            t.mh_step(t.propose(S, SAMPLING_SEED, 0), st, SAMPLING_SEED)
            n0 = st.n_accept.clone()
            t.mh_step(t.propose(S, SAMPLING_SEED, S), st, SAMPLING_SEED)
            ev[2].record()
            torch.cuda.synchronize()
            acc = (st.n_accept - n0).cpu().numpy() / S
            print(json.dumps({"sweep": "acceptance", "beta": beta, "chi": chi, "L": L, "precision": args.prec,
                              "realizations": 16, "samples": S, "acceptance_mean": float(acc.mean()),
                              "acceptance_sem": float(acc.std() / np.sqrt(acc.size)),
                              "env_build_s": ev[0].elapsed_time(ev[1]) / 1e3,
                              "status": int(t.device_status()[0])}), flush=True)
            del t, J
            torch.cuda.empty_cache()
    # the paper's configuration at L = 1024
    L, beta, chi, n_real = 1024, 1.0, 8, 64
    wl = Workload("paper_L1024_beta1_chi8", [L] * n_real, beta, chi, S)
    J = torch.from_numpy(wl.packed_J()).cuda()
    t = P.TNMC(wl.Ls, chi, beta, args.prec, max_samples=S)
    st = t.mh_init_empty()
    t.build_envs(J)
    t.mh_step(t.propose(S, SAMPLING_SEED, 0), st, SAMPLING_SEED)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    n0 = st.n_accept.clone()
    ev[0].record()
    t.build_envs(J)
    ev[1].record()
    props = t.propose(S, SAMPLING_SEED, S)
    ev[2].record()
    t.mh_step(props, st, SAMPLING_SEED)
    ev[3].record()
    torch.cuda.synchronize()
    acc = float((st.n_accept - n0).sum().item()) / (S * n_real)
    env_s, prop_s, mh_s = (ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3,
                           ev[2].elapsed_time(ev[3]) / 1e3)
    step_s = env_s + prop_s + mh_s
    # 10^3 realizations x 10^3 accepted samples: environments once per realization,
    # proposals in rounds of S per realization until 10^3 are accepted
    waves = int(np.ceil(1000 / min(n_real, 148)))
    hours = (waves * env_s + 1000 * 1000 / acc / (S * n_real) * (prop_s + mh_s)) / 3600
    print(json.dumps({"sweep": "paper_configuration", "L": L, "beta": beta, "chi": chi,
                      "precision": args.prec, "realizations": n_real, "samples": S,
                      "acceptance": acc, "env_build_s": env_s, "proposals_s": prop_s, "mh_s": mh_s,
                      "accepted_per_s": acc * S * n_real / step_s,
                      "projected_hours_1000x1000": hours,
                      "projected_hours_1000x1000_proposals":
                          (waves * env_s + 1000 * 1000 / (S * n_real) * (prop_s + mh_s)) / 3600,
                      "paper_hours_1000x1000": 3.3, "status": int(t.device_status()[0])}), flush=True)


def run_nishimori(args):
    """Random-bond Ising model on the Nishimori line: +-J bonds antiferromagnetic with
    probability p, beta with
    exp(-2 beta) = p / (1 - p). Per (p, L), 32 realizations, S proposals each: the
    importance-sampling observables (tnmc_observables) averaged over disorder, with the
    exact identity [<E>] = -N_B (1 - 2p) as a check, and the IS log Z against the
    boundary-MPS log Z of the same environments.
    """
    import torch
    import paper_2509_19006_b300 as P
    from workloads import Workload
    S, n_real, chi = 256, 32, 16
    for p in (0.05, 0.1):
        beta = 0.5 * float(np.log((1.0 - p) / p))
        for L in (16, 32, 64):
            wl = Workload(f"nishimori_p{p}_L{L}", [L] * n_real, beta, chi, S, p=p, base_seed=9000)
            J = torch.from_numpy(wl.packed_J()).cuda()
            t = P.TNMC(wl.Ls, chi, beta, args.prec, max_samples=S)
            t.build_envs(J)
            lz = t.log_z().cpu().numpy()
            obs = t.observables(t.propose(S, SAMPLING_SEED, 0)).cpu().numpy()
            nb = 2 * L * (L - 1)
            e_bond = obs[:, 2] * L * L / nb
            sem = lambda x: float(np.std(x) / np.sqrt(x.size))
            print(json.dumps({"nishimori": True, "p": p, "beta": beta, "L": L, "chi": chi,
                              "precision": args.prec, "realizations": n_real, "samples": S,
                              "energy_per_bond": float(e_bond.mean()), "energy_per_bond_sem": sem(e_bond),
                              "energy_per_bond_exact": -(1 - 2 * p),
                              "q2": float(obs[:, 3].mean()), "q2_sem": sem(obs[:, 3]),
                              "binder": float(obs[:, 5].mean()), "binder_sem": sem(obs[:, 5]),
                              "ess_mean": float(obs[:, 1].mean()),
                              "is_minus_bmps_log_z": float((obs[:, 0] - lz).mean()),
                              "is_minus_bmps_log_z_sem": sem(obs[:, 0] - lz),
                              "status": int(t.device_status()[0])}), flush=True)
            del t, J
            torch.cuda.empty_cache()


def run_serial_vs_batch(args):
    """The gain of batching (the paper's R1, Eq. 11, measured with this code on one GPU).

    Serial: one realization, its environments, then proposals one at a time (S = 1 per
    call), each followed by its MH step. Batched: n realizations at once and S proposals per
    call. Both at L, beta = 1, chi = 8 (the paper's speed-up setting, at a size that runs in
    seconds). Reported: time per proposal in each mode, the environment time per
    realization, and the ratio of the two times for n x S proposals.
    """
    import torch
    import paper_2509_19006_b300 as P
    from workloads import Workload
    L, beta, chi, n_real, S, n_serial = args.rs_L, 1.0, 8, 64, 256, 32
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # serial
    wl1 = Workload("serial", [L], beta, chi, 1)
    J1 = torch.from_numpy(wl1.packed_J()).cuda()
    t1 = P.TNMC(wl1.Ls, chi, beta, args.prec, max_samples=1)
    t1.build_envs(J1)
    st1 = t1.mh_init_empty()
    torch.cuda.synchronize()
    e0, e1, e2 = ev(), ev(), ev()
    e0.record()
    t1.build_envs(J1)
    e1.record()
    for k in range(n_serial):
        t1.mh_step(t1.propose(1, SAMPLING_SEED, k), st1, SAMPLING_SEED)
    e2.record()
    torch.cuda.synchronize()
    env1 = e0.elapsed_time(e1) / 1e3
    per_prop_serial = e1.elapsed_time(e2) / 1e3 / n_serial
    # batched
    wl = Workload("batched", [L] * n_real, beta, chi, S)
    J = torch.from_numpy(wl.packed_J()).cuda()
    t = P.TNMC(wl.Ls, chi, beta, args.prec, max_samples=S)
    t.build_envs(J)
    st = t.mh_init_empty()
    torch.cuda.synchronize()
    f0, f1, f2 = ev(), ev(), ev()
    f0.record()
    t.build_envs(J)
    f1.record()
    t.mh_step(t.propose(S, SAMPLING_SEED, 0), st, SAMPLING_SEED)
    f2.record()
    torch.cuda.synchronize()
    env_b = f0.elapsed_time(f1) / 1e3
    per_prop_batch = f1.elapsed_time(f2) / 1e3 / (n_real * S)
    t_serial = n_real * (env1 + S * per_prop_serial)
    t_batch = env_b + n_real * S * per_prop_batch
    print(json.dumps({"serial_vs_batch": True, "L": L, "beta": beta, "chi": chi, "precision": args.prec,
                      "realizations": n_real, "samples": S,
                      "serial": {"env_build_s": env1, "s_per_proposal": per_prop_serial},
                      "batched": {"env_build_s": env_b, "s_per_proposal": per_prop_batch},
                      "time_serial_s": t_serial, "time_batched_s": t_batch,
                      "ratio": t_serial / t_batch}), flush=True)


def run_env_once(args, wl):
    """Build the environments of the workload once (a target for profiler captures)."""
    import torch
    import paper_2509_19006_b300 as P
    J = torch.from_numpy(wl.packed_J()).cuda()
    t = P.TNMC(wl.Ls, wl.chi, wl.beta, args.prec, max_samples=wl.S, cutoff=args.cutoff, q=wl.q)
    if args.build_variant >= 0:
        t.set_build_variant(args.build_variant)
    t.build_envs(J)
    lz = t.log_z()
    torch.cuda.synchronize()
    st, flags = t.device_status()
    print(json.dumps({"workload": wl.name, "precision": args.prec, "status": int(st),
                      "log_z_0": float(lz[0].item())}), flush=True)
    if st != 0 and st != 4:
        sys.exit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp64", "fp32", "tf32", "bf16", "mixed", "dfloat"], default="fp32")
    ap.add_argument("--workload", default="L256")
    ap.add_argument("--cutoff", type=float, default=0.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--ref-acceptance", type=float, default=None,
                    help="acceptance credited to the oracle (default: the measured value for the workload)")
    ap.add_argument("--tune-rows", type=int, default=6,
                    help="rows below the lattice's middle the build autotuner times per layout "
                         "(0: no autotuning)")
    ap.add_argument("--build-variant", type=int, default=-1,
                    help="--env-once: build with this layout (tnmc_set_build_variant) instead of the default")
    ap.add_argument("--arms", default=None,
                    help="comparison arms 'prec:steps,...' timed after the primary line (default for "
                         "the L256 workload: fp64:1,dfloat:2; '' for none)")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="steps of the end-to-end leg (host buffers), at most --steps")
    ap.add_argument("--ckpt", type=int, default=-1,
                    help="cache every K-th environment row (default: 32 where the full cache "
                         "does not fit in 60 %% of the free device memory, else off)")
    ap.add_argument("--learned", action="store_true",
                    help="train the learned correction (setup) and time the corrected steps")
    ap.add_argument("--teacher-chi", type=int, default=32)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--sweep", action="store_true",
                    help="acceptance against L at the paper's (beta, chi), and its L=1024 configuration")
    ap.add_argument("--sweep-sizes", default="16,32,64,128,256,512,1024")
    ap.add_argument("--serial-vs-batch", action="store_true",
                    help="time serial (one realization, one proposal at a time) against batched")
    ap.add_argument("--rs-L", type=int, default=256)
    ap.add_argument("--nishimori", action="store_true",
                    help="random-bond Ising model on the Nishimori line: observables and the energy identity")
    ap.add_argument("--env-once", action="store_true",
                    help="build the environments once and exit (for profiler captures)")
    args = ap.parse_args()
    wl = config(args.workload)
    if args.arms is None:
        args.arms = "fp64:1,dfloat:2" if args.workload == "L256" and args.impl == "ours" else ""
    if args.sweep:
        run_sweep(args)
    elif args.serial_vs_batch:
        run_serial_vs_batch(args)
    elif args.nishimori:
        run_nishimori(args)
    elif args.env_once:
        run_env_once(args, wl)
    elif args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
