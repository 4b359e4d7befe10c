"""Weak-scaling sharding across ranks, run as two gloo processes on CPU.

Each rank owns a full batch of realizations with its own disorder seeds (no
collective on the data path); only the final reduction of accepted counts and
the slowest rank's time crosses ranks, as in bench.py. The oracle stands in
for the GPU path so the host-side logic runs anywhere.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from workloads import Workload


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import bmps, mh, philox, sampler
    wl = Workload("tiny", [4, 3], 0.8, 4, 16)
    wl.base_seed = wl.base_seed + rank * 100000        # the rank's own disorder, as in bench.py
    accepted, first_bonds = 0, None
    for n in range(wl.n_real):
        Jh, Jv = wl.realization(n)
        if n == 0:
            first_bonds = np.concatenate([Jh.ravel(), Jv.ravel()])
        rows = bmps.build_envs(Jh, Jv, wl.beta, wl.chi)
        s0 = philox.init_spins(wl.Ls[n], n, 42)
        lq0, E0, _ = sampler.score(rows, Jh, Jv, wl.beta, s0[None])
        props = sampler.propose(rows, Jh, Jv, wl.beta, wl.S, 42, 0, n)[:3]
        _, acc, _, _ = mh.chain((s0, lq0[0], E0[0]), props, wl.beta, 42, 0, n)
        accepted += int(acc.sum())
    t = torch.tensor([float(accepted), float(rank + 1)], dtype=torch.float64)
    tot = t.clone(); dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    mx = t.clone(); dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    bonds = torch.from_numpy(first_bonds.astype(np.float64))
    gathered = [torch.zeros_like(bonds) for _ in range(world)]
    dist.all_gather(gathered, bonds)
    out[rank] = (accepted, tot[0].item(), mx[1].item(),
                 not torch.equal(gathered[0], gathered[1]))
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][1] == res[0][0] + res[1][0]          # whole-job accepted = sum over ranks
    assert res[0][2] == res[1][2] == 2.0               # max over ranks (time stand-in)
    assert res[0][3] and res[1][3]                     # ranks drew different disorder
