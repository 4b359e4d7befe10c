"""Realizations sharded over ranks (two gloo processes on CPU).

The product's host logic decides the shards (``shard.lpt_partition``: longest
processing time first on the build cost) and gathers the per-realization
results (``shard.gather``). Each rank computes its realizations with its
realizations' global indices as their random-number stream ids, as a rank's
``TNMC`` handle does after ``set_realization_ids``; the oracle stands in for the
GPU here so that the ranks run anywhere. Checked: the shards cover the set
exactly once, the loads are balanced, and every realization's results at world
size 2 equal those at world size 1.
"""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_19006_b300 import shard
from workloads import draw_bonds

LS = [4, 3, 5, 2, 4, 3, 5, 1]
CHI, BETA, S, SEED = 4, 0.8, 16, 42


def _results(ids):
    """(log Z, accepted count) of the realizations ``ids`` of the set, by the oracle."""
    from oracle import bmps, mh, philox, sampler
    out = []
    for g in ids:
        L = LS[g]
        Jh, Jv = draw_bonds(L, 1000 + g, "pmj")          # disorder seeded by the global index
        rows = bmps.build_envs(Jh, Jv, BETA, CHI)
        s0 = philox.init_spins(L, g, SEED)                # random numbers keyed by the global index
        lq0, E0, _ = sampler.score(rows, Jh, Jv, BETA, s0[None])
        props = sampler.propose(rows, Jh, Jv, BETA, S, SEED, 0, g)[:3]
        _, acc, _, _ = mh.chain((s0, lq0[0], E0[0]), props, BETA, SEED, 0, g)
        out.append([bmps.log_z(rows), float(acc.sum())])
    return np.array(out, dtype=np.float64).reshape(len(ids), 2)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shards = shard.lpt_partition(LS, CHI, world)
    mine = shards[rank]
    full = shard.gather(dist, len(LS), mine, _results(mine))
    out[rank] = (shards, full.numpy())
    dist.destroy_process_group()


def test_lpt_partition_covers_and_balances():
    Ls = [256] * 64
    for world in (1, 2, 3, 8):
        sh = shard.lpt_partition(Ls, 64, world)
        assert sorted(i for s in sh for i in s) == list(range(64))
        assert max(map(len, sh)) - min(map(len, sh)) <= 1
    rng = np.random.default_rng(7)
    Ls = [int(x) for x in rng.choice([32, 48, 64, 96, 128], size=200)]
    sh = shard.lpt_partition(Ls, 32, 4)
    assert sorted(i for s in sh for i in s) == list(range(200))
    loads = [sum(shard.build_cost(Ls[i], 32) for i in s) for s in sh]
    # Graham's bound for LPT: makespan <= (4/3 - 1/(3m)) OPT, and OPT >= mean load
    assert max(loads) <= (4 / 3) * (sum(loads) / 4) + max(shard.build_cost(L, 32) for L in Ls)
    assert max(loads) / min(loads) < 1.05
    # the cost model: chi caps the bond only once 2^(L/2) exceeds it
    assert shard.build_cost(4, 64) == 16 * 4 ** 3 and shard.build_cost(128, 8) == 128 ** 2 * 8 ** 3


def test_two_ranks_equal_one_rank():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    shards = res[0][0]
    assert res[1][0] == shards
    assert sorted(shards[0] + shards[1]) == list(range(len(LS)))     # exactly once
    assert not set(shards[0]) & set(shards[1])
    one = _results(list(range(len(LS))))                             # world size 1
    np.testing.assert_array_equal(res[0][1], one)
    np.testing.assert_array_equal(res[1][1], one)
    assert one[:, 1].sum() > 0
