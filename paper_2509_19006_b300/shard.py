"""Realizations over ranks: one process per GPU, each with a shard of the batch.

Disorder realizations are independent (Sec. 3.4 batches them as a leading
dimension), so a set of realizations splits over GPUs with no exchange on the
data path. Each rank builds, samples and scores its own shard; only the
per-realization results (log Z, accepted counts) are gathered at the end.

* ``lpt_partition`` assigns realizations to ranks by longest processing time
  first (Graham, 1969) on the cost of the environment build, which dominates a
  step: L^2 sites per row sweep, each a QR and an SVD of cost ~ D^3 for a bond of
  dimension D = min(chi, 2^floor(L/2)).
* A rank's handle names its realizations by their indices in the whole set
  (``TNMC.set_realization_ids``), so the random numbers of realization g do not
  depend on how many ranks there are or which one holds g.
* ``gather`` puts every rank's per-realization values back in global order.
"""
from __future__ import annotations

from typing import List, Sequence


def build_cost(L: int, chi: int) -> float:
    """Relative cost of one realization's environments: L^2 site steps of O(D^3)."""
    d = min(int(chi), 2 ** min(int(L) // 2, 30))
    return float(L) * float(L) * float(d) ** 3


def lpt_partition(Ls: Sequence[int], chi: int, world: int) -> List[List[int]]:
    """Global indices of the realizations each rank owns (each list ascending).

    Realizations in decreasing cost (ties: lower index first) go one at a time to
    the rank with the least cost so far (ties: lower rank). Every index lands on
    exactly one rank; with equal sizes the ranks get equal counts (+-1).
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(Ls)), key=lambda n: (-build_cost(Ls[n], chi), n))
    load = [0.0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for n in order:
        k = min(range(world), key=lambda r: (load[r], r))
        shards[k].append(n)
        load[k] += build_cost(Ls[n], chi)
    return [sorted(s) for s in shards]


def gather(dist, n_total: int, ids: Sequence[int], values, device=None):
    """All ranks' per-realization values in global order (float64 tensor [n_total, ...]).

    ``values`` is this rank's tensor [len(ids), ...] for the realizations ``ids``;
    ``dist`` is ``torch.distributed`` (initialised) or None for one process. A sum
    over ranks of zero-padded copies: each realization is owned by exactly one rank.
    """
    import torch
    vals = torch.as_tensor(values, dtype=torch.float64, device=device)
    full = torch.zeros((n_total,) + tuple(vals.shape[1:]), dtype=torch.float64, device=vals.device)
    if len(ids):
        full[torch.as_tensor(list(ids), dtype=torch.long, device=vals.device)] = vals
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(full, op=dist.ReduceOp.SUM)
    return full
