"""Multi-GPU form of the sampler: independent ligand shards, one process per GPU.

Ligands are independent units, so a run splits them across ranks with no exchange on the
data path.  The pocket and parameters are replicated; each rank packs and samples its own
shard with random-stream ids that do not depend on the split (`lig_base` = the shard's
first global ligand id when shards are contiguous, or per-ligand ids when they are not).
The only communication is outside the hot path: a max over ranks of the timed region and,
if wanted, a host-side gather of the per-ligand top-k results.
"""
from __future__ import annotations

import numpy as np


def shard_contiguous(n_lig: int, rank: int, world: int) -> np.ndarray:
    """Ligands [start, stop) of `rank` in a contiguous split (sizes differ by at most one)."""
    start = (n_lig * rank) // world
    stop = (n_lig * (rank + 1)) // world
    return np.arange(start, stop, dtype=np.int64)


def shard_lpt(costs, world: int) -> list:
    """Longest-processing-time-first split: ligands by decreasing cost, each to the rank
    with the least assigned cost (ties: lower rank).  Deterministic; returns one sorted
    index array per rank."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    out = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(load))
        out[r].append(int(i))
        load[r] += costs[i]
    return [np.array(sorted(o), dtype=np.int64) for o in out]


def ligand_cost(n_atoms, n_tor, n_pairs=None) -> np.ndarray:
    """Relative sampling cost of ligands (atoms dominate through the pocket pairs).  Without
    intra-pair counts, L (L - 1) / 2 stands in for them."""
    n_atoms = np.asarray(n_atoms, dtype=np.float64)
    if n_pairs is None:
        n_pairs = n_atoms * (n_atoms - 1) / 2
    return 60.0 * n_atoms + 2.0 * np.asarray(n_pairs) + 20.0 * np.asarray(n_tor) + 10.0


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (measurement only; identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def merge_topk(parts):
    """Per-shard (global ligand ids, top-k pose indices, energies) -> one set in global ligand
    order."""
    ids = np.concatenate([np.asarray(p[0]) for p in parts])
    order = np.argsort(ids, kind="stable")
    return (ids[order], np.concatenate([np.asarray(p[1]) for p in parts])[order],
            np.concatenate([np.asarray(p[2]) for p in parts])[order])


def gather_topk(global_ids, idx, energies):
    """Rank 0 receives every rank's (global ligand ids, top-k pose indices, energies) and
    returns them in global ligand order; other ranks return None."""
    import torch.distributed as dist
    item = (np.asarray(global_ids), np.asarray(idx), np.asarray(energies))
    if not (dist.is_available() and dist.is_initialized()):
        parts = [item]
    else:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, item)
        if dist.get_rank() != 0:
            return None
    return merge_topk(parts)


def rank_world(rank=None, world=None):
    """(rank, world size): the given values, else the process group's, else (0, 1)."""
    if rank is not None and world is not None:
        return int(rank), int(world)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def screen_shards(n_atoms, n_tor, run_shard, rank=None, world=None, gather=True):
    """Screening of one ligand set split over ranks (one process per GPU): the ligands are
    split by shard_lpt on ligand_cost; this rank runs run_shard(ids) on its own global ligand
    ids (sorted) and gets (top-k pose indices [n, k], energies [n, k]) back; with gather, rank
    0 receives every shard's results in global ligand order (other ranks get None), else each
    rank returns its own (ids, idx, energies).  No collective touches the sampling itself."""
    rank, world = rank_world(rank, world)
    mine = shard_lpt(ligand_cost(n_atoms, n_tor), world)[rank]
    idx, e = run_shard(mine)
    if not gather:
        return mine, np.asarray(idx), np.asarray(e)
    return gather_topk(mine, idx, e)
