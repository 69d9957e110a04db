"""Multi-process sharding on CPU (gloo, world size 2): shard, sample each shard with the
oracle, gather top-k on rank 0 and compare with a single-process run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_24186_b300 import parallel, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run_shard(lig_ids, ligs, pk, seed, P, S):
    import oracle
    op = oracle.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    cfg = oracle.sample_cfg(steps=S, mc_loops=3, seed=seed)
    tops, es = [], []
    for gid in lig_ids:
        lg = ligs[gid]
        st, ol = oracle.pack(lg.xyz, lg.type, lg.bonds, lg.rotatable)
        dof, e, _ = oracle.sample_ligand(cfg, op, pk.xyz, pk.type, ol, int(gid), P)
        X = np.stack([oracle.fk(ol, dof[p]) for p in range(P)])
        idx, _ = oracle.topk(e, X, 3, 1.0)
        tops.append(idx)
        es.append(e[np.maximum(idx, 0)])
    return np.array(tops), np.array(es)


def _ligands():
    rng = np.random.default_rng(3)
    return [synth.gen_ligand(rng, int(rng.integers(6, 14)), int(rng.integers(0, 3))) for _ in range(7)]


def _worker(rank, world, port, out_path):
    """One rank of the sharded screening host logic (parallel.screen_shards, the logic
    api.screen_sharded runs around its GPU calls), with the oracle standing in for the
    rank's GPU sampling of its shard."""
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workload("single_ligand")
    ligs = _ligands()
    seen = []

    def run_shard(ids):
        seen.append(np.asarray(ids))
        return _run_shard(ids, ligs, w.pocket, 11, 6, 4)

    got = parallel.screen_shards([len(l.type) for l in ligs], [l.n_tor for l in ligs], run_shard)
    t = parallel.max_over_ranks(float(rank + 1))
    mine = parallel.gather_topk(seen[0], np.zeros((len(seen[0]), 1)), np.zeros((len(seen[0]), 1)))
    if rank == 0:
        np.savez(out_path, ids=got[0], idx=got[1], e=got[2], tmax=t, shard_ids=mine[0])
    else:
        assert got is None and mine is None
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_all_ligands_once():
    costs = np.random.default_rng(0).uniform(1, 10, 101)
    for world in (1, 2, 3, 8):
        parts = parallel.shard_lpt(costs, world)
        allids = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allids, np.arange(101))
        loads = [costs[p].sum() for p in parts]
        assert max(loads) - min(loads) <= costs.max() + 1e-9
        cont = [parallel.shard_contiguous(101, r, world) for r in range(world)]
        np.testing.assert_array_equal(np.concatenate(cont), np.arange(101))


def test_two_rank_gloo_matches_single_process(tmp_path):
    out = str(tmp_path / "r0.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    r = np.load(out)
    assert r["tmax"] == 2.0
    np.testing.assert_array_equal(r["shard_ids"], np.arange(7))   # every ligand on exactly one rank
    w = synth.workload("single_ligand")
    ligs = _ligands()
    tops, es = _run_shard(np.arange(7), ligs, w.pocket, 11, 6, 4)
    np.testing.assert_array_equal(r["ids"], np.arange(7))
    np.testing.assert_array_equal(r["idx"], tops)
    np.testing.assert_array_equal(r["e"], es)
