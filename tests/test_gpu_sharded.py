"""Sharded screening (api.screen_sharded): the batched-screening ligands split over two
ranks by longest-processing-time, each shard sampled with the ligands' global indices as
random-stream ids, and the shards' top-k merged in global order equal one unsplit run bit
for bit.  The two ranks run one after the other in this process (the library call is the
same on each rank; the host gather is covered with gloo on CPU)."""
import numpy as np
import pytest
import torch

from paper_2510_24186_b300 import api, parallel, synth

pytestmark = pytest.mark.gpu


def test_two_shards_merge_to_the_unsplit_result():
    w = synth.workload("batched_screening", n_lig=24)
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    P, S, k = 64, 12, 5
    parts = [api.screen_sharded(pk, w.ligands, P, S, k, seed=21, mc_loops=4, rank=r, world=2, gather=False)
             for r in range(2)]
    assert len(parts[0][0]) and len(parts[1][0])
    assert not set(parts[0][0]) & set(parts[1][0])
    ids, idx, e = parallel.merge_topk(parts)
    whole = api.screen_sharded(pk, w.ligands, P, S, k, seed=21, mc_loops=4, rank=0, world=1)
    np.testing.assert_array_equal(ids, np.arange(24))
    np.testing.assert_array_equal(whole[0], ids)
    np.testing.assert_array_equal(whole[1], idx)
    np.testing.assert_array_equal(whole[2], e)      # bit for bit
    # and the unsplit run equals a plain batch sampled with ligand ids 0..23
    b = api.Batch.from_ligands(pk, w.ligands)
    out = api.sample(pk, b, P, S, mc_loops=4, seed=21)
    i2, e2 = api.topk(b, out["energy"], out["dof"], k, 1.0)
    np.testing.assert_array_equal(i2.cpu().numpy(), idx)
    np.testing.assert_array_equal(e2.cpu().numpy(), e)


def _rank_main(rank, world, port, out_path):
    """One rank of a two-process run on this one GPU: the shard's sampling is this rank's
    own library call, the top-k gather goes through a gloo process group."""
    import os
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.workload("batched_screening", n_lig=24)
        sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff)
        pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
        got = api.screen_sharded(pk, w.ligands, 64, 12, 5, seed=21, mc_loops=4)
        if rank == 0:
            np.savez(out_path, ids=got[0], idx=got[1], e=got[2])
        else:
            assert got is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_processes_gather_the_unsplit_result(tmp_path):
    """Two processes (ranks) share the GPU; no kernel of one waits on the other.  Rank 0's
    gathered top-k equals the unsplit single-process run bit for bit."""
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = str(tmp_path / "r0.npz")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    r = np.load(out)
    w = synth.workload("batched_screening", n_lig=24)
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    whole = api.screen_sharded(pk, w.ligands, 64, 12, 5, seed=21, mc_loops=4, rank=0, world=1)
    np.testing.assert_array_equal(r["ids"], whole[0])
    np.testing.assert_array_equal(r["idx"], whole[1])
    np.testing.assert_array_equal(r["e"], whole[2])
