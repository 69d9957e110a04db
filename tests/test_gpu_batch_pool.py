"""Freed batches hand their device block to the next batch (trids_free_batch pools it): a
batch packed into a reused block, whose bytes still hold another batch's arrays, samples,
ranks and screens exactly like the same batch packed into a fresh block, and the screening
stream (which frees every batch on its packing thread) gives each batch the same results as
a batch sampled on its own."""
import numpy as np
import pytest
import torch

from paper_2510_24186_b300 import api, synth

pytestmark = pytest.mark.gpu

P, S, K = 64, 12, 5


def _setup():
    w = synth.workload("batched_screening", n_lig=40)
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    return w, pk


def _run(pk, b, lig_base=0):
    out = api.sample(pk, b, P, S, mc_loops=4, seed=33, lig_base=lig_base)
    idx, e = api.topk(b, out["energy"], out["dof"], K, 1.0)
    torch.cuda.synchronize()
    return out["energy"].cpu().numpy(), out["dof"].cpu().numpy(), idx.cpu().numpy(), e.cpu().numpy()


def test_reused_block_samples_like_a_fresh_one():
    w, pk = _setup()
    small = synth.concat_ligands(w.ligands[24:36])
    big = synth.concat_ligands(w.ligands[:24])
    b = api.Batch(pk, *small)            # packed while no block of this size need be pooled
    ref = _run(pk, b)
    b.close()
    other = api.Batch(pk, *big)          # the larger batch fills its own block with its arrays
    _run(pk, other)
    other.close()                        # ... and leaves it (and the first one) to the pool
    again = api.Batch(pk, *small)        # takes a pooled block that held the other arrays
    got = _run(pk, again)
    again.close()
    for r, g in zip(ref, got):
        np.testing.assert_array_equal(r, g)   # bit for bit


def test_stream_of_batches_matches_batches_sampled_alone():
    w, pk = _setup()
    spans = [(0, 10), (10, 25), (25, 31), (31, 40)]
    batches = [synth.concat_ligands(w.ligands[a:b]) for a, b in spans]
    got = list(api.screen_stream(pk, batches, P, S, K, seed=33, mc_loops=4))
    assert [g[0] for g in got] == [a for a, _ in spans]
    for (a, _), arrays, (base, idx, e) in zip(spans, batches, got):
        b = api.Batch(pk, *arrays)
        _, _, ri, re = _run(pk, b, lig_base=a)
        b.close()
        np.testing.assert_array_equal(idx, ri)
        np.testing.assert_array_equal(e, re)
