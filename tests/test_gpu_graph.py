"""The persistent sampler's CUDA graph (Sec. 4 item 2: repeated operators kept on the GPU as
a graph) is built once per launch shape and replayed: a new seed, other buffers, a resumed
step range or another batch of the same shape update its nodes, and every replay gives
the same bits as a plain launch with the same arguments."""
import numpy as np
import pytest
import torch

from paper_2510_24186_b300 import api, synth

pytestmark = pytest.mark.gpu


def _setup():
    w = synth.workload("batched_screening", n_lig=12)
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    arrays = synth.concat_ligands(w.ligands)
    return w, pk, arrays


def _same(a, b):
    return torch.equal(a["energy"], b["energy"]) and torch.equal(a["dof"], b["dof"])


@pytest.mark.parametrize("explicit_stream", [False, True], ids=["default_stream", "side_stream"])
def test_graph_is_built_once_and_replayed_with_new_arguments(explicit_stream):
    w, pk, arrays = _setup()
    b1 = api.Batch(pk, *arrays)
    P, S = 64, 12
    st = torch.cuda.Stream() if explicit_stream else None
    kw = dict(mc_loops=4, stream=st)
    s0 = pk.graph_stats()
    api.sample(pk, b1, P, S, seed=11, **kw)
    g12 = api.sample(pk, b1, P, S, seed=12, **kw)
    ref12 = api.sample(pk, b1, P, S, seed=12, use_graph=False, **kw)
    torch.cuda.synchronize()
    assert _same(g12, ref12)
    s1 = pk.graph_stats()
    assert s1["instantiations"] == s0["instantiations"] + 1
    assert s1["updates"] >= s0["updates"] + 1 and s1["launches"] == s0["launches"] + 2
    # another batch of the same shape (the same ligands) replays the same graph
    b2 = api.Batch(pk, *arrays)
    g12b = api.sample(pk, b2, P, S, seed=12, **kw)
    # a resumed step range through the graph equals one plain pass
    half = api.sample(pk, b1, P, S, seed=13, step_end=7, **kw)
    rest = api.sample(pk, b1, P, S, seed=13, step_begin=7, dof=half["dof"], state=half["state"],
                      energy=half["energy"], **kw)
    ref13 = api.sample(pk, b1, P, S, seed=13, use_graph=False, **kw)
    # other ligand ids
    g_lb = api.sample(pk, b1, P, S, seed=12, lig_base=100, **kw)
    ref_lb = api.sample(pk, b1, P, S, seed=12, lig_base=100, use_graph=False, **kw)
    torch.cuda.synchronize()
    assert _same(g12b, ref12)
    assert _same(rest, ref13)
    assert _same(g_lb, ref_lb) and not torch.equal(g_lb["energy"], ref12["energy"])
    s2 = pk.graph_stats()
    assert s2["instantiations"] == s1["instantiations"]
    assert s2["launches"] == s1["launches"] + 4
    assert s2["updates"] == s1["updates"] + 4
    assert api.sync(b1, P, rest["state"], timeout_ms=60000) == 0


def test_graph_is_rebuilt_when_the_launch_shape_changes():
    w, pk, arrays = _setup()
    b = api.Batch(pk, *arrays)
    s0 = pk.graph_stats()
    api.sample(pk, b, 64, 6, mc_loops=2, seed=1, warps_per_block=20)
    api.sample(pk, b, 64, 6, mc_loops=2, seed=1, warps_per_block=16)
    o = api.sample(pk, b, 64, 6, mc_loops=2, seed=1, warps_per_block=16)
    ref = api.sample(pk, b, 64, 6, mc_loops=2, seed=1, warps_per_block=16, use_graph=False)
    torch.cuda.synchronize()
    s1 = pk.graph_stats()
    assert s1["instantiations"] == s0["instantiations"] + 2
    assert _same(o, ref)
