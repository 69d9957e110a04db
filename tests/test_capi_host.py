"""Host-side checks of libtrids that need no GPU: exports, packing, argument errors."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2510_24186_b300 import _lib, api, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "trids.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(trids_\w+)\s*\(", hdr, re.M))
    assert declared == set(_lib.EXPORTS)
    L = _lib.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert L.trids_version() >= 100


def test_host_pack_matches_oracle_bit_exact(orc):
    rng = np.random.default_rng(21)
    ligs = [synth.workload("single_ligand").ligands[0]]
    ligs += [synth.gen_ligand(rng, int(rng.integers(1, 71)), int(rng.integers(0, 21))) for _ in range(60)]
    ligs += [synth.gen_ligand(rng, 70, 20), synth.gen_ligand(rng, 1, 0), synth.gen_ligand(rng, 2, 0)]
    for lg in ligs:
        a = api.pack_topology(lg.xyz, lg.type, lg.bonds, lg.rotatable)
        st, ol = orc.pack(lg.xyz.astype(np.float32).astype(np.float64), lg.type, lg.bonds, lg.rotatable)
        assert st == 0
        np.testing.assert_array_equal(a, orc.topology(ol))


@pytest.mark.parametrize("case", ["ring_rot", "disconnected", "dup", "type", "nan", "big", "self", "empty"])
def test_host_pack_rejects_bad_ligands(case):
    lg = synth.workload("single_ligand").ligands[0]
    xyz, t, b, r = lg.xyz.copy(), lg.type.copy(), lg.bonds.copy(), lg.rotatable.copy()
    if case == "ring_rot":
        b = np.vstack([b, [[0, 9]]]) if not any((b == [0, 9]).all(1)) else b
        r = np.concatenate([r, [1]])
    elif case == "disconnected":
        b, r = b[1:], r[1:]
    elif case == "dup":
        b, r = np.vstack([b, b[:1]]), np.concatenate([r, [0]])
    elif case == "type":
        t[0] = 8
    elif case == "nan":
        xyz[1, 1] = np.inf
    elif case == "big":
        big = synth.gen_ligand(np.random.default_rng(0), 71, 0)
        xyz, t, b, r = big.xyz, big.type, big.bonds, big.rotatable
    elif case == "self":
        b = np.vstack([b, [[3, 3]]])
        r = np.concatenate([r, [0]])
    elif case == "empty":                       # a ligand without atoms
        xyz, t = np.zeros((0, 3), np.float32), np.zeros(0, np.int32)
        b, r = np.zeros((0, 2), np.int32), np.zeros(0, np.uint8)
    with pytest.raises(_lib.TridsError) as e:
        api.pack_topology(xyz, t, b, r)
    assert e.value.code == _lib.EINVAL
    assert _lib.lib().trids_last_error().decode() != ""


def test_null_arguments_are_rejected_without_a_gpu():
    L = _lib.lib()
    assert L.trids_score_grad(None, None, 1, None, None, None, None, None, None, None, None, None) == _lib.EINVAL
    assert L.trids_sample(None, None, None, None, None, None, None) == _lib.EINVAL
    assert L.trids_topk(None, 1, None, None, 1, 1.0, None, None, None) == _lib.EINVAL
    assert L.trids_state_floats(None, 4) == 0
    out = C.c_void_p()
    assert L.trids_pack_ligands(None, 1, None, None, None, None, None, None, C.byref(out)) == _lib.EINVAL
    assert out.value is None


def test_new_entry_points_reject_null_handles_without_a_gpu():
    L = _lib.lib()
    assert L.trids_set_residues(None, 4, None) == _lib.EINVAL
    assert L.trids_set_mdn(None, 4, 2, None, None) == _lib.EINVAL
    assert L.trids_build_maps(None, 0.375, 8.0, None) == _lib.EINVAL
    lo = (C.c_float * 3)()
    h = C.c_float()
    n = (C.c_int32 * 3)()
    assert L.trids_maps_info(None, C.byref(lo), C.byref(h), C.byref(n)) == _lib.EINVAL
    assert L.trids_set_boxes(None, 1, None, None) == _lib.EINVAL
    assert L.trids_screen_energy(None, None, 1, 1, None, None, None, None) == _lib.EINVAL
    assert b"NULL" in L.trids_last_error()
    v = C.c_int64(-1)
    assert L.trids_graph_stats(None, C.byref(v), None, None) == _lib.EINVAL and v.value == -1
    assert L.trids_set_stream_ids(None, None) == _lib.EINVAL


def test_sharded_screening_host_logic_on_one_process():
    """parallel.screen_shards without a process group: world 1 runs the whole set as one
    shard; an explicit rank/world runs that rank's longest-processing-time shard, and the
    shards of all ranks cover the set once."""
    import numpy as np
    from paper_2510_24186_b300 import parallel
    n_atoms = [12, 40, 25, 33, 18, 60, 27]
    n_tor = [1, 9, 3, 4, 2, 15, 5]
    seen = []

    def run(ids):
        seen.append(list(ids))
        return np.array([[i, -1] for i in ids]), np.array([[-float(i), np.nan] for i in ids])

    ids, idx, e = parallel.screen_shards(n_atoms, n_tor, run)
    assert list(ids) == list(range(7)) and seen[-1] == list(range(7))
    assert idx[:, 0].tolist() == list(range(7))
    parts = [parallel.screen_shards(n_atoms, n_tor, run, rank=r, world=3, gather=False) for r in range(3)]
    assert sorted(sum((list(p[0]) for p in parts), [])) == list(range(7))
    merged = parallel.merge_topk(parts)
    assert merged[0].tolist() == list(range(7)) and merged[1][:, 0].tolist() == list(range(7))
    loads = [parallel.ligand_cost(np.array(n_atoms)[p[0]], np.array(n_tor)[p[0]]).sum() for p in parts]
    assert max(loads) - min(loads) <= parallel.ligand_cost(n_atoms, n_tor).max()


def test_python_api_fails_loudly_without_cuda():
    """There is no CPU fallback: the product path raises when no CUDA device is present."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2510_24186_b300 import api, synth
    w = synth.workload("single_ligand")
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    with pytest.raises(RuntimeError, match="CUDA"):
        api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)


@pytest.mark.parametrize("n_atoms", [0, -1, 8192])
def test_pocket_size_outside_the_limits_is_rejected_without_a_gpu(n_atoms):
    """An empty pocket and one beyond the 13-bit candidate index fail on the host, before
    any device work."""
    from paper_2510_24186_b300 import api
    L = _lib.lib()
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    n = max(n_atoms, 1)
    xyz = np.zeros((n, 3), np.float32)
    ty = np.zeros(n, np.int32)
    c, size = (C.c_float * 3)(0, 0, 0), (C.c_float * 3)(22.5, 22.5, 22.5)
    cp = sp.to_c()
    out = C.c_void_p()
    rc = L.trids_make_pocket(xyz.ctypes.data, ty.ctypes.data, n_atoms, C.byref(c), C.byref(size), 0.0,
                             C.byref(cp), C.byref(out))
    assert rc == _lib.EINVAL and out.value is None
    assert b"atoms" in L.trids_last_error()
