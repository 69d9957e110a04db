"""Input generators: the ligand recipe's invariants hold for both ways of drawing candidate
placements, and the indexed ligand set (the 100,000-ligand screening stream) does not depend
on how many worker processes build it."""
import numpy as np
import pytest

from paper_2510_24186_b300 import synth


@pytest.mark.parametrize("vector_tries", [False, True])
def test_ligand_recipe_invariants(vector_tries):
    rng = np.random.default_rng(5)
    for _ in range(40):
        L, T = int(rng.integers(2, 71)), int(rng.integers(0, 21))
        lg = synth.gen_ligand(rng, L, T, synth.DRUGLIKE_MIX, vector_tries=vector_tries)
        assert lg.xyz.shape == (L, 3) and len(lg.bonds) == L - 1
        d = np.linalg.norm(lg.xyz[lg.bonds[:, 0]] - lg.xyz[lg.bonds[:, 1]], axis=1)
        np.testing.assert_allclose(d, synth.BOND, atol=1e-9)
        bonded = np.zeros((L, L), dtype=bool)
        bonded[lg.bonds[:, 0], lg.bonds[:, 1]] = bonded[lg.bonds[:, 1], lg.bonds[:, 0]] = True
        dist = np.linalg.norm(lg.xyz[:, None] - lg.xyz[None], axis=2)
        off = ~bonded & ~np.eye(L, dtype=bool)
        assert (dist[off] >= 2.0 - 1e-9).all()
        deg = np.bincount(lg.bonds.ravel(), minlength=L)
        assert deg.max() <= 4
        rot = lg.bonds[lg.rotatable.astype(bool)]
        assert ((deg[rot[:, 0]] >= 2) & (deg[rot[:, 1]] >= 2)).all()
        assert lg.n_tor == min(T, int(((deg[lg.bonds[:, 0]] >= 2) & (deg[lg.bonds[:, 1]] >= 2)).sum()))
        # each atom's angle to its parent's earlier neighbour stays near tetrahedral
        for a, b in lg.bonds:
            for c in np.nonzero(bonded[a])[0]:
                if c != b and c < b:
                    u, v = lg.xyz[b] - lg.xyz[a], lg.xyz[c] - lg.xyz[a]
                    ang = np.degrees(np.arccos(np.dot(u, v) / np.linalg.norm(u) / np.linalg.norm(v)))
                    assert 95.0 < ang < 125.0


def test_indexed_set_does_not_depend_on_the_worker_count():
    args = (1004, 240, (10, 70), (0, 20), synth.DRUGLIKE_MIX, np.zeros(3))
    one = synth._ligand_set_indexed(*args, workers=1)
    many = synth._ligand_set_indexed(*args, workers=4, min_parallel=0)
    assert len(one) == len(many) == 240
    for a, b in zip(one, many):
        assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.bonds, b.bonds)
        assert np.array_equal(a.type, b.type) and np.array_equal(a.rotatable, b.rotatable)
    head = synth.workload("screening_stream", n_lig=30).ligands
    assert all(np.array_equal(a.xyz, b.xyz) for a, b in zip(one[:30], head))
