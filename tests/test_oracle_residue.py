"""Pins of the oracle's residue-level E_MDN (term set 2) against closed forms, a
numpy brute force of the residue minimum, central differences and invariants."""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2510_24186_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MDN_ONLY = (1.0, 0.0, 0.0, 0.0, 0.0)


def res_params(orc, w=synth.TRIDS_WEIGHTS, cutoff=10.0):
    return orc.make_params(2, synth.TYPE_RADIUS, synth.TYPE_FLAGS, w, cutoff)


def _rows():
    out = []
    for line in open(os.path.join(GOLDEN, "residue_mdn.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        atoms, kern, e, g = line.split("|")
        out.append((atoms.split(), kern.split(), e.strip(), g.split()))
    return out


def _ev(s):
    return eval(s, {"exp": math.exp})


@pytest.mark.parametrize("row", _rows())
def test_residue_mdn_closed_forms(orc, row):
    atoms, kern, e, g = row
    res = [int(a.split(":")[0]) for a in atoms]
    xyz = np.array([[float(v) for v in a.split(":")[1].split(",")] for a in atoms])
    n_res = max(res) + 1
    prm = np.zeros((1, n_res, 2, 3))
    count = [0] * n_res
    for k in kern:
        r = int(k.split(":")[0])
        prm[0, r, count[r]] = [float(v) for v in k.split(":")[1].split(",")]
        count[r] += 1
    st, lg = orc.pack(np.zeros((1, 3)), [1], np.zeros((0, 2)), [])
    p = res_params(orc, MDN_ONLY)
    st, ev = orc.score(p, xyz, np.ones(len(res), np.int32), lg, np.array([0, 0, 0, 1, 0, 0, 0.0]),
                       orc.mdn(res, prm))
    assert st == 0
    assert ev.e_total == pytest.approx(_ev(e), abs=1e-14)
    np.testing.assert_allclose(ev.g_dof[:3], [_ev(v) for v in g], atol=1e-14)
    assert ev.g_w[0] == pytest.approx(_ev(e), abs=1e-14)


def _system(seed, n_lig_atoms=18, n_tor=4, M=160, K=3):
    rng = np.random.default_rng(seed)
    pk = synth.gen_pocket(rng, M, np.zeros(3), r_out=10.0)
    res = synth.gen_residues(rng, pk.xyz)
    lig = synth.gen_ligand(rng, n_lig_atoms, n_tor)
    prm = synth.gen_mdn(rng, n_lig_atoms, int(res.max()) + 1, K).astype(np.float64)
    return rng, pk, res, lig, prm


def test_residue_minimum_matches_numpy_brute_force(orc):
    """E_MDN from the oracle equals a direct numpy evaluation of the definition on the
    oracle's world coordinates (distance matrix, per-residue minimum, kernel sum)."""
    for seed in (1, 2, 3):
        rng, pk, res, lig, prm = _system(seed)
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        p = res_params(orc, MDN_ONLY, cutoff=0.01)   # atom pairs out of range: E = E_MDN
        for _ in range(4):
            q = rng.normal(size=4)
            dof = np.concatenate([rng.uniform(-3, 3, 3), q / np.linalg.norm(q),
                                  rng.uniform(-math.pi, math.pi, lg.n_tor)])
            st, ev = orc.score(p, pk.xyz, pk.type, lg, dof, orc.mdn(res, prm))
            x = np.array(ev.x)[:lg.n_atoms]
            D = np.linalg.norm(x[:, None, :] - pk.xyz[None, :, :], axis=2)
            E = 0.0
            npairs = 0
            for i in range(lg.n_atoms):
                kin = lg.perm[i]                     # the kernels are given in input atom order
                for r in range(prm.shape[1]):
                    d = D[i, res == r].min()
                    if d < 5.0:
                        pi_, mu, sg = prm[kin, r, :, 0], prm[kin, r, :, 1], prm[kin, r, :, 2]
                        E -= float(np.sum(pi_ * np.exp(-(d - mu) ** 2 / (2 * sg ** 2))))
                        npairs += 1
            assert npairs > 10
            assert ev.n_res_pairs == npairs
            assert ev.e_total == pytest.approx(E, rel=1e-12, abs=1e-12)


def test_residue_mdn_gradient_matches_central_differences(orc):
    """dE/d(t, q, theta) with the residue term on (full E_dock weights)."""
    for seed in (4, 5):
        rng, pk, res, lig, prm = _system(seed)
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        md = orc.mdn(res, prm)
        p = res_params(orc)
        for _ in range(3):
            q = rng.normal(size=4) * rng.uniform(0.5, 2.0)
            dof = np.concatenate([rng.uniform(-3, 3, 3), q, rng.uniform(-math.pi, math.pi, lg.n_tor)])
            st, ev = orc.score(p, pk.xyz, pk.type, lg, dof, md)
            assert ev.n_res_pairs > 0
            g = np.array(ev.g_dof[:7 + lg.n_tor])
            for j in range(7 + lg.n_tor):
                def fd(h):
                    dp, dm = dof.copy(), dof.copy()
                    dp[j] += h
                    dm[j] -= h
                    return (orc.score(p, pk.xyz, pk.type, lg, dp, md)[1].e_total
                            - orc.score(p, pk.xyz, pk.type, lg, dm, md)[1].e_total) / (2 * h)
                f1, f2 = fd(1e-4), fd(5e-5)
                if abs(f1 - f2) > 1e-3 * (1 + abs(f1)):    # a cutoff, kink or argmin switch
                    continue
                rich = (4 * f2 - f1) / 3
                assert rich == pytest.approx(g[j], rel=1e-7, abs=1e-7), j


def test_residue_mdn_rigid_motion_of_whole_complex(orc):
    rng, pk, res, lig, prm = _system(6)
    st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
    md = orc.mdn(res, prm)
    p = res_params(orc)
    for _ in range(3):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        dof = np.concatenate([rng.uniform(-3, 3, 3), q, rng.uniform(-math.pi, math.pi, lg.n_tor)])
        st, ev = orc.score(p, pk.xyz, pk.type, lg, dof, md)
        Q = Rotation.random(random_state=int(rng.integers(1 << 30)))
        s = rng.normal(size=3) * 5
        qq = Q.as_quat()
        qq = np.array([qq[3], qq[0], qq[1], qq[2]])
        qn = np.array([qq[0] * q[0] - qq[1:] @ q[1:]] + list(qq[0] * q[1:] + q[0] * qq[1:] + np.cross(qq[1:], q[1:])))
        dof2 = np.concatenate([Q.apply(dof[:3]) + s, qn, dof[7:]])
        st, ev2 = orc.score(p, Q.apply(pk.xyz) + s, pk.type, lg, dof2, md)
        assert ev.n_res_pairs > 0
        assert ev2.e_total == pytest.approx(ev.e_total, rel=1e-10, abs=1e-10)
        gx = np.array(ev.g_x)[:lg.n_atoms]
        np.testing.assert_allclose(np.array(ev2.g_x)[:lg.n_atoms], Q.apply(gx), atol=1e-9)


def test_residue_term_needs_its_inputs_and_other_sets_ignore_them(orc):
    rng, pk, res, lig, prm = _system(7)
    st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
    dof = np.concatenate([np.zeros(3), [1, 0, 0, 0], np.zeros(lg.n_tor)])
    st, _ = orc.score(res_params(orc), pk.xyz, pk.type, lg, dof)
    assert st != 0
    p1 = orc.make_params(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0)
    _, a = orc.score(p1, pk.xyz, pk.type, lg, dof)
    _, b = orc.score(p1, pk.xyz, pk.type, lg, dof, orc.mdn(res, prm))
    assert a.e_total == b.e_total and b.n_res_pairs == 0
    # term set 2 = term set 1 without the atom-pair E_MDN (gmm all zero) + the residue sum
    _, c = orc.score(res_params(orc), pk.xyz, pk.type, lg, dof, orc.mdn(res, prm))
    _, m = orc.score(res_params(orc, MDN_ONLY, cutoff=0.01), pk.xyz, pk.type, lg, dof, orc.mdn(res, prm))
    assert c.e_total == pytest.approx(a.e_total + m.e_total, rel=1e-12, abs=1e-12)
