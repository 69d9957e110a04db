"""Pins of the FP64 oracle against things other than itself.

Each check ties one oracle function to a closed form, a library routine, an
independent algorithm, an invariant or brute force, so that a dropped term, a
wrong sign or index, or a transposed operand fails somewhere here.
"""
import ctypes as C
import itertools
import math
import os

import networkx as nx
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2510_24186_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def vina_params(orc, cutoff=8.0):
    return orc.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, cutoff)


def trids_params(orc, rng=None, cutoff=10.0, K=2):
    rng = rng or np.random.default_rng(7)
    gmm = np.zeros((8, 8, K, 3))
    gmm[..., 0] = rng.uniform(0.2, 1.0, (8, 8, K))
    gmm[..., 1] = rng.uniform(2.0, 4.5, (8, 8, K))
    gmm[..., 2] = rng.uniform(0.4, 1.2, (8, 8, K))
    return orc.make_params(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, cutoff, gmm=gmm)


def small_ligands(n=6, seed=3):
    rng = np.random.default_rng(seed)
    out = [synth.workload("single_ligand").ligands[0]]
    for _ in range(n):
        out.append(synth.gen_ligand(rng, int(rng.integers(6, 30)), int(rng.integers(0, 6))))
    return out


def random_dof(rng, T, box=8.0):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    return np.concatenate([rng.uniform(-box, box, 3), q, rng.uniform(-math.pi, math.pi, T)])


# --------------------------------------------------------------------------- Philox
def _curand():
    for name in ("libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so.10", "libcurand.so"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    pytest.fail("cuRAND host library not found; it is the reference for the Philox pin")


@pytest.mark.parametrize("seed,offset", [(0, 0), (1234567, 0), (0xDEADBEEFCAFEF00D, 4 * 65530),
                                         (42, 4 * ((1 << 48) + (3 << 16) + 7)), (99, 4 * ((5 << 48) + 123))])
def test_philox_matches_curand_host_generator(orc, seed, offset):
    """Oracle Philox4x32-10 vs cuRAND's host PHILOX4_32_10 generator.  Observed layout of
    that generator: key = seed, block B of the output stream has counter
    (B >> 16 low word, B >> 48, B & 0xffff, 0); offset counts 32-bit outputs.  This
    exercises counter words 0-2 and both key words, which are the words the sampler uses."""
    cr = _curand()
    gen = C.c_void_p()
    assert cr.curandCreateGeneratorHost(C.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, C.c_ulonglong(offset)) == 0
        n = 64
        buf = (C.c_uint32 * n)()
        assert cr.curandGenerate(gen, buf, C.c_size_t(n)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    got = []
    for b in range(n // 4):
        blk = offset // 4 + b
        got += orc.philox([(blk >> 16) & 0xFFFFFFFF, blk >> 48, blk & 0xFFFF, 0], key)
    assert got == list(buf)


def test_uniform_draws_in_unit_interval(orc):
    w = [orc.lib().or_rand_word(5, 1, p, 2, 1, n) for p in range(50) for n in range(6)]
    u = np.array([(x >> 8) / 16777216.0 for x in w])
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.05


# --------------------------------------------------------------------------- rotations
def test_rodrigues_matches_scipy(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        th = rng.uniform(-math.pi, math.pi)
        np.testing.assert_allclose(orc.rot(u, th), Rotation.from_rotvec(u * th).as_matrix(), atol=1e-14)


def test_quaternion_matrix_matches_scipy(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        q = rng.normal(size=4) * rng.uniform(0.3, 3.0)  # un-normalised on purpose
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(orc.quat_mat(q), ref, atol=1e-14)


# --------------------------------------------------------------------------- pair terms
def _golden_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "terms.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, vals, ders = line.split("|")
        ts, ti, tj, r = head.split()
        rows.append((int(ts), int(ti), int(tj), float(r), vals.split(), ders.split()))
    return rows


def _ev(s):
    return None if s == "X" else eval(s, {"exp": math.exp, "log": math.log})


@pytest.mark.parametrize("row", _golden_rows())
def test_pair_terms_closed_forms(orc, row):
    ts, ti, tj, r, vals, ders = row
    p = vina_params(orc) if ts == 0 else orc.make_params(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS,
                                                         synth.TRIDS_WEIGHTS, 10.0)
    e, dr, _ = orc.pair(p, ti, tj, r)
    for t in range(5):
        if _ev(vals[t]) is not None:
            assert e[t] == pytest.approx(_ev(vals[t]), abs=1e-12), f"term {t}"
        if _ev(ders[t]) is not None:
            assert dr[t] == pytest.approx(_ev(ders[t]), abs=1e-12), f"d term {t}"


def test_gmm_term_closed_form(orc):
    """E_MDN pair = -sum_k pi_k exp(-(r-mu_k)^2/(2 sigma_k^2)) for r < 5 (Sec. 2, Eqs. P(d), E_MDN)."""
    gmm = np.zeros((8, 8, 2, 3))
    gmm[2, 4, 0] = (0.7, 3.0, 0.5)
    gmm[2, 4, 1] = (0.2, 4.0, 1.0)
    p = orc.make_params(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0, gmm=gmm)
    e, dr, _ = orc.pair(p, 2, 4, 3.0)
    assert e[0] == pytest.approx(-(0.7 + 0.2 * math.exp(-0.5)), abs=1e-14)
    assert dr[0] == pytest.approx(-0.2 * math.exp(-0.5), abs=1e-14)
    e, _, _ = orc.pair(p, 2, 4, 3.5)
    assert e[0] == pytest.approx(-(0.7 * math.exp(-0.5) + 0.2 * math.exp(-0.125)), abs=1e-14)
    e, _, _ = orc.pair(p, 2, 4, 5.0)  # cutoff 5 A, strict
    assert e[0] == 0.0
    e, _, _ = orc.pair(p, 2, 4, 3.0, inter=False)  # intra pairs carry no MDN term
    assert e[0] == 0.0


@pytest.mark.parametrize("ts", [0, 1])
def test_one_atom_pair_energy_is_weighted_terms(orc, ts):
    """A one-atom ligand and a one-atom pocket: E = sum_t w_t f_t(r) exactly."""
    p = vina_params(orc) if ts == 0 else trids_params(orc)
    w = synth.VINA_WEIGHTS if ts == 0 else synth.TRIDS_WEIGHTS
    for ti, tj, r in [(0, 7, 3.3), (3, 5, 2.9), (6, 6, 4.4), (1, 2, 7.9)]:
        st, lg = orc.pack(np.zeros((1, 3)), [ti], np.zeros((0, 2)), [])
        assert st == 0
        dof = np.array([r, 0, 0, 1, 0, 0, 0.0])
        st, ev = orc.score(p, np.zeros((1, 3)), np.array([tj]), lg, dof)
        e, dr, _ = orc.pair(p, ti, tj, r)
        assert ev.e_total == pytest.approx(float(np.dot(w, e)), abs=1e-14)
        assert ev.g_dof[0] == pytest.approx(float(np.dot(w, dr)), abs=1e-14)
        np.testing.assert_allclose(list(ev.g_w), e, atol=1e-14)


# --------------------------------------------------------------------------- pack
def _nx_expected(lig):
    """Brute-force topology from networkx: fragments, root, BFS torsions, DFS layout."""
    n = len(lig.type)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(map(tuple, lig.bonds))
    H = nx.Graph()
    H.add_nodes_from(range(n))
    H.add_edges_from(tuple(b) for b, r in zip(lig.bonds, lig.rotatable) if not r)
    comps = sorted((sorted(c) for c in nx.connected_components(H)), key=lambda c: c[0])
    fid = {a: i for i, c in enumerate(comps) for a in c}
    F = nx.Graph()
    F.add_nodes_from(range(len(comps)))
    for (a, b), r in zip(lig.bonds, lig.rotatable):
        if r:
            F.add_edge(fid[a], fid[b], atoms={fid[a]: a, fid[b]: b})
    ecc = nx.eccentricity(F) if len(comps) > 1 else {0: 0}
    root = min(range(len(comps)), key=lambda f: (ecc[f], comps[f][0]))
    order, par = [root], {root: None}
    for u in order:
        for v in sorted(F.neighbors(u), key=lambda f: comps[f][0]):
            if v not in par:
                par[v] = u
                order.append(v)
    tor = {f: k - 1 for k, f in enumerate(order)}  # child fragment -> torsion index
    pre = []

    def dfs(u):
        pre.append(u)
        for v in sorted((v for v in F.neighbors(u) if par.get(v) == u), key=lambda f: comps[f][0]):
            dfs(v)
    dfs(root)
    perm = [a for f in pre for a in comps[f]]
    new = {a: i for i, a in enumerate(perm)}
    frag = [0 if fid[a] == root else tor[fid[a]] + 1 for a in perm]
    T = len(comps) - 1
    tors = []
    for f in order[1:]:
        p = par[f]
        at = F.edges[p, f]["atoms"]
        desc = nx.descendants(nx.bfs_tree(F, root), f) | {f}
        idx = sorted(new[a] for g in desc for a in comps[g])
        assert idx == list(range(idx[0], idx[-1] + 1)), "moving subtree not contiguous"
        tors.append((new[at[p]], new[at[f]], -1 if p == root else tor[p], idx[0], idx[-1] + 1))
    sp = dict(nx.all_pairs_shortest_path_length(G))
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)
             if frag[i] != frag[j] and sp[perm[i]][perm[j]] >= 4]
    out = [n, T, len(pairs)] + perm + frag + [v for t in tors for v in t] + [v for pr in pairs for v in pr]
    return np.array(out, dtype=np.int32)


def test_pack_matches_networkx_brute_force(orc):
    rng = np.random.default_rng(11)
    ligs = small_ligands(8) + [synth.gen_ligand(rng, 70, 20), synth.gen_ligand(rng, 1, 0),
                                synth.gen_ligand(rng, 2, 0), synth.gen_ligand(rng, 60, 15)]
    for lig in ligs:
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        assert st == 0
        np.testing.assert_array_equal(orc.topology(lg), _nx_expected(lig))
        assert lg.n_tor == lig.n_tor


def test_pack_rejects_bad_inputs(orc):
    lig = synth.workload("single_ligand").ligands[0]
    # rotatable bond that closes a ring: add a ring bond and flag one ring edge
    bonds = np.vstack([lig.bonds, [[0, 5]]]) if not any((lig.bonds == [0, 5]).all(1)) else lig.bonds
    rot = np.concatenate([lig.rotatable, [1]])
    assert orc.pack(lig.xyz, lig.type, bonds, rot)[0] != 0
    # disconnected
    assert orc.pack(lig.xyz, lig.type, lig.bonds[1:], lig.rotatable[1:])[0] != 0
    # duplicate bond
    assert orc.pack(lig.xyz, lig.type, np.vstack([lig.bonds, lig.bonds[:1]]),
                    np.concatenate([lig.rotatable, [0]]))[0] != 0
    # type out of range, NaN coordinate
    t = lig.type.copy()
    t[3] = 8
    assert orc.pack(lig.xyz, t, lig.bonds, lig.rotatable)[0] != 0
    x = lig.xyz.copy()
    x[2, 1] = np.nan
    assert orc.pack(x, lig.type, lig.bonds, lig.rotatable)[0] != 0
    # too many atoms
    rng = np.random.default_rng(0)
    big = synth.gen_ligand(rng, 71, 0)
    assert orc.pack(big.xyz, big.type, big.bonds, big.rotatable)[0] != 0


# --------------------------------------------------------------------------- FK
def test_fk_frames_match_brute_rodrigues(orc):
    rng = np.random.default_rng(4)
    for lig in small_ligands(10):
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        for _ in range(5):
            dof = random_dof(rng, lg.n_tor)
            np.testing.assert_allclose(orc.fk(lg, dof), orc.fk(lg, dof, brute=True), atol=1e-12)


def test_fk_identity_and_invariants(orc):
    rng = np.random.default_rng(5)
    for lig in small_ligands(6):
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        perm = np.array(lg.perm[:lg.n_atoms])
        y = lig.xyz[perm]
        c = np.array(lg.c[:])
        # theta = 0, q = identity, t = c reproduces the input geometry
        dof0 = np.concatenate([c, [1, 0, 0, 0], np.zeros(lg.n_tor)])
        np.testing.assert_allclose(orc.fk(lg, dof0), y, atol=1e-12)
        frag = np.array(lg.frag[:lg.n_atoms])
        inv = {tuple(sorted(b)) for b in lig.bonds}
        for _ in range(4):
            x = orc.fk(lg, random_dof(rng, lg.n_tor))
            for a, b in lig.bonds:  # bond lengths preserved
                ia, ib = np.nonzero(perm == a)[0][0], np.nonzero(perm == b)[0][0]
                assert np.linalg.norm(x[ia] - x[ib]) == pytest.approx(np.linalg.norm(y[ia] - y[ib]), abs=1e-12)
            for f in set(frag.tolist()):  # rigid fragments stay rigid
                ix = np.nonzero(frag == f)[0]
                dx = np.linalg.norm(x[ix][:, None] - x[ix][None], axis=2)
                dy = np.linalg.norm(y[ix][:, None] - y[ix][None], axis=2)
                np.testing.assert_allclose(dx, dy, atol=1e-12)
        del inv


# --------------------------------------------------------------------------- energy
@pytest.mark.parametrize("ts", [0, 1])
def test_rigid_motion_of_whole_complex(orc, ts):
    w = synth.workload("single_ligand")
    p = vina_params(orc) if ts == 0 else trids_params(orc)
    lig = w.ligands[0]
    st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
    rng = np.random.default_rng(6)
    for _ in range(4):
        dof = random_dof(rng, lg.n_tor, box=4.0)
        st, ev = orc.score(p, w.pocket.xyz, w.pocket.type, lg, dof)
        Q = Rotation.random(random_state=int(rng.integers(1 << 30)))
        s = rng.normal(size=3) * 5
        qQ = Q.as_quat()  # x y z w
        qQ = np.array([qQ[3], qQ[0], qQ[1], qQ[2]])
        q = dof[3:7]
        qn = np.array([qQ[0] * q[0] - qQ[1:] @ q[1:]]
                      + list(qQ[0] * q[1:] + q[0] * qQ[1:] + np.cross(qQ[1:], q[1:])))
        dof2 = np.concatenate([Q.apply(dof[:3]) + s, qn, dof[7:]])
        st, ev2 = orc.score(p, Q.apply(w.pocket.xyz) + s, w.pocket.type, lg, dof2)
        assert ev2.e_total == pytest.approx(ev.e_total, rel=1e-10, abs=1e-10)
        np.testing.assert_allclose(np.array(ev2.x)[:lg.n_atoms], Q.apply(np.array(ev.x)[:lg.n_atoms]) + s,
                                   atol=1e-10)


def test_intra_energy_rigid_invariance_and_zero_net_force(orc):
    p = vina_params(orc)
    rng = np.random.default_rng(8)
    for lig in small_ligands(5):
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        th = rng.uniform(-math.pi, math.pi, lg.n_tor)
        e0 = None
        for _ in range(3):
            q = rng.normal(size=4)
            dof = np.concatenate([rng.normal(size=3) * 10, q / np.linalg.norm(q), th])
            st, ev = orc.score(p, np.zeros((0, 3)), np.zeros(0, np.int32), lg, dof)
            assert ev.e_inter == 0
            e0 = ev.e_intra if e0 is None else e0
            assert ev.e_intra == pytest.approx(e0, rel=1e-12, abs=1e-12)
            scale = 1 + np.abs(np.array(ev.g_x)[:lg.n_atoms]).sum()
            np.testing.assert_allclose(ev.g_dof[:3], 0, atol=1e-12 * scale)   # net force
            np.testing.assert_allclose(ev.tau[:], 0, atol=1e-11 * scale)      # net torque


def _fd_check(orc, p, pk, lg, dof, rng, h=1e-4):
    st, ev = orc.score(p, pk.xyz, pk.type, lg, dof)
    g = np.array(ev.g_dof[:7 + lg.n_tor])
    bad = []
    for j in range(7 + lg.n_tor):
        def fd(hh):
            dp, dm = dof.copy(), dof.copy()
            dp[j] += hh
            dm[j] -= hh
            return (orc.score(p, pk.xyz, pk.type, lg, dp)[1].e_total
                    - orc.score(p, pk.xyz, pk.type, lg, dm)[1].e_total) / (2 * hh)
        f1, f2 = fd(h), fd(h / 2)
        if abs(f1 - f2) > 1e-3 * (1 + abs(f1)):   # a cutoff or kink inside the stencil
            continue
        rich = (4.0 * f2 - f1) / 3.0               # Richardson: cancels the h^2 error term
        if abs(rich - g[j]) > 1e-7 * (1 + abs(g[j])):
            bad.append((j, rich, g[j]))
    return bad


@pytest.mark.parametrize("ts", [0, 1])
def test_dof_gradient_matches_central_differences(orc, ts):
    """FP64 central differences (h = 1e-4) of E w.r.t. t, q (through E(q/|q|)) and theta."""
    w = synth.workload("single_ligand")
    p = vina_params(orc) if ts == 0 else trids_params(orc)
    rng = np.random.default_rng(9)
    for lig in small_ligands(3):
        st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
        for _ in range(3):
            dof = random_dof(rng, lg.n_tor, box=6.0)
            dof[3:7] *= rng.uniform(0.5, 2.0)  # off the unit sphere: dE/dq is for E(q/|q|)
            assert _fd_check(orc, p, w.pocket, lg, dof, rng) == []


@pytest.mark.parametrize("ts", [0, 1])
def test_parameter_gradients(orc, ts):
    """dE/dw_t equals the per-term sums (E is linear in w); dE/dR_a matches FD in R_a."""
    w = synth.workload("single_ligand")
    rng = np.random.default_rng(10)
    lig = w.ligands[0]
    st, lg = orc.pack(lig.xyz, lig.type, lig.bonds, lig.rotatable)
    dof = random_dof(rng, lg.n_tor, box=4.0)
    base = vina_params(orc) if ts == 0 else trids_params(orc)
    st, ev = orc.score(base, w.pocket.xyz, w.pocket.type, lg, dof)
    W = list(synth.VINA_WEIGHTS if ts == 0 else synth.TRIDS_WEIGHTS)
    for t in range(5):
        W2 = list(W)
        W2[t] += 1.0
        p2 = vina_params(orc) if ts == 0 else trids_params(orc)
        p2.w[t] = W2[t]
        e2 = orc.score(p2, w.pocket.xyz, w.pocket.type, lg, dof)[1].e_total
        assert e2 - ev.e_total == pytest.approx(ev.g_w[t], rel=1e-9, abs=1e-10)
    for a in range(8):
        vals = []
        for hh in (1e-4, 5e-5):
            pp = vina_params(orc) if ts == 0 else trids_params(orc)
            pm = vina_params(orc) if ts == 0 else trids_params(orc)
            pp.radius[a] += hh
            pm.radius[a] -= hh
            ep = orc.score(pp, w.pocket.xyz, w.pocket.type, lg, dof)[1].e_total
            em = orc.score(pm, w.pocket.xyz, w.pocket.type, lg, dof)[1].e_total
            vals.append((ep - em) / (2 * hh))
        if abs(vals[0] - vals[1]) > 1e-6 * (1 + abs(vals[0])):
            continue
        assert vals[0] == pytest.approx(ev.g_R[a], rel=1e-6, abs=1e-7)


def test_torsion_with_axis_atom_only_has_zero_gradient(orc):
    """A torsion whose moving side is one atom lying on the bond axis cannot change E."""
    xyz = np.array([[0, 0, 0], [1.5, 0, 0], [3.0, 0.0, 0.0], [-0.5, 1.4, 0]])
    st, lg = orc.pack(xyz, [0, 1, 2, 3], [[0, 1], [1, 2], [0, 3]], [0, 1, 0])
    assert st == 0 and lg.n_tor == 1
    p = vina_params(orc)
    pk = np.array([[2.0, 3.0, 1.0], [4.0, -2.0, 0.5]])
    rng = np.random.default_rng(1)
    for _ in range(5):
        st, ev = orc.score(p, pk, np.array([0, 5]), lg, random_dof(rng, 1, 1.0))
        assert abs(ev.g_dof[7]) < 1e-12


# --------------------------------------------------------------------------- sampling
def test_metropolis_beta_gives_half_acceptance_at_10(orc):
    """beta = 0.069 makes the acceptance probability 0.5 at dE = 10 (Sec. 2)."""
    assert math.exp(-0.069 * 10) == pytest.approx(0.5, abs=0.002)
    assert orc.metropolis_accept(3.0, 3.0 + 1e-9, 0.069, 0.999999)
    assert orc.metropolis_accept(-5.0, 0.0, 0.069, 0.9999)
    assert not orc.metropolis_accept(10.0, 0.0, 0.069, 0.51)
    assert orc.metropolis_accept(10.0, 0.0, 0.069, 0.49)
    # empirical rate over the Philox draws
    us = [orc.metropolis_u(77, 0, p, l) for p in range(400) for l in range(1, 8)]
    rate = np.mean([orc.metropolis_accept(10.0, 0.0, 0.069, u) for u in us])
    assert rate == pytest.approx(0.5016, abs=0.03)


def test_init_pose_ranges_and_uniform_rotation(orc):
    cfg = orc.sample_cfg(seed=123, box_lo=(-1, -2, -3), box_hi=(4, 5, 6))
    dofs = np.array([orc.init_pose(cfg, 5, 3, p) for p in range(4000)])
    assert (dofs[:, :3] >= [-1, -2, -3]).all() and (dofs[:, :3] < [4, 5, 6]).all()
    np.testing.assert_allclose(np.linalg.norm(dofs[:, 3:7], axis=1), 1, atol=1e-14)
    assert (dofs[:, 7:] >= -math.pi).all() and (dofs[:, 7:] < math.pi).all()
    # Haar-uniform rotations: E[R] = 0 and E[q_i^2] = 1/4
    R = Rotation.from_quat(dofs[:, [4, 5, 6, 3]]).as_matrix()
    assert np.abs(R.mean(axis=0)).max() < 0.05
    np.testing.assert_allclose((dofs[:, 3:7] ** 2).mean(axis=0), 0.25, atol=0.02)


def test_perturb_changes_exactly_one_variable(orc):
    cfg = orc.sample_cfg(seed=9)
    T = 4
    counts = np.zeros(6 + T)
    for p in range(3000):
        dof = orc.init_pose(cfg, T, 0, p)
        c, d2 = orc.perturb(cfg, T, 0, p, 1 + p % 7, dof)
        counts[c] += 1
        changed = np.nonzero(np.abs(d2 - dof) > 0)[0].tolist()
        if c < 3:
            assert changed == [c]
        elif c < 6:
            assert set(changed) <= {3, 4, 5, 6}
            # the rotation is about world axis e_(c-3): that axis is left fixed
            R0 = orc.quat_mat(dof[3:7])
            R1 = orc.quat_mat(d2[3:7])
            e = np.eye(3)[c - 3]
            np.testing.assert_allclose(R1 @ R0.T @ e, e, atol=1e-12)
        else:
            assert changed == [7 + c - 6]
    assert counts.min() > 3000 / (6 + T) * 0.75


def test_adam_step_matches_torch(orc):
    """The t and theta parts of the update equal torch.optim.Adam; the rotation part applies
    the same step as a left-multiplied rotation vector."""
    import torch
    cfg = orc.sample_cfg(lr=0.1, box_lo=(-100,) * 3, box_hi=(100,) * 3)
    rng = np.random.default_rng(12)
    T = 3
    dof = random_dof(rng, T, 2.0)
    dof[7:] *= 0.2
    x = torch.tensor(np.concatenate([dof[:3], np.zeros(3), dof[7:]]), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([x], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros(6 + T), np.zeros(6 + T)
    d = dof.copy()
    for step in range(1, 8):
        g = rng.normal(size=6 + T) * 3
        before = x.detach().clone().numpy()
        x.grad = torch.tensor(g)
        opt.step()
        after = x.detach().numpy()
        q_prev = d[3:7].copy()
        orc.adam_step(cfg, T, step, g, m, v, d)
        np.testing.assert_allclose(d[:3], after[:3], atol=1e-12)
        np.testing.assert_allclose(d[7:], after[6:], atol=1e-12)
        dw = after[3:6] - before[3:6]
        expect = Rotation.from_rotvec(dw) * Rotation.from_quat([q_prev[1], q_prev[2], q_prev[3], q_prev[0]])
        qe = expect.as_quat()
        qe = np.array([qe[3], qe[0], qe[1], qe[2]])
        assert min(np.abs(d[3:7] - qe).max(), np.abs(d[3:7] + qe).max()) < 1e-12


def test_single_atom_sampler_is_textbook_adam(orc):
    """0 torsions, 1 atom, one loop: the sampler is plain Adam on the atom position
    (S evaluations, S-1 updates)."""
    import torch
    p = vina_params(orc)
    st, lg = orc.pack(np.zeros((1, 3)), [0], np.zeros((0, 2)), [])
    pk = np.array([[0.0, 0.0, 0.0]])
    pt = np.array([7], dtype=np.int32)
    S = 25
    cfg = orc.sample_cfg(steps=S, mc_loops=1, seed=3, box_lo=(-3,) * 3, box_hi=(3,) * 3)
    dof_fin, e_fin, _ = orc.sample_ligand(cfg, p, pk, pt, lg, 0, 1)
    x0 = orc.init_pose(cfg, 0, 0, 0)
    x = torch.tensor(x0[:3], requires_grad=True)
    opt = torch.optim.Adam([x], lr=0.1)
    for _ in range(S - 1):
        d = np.concatenate([x.detach().numpy(), x0[3:7]])
        g = np.array(orc.score(p, pk, pt, lg, d)[1].g_dof[:3])
        x.grad = torch.tensor(g)
        opt.step()
        with torch.no_grad():
            x.clamp_(-3, 3)
    np.testing.assert_allclose(dof_fin[0, :3], x.detach().numpy(), atol=1e-12)
    d = np.concatenate([x.detach().numpy(), x0[3:7]])
    assert e_fin[0] == pytest.approx(orc.score(p, pk, pt, lg, d)[1].e_total, abs=1e-12)


def test_loop_schedule(orc):
    for S, Lm in [(30, 8), (50, 8), (5, 8), (8, 8), (100, 7)]:
        n = [orc.loop_steps(S, Lm, l) for l in range(Lm)]
        assert sum(n) == S and max(n) - min(n) <= 1 and n == sorted(n, reverse=True)


# --------------------------------------------------------------------------- top-k
def _brute_topk(E, X, k, rho):
    """Lexicographically first maximal conflict-free set in (E, index) order, by enumeration."""
    P, L = X.shape[:2]
    order = sorted((i for i in range(P) if np.isfinite(E[i])), key=lambda i: (E[i], i))
    conf = lambda a, b: ((X[a] - X[b]) ** 2).sum() < rho * rho * L
    best = None
    for r in range(len(order) + 1):
        for sub in itertools.combinations(order, r):   # combinations keep the order
            if any(conf(a, b) for a, b in itertools.combinations(sub, 2)):
                continue
            if any(all(not conf(o, s) for s in sub) for o in order if o not in sub):
                continue  # not maximal
            pos = [order.index(s) for s in sub]
            if best is None or pos < best[0]:
                best = (pos, list(sub))
    out = best[1][:k]
    return out + [-1] * (k - len(out))


def test_topk_matches_brute_force(orc):
    rng = np.random.default_rng(13)
    for trial in range(40):
        P, L = int(rng.integers(1, 8)), 3
        base = rng.normal(size=(3, L, 3)) * 2
        X = base[rng.integers(0, 3, P)] + rng.normal(size=(P, L, 3)) * rng.choice([0.05, 0.8])
        E = rng.integers(-3, 3, P).astype(float)  # many ties
        if trial % 5 == 0:
            E[0] = np.nan
        k = int(rng.integers(1, 5))
        idx, _ = orc.topk(E, X, k, 1.0)
        assert idx.tolist() == _brute_topk(E, X, k, 1.0)
    # rho = 0 disables dedupe: plain (E, index) order
    E = np.array([2.0, 1.0, 1.0, 0.5])
    X = np.zeros((4, 2, 3))
    assert orc.topk(E, X, 3, 0.0)[0].tolist() == [3, 1, 2]


def test_screen_energy_values_and_identities(orc):
    """E_screen (Sec. 2, virtual screening) divides the docking score by 1 + w_tor N_tor:
    values worked by hand at the paper's w_tor = 0.01, the identities at w_tor = 0 and at
    N_tor = 0, and the direction of the penalty (more torsions, less negative score)."""
    assert orc.screen_energy(-10.5, 0.01, 5) == pytest.approx(-10.0, rel=1e-14)      # 1.05
    assert orc.screen_energy(-12.0, 0.01, 20) == pytest.approx(-10.0, rel=1e-14)     # 1.20
    assert orc.screen_energy(4.4, 0.01, 10) == pytest.approx(4.0, rel=1e-14)         # 1.10
    assert orc.screen_energy(-7.25, 0.0, 13) == -7.25
    assert orc.screen_energy(-7.25, 0.01, 0) == -7.25
    vals = [orc.screen_energy(-9.0, 0.01, t) for t in range(21)]
    assert all(a < b for a, b in zip(vals, vals[1:]))


def test_multiple_boxes_assign_pose_p_to_box_p_mod_n(orc):
    """Several docking boxes: init, perturbation and the Adam clamp of pose p use box p mod n."""
    lo = np.array([[-30, -5, -5], [10, 10, 10], [-2, 20, -40]], dtype=float)
    hi = lo + np.array([[4, 4, 4], [2, 3, 4], [5, 5, 5]], dtype=float)
    cfg = orc.sample_cfg(seed=5, box_lo=lo, box_hi=hi, lr=5.0)
    T = 2
    rng = np.random.default_rng(0)
    for p in range(30):
        b = p % 3
        d = orc.init_pose(cfg, T, 1, p)
        assert (d[:3] >= lo[b]).all() and (d[:3] < hi[b]).all()
        for loop in range(1, 6):
            c, d2 = orc.perturb(cfg, T, 1, p, loop, d)
            assert (d2[:3] >= lo[b]).all() and (d2[:3] <= hi[b]).all()
        m, v = np.zeros(6 + T), np.zeros(6 + T)
        g = rng.normal(size=6 + T) * 100
        orc.adam_step(cfg, T, 1, g, m, v, d, pose=p)
        assert (d[:3] >= lo[b]).all() and (d[:3] <= hi[b]).all()
