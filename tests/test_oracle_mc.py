"""Pins of the oracle's Monte-Carlo orchestration (Sec. 2 "Conformation sampling", Fig. 2).

Two links tie ``or_sample_pose`` / ``or_sample_ligand`` to something other than themselves:

1. A one-atom, two-loop trajectory worked out independently of the oracle's sampler, score
   and update code: the Vina-form terms in closed form (numpy), torch.optim.Adam with a box
   clamp (a fresh optimiser for each loop, so the moments restart), the perturbation and the
   Metropolis test computed from the stated rules on raw Philox words (the Philox itself is
   pinned against cuRAND).  Seeds are chosen so that one case rejects (the state and energy
   saved before the perturbation come back) and one accepts after a translation jump (where
   keeping the old moments would give a different result).  The helper ``McPose`` must
   reproduce these trajectories evaluation by evaluation.
2. ``McPose`` (the same helper the GPU trace checker uses) composed from the separately
   pinned pieces must reproduce the C sampler bit for bit: 1-atom T = 0 and T = 3-5 ligands,
   2 and 8 Monte-Carlo loops, with rejections, acceptances and all three kinds of
   perturbation occurring.
"""
import math

import numpy as np
import pytest

from paper_2510_24186_b300 import synth

from mc_replay import McPose, replay

torch = pytest.importorskip("torch")

# one ligand atom of type C_P (radius 1.9, no flags) against one pocket atom of type C_P at
# the origin; deep enough weights that a jump into the repulsive core is rejected
W_HAND = (-1.0, -0.5, 10.0, -0.0351, -0.587)
R_SUM = 3.8
BOX = 3.0


def _word(orc, seed, lig, pose, loop, purpose, n):
    return orc.lib().or_rand_word(seed, lig, pose, loop, purpose, n)


def _u01(w):
    return (w >> 8) * 2.0 ** -24


def _hand_energy(t):
    """E and dE/dt of the one-atom system: Vina-form terms on d = r - R_sum (no hydrophobic
    or H-bond pair: C_P carries no flags), inside the 8 A cutoff."""
    r = float(np.linalg.norm(t))
    if r >= 8.0:
        return 0.0, np.zeros(3)
    d = r - R_SUM
    g1, g2 = math.exp(-(d / 0.5) ** 2), math.exp(-((d - 3.0) / 2.0) ** 2)
    rep = d * d if d < 0 else 0.0
    e = W_HAND[0] * g1 + W_HAND[1] * g2 + W_HAND[2] * rep
    de = W_HAND[0] * g1 * (-8.0 * d) + W_HAND[1] * g2 * (-(d - 3.0) / 2.0) + W_HAND[2] * (2.0 * d if d < 0 else 0.0)
    return e, de * np.asarray(t) / r


def _hand_trajectory(orc, seed, S, reset_moments=True):
    """The two-loop trajectory of pose 0 of ligand 0, worked out without the oracle's sampler.
    Returns (evaluated (t, E) list, final t, final E, perturbed variable, accepted)."""
    lo, hi = -BOX, BOX
    n0 = S // 2 + S % 2
    n1 = S // 2
    # A1: t_d = lo + u (hi - lo) from words 0-2 of the init stream
    t = np.array([lo + _u01(_word(orc, seed, 0, 0, 0, 0, d)) * (hi - lo) for d in range(3)])
    evals = []
    x = torch.tensor(t, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([x], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
    for j in range(n0):
        e, g = _hand_energy(x.detach().numpy())
        evals.append((x.detach().numpy().copy(), e))
        if j < n0 - 1:
            x.grad = torch.tensor(g)
            opt.step()
            with torch.no_grad():
                x.clamp_(lo, hi)
    t_saved, e_saved = x.detach().numpy().copy(), evals[-1][1]
    # loop 1: one of the 6 variables from word 0, its new value from word 1
    c = ((_word(orc, seed, 0, 0, 1, 1, 0) >> 8) * 6) >> 24
    u1 = _u01(_word(orc, seed, 0, 0, 1, 1, 1))
    t1 = t_saved.copy()
    if c < 3:
        t1[c] = lo + u1 * (hi - lo)
    # a rotation (c >= 3) does not move a one-atom ligand about its own centroid
    with torch.no_grad():
        x.copy_(torch.tensor(t1))
    if reset_moments:
        opt = torch.optim.Adam([x], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
    for j in range(n1):
        e, g = _hand_energy(x.detach().numpy())
        evals.append((x.detach().numpy().copy(), e))
        if j < n1 - 1:
            x.grad = torch.tensor(g)
            opt.step()
            with torch.no_grad():
                x.clamp_(lo, hi)
    e1 = evals[-1][1]
    u = _u01(_word(orc, seed, 0, 0, 1, 2, 0))
    accepted = u < math.exp(-0.069 * (e1 - e_saved))
    if accepted:
        return evals, x.detach().numpy().copy(), e1, c, True
    return evals, t_saved, e_saved, c, False


def _setup(orc, S, seed):
    p = orc.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, W_HAND, 8.0)
    st, lg = orc.pack(np.zeros((1, 3)), [1], np.zeros((0, 2)), [])
    assert st == 0
    pk = np.zeros((1, 3))
    pt = np.array([1], dtype=np.int32)
    cfg = orc.sample_cfg(steps=S, mc_loops=2, seed=seed, box_lo=(-BOX,) * 3, box_hi=(BOX,) * 3)
    return p, lg, pk, pt, cfg


def _find_seed(orc, S, want_accept):
    for seed in range(1, 400):
        evals, t_fin, e_fin, c, acc = _hand_trajectory(orc, seed, S)
        if c >= 3 or acc != want_accept:
            continue
        if not want_accept and evals[S // 2 + S % 2][1] - evals[S // 2 + S % 2 - 1][1] < 5.0:
            continue          # want a clear rejection: the jump lands well uphill
        return seed
    pytest.fail("no seed with the wanted Metropolis outcome")


@pytest.mark.parametrize("want_accept", [False, True], ids=["rejected", "accepted"])
def test_two_loop_one_atom_trajectory_worked_by_hand(orc, want_accept):
    S = 8
    seed = _find_seed(orc, S, want_accept)
    evals, t_fin, e_fin, c, acc = _hand_trajectory(orc, seed, S)
    p, lg, pk, pt, cfg = _setup(orc, S, seed)
    rec = []
    mc, fin, e = replay(cfg, p, pk, pt, lg, 0, 0, S, 2, seed, record=rec)
    assert len(rec) == S
    for (ta, ea), (da, eb) in zip(evals, rec):
        np.testing.assert_allclose(da[:3], ta, atol=1e-10)
        assert eb == pytest.approx(ea, abs=1e-10)
    assert mc.accepted == [(1, want_accept)] and mc.perturbed == [(1, c)]
    np.testing.assert_allclose(fin[:3], t_fin, atol=1e-10)
    assert e == pytest.approx(e_fin, abs=1e-10)
    # the C sampler returns the same pose
    dof_c, e_c, _ = orc.sample_ligand(cfg, p, pk, pt, lg, 0, 1)
    np.testing.assert_allclose(dof_c[0, :3], t_fin, atol=1e-10)
    assert e_c[0] == pytest.approx(e_fin, abs=1e-10)
    n0 = S // 2 + S % 2
    if not want_accept:
        # the rejection brings back the state and energy saved before the perturbation
        np.testing.assert_array_equal(fin[:3], rec[n0 - 1][0][:3])
        assert e == rec[n0 - 1][1]
        assert e_c[0] == e
    else:
        # the moments restart at the loop start: carrying them over would end elsewhere
        _, t_keep, _, _, _ = _hand_trajectory(orc, seed, S, reset_moments=False)
        assert np.abs(t_keep - t_fin).max() > 1e-6
        np.testing.assert_allclose(fin[:3], rec[-1][0][:3], atol=0)


def _ligands():
    rng = np.random.default_rng(23)
    out = [synth.Ligand(xyz=np.zeros((1, 3)), type=np.array([3], dtype=np.int32),
                        bonds=np.zeros((0, 2), dtype=np.int32), rotatable=np.zeros(0, dtype=np.uint8), n_tor=0)]
    for T in (3, 4, 5):
        out.append(synth.gen_ligand(rng, int(rng.integers(10, 18)), T))
    return out


@pytest.mark.parametrize("Lmc,S", [(2, 9), (8, 20)])
def test_sampler_equals_replay_of_pinned_pieces(orc, Lmc, S):
    """or_sample_ligand == McPose driven by or_score, bit for bit (final state and energy of
    every pose), for 1-atom and T = 3-5 ligands; both branches of the Metropolis test and all
    three kinds of perturbation must occur."""
    w = synth.workload("single_ligand")
    p = orc.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    pxyz = w.pocket.xyz.astype(np.float64)
    ptype = w.pocket.type.astype(np.int32)
    lo, hi = w.box_center - w.box_size / 2, w.box_center + w.box_size / 2
    P = 6
    acc_seen, kinds = set(), set()
    for li, lig in enumerate(_ligands()):
        st, ol = orc.pack(lig.xyz.astype(np.float64), lig.type, lig.bonds, lig.rotatable)
        assert st == 0 and ol.n_tor == (0 if li == 0 else (2 + li))
        cfg = orc.sample_cfg(steps=S, mc_loops=Lmc, seed=31 + li, box_lo=lo, box_hi=hi, beta=0.069)
        dof_c, e_c, _ = orc.sample_ligand(cfg, p, pxyz, ptype, ol, 40 + li, P)
        for pose in range(P):
            mc, fin, e = replay(cfg, p, pxyz, ptype, ol, 40 + li, pose, S, Lmc, 31 + li)
            assert np.array_equal(fin, dof_c[pose]), (li, pose)
            assert e == e_c[pose] or (math.isnan(e) and math.isnan(e_c[pose]))
            acc_seen |= {a for _, a in mc.accepted}
            kinds |= {0 if c < 3 else (1 if c < 6 else 2) for _, c in mc.perturbed}
    assert acc_seen == {True, False}
    assert kinds == {0, 1, 2}


def _oracle_trace(orc, cfg, p, pxyz, ptype, ol, lig, P, S, Lmc, seed):
    """An FP64 sampler trace in the GPU's record layout ([S][pose][2 D]: state, then E, dE/dt,
    tau, dE/dtheta at offset D = 7 + T) and the returned states and energies."""
    T = ol.n_tor
    D = 7 + T
    trace = np.zeros((S, P, 2 * D))
    fin = np.zeros((1, P, D))
    efin = np.zeros((1, P))
    for pose in range(P):
        mc = McPose(cfg, T, lig, pose, S, Lmc, seed)
        dof = mc.start()
        s = 0
        while dof is not None:
            st, ev = orc.score(p, pxyz, ptype, ol, dof)
            g = np.concatenate([np.array(ev.g_dof[:3]), np.array(ev.tau[:]), np.array(ev.g_dof[7:7 + T])])
            trace[s, pose, :D] = dof
            trace[s, pose, D] = ev.e_total
            trace[s, pose, D + 1:D + 7] = g[:6]
            trace[s, pose, D + 7:D + 7 + T] = g[6:]
            dof = mc.step(dof, ev.e_total, g)
            s += 1
        fin[0, pose] = mc.final
        efin[0, pose] = np.float32(mc.e_cur)
    return trace, fin, efin


def test_trace_checker_follows_the_sampler_and_catches_a_wrong_step(orc):
    """The GPU trace checker, fed the FP64 sampler's own trace, passes with every state
    reproduced; a trace whose post-loop state was not restored after a rejection, or whose
    update used a stale gradient, fails."""
    from parity_util import check_trace
    w = synth.workload("single_ligand")
    p = orc.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    pxyz = w.pocket.xyz.astype(np.float64)
    ptype = w.pocket.type.astype(np.int32)
    lo, hi = w.box_center - w.box_size / 2, w.box_center + w.box_size / 2
    lig = _ligands()[2]
    st, ol = orc.pack(lig.xyz.astype(np.float64), lig.type, lig.bonds, lig.rotatable)
    S, Lmc, seed, P = 12, 4, 77, 4
    cfg = orc.sample_cfg(steps=S, mc_loops=Lmc, seed=seed, box_lo=lo, box_hi=hi)
    trace, fin, efin = _oracle_trace(orc, cfg, p, pxyz, ptype, ol, 0, P, S, Lmc, seed)
    res = check_trace(trace, list(range(P)), P, [ol], pxyz, ptype, p, cfg, S, Lmc, seed, fin, efin)
    assert not res.fails and res.n == S * P and res.s_err < 1e-7   # acos resolution of the angle
    # a rejected loop whose state was not restored
    rej = None
    for pose in range(P):
        mc = McPose(cfg, ol.n_tor, 0, pose, S, Lmc, seed)
        d = mc.start()
        s = 0
        while d is not None:
            st_, ev = orc.score(p, pxyz, ptype, ol, d)
            g = np.concatenate([np.array(ev.g_dof[:3]), np.array(ev.tau[:]), np.array(ev.g_dof[7:7 + ol.n_tor])])
            d = mc.step(d, ev.e_total, g)
            if mc.accepted and mc.accepted[-1][1] is False and rej is None and d is not None:
                rej = (pose, s)
            s += 1
    assert rej is not None, "the seed gives no rejection before the last loop"
    pose, s = rej
    bad = trace.copy()
    bad[s + 1, pose, :7 + ol.n_tor] = trace[s, pose, :7 + ol.n_tor]   # kept the rejected loop's state
    res = check_trace(bad, list(range(P)), P, [ol], pxyz, ptype, p, cfg, S, Lmc, seed, fin, efin)
    assert res.fails
    # an update from the wrong gradient
    bad = trace.copy()
    D = 7 + ol.n_tor
    bad[1, 0, D + 1:D + 4] *= 1.5
    res = check_trace(bad, list(range(P)), P, [ol], pxyz, ptype, p, cfg, S, Lmc, seed, fin, efin)
    assert res.fails
