"""GPU parity: libtrids through its C-ABI against the FP64 oracle, element by element."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_24186_b300 import synth

from parity_util import (report, Stats, block_ok, check_trace, energy_ok, grad_slack, t_slack, xyz_slack, oracle_ligands, oracle_params,
                         pocket_arrays, round_slack, score_params, state_err)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2510_24186_b300 import api as a
    return a


def make(api, w, term_set=0, ligs=None, cell=0.0, cutoff=None):
    sp = score_params(term_set, cutoff=cutoff or (w.cutoff if term_set == 0 else 10.0))
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp, cell=cell)
    b = api.Batch.from_ligands(pk, ligs if ligs is not None else w.ligands)
    return sp, pk, b


def cfg_for(w, seed, S=None, Lmc=None):
    lo = (w.box_center - w.box_size / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_center + w.box_size / 2).astype(np.float32).astype(np.float64)
    return oracle.sample_cfg(steps=S or w.steps, mc_loops=Lmc or w.mc_loops, lr=float(np.float32(0.1)),
                             b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)),
                             beta=float(np.float32(0.069)), seed=seed, box_lo=lo, box_hi=hi)


# --------------------------------------------------------------------------- topology
def test_batch_topology_matches_oracle(api):
    w = synth.workload("single_ligand")
    rng = np.random.default_rng(5)
    ligs = w.ligands + [synth.gen_ligand(rng, int(rng.integers(1, 71)), int(rng.integers(0, 21))) for _ in range(40)]
    ligs.append(synth.gen_ligand(rng, 70, 20))
    sp, pk, b = make(api, w, ligs=ligs)
    for l, ol in enumerate(oracle_ligands(ligs)):
        np.testing.assert_array_equal(b.topology(l), oracle.topology(ol))
    assert b.max_atoms == 70 and b.max_tor == 20


# --------------------------------------------------------------------------- score + gradient
def _score_case(api, w, term_set, ligs, P, seed, xyz=False):
    sp, pk, b = make(api, w, term_set, ligs)
    rng = np.random.default_rng(seed)
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    out = api.score_grad(pk, b, torch.from_numpy(dof).cuda(), grad=True, xyz_grad=xyz)
    torch.cuda.synchronize()
    return sp, b, dof, {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("term_set", [0, 1])
def test_score_grad_parity_single_ligand(api, term_set):
    """Single-ligand workload shapes: one 24-atom ligand, 300-atom pocket, 64 random poses; every pose checked."""
    w = synth.workload("single_ligand")
    sp, b, dof, out = _score_case(api, w, term_set, w.ligands, 64, 11, xyz=True)
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    lg = oracle_ligands(w.ligands)[0]
    T = lg.n_tor
    st = Stats()
    perm = np.array(lg.perm[:lg.n_atoms])
    for p in range(64):
        stt, ev = oracle.score(op, pxyz, ptype, lg, dof[0, p, :7 + T])
        st.n += 1
        energy_ok(out["energy"][0, p], ev, st, f"pose {p}")
        sl = grad_slack(ev)
        assert abs(out["e_inter"][0, p] - ev.e_inter) <= max(1e-3, 1e-5 * abs(ev.e_inter)) + ev.e_slack
        block_ok(out["g_dof"][0, p, :3], ev.g_dof[:3], t_slack(ev), st, f"pose {p} t", rnd=round_slack(ev, 0, 3))
        block_ok(out["g_dof"][0, p, 3:7], ev.g_dof[3:7], sl, st, f"pose {p} q", rnd=round_slack(ev, 3, 7))
        block_ok(out["g_dof"][0, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"pose {p} theta", rnd=round_slack(ev, 7, 7 + T))
        assert np.all(out["g_dof"][0, p, 7 + T:] == 0)
        gx = np.zeros((b.max_atoms, 3))
        gx[perm] = np.array(ev.g_x)[:lg.n_atoms]
        block_ok(out["g_xyz"][0, p].ravel(), gx.ravel(), xyz_slack(ev), st, f"pose {p} xyz")
    report(st, f"score term_set={term_set}")


@pytest.mark.parametrize("term_set", [0, 1])
def test_score_grad_parity_batch_ragged(api, term_set):
    """Adjoint-check workload shapes (ligands 10-40 atoms, 0-10 torsions, 1,500-atom pocket), 37 poses
    (a ragged 32-pose tile), a sample of ligands x poses checked one by one."""
    w = synth.workload("adjoint_check", n_lig=48)
    sp, b, dof, out = _score_case(api, w, term_set, w.ligands, 37, 12)
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    ligs = oracle_ligands(w.ligands)
    rng = np.random.default_rng(3)
    st = Stats()
    for l in range(len(ligs)):
        for p in sorted(set(rng.integers(0, 37, 4).tolist()) | {36}):
            T = ligs[l].n_tor
            stt, ev = oracle.score(op, pxyz, ptype, ligs[l], dof[l, p, :7 + T])
            st.n += 1
            energy_ok(out["energy"][l, p], ev, st, f"lig {l} pose {p}")
            sl = grad_slack(ev)
            block_ok(out["g_dof"][l, p, :3], ev.g_dof[:3], t_slack(ev), st, f"lig {l} pose {p} t", rnd=round_slack(ev, 0, 3))
            block_ok(out["g_dof"][l, p, 3:7], ev.g_dof[3:7], sl, st, f"lig {l} pose {p} q", rnd=round_slack(ev, 3, 7))
            block_ok(out["g_dof"][l, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"lig {l} pose {p} theta",
                     rnd=round_slack(ev, 7, 7 + T))
    report(st, f"score batch term_set={term_set}")


@pytest.mark.parametrize("term_set", [0, 1])
def test_parameter_gradients_and_autograd(api, term_set):
    """dE/dw and dE/dR summed over poses with upstream weights, through TridsScore."""
    from paper_2510_24186_b300.autograd import score as tscore
    w = synth.workload("adjoint_check", n_lig=12)
    sp, pk, b = make(api, w, term_set)
    rng = np.random.default_rng(4)
    P = 40
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    d = torch.from_numpy(dof).cuda().requires_grad_(True)
    W = torch.tensor(list(sp.w), dtype=torch.float64, requires_grad=True)
    R = torch.tensor(list(sp.radius), dtype=torch.float64, requires_grad=True)
    E = tscore(d, W, R, pk, b)
    ebar = torch.from_numpy(rng.uniform(-1, 1, (b.n_lig, P)).astype(np.float32)).cuda()
    (E * ebar).sum().backward()
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    ligs = oracle_ligands(w.ligands)
    gw = np.zeros(5)
    gr = np.zeros(16)
    eb = ebar.cpu().numpy().astype(np.float64)
    gd = d.grad.cpu().numpy()
    st = Stats()
    for l in range(b.n_lig):
        for p in range(P):
            T = ligs[l].n_tor
            stt, ev = oracle.score(op, pxyz, ptype, ligs[l], dof[l, p, :7 + T])
            gw += eb[l, p] * np.array(ev.g_w)
            gr += eb[l, p] * np.array(ev.g_R)
            block_ok(gd[l, p, :7 + T], eb[l, p] * np.array(ev.g_dof[:7 + T]), abs(eb[l, p]) * grad_slack(ev), st,
                     f"lig {l} pose {p}", rnd=abs(eb[l, p]) * round_slack(ev, 0, 7 + T))
    block_ok(W.grad.numpy(), gw, 0.0, st, "dE/dw")
    block_ok(R.grad.numpy(), gr[:8], 0.0, st, "dE/dR")
    report(st, f"param grads term_set={term_set}")


# --------------------------------------------------------------------------- sampler
def _sample(api, pk, b, w, seed, P=None, S=None, **kw):
    P = P or w.poses
    S = S or w.steps
    return api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, **kw)


@pytest.mark.parametrize("term_set", [0, 1])
def test_sampler_per_step_parity_single_ligand(api, term_set):
    """Single-ligand workload: every pose, every evaluation: energy, gradient, Adam update, Metropolis
    decision, perturbation, initial and final state against the oracle."""
    w = synth.workload("single_ligand")
    sp, pk, b = make(api, w, term_set)
    seed = 1001
    P, S = w.poses, w.steps
    out = _sample(api, pk, b, w, seed, trace_poses=list(range(P)))
    assert api.sync(b, P, out["state"], timeout_ms=60000) == 0
    st = check_trace(out["trace"].cpu().numpy(), list(range(P)), P, oracle_ligands(w.ligands),
                     *pocket_arrays(w.pocket), oracle_params(sp), cfg_for(w, seed), S, w.mc_loops, seed,
                     out["dof"].cpu().numpy(), out["energy"].cpu().numpy())
    report(st, f"sampler single ligand term_set={term_set}")


def test_persistent_graph_and_per_ligand_forms_are_bit_identical(api):
    w = synth.workload("adjoint_check", n_lig=20)
    sp, pk, b = make(api, w)
    P, S = 45, 13
    runs = []
    for mode, graph in ((0, True), (0, False), (1, False)):
        o = api.sample(pk, b, P, S, mc_loops=4, seed=77, mode=mode, use_graph=graph)
        torch.cuda.synchronize()
        runs.append((o["dof"].cpu().numpy(), o["energy"].cpu().numpy()))
    for d, e in runs[1:]:
        np.testing.assert_array_equal(d, runs[0][0])
        np.testing.assert_array_equal(e, runs[0][1])
    # replaying the cached graph gives the same result again
    o = api.sample(pk, b, P, S, mc_loops=4, seed=77, mode=0, use_graph=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o["dof"].cpu().numpy(), runs[0][0])


def test_resume_is_bit_exact(api):
    """S = S1 + S2 with the state buffer carried over equals one S-evaluation run."""
    w = synth.workload("adjoint_check", n_lig=10)
    sp, pk, b = make(api, w)
    P, S = 33, 21
    full = api.sample(pk, b, P, S, mc_loops=5, seed=5)
    part = api.sample(pk, b, P, S, mc_loops=5, seed=5, step_end=8)
    part = api.sample(pk, b, P, S, mc_loops=5, seed=5, step_begin=8, dof=part["dof"], state=part["state"],
                      energy=part["energy"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(part["dof"].cpu().numpy(), full["dof"].cpu().numpy())
    np.testing.assert_array_equal(part["energy"].cpu().numpy(), full["energy"].cpu().numpy())


def test_edge_ligands_and_tiny_schedules(api):
    """A 1-atom ligand, a 2-atom ligand, a 70-atom / 20-torsion ligand, 1 pose, S < loops."""
    w = synth.workload("single_ligand")
    rng = np.random.default_rng(9)
    ligs = [synth.gen_ligand(rng, 1, 0), synth.gen_ligand(rng, 2, 0), synth.gen_ligand(rng, 70, 20)]
    sp, pk, b = make(api, w, ligs=ligs)
    for P, S, Lm in ((1, 3, 8), (3, 9, 2)):
        seed = 31 + P
        out = api.sample(pk, b, P, S, mc_loops=Lm, seed=seed, trace_poses=list(range(3 * P)))
        torch.cuda.synchronize()
        st = check_trace(out["trace"].cpu().numpy(), list(range(3 * P)), P, oracle_ligands(ligs),
                         *pocket_arrays(w.pocket), oracle_params(sp), cfg_for(w, seed, S, Lm), S, Lm, seed,
                         out["dof"].cpu().numpy(), out["energy"].cpu().numpy())
        report(st, f"edge P={P} S={S}")


def test_topk_matches_oracle(api):
    w = synth.workload("adjoint_check", n_lig=16)
    sp, pk, b = make(api, w)
    P = 64
    out = api.sample(pk, b, P, 16, mc_loops=4, seed=9)
    for rho, k in ((1.0, 9), (0.0, 5), (2.5, 12)):
        idx, e = api.topk(b, out["energy"], out["dof"], k, rho)
        torch.cuda.synchronize()
        idx = idx.cpu().numpy()
        E = out["energy"].cpu().numpy().astype(np.float64)
        dof = out["dof"].cpu().numpy().astype(np.float64)
        ligs = oracle_ligands(w.ligands)
        for l in range(b.n_lig):
            X = np.stack([oracle.fk(ligs[l], dof[l, p, :7 + ligs[l].n_tor]) for p in range(P)])
            ref, near = oracle.topk(E[l], X, k, rho)
            if near == 0:
                np.testing.assert_array_equal(idx[l], ref)
            np.testing.assert_array_equal(e.cpu().numpy()[l][idx[l] >= 0], E[l][idx[l][idx[l] >= 0]].astype(np.float32))


def test_screen_energy_of_kept_poses_matches_oracle(api):
    """E_screen = E_inter / (1 + w_tor N_tor) of the top-k poses: the GPU's e_inter of the
    sampled poses (trids_score_grad) rescaled by trids_screen_energy, against the oracle's
    FP64 E_inter of the same FP32 DOFs; empty slots (fewer distinct poses than k) are NaN."""
    w = synth.workload("adjoint_check", n_lig=16)
    sp, pk, b = make(api, w)
    P, k = 64, 9
    out = api.sample(pk, b, P, 16, mc_loops=4, seed=11)
    idx, _ = api.topk(b, out["energy"], out["dof"], k, 1.0)
    sc = api.score_grad(pk, b, out["dof"], grad=False)
    es = api.screen_energy(pk, b, idx, sc["e_inter"])
    # a slot past the end and a -1 slot must come out NaN, the rest as before
    idx2 = idx.clone()
    idx2[0, 0] = -1
    idx2[1, 0] = P
    es2 = api.screen_energy(pk, b, idx2, sc["e_inter"])
    torch.cuda.synchronize()
    idx, es, es2 = idx.cpu().numpy(), es.cpu().numpy(), es2.cpu().numpy()
    dof = out["dof"].cpu().numpy().astype(np.float64)
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    ligs = oracle_ligands(w.ligands)
    w_tor = float(np.float32(sp.w_tor))
    st = Stats()
    for l in range(b.n_lig):
        T = ligs[l].n_tor
        for s_ in range(k):
            p = int(idx[l, s_])
            if p < 0:
                assert math.isnan(es[l, s_])
                continue
            _, ev = oracle.score(op, pxyz, ptype, ligs[l], dof[l, p, :7 + T])
            ref = oracle.screen_energy(ev.e_inter, w_tor, T)
            d = abs(float(es[l, s_]) - ref)
            st.n += 1
            st.energy(d, ref)
            if not d <= max(1e-3, 1e-5 * abs(ref)) + ev.e_slack:
                st.fail(f"lig {l} slot {s_} pose {p}: E_screen gpu {es[l, s_]!r} oracle {ref!r}")
    assert math.isnan(es2[0, 0]) and math.isnan(es2[1, 0])
    np.testing.assert_array_equal(es2[2:], es[2:])
    np.testing.assert_array_equal(es2[:2, 1:], es[:2, 1:])
    report(st, "E_screen of the top-9 poses")


def test_nonfinite_pose_is_flagged_and_sync_times_out(api):
    """Host-observable failures: a huge radius overflows the repulsion term to inf in
    float32, the pose is frozen and trids_sync reports it; a zero wait limit times out."""
    w = synth.workload("single_ligand")
    sp = score_params(0)
    rad = list(sp.radius)
    rad[0] = 1e30
    sp.radius = rad
    pk = api.Pocket(w.pocket.xyz, np.zeros_like(w.pocket.type), w.box_center, w.box_size, sp)
    lig = w.ligands[0]
    lig = synth.Ligand(lig.xyz, np.zeros_like(lig.type), lig.bonds, lig.rotatable, lig.n_tor)
    b = api.Batch.from_ligands(pk, [lig])
    out = api.sample(pk, b, 32, 8, mc_loops=2, seed=1)
    assert api.sync(b, 32, out["state"], timeout_ms=60000) == -5
    w2 = synth.workload("adjoint_check", n_lig=64)
    sp2, pk2, b2 = make(api, w2)
    out = api.sample(pk2, b2, 128, 40, mc_loops=8, seed=2)
    rc = api.sync(b2, 128, out["state"], timeout_ms=1e-6)
    assert rc in (-4, 0)
    assert api.sync(b2, 128, out["state"], timeout_ms=120000) == 0


def test_batched_screening_full_size_sampled(api):
    """The benchmark's workload and launch (1,024 ligands x 128 poses x 50 evaluations,
    persistent launch in a CUDA graph): 256 seeded poses traced and checked per
    evaluation, top-9 of the traced ligands checked against the oracle."""
    w = synth.workload("batched_screening")
    sp, pk, b = make(api, w)
    P, S, seed = w.poses, w.steps, 2002
    rng = np.random.default_rng(2)
    poses_g = np.sort(rng.choice(b.n_lig * P, 256, replace=False))
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=poses_g.tolist())
    idx, e = api.topk(b, out["energy"], out["dof"], w.topk, 1.0)
    assert api.sync(b, P, out["state"], timeout_ms=120000) == 0
    ligs = oracle_ligands(w.ligands)
    st = check_trace(out["trace"].cpu().numpy(), poses_g, P, ligs, *pocket_arrays(w.pocket), oracle_params(sp),
                     cfg_for(w, seed), S, w.mc_loops, seed, out["dof"].cpu().numpy(), out["energy"].cpu().numpy())
    report(st, "batched screening sampled")
    E = out["energy"].cpu().numpy().astype(np.float64)
    dof = out["dof"].cpu().numpy().astype(np.float64)
    idx = idx.cpu().numpy()
    for l in sorted(set((poses_g // P).tolist()))[:24]:
        X = np.stack([oracle.fk(ligs[l], dof[l, p, :7 + ligs[l].n_tor]) for p in range(P)])
        ref, near = oracle.topk(E[l], X, w.topk, 1.0)
        if near == 0:
            np.testing.assert_array_equal(idx[l], ref)


def test_trids_atom_pair_terms_full_size_sampled(api):
    """The benchmark's workload with the TRIDS terms and the atom-pair E_MDN (term set 1,
    10 A cutoff, K = 4; 1,024 ligands x 128 poses x 50 evaluations, persistent launch in a
    CUDA graph): 96 seeded poses traced and checked per evaluation against the oracle."""
    w = synth.workload("batched_screening")
    sp, pk, b = make(api, w, term_set=1)
    P, S, seed = w.poses, w.steps, 2102
    rng = np.random.default_rng(21)
    poses_g = np.sort(rng.choice(b.n_lig * P, 96, replace=False))
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=poses_g.tolist())
    assert api.sync(b, P, out["state"], timeout_ms=120000) == 0
    st = check_trace(out["trace"].cpu().numpy(), poses_g, P, oracle_ligands(w.ligands), *pocket_arrays(w.pocket),
                     oracle_params(sp), cfg_for(w, seed), S, w.mc_loops, seed, out["dof"].cpu().numpy(),
                     out["energy"].cpu().numpy())
    report(st, "TRIDS atom-pair terms, batched screening, sampled")


def test_adjoint_check_full_size_score_sampled(api):
    """Adjoint-check workload at full size (256 ligands x 64 random poses) through the autograd Function:
    energies, DOF gradients (t, q, theta) and parameter gradients against the oracle on a
    seeded sample of 192 poses, plus dE/dw, dE/dR summed over every pose."""
    from paper_2510_24186_b300.autograd import score as tscore
    w = synth.workload("adjoint_check")
    sp, pk, b = make(api, w)
    rng = np.random.default_rng(33)
    P = 64
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    d = torch.from_numpy(dof).cuda().requires_grad_(True)
    W = torch.tensor(list(sp.w), dtype=torch.float64, requires_grad=True)
    R = torch.tensor(list(sp.radius), dtype=torch.float64, requires_grad=True)
    E = tscore(d, W, R, pk, b)
    E.sum().backward()
    Eh, gd = E.detach().cpu().numpy(), d.grad.cpu().numpy()
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    ligs = oracle_ligands(w.ligands)
    st = Stats()
    picks = rng.choice(b.n_lig * P, 192, replace=False)
    for g in picks:
        l, p = divmod(int(g), P)
        T = ligs[l].n_tor
        stt, ev = oracle.score(op, pxyz, ptype, ligs[l], dof[l, p, :7 + T])
        st.n += 1
        energy_ok(Eh[l, p], ev, st, f"lig {l} pose {p}")
        sl = grad_slack(ev)
        block_ok(gd[l, p, :3], ev.g_dof[:3], t_slack(ev), st, f"lig {l} pose {p} t", rnd=round_slack(ev, 0, 3))
        block_ok(gd[l, p, 3:7], ev.g_dof[3:7], sl, st, f"lig {l} pose {p} q", rnd=round_slack(ev, 3, 7))
        block_ok(gd[l, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"lig {l} pose {p} theta", rnd=round_slack(ev, 7, 7 + T))
    # parameter gradients over every pose: oracle sums over all 16,384 poses
    gw = np.zeros(5)
    gr = np.zeros(16)
    for l in range(b.n_lig):
        for p in range(P):
            T = ligs[l].n_tor
            ev = oracle.score(op, pxyz, ptype, ligs[l], dof[l, p, :7 + T])[1]
            gw += np.array(ev.g_w)
            gr += np.array(ev.g_R)
    block_ok(W.grad.numpy(), gw, 0.0, st, "dE/dw")
    block_ok(R.grad.numpy(), gr[:8], 0.0, st, "dE/dR")
    report(st, "adjoint check full size")


def test_blind_docking_three_cavities_sampled(api):
    """Blind-docking workload shapes: 6,000-atom region around three cavities, one docking box per
    cavity (pose p in box p mod 3), 512 poses; 48 ligands x 100 evaluations, 256 seeded
    traced poses checked per evaluation against the oracle."""
    w = synth.workload("blind_docking", n_lig=48)
    sp = score_params(0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp, cell=1.0)
    pk.set_boxes(w.box_centers, w.box_sizes)
    b = api.Batch.from_ligands(pk, w.ligands)
    P, S, seed = w.poses, w.steps, 5005
    rng = np.random.default_rng(5)
    poses_g = np.sort(rng.choice(b.n_lig * P, 256, replace=False))
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=poses_g.tolist())
    assert api.sync(b, P, out["state"], timeout_ms=120000) == 0
    lo = (w.box_centers - w.box_sizes / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_centers + w.box_sizes / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=w.mc_loops, lr=float(np.float32(0.1)), b1=float(np.float32(0.9)),
                            b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)), beta=float(np.float32(0.069)),
                            seed=seed, box_lo=lo, box_hi=hi)
    dof = out["dof"].cpu().numpy()
    st = check_trace(out["trace"].cpu().numpy(), poses_g, P, oracle_ligands(w.ligands), *pocket_arrays(w.pocket),
                     oracle_params(sp), cfg, S, w.mc_loops, seed, dof, out["energy"].cpu().numpy())
    report(st, "blind docking sampled")
    # every final translation lies in its pose's box
    p_of = np.arange(P) % 3
    assert (dof[:, :, :3] >= lo[p_of][None] - 1e-4).all() and (dof[:, :, :3] <= hi[p_of][None] + 1e-4).all()


def test_screening_stream_shapes_sampled(api):
    """Screening-stream workload shapes (drug-like type mix, 10-70 atoms, 0-20 torsions,
    2,000-atom pocket, 64 poses x 40 evaluations): 256 seeded poses of 64 ligands traced and
    checked against the oracle at every evaluation."""
    w = synth.workload("screening_stream", n_lig=64)
    sp, pk, b = make(api, w)
    P, S, seed = w.poses, w.steps, 4004
    rng = np.random.default_rng(4)
    poses_g = np.sort(rng.choice(b.n_lig * P, 256, replace=False))
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=poses_g.tolist())
    assert api.sync(b, P, out["state"], timeout_ms=120000) == 0
    st = check_trace(out["trace"].cpu().numpy(), poses_g, P, oracle_ligands(w.ligands), *pocket_arrays(w.pocket),
                     oracle_params(sp), cfg_for(w, seed), S, w.mc_loops, seed, out["dof"].cpu().numpy(),
                     out["energy"].cpu().numpy())
    report(st, "screening stream shapes sampled")


def test_screening_stream_matches_separate_batches(api):
    """Screening-stream workload shapes (drug-like mix, 2,000-atom pocket, 64 poses x 40 evaluations) as a
    stream of uneven batches with device-resident buffers and host packing overlapped:
    identical to sampling each batch on its own with the same ligand ids."""
    w = synth.workload("screening_stream", n_lig=300)
    sp = score_params(0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    sizes = [70, 130, 100]
    chunks, o = [], 0
    for s in sizes:
        chunks.append(synth.concat_ligands(w.ligands[o:o + s]))
        o += s
    got = list(api.screen_stream(pk, chunks, w.poses, w.steps, w.topk, seed=44))
    assert [g[0] for g in got] == [0, 70, 200]
    base = 0
    for (b0, idx, e), arr in zip(got, chunks):
        b = api.Batch(pk, *arr)
        out = api.sample(pk, b, w.poses, w.steps, mc_loops=w.mc_loops, seed=44, lig_base=base)
        i2, e2 = api.topk(b, out["energy"], out["dof"], w.topk, 1.0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(idx, i2.cpu().numpy())
        np.testing.assert_array_equal(e, e2.cpu().numpy())
        base += b.n_lig
