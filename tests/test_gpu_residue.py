"""GPU parity of the residue-level E_MDN (term set 2) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2510_24186_b300 import synth

from parity_util import (report, Stats, block_ok, check_trace, energy_ok, grad_slack, t_slack, xyz_slack, oracle_ligands, oracle_params,
                         pocket_arrays, round_slack)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2510_24186_b300 import api as a
    return a


def res_setup(api, w, ligs, K=4, seed=21, cell=0.0):
    """Pocket with seeded residues, batch with seeded per-pair kernels; the oracle's inputs
    hold the same float32 values."""
    sp = api.ScoreParams(2, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp, cell=cell)
    rng = np.random.default_rng(seed)
    res = synth.gen_residues(rng, w.pocket.xyz)
    pk.set_residues(res)
    b = api.Batch.from_ligands(pk, ligs)
    mdn = synth.gen_mdn(rng, int(b.n_atoms.sum()), int(res.max()) + 1, K)
    b.set_mdn(torch.from_numpy(mdn).cuda())
    offs = np.concatenate([[0], np.cumsum(b.n_atoms)])
    mds = [oracle.mdn(res, mdn[offs[l]:offs[l + 1]].astype(np.float64)) for l in range(len(ligs))]
    return sp, pk, b, mds


def _check_pose(st, out, l, p, ev, T, what):
    energy_ok(out["energy"][l, p], ev, st, what)
    sl = grad_slack(ev)
    block_ok(out["g_dof"][l, p, :3], ev.g_dof[:3], t_slack(ev), st, f"{what} t", rnd=round_slack(ev, 0, 3))
    block_ok(out["g_dof"][l, p, 3:7], ev.g_dof[3:7], sl, st, f"{what} q", rnd=round_slack(ev, 3, 7))
    block_ok(out["g_dof"][l, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"{what} theta", rnd=round_slack(ev, 7, 7 + T))


def test_residue_score_parity_single_ligand(api):
    """Single-ligand workload shapes with residues: every one of 64 random poses, energy, DOF and atom gradients."""
    w = synth.workload("single_ligand")
    sp, pk, b, mds = res_setup(api, w, w.ligands)
    rng = np.random.default_rng(31)
    P = 64
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    out = api.score_grad(pk, b, torch.from_numpy(dof).cuda(), grad=True, xyz_grad=True)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    lg = oracle_ligands(w.ligands)[0]
    perm = np.array(lg.perm[:lg.n_atoms])
    st = Stats()
    n_res_pairs = 0
    for p in range(P):
        _, ev = oracle.score(op, pxyz, ptype, lg, dof[0, p, :7 + lg.n_tor], mds[0])
        st.n += 1
        n_res_pairs += ev.n_res_pairs
        _check_pose(st, out, 0, p, ev, lg.n_tor, f"pose {p}")
        gx = np.zeros((b.max_atoms, 3))
        gx[perm] = np.array(ev.g_x)[:lg.n_atoms]
        block_ok(out["g_xyz"][0, p].ravel(), gx.ravel(), xyz_slack(ev), st, f"pose {p} xyz")
    assert n_res_pairs > 100 * P
    report(st, "residue score single ligand")


def test_residue_score_parity_batch_and_param_grads(api):
    """Adjoint-check workload shapes (1,500-atom pocket with ~220 residues), 24 ligands x 37 poses (a
    ragged tile), sampled poses; dE/dw summed with upstream weights through autograd."""
    from paper_2510_24186_b300.autograd import score as tscore
    w = synth.workload("adjoint_check", n_lig=24)
    sp, pk, b, mds = res_setup(api, w, w.ligands, K=6)
    rng = np.random.default_rng(32)
    P = 37
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    out = api.score_grad(pk, b, torch.from_numpy(dof).cuda(), grad=True)
    d = torch.from_numpy(dof).cuda().requires_grad_(True)
    W = torch.tensor(list(sp.w), dtype=torch.float64, requires_grad=True)
    R = torch.tensor(list(sp.radius), dtype=torch.float64, requires_grad=True)
    E = tscore(d, W, R, pk, b)
    ebar = torch.from_numpy(rng.uniform(-1, 1, (b.n_lig, P)).astype(np.float32)).cuda()
    (E * ebar).sum().backward()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    eb = ebar.cpu().numpy().astype(np.float64)
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(w.pocket)
    ligs = oracle_ligands(w.ligands)
    st = Stats()
    gw = np.zeros(5)
    gr = np.zeros(16)
    for l in range(b.n_lig):
        T = ligs[l].n_tor
        for p in range(P):
            _, ev = oracle.score(op, pxyz, ptype, ligs[l], dof[l, p, :7 + T], mds[l])
            gw += eb[l, p] * np.array(ev.g_w)
            gr += eb[l, p] * np.array(ev.g_R)
            if p % 5 == 0 or p == P - 1:
                st.n += 1
                _check_pose(st, out, l, p, ev, T, f"lig {l} pose {p}")
    block_ok(W.grad.numpy(), gw, 0.0, st, "dE/dw")
    block_ok(R.grad.numpy(), gr[:8], 0.0, st, "dE/dR")
    report(st, "residue score batch + param grads")


def test_residue_sampler_per_step_parity_single_ligand(api):
    """Single-ligand workload with residues: every pose and evaluation against the oracle (energy,
    gradient, Adam update, Metropolis, perturbation, final state); persistent and
    per-ligand forms bit-identical."""
    w = synth.workload("single_ligand")
    sp, pk, b, mds = res_setup(api, w, w.ligands)
    seed = 1201
    P, S = w.poses, w.steps
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=list(range(P)))
    assert api.sync(b, P, out["state"], timeout_ms=60000) == 0
    lo = (w.box_center - w.box_size / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_center + w.box_size / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=w.mc_loops, lr=float(np.float32(0.1)), b1=float(np.float32(0.9)),
                            b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)),
                            beta=float(np.float32(0.069)), seed=seed, box_lo=lo, box_hi=hi)
    st = check_trace(out["trace"].cpu().numpy(), list(range(P)), P, oracle_ligands(w.ligands),
                     *pocket_arrays(w.pocket), oracle_params(sp), cfg, S, w.mc_loops, seed,
                     out["dof"].cpu().numpy(), out["energy"].cpu().numpy(), mds=mds)
    report(st, "residue sampler single ligand")
    o2 = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, mode=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o2["dof"].cpu().numpy(), out["dof"].cpu().numpy())
    np.testing.assert_array_equal(o2["energy"].cpu().numpy(), out["energy"].cpu().numpy())


def test_residue_inputs_are_checked(api):
    from paper_2510_24186_b300._lib import TridsError
    w = synth.workload("single_ligand")
    sp = api.ScoreParams(2, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    dof = torch.zeros((1, 4, b.dof_stride), device="cuda")
    dof[..., 3] = 1
    with pytest.raises(TridsError, match="trids_set_residues"):
        api.score_grad(pk, b, dof)
    res = synth.gen_residues(np.random.default_rng(1), w.pocket.xyz)
    pk.set_residues(res)
    with pytest.raises(TridsError, match="trids_set_mdn"):
        api.score_grad(pk, b, dof)
    n_res = int(res.max()) + 1
    bad = torch.from_numpy(synth.gen_mdn(np.random.default_rng(2), int(b.n_atoms.sum()), n_res, 2)).cuda()
    bad[0, 0, 1, 2] = 0.0   # sigma = 0
    with pytest.raises(TridsError, match="sigma"):
        b.set_mdn(bad)
    other = torch.from_numpy(synth.gen_mdn(np.random.default_rng(2), int(b.n_atoms.sum()), n_res + 1, 2)).cuda()
    b.set_mdn(other)
    with pytest.raises(TridsError, match="residues"):
        api.score_grad(pk, b, dof)
    with pytest.raises(TridsError):
        pk.set_residues(np.full(len(res), -1))
    big = np.arange(len(res)) % 200
    big[:64] = 0                                  # one residue of 64 atoms: above the 63-atom limit
    with pytest.raises(TridsError, match="more than 63"):
        pk.set_residues(big)
    small = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size,
                       api.ScoreParams(2, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 4.0))
    with pytest.raises(TridsError, match="cutoff"):
        small.set_residues(res)


def test_residue_full_size_sampled(api):
    """The batched-screening workload with the paper's residue-level E_MDN (1,024 ligands x
    128 poses x 50 evaluations, about 220 residues, K = 4, persistent launch in a CUDA
    graph): 96 seeded poses traced and checked per evaluation against the oracle."""
    w = synth.workload("batched_screening")
    sp, pk, b, mds = res_setup(api, w, w.ligands, K=4, seed=2202)
    P, S, seed = w.poses, w.steps, 2203
    rng = np.random.default_rng(22)
    poses_g = np.sort(rng.choice(b.n_lig * P, 96, replace=False))
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=poses_g.tolist())
    assert api.sync(b, P, out["state"], timeout_ms=120000) == 0
    lo = (w.box_center - w.box_size / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_center + w.box_size / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=w.mc_loops, lr=float(np.float32(0.1)), b1=float(np.float32(0.9)),
                            b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)),
                            beta=float(np.float32(0.069)), seed=seed, box_lo=lo, box_hi=hi)
    st = check_trace(out["trace"].cpu().numpy(), poses_g, P, oracle_ligands(w.ligands), *pocket_arrays(w.pocket),
                     oracle_params(sp), cfg, S, w.mc_loops, seed, out["dof"].cpu().numpy(),
                     out["energy"].cpu().numpy(), mds=mds)
    report(st, "residue E_MDN, batched screening, sampled")
