"""GPU parity of the grid-map form (trids_build_maps) against the FP64 oracle's map form,
plus the map rules: rebuild after new parameters, no parameter gradients with maps."""
import numpy as np
import pytest

import oracle
from paper_2510_24186_b300 import synth

from parity_util import (report, Stats, block_ok, check_trace, energy_ok, grad_slack, t_slack, oracle_ligands, oracle_params,
                         pocket_arrays, round_slack, score_params)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2510_24186_b300 import api as a
    return a


def oracle_maps(pk):
    lo, h, n = pk.maps_info()
    return oracle.maps(lo.astype(np.float64), float(np.float32(h)), n)


@pytest.mark.parametrize("term_set", [0, 1])
def test_map_score_parity(api, term_set):
    """Single-ligand workload shapes, 64 random poses, maps at 0.375 A over the box + 4 A (some atoms fall
    outside and keep the direct sum)."""
    w = synth.workload("single_ligand")
    sp = score_params(term_set, cutoff=w.cutoff if term_set == 0 else 10.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    pk.build_maps(0.375, 4.0)
    b = api.Batch.from_ligands(pk, w.ligands)
    rng = np.random.default_rng(51)
    P = 64
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    out = api.score_grad(pk, b, torch.from_numpy(dof).cuda(), grad=True)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    op = oracle_params(sp)
    mp = oracle_maps(pk)
    pxyz, ptype = pocket_arrays(w.pocket)
    lg = oracle_ligands(w.ligands)[0]
    T = lg.n_tor
    st = Stats()
    mapped = 0
    for p in range(P):
        _, ev = oracle.score(op, pxyz, ptype, lg, dof[0, p, :7 + T], mp=mp)
        mapped += ev.n_map_atoms
        st.n += 1
        energy_ok(out["energy"][0, p], ev, st, f"pose {p}")
        sl = grad_slack(ev)
        block_ok(out["g_dof"][0, p, :3], ev.g_dof[:3], t_slack(ev), st, f"pose {p} t", rnd=round_slack(ev, 0, 3))
        block_ok(out["g_dof"][0, p, 3:7], ev.g_dof[3:7], sl, st, f"pose {p} q", rnd=round_slack(ev, 3, 7))
        block_ok(out["g_dof"][0, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"pose {p} th", rnd=round_slack(ev, 7, 7 + T))
    assert 0 < mapped < P * lg.n_atoms      # both forms occur
    report(st, f"map score term_set={term_set}")


def test_map_sampler_per_step_parity_single_ligand(api):
    w = synth.workload("single_ligand")
    sp = score_params(0, cutoff=w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    pk.build_maps(0.375, 8.0)
    b = api.Batch.from_ligands(pk, w.ligands)
    seed, P, S = 1401, 32, w.steps
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=list(range(P)))
    assert api.sync(b, P, out["state"], timeout_ms=60000) == 0
    lo = (w.box_center - w.box_size / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_center + w.box_size / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=w.mc_loops, lr=float(np.float32(0.1)), b1=float(np.float32(0.9)),
                            b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)),
                            beta=float(np.float32(0.069)), seed=seed, box_lo=lo, box_hi=hi)
    st = check_trace(out["trace"].cpu().numpy(), list(range(P)), P, oracle_ligands(w.ligands),
                     *pocket_arrays(w.pocket), oracle_params(sp), cfg, S, w.mc_loops, seed,
                     out["dof"].cpu().numpy(), out["energy"].cpu().numpy(), mp=oracle_maps(pk))
    report(st, "map sampler single ligand")
    o2 = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, mode=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o2["dof"].cpu().numpy(), out["dof"].cpu().numpy())


def test_map_rules(api):
    from paper_2510_24186_b300._lib import TridsError
    w = synth.workload("single_ligand")
    sp = score_params(0, cutoff=w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    dof = torch.zeros((1, 8, b.dof_stride), device="cuda")
    dof[..., 3] = 1
    e_direct = api.score_grad(pk, b, dof)["energy"].clone()
    pk.build_maps(0.375, 8.0)
    lo, h, n = pk.maps_info()
    assert h == pytest.approx(0.375) and min(n) > 2
    with pytest.raises(TridsError, match="direct scoring"):
        api.score_grad(pk, b, dof, param_grad=True)
    pk.set_params(sp)
    with pytest.raises(TridsError, match="trids_build_maps"):
        api.score_grad(pk, b, dof)
    pk.build_maps(0.375, 8.0)
    e_map = api.score_grad(pk, b, dof)["energy"]
    pk.build_maps(0.0, 0.0)
    assert pk.maps_info()[2] == (0, 0, 0)
    e_again = api.score_grad(pk, b, dof)["energy"]
    torch.cuda.synchronize()
    assert torch.equal(e_again, e_direct)
    assert torch.allclose(e_map, e_direct, rtol=0.05, atol=0.5)
    with pytest.raises(TridsError):
        pk.build_maps(0.01, 8.0)


def test_maps_with_residue_terms(api):
    """Term set 2 with grid maps: the maps hold the atom-pair physics terms, the residue-level
    E_MDN stays direct; every pose checked against the oracle's map form with residues."""
    w = synth.workload("single_ligand")
    sp = api.ScoreParams(2, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    rng = np.random.default_rng(61)
    res = synth.gen_residues(rng, w.pocket.xyz)
    pk.set_residues(res)
    pk.build_maps(0.375, 6.0)
    b = api.Batch.from_ligands(pk, w.ligands)
    mdn = synth.gen_mdn(rng, int(b.n_atoms.sum()), int(res.max()) + 1, 3)
    b.set_mdn(torch.from_numpy(mdn).cuda())
    P = 48
    dof = synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2, w.box_center + w.box_size / 2,
                            b.dof_stride)
    out = api.score_grad(pk, b, torch.from_numpy(dof).cuda(), grad=True)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    op = oracle_params(sp)
    mp = oracle_maps(pk)
    md = oracle.mdn(res, mdn.astype(np.float64))
    pxyz, ptype = pocket_arrays(w.pocket)
    lg = oracle_ligands(w.ligands)[0]
    T = lg.n_tor
    st = Stats()
    mapped = res_pairs = 0
    for p in range(P):
        _, ev = oracle.score(op, pxyz, ptype, lg, dof[0, p, :7 + T], md, mp)
        mapped += ev.n_map_atoms
        res_pairs += ev.n_res_pairs
        st.n += 1
        energy_ok(out["energy"][0, p], ev, st, f"pose {p}")
        sl = grad_slack(ev)
        block_ok(out["g_dof"][0, p, :3], ev.g_dof[:3], t_slack(ev), st, f"pose {p} t", rnd=round_slack(ev, 0, 3))
        block_ok(out["g_dof"][0, p, 3:7], ev.g_dof[3:7], sl, st, f"pose {p} q", rnd=round_slack(ev, 3, 7))
        block_ok(out["g_dof"][0, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"pose {p} th", rnd=round_slack(ev, 7, 7 + T))
    assert mapped > 0 and res_pairs > 0
    report(st, "maps + residue E_MDN")
