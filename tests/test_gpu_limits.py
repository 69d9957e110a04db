"""GPU parity at the size limits: the largest pocket the candidate entries encode (8,191
atoms, 13-bit indices) with the largest ligands (70 atoms, 20 torsions), the smallest
ones, and a ragged pose count; energies, gradients and a per-step sampler trace."""
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


@pytest.fixture(scope="module")
def big(api):
    rng = np.random.default_rng(8191)
    pocket = synth.gen_pocket(rng, 8191, np.zeros(3))
    ligs = [synth.gen_ligand(rng, 70, 20), synth.gen_ligand(rng, 70, 20), synth.gen_ligand(rng, 1, 0),
            synth.gen_ligand(rng, 2, 0), synth.gen_ligand(rng, 37, 9)]
    sp = score_params(0, cutoff=8.0)
    box_c, box_s = np.zeros(3), np.full(3, 22.5)
    pk = api.Pocket(pocket.xyz, pocket.type, box_c, box_s, sp)
    b = api.Batch.from_ligands(pk, ligs)
    return pocket, ligs, sp, pk, b, box_c, box_s


def test_max_pocket_score_parity(api, big):
    pocket, ligs, sp, pk, b, box_c, box_s = big
    assert len(pocket.type) == 8191 and b.max_atoms == 70 and b.max_tor == 20
    rng = np.random.default_rng(3)
    P = 33
    dof = synth.random_dofs(rng, b.n_tor, P, box_c - box_s / 2, box_c + box_s / 2, b.dof_stride)
    out = api.score_grad(pk, b, torch.from_numpy(dof).cuda(), grad=True)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    op = oracle_params(sp)
    pxyz, ptype = pocket_arrays(pocket)
    ols = oracle_ligands(ligs)
    st = Stats()
    for l, ol in enumerate(ols):
        T = ol.n_tor
        for p in (0, 5, 17, 31, 32):
            _, ev = oracle.score(op, pxyz, ptype, ol, dof[l, p, :7 + T])
            st.n += 1
            energy_ok(out["energy"][l, p], ev, st, f"lig {l} pose {p}")
            sl = grad_slack(ev)
            block_ok(out["g_dof"][l, p, :3], ev.g_dof[:3], t_slack(ev), st, f"lig {l} pose {p} t", rnd=round_slack(ev, 0, 3))
            block_ok(out["g_dof"][l, p, 3:7], ev.g_dof[3:7], sl, st, f"lig {l} pose {p} q", rnd=round_slack(ev, 3, 7))
            block_ok(out["g_dof"][l, p, 7:7 + T], ev.g_dof[7:7 + T], sl, st, f"lig {l} pose {p} theta",
                     rnd=round_slack(ev, 7, 7 + T))
    report(st, "max pocket score")


def test_max_pocket_sampler_trace(api, big):
    pocket, ligs, sp, pk, b, box_c, box_s = big
    P, S, Lm, seed = 8, 12, 3, 4242
    slots = [l * P + p for l in range(len(ligs)) for p in (0, 7)]
    out = api.sample(pk, b, P, S, mc_loops=Lm, seed=seed, trace_poses=slots)
    assert api.sync(b, P, out["state"], timeout_ms=60000) == 0
    lo = (box_c - box_s / 2).astype(np.float32).astype(np.float64)
    hi = (box_c + box_s / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=Lm, lr=float(np.float32(0.1)), b1=float(np.float32(0.9)),
                            b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)), beta=float(np.float32(0.069)),
                            seed=seed, box_lo=lo, box_hi=hi)
    st = check_trace(out["trace"].cpu().numpy(), slots, P, oracle_ligands(ligs), *pocket_arrays(pocket),
                     oracle_params(sp), cfg, S, Lm, seed, out["dof"].cpu().numpy(), out["energy"].cpu().numpy())
    report(st, "max pocket sampler")


def test_pocket_size_limit_is_enforced(api):
    from paper_2510_24186_b300._lib import TridsError
    rng = np.random.default_rng(1)
    xyz = rng.uniform(-60, 60, (8192, 3))
    with pytest.raises(TridsError, match="8191"):
        api.Pocket(xyz, np.zeros(8192, np.int32), np.zeros(3), np.full(3, 10.0), score_params(0))


def test_empty_and_degenerate_sizes_are_rejected(api):
    """Empty inputs and sizes outside the documented ranges fail with TRIDS_EINVAL on the
    host, before any launch, and leave the pocket and the batch usable: a batch without
    ligands, a ligand without atoms, zero poses, zero evaluations or loops, an empty step
    range, k outside 1..64; a stream without batches yields nothing."""
    from paper_2510_24186_b300 import _lib
    w = synth.workload("single_ligand")
    sp = score_params(0, cutoff=8.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    lig = w.ligands[0]

    def einval(fn, *a, **kw):
        with pytest.raises(_lib.TridsError) as e:
            fn(*a, **kw)
        assert e.value.code == _lib.EINVAL, e.value
        return str(e.value)

    einval(api.Batch, pk, np.zeros(0), np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros((0, 2)), np.zeros(0))
    msg = einval(api.Batch, pk, [len(lig.type), 0], lig.xyz, lig.type, [len(lig.bonds), 0], lig.bonds,
                 lig.rotatable)
    assert "ligand 1" in msg
    b = api.Batch.from_ligands(pk, w.ligands)
    P, S = 8, 4
    bufs = {"dof": torch.zeros(b.n_lig, P, b.dof_stride, device="cuda"),
            "state": torch.zeros(b.state_floats(P), device="cuda"),
            "energy": torch.empty(b.n_lig, P, device="cuda")}
    for kw in ({"poses": 0, "steps": S}, {"poses": P, "steps": 0}, {"poses": P, "steps": S, "mc_loops": 0},
               {"poses": P, "steps": S, "step_begin": 2, "step_end": 2}):
        einval(api.sample, pk, b, seed=3, **kw, **bufs)
    einval(api.score_grad, pk, b, torch.zeros(b.n_lig, 0, b.dof_stride, device="cuda"))
    out = api.sample(pk, b, P, S, mc_loops=2, seed=3, **bufs)
    for k in (0, 65):
        einval(api.topk, b, out["energy"], out["dof"], k)
    idx, e = api.topk(b, out["energy"], out["dof"], 3)
    torch.cuda.synchronize()
    assert idx.shape == (b.n_lig, 3) and bool(torch.isfinite(e[:, 0]).all())
    assert (idx[:, 0] >= 0).all() and (idx < P).all()
    assert list(api.screen_stream(pk, [], P, S, 3)) == []
