"""GPU parity of the update rules other than Adam (Table S5): per-evaluation trace of
the single-ligand workload against the oracle, which applies its FP64 rule to the GPU's state and gradient."""
import numpy as np
import pytest

import oracle
from paper_2510_24186_b300 import synth

from parity_util import check_trace, report, oracle_ligands, oracle_params, pocket_arrays, score_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

f32 = lambda x: float(np.float32(x))

RULES = [
    ("adamw", dict(lr=0.1, weight_decay=0.01)),
    ("rmsprop", dict(lr=0.02, alpha=0.99)),
    ("adagrad", dict(lr=0.1, eps=1e-10)),
    ("sgd", dict(lr=0.005, momentum=0.9)),
    ("sgd", dict(lr=0.002, momentum=0.0)),
]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2510_24186_b300 import api as a
    return a


@pytest.mark.parametrize("name,hp", RULES, ids=[f"{n}-{i}" for i, (n, _) in enumerate(RULES)])
def test_update_rule_per_step_parity(api, name, hp):
    w = synth.workload("single_ligand")
    sp = score_params(0, cutoff=w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    seed, P, S = 1301, 32, w.steps
    kw = dict(lr=0.1, eps=1e-8, weight_decay=0.01, momentum=0.0, alpha=0.99)
    kw.update(hp)
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=list(range(P)), optimizer=name, **kw)
    assert api.sync(b, P, out["state"], timeout_ms=60000) == 0
    lo = (w.box_center - w.box_size / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_center + w.box_size / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=w.mc_loops, lr=f32(kw["lr"]), b1=f32(0.9), b2=f32(0.999),
                            eps=f32(kw["eps"]), beta=f32(0.069), seed=seed, box_lo=lo, box_hi=hi, optimizer=name,
                            weight_decay=f32(kw["weight_decay"]), momentum=f32(kw["momentum"]),
                            alpha=f32(kw["alpha"]))
    st = check_trace(out["trace"].cpu().numpy(), list(range(P)), P, oracle_ligands(w.ligands),
                     *pocket_arrays(w.pocket), oracle_params(sp), cfg, S, w.mc_loops, seed,
                     out["dof"].cpu().numpy(), out["energy"].cpu().numpy())
    report(st, f"{name} {hp}")
    # the persistent launch and the plain per-ligand form agree bit for bit
    o2 = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, mode=1, optimizer=name, **kw)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o2["dof"].cpu().numpy(), out["dof"].cpu().numpy())


def test_unknown_update_rule_is_rejected(api):
    from paper_2510_24186_b300 import _lib
    w = synth.workload("single_ligand")
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, score_params(0))
    b = api.Batch.from_ligands(pk, w.ligands)
    _lib.OPTIMIZERS["bogus"] = 9
    try:
        with pytest.raises(_lib.TridsError, match="optimizer"):
            api.sample(pk, b, 4, 3, optimizer="bogus")
    finally:
        del _lib.OPTIMIZERS["bogus"]
    with pytest.raises(_lib.TridsError, match="momentum"):
        api.sample(pk, b, 4, 3, optimizer="sgd", momentum=1.0)


def test_type_both_hydrophobic_and_hbonding_uses_both_flag_terms(api):
    """The plain sampler evaluates one flag term per ligand atom (a type is hydrophobic or
    H-bonding or neither).  A parameter set with a type that is both runs the general
    kernels, which evaluate both terms; the per-evaluation trace still matches the oracle,
    and the same ligands under ordinary flags still run the plain kernels bit-identically
    to the plain per-ligand form."""
    w = synth.workload("single_ligand")
    flags = list(synth.TYPE_FLAGS)
    flags[0] = 1 | 2                      # C_H: hydrophobic and donor
    flags[7] = 1 | 4                      # Cl_H: hydrophobic and acceptor
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, flags, synth.VINA_WEIGHTS, w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    seed, P, S = 1302, 32, w.steps
    out = api.sample(pk, b, P, S, mc_loops=w.mc_loops, seed=seed, trace_poses=list(range(P)))
    assert api.sync(b, P, out["state"], timeout_ms=60000) == 0
    lo = (w.box_center - w.box_size / 2).astype(np.float32).astype(np.float64)
    hi = (w.box_center + w.box_size / 2).astype(np.float32).astype(np.float64)
    cfg = oracle.sample_cfg(steps=S, mc_loops=w.mc_loops, lr=f32(0.1), b1=f32(0.9), b2=f32(0.999), eps=f32(1e-8),
                            beta=f32(0.069), seed=seed, box_lo=lo, box_hi=hi)
    st = check_trace(out["trace"].cpu().numpy(), list(range(P)), P, oracle_ligands(w.ligands),
                     *pocket_arrays(w.pocket), oracle_params(sp), cfg, S, w.mc_loops, seed,
                     out["dof"].cpu().numpy(), out["energy"].cpu().numpy())
    report(st, "types both hydrophobic and H-bonding")
    # the oracle sees pairs that need both terms: hydrophobic and H-bond energies together
    ol = oracle_ligands(w.ligands)[0]
    assert any(ol.type[i] in (0, 7) for i in range(ol.n_atoms))
