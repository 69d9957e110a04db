"""Pins of the oracle's update rules (Adam, AdamW, RMSprop, Adagrad, SGD; Sec. 2 and
Table S5) against torch.optim on float64 tensors.

The parameter vector torch sees is (t - box centre, rotation vector, theta).  The
rotation vector is reset to zero before every step (the sampler re-centres the
tangent at the current orientation), so torch's step on it is the rotation the
oracle applies on the left of q."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

torch = pytest.importorskip("torch")

CASES = [
    ("adam", lambda x: torch.optim.Adam([x], lr=0.1, betas=(0.9, 0.999), eps=1e-8), {}),
    ("adamw", lambda x: torch.optim.AdamW([x], lr=0.1, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.05),
     {"weight_decay": 0.05}),
    ("rmsprop", lambda x: torch.optim.RMSprop([x], lr=0.01, alpha=0.95, eps=1e-8), {"alpha": 0.95}),
    ("adagrad", lambda x: torch.optim.Adagrad([x], lr=0.1, eps=1e-10), {"eps": 1e-10}),
    ("sgd", lambda x: torch.optim.SGD([x], lr=0.02), {}),
    ("sgd_momentum", lambda x: torch.optim.SGD([x], lr=0.02, momentum=0.9), {"momentum": 0.9}),
]


@pytest.mark.parametrize("name,make,extra", CASES, ids=[c[0] for c in CASES])
def test_update_rules_match_torch_optim(orc, name, make, extra):
    opt_name = "sgd" if name.startswith("sgd") else name
    lr = {"rmsprop": 0.01, "sgd": 0.02, "sgd_momentum": 0.02}.get(name, 0.1)
    centre = np.array([3.0, -2.0, 5.0])
    kw = dict(lr=lr, box_lo=tuple(centre - 100), box_hi=tuple(centre + 100), optimizer=opt_name)
    kw.update(extra)
    cfg = orc.sample_cfg(**kw)
    rng = np.random.default_rng(41)
    T = 3
    q = rng.normal(size=4)
    dof = np.concatenate([centre + rng.uniform(-2, 2, 3), q / np.linalg.norm(q), rng.uniform(-0.5, 0.5, T)])
    x = torch.tensor(np.concatenate([dof[:3] - centre, np.zeros(3), dof[7:]]), dtype=torch.float64,
                     requires_grad=True)
    opt = make(x)
    m, v = np.zeros(6 + T), np.zeros(6 + T)
    d = dof.copy()
    for step in range(1, 9):
        g = rng.normal(size=6 + T) * 3
        with torch.no_grad():
            x[3:6] = 0.0
        x.grad = torch.tensor(g)
        opt.step()
        after = x.detach().numpy().copy()
        q_prev = d[3:7].copy()
        orc.opt_step(cfg, T, step, g, m, v, d)
        np.testing.assert_allclose(d[:3] - centre, after[:3], atol=1e-12)
        np.testing.assert_allclose(d[7:], after[6:], atol=1e-12)
        expect = Rotation.from_rotvec(after[3:6]) * Rotation.from_quat([q_prev[1], q_prev[2], q_prev[3], q_prev[0]])
        qe = expect.as_quat()
        qe = np.array([qe[3], qe[0], qe[1], qe[2]])
        assert min(np.abs(d[3:7] - qe).max(), np.abs(d[3:7] + qe).max()) < 1e-12


@pytest.mark.parametrize("name,make,extra", CASES, ids=[c[0] for c in CASES])
def test_single_atom_sampler_is_the_textbook_optimizer(orc, name, make, extra):
    """0 torsions, 1 atom, one loop: the sampler is the plain optimizer on the atom position
    (S evaluations, S-1 updates, t clamped into the box)."""
    from paper_2510_24186_b300 import synth
    opt_name = "sgd" if name.startswith("sgd") else name
    lr = {"rmsprop": 0.01, "sgd": 0.02, "sgd_momentum": 0.02}.get(name, 0.1)
    p = orc.make_params(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    st, lg = orc.pack(np.zeros((1, 3)), [0], np.zeros((0, 2)), [])
    pk = np.array([[0.0, 0.0, 0.0]])
    pt = np.array([7], dtype=np.int32)
    S = 25
    kw = dict(steps=S, mc_loops=1, seed=3, box_lo=(-3,) * 3, box_hi=(3,) * 3, lr=lr, optimizer=opt_name)
    kw.update(extra)
    cfg = orc.sample_cfg(**kw)
    dof_fin, e_fin, _ = orc.sample_ligand(cfg, p, pk, pt, lg, 0, 1)
    x0 = orc.init_pose(cfg, 0, 0, 0)
    x = torch.tensor(x0[:3], requires_grad=True)
    opt = make(x)
    for _ in range(S - 1):
        d = np.concatenate([x.detach().numpy(), x0[3:7]])
        x.grad = torch.tensor(np.array(orc.score(p, pk, pt, lg, d)[1].g_dof[:3]))
        opt.step()
        with torch.no_grad():
            x.clamp_(-3, 3)
    np.testing.assert_allclose(dof_fin[0, :3], x.detach().numpy(), atol=1e-11)
    assert math.isfinite(e_fin[0])
