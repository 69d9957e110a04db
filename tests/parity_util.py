"""Shared helpers of the GPU parity tests: build inputs, run the oracle, compare.

Tolerances (stated for the method's FP32 results against the FP64 oracle):
  energy    |dE| <= max(1e-3 kcal/mol, 1e-5 |E|) + straddle slack
  gradient  per block (t, rotation, torsions): |g - g_ref| / max(|g_ref|, 1e-3) <= 1e-3,
            plus slack for pairs sitting on a cutoff or kink, plus the FP32 rounding bound
            4 * 2^-24 * (sum over the block's DOFs of the oracle's condition magnitudes,
            sum over atoms of |lever| * sum of |dE/dr| of the atom's pairs): a gradient that is
            a small difference of large terms cannot be closer than this in float32
  states    t and theta within 1e-4 (theta on the circle), q within 1e-4 as a rotation
Integer results (topology, top-k indices, perturbed variable, acceptance decisions)
must match exactly, except decisions the oracle marks as near ties.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import oracle
from paper_2510_24186_b300 import synth

E_ABS, E_REL, G_REL, G_FLOOR, S_TOL = 1e-3, 1e-5, 1e-3, 1e-3, 1e-4


def score_params(term_set=0, cutoff=8.0, seed=7, K=2):
    from paper_2510_24186_b300 import api
    if term_set == 0:
        return api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, cutoff)
    return api.ScoreParams(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, cutoff, gmm=gmm_table(seed, K))


def gmm_table(seed=7, K=2):
    rng = np.random.default_rng(seed)
    g = np.zeros((8, 8, K, 3))
    g[..., 0] = rng.uniform(0.2, 1.0, (8, 8, K))
    g[..., 1] = rng.uniform(2.0, 4.5, (8, 8, K))
    g[..., 2] = rng.uniform(0.4, 1.2, (8, 8, K))
    return g.astype(np.float32).astype(np.float64)


def oracle_params(sp):
    """Oracle parameter block holding the same float32 values the GPU uses."""
    f = lambda v: [float(np.float32(x)) for x in v]
    return oracle.make_params(sp.term_set, f(sp.radius), sp.flags, f(sp.w), float(np.float32(sp.cutoff)),
                              float(np.float32(sp.w_tor)), gmm=None if sp.gmm is None else np.asarray(sp.gmm))


def oracle_ligands(ligs):
    out = []
    for lg in ligs:
        st, ol = oracle.pack(lg.xyz.astype(np.float32).astype(np.float64), lg.type, lg.bonds, lg.rotatable)
        assert st == 0
        out.append(ol)
    return out


def pocket_arrays(pk):
    return pk.xyz.astype(np.float32).astype(np.float64), pk.type.astype(np.int32)


@dataclasses.dataclass
class Stats:
    """Worst and 99th-percentile errors of one parity check, plus its failures."""
    n: int = 0
    e_abs: float = 0.0
    e_rel: float = 0.0
    g_rel: float = 0.0
    s_err: float = 0.0
    straddles: int = 0
    near_ties: int = 0
    n_grad: int = 0            # gradient block checks
    e_allow: int = 0           # energy checks that pass only through the straddle allowance
    g_straddle: int = 0        # gradient blocks that need the straddle allowance
    g_round: int = 0           # gradient blocks that need only the float32 rounding allowance
    fails: list = dataclasses.field(default_factory=list)
    g_worst: str = ""
    e_abs_all: list = dataclasses.field(default_factory=list)
    g_rel_all: list = dataclasses.field(default_factory=list)
    s_err_all: list = dataclasses.field(default_factory=list)

    def fail(self, msg):
        if len(self.fails) < 20:
            self.fails.append(msg)

    def energy(self, d, ref):
        self.e_abs = max(self.e_abs, d)
        self.e_rel = max(self.e_rel, d / max(abs(ref), 1e-30))
        self.e_abs_all.append(d)

    def grad(self, r, what=""):
        if r > self.g_rel:
            self.g_worst = what
        self.g_rel = max(self.g_rel, r)
        self.g_rel_all.append(r)

    def state(self, e):
        self.s_err = max(self.s_err, e)
        self.s_err_all.append(e)

    @staticmethod
    def _p99(v):
        return float(np.percentile(v, 99)) if len(v) else 0.0

    def summary(self, what):
        return (f"[{what}] n={self.n} |dE| max {self.e_abs:.3e} p99 {self._p99(self.e_abs_all):.3e}, "
                f"rel dE max {self.e_rel:.3e}; grad rel max {self.g_rel:.3e} p99 {self._p99(self.g_rel_all):.3e}; "
                f"state err max {self.s_err:.3e} p99 {self._p99(self.s_err_all):.3e}; straddles={self.straddles} "
                f"near ties={self.near_ties}; passing only through an allowance: energy {self.e_allow}/{self.n}, "
                f"gradient blocks {self.g_straddle + self.g_round}/{self.n_grad} (straddle {self.g_straddle}, "
                f"float32 rounding {self.g_round})" + (f"; worst gradient block: {self.g_worst}" if self.g_worst else ""))


def report(st: Stats, what):
    """Print the check's max and p99 errors (pytest -s shows them); fail on any recorded failure."""
    print("\n" + st.summary(what))
    assert not st.fails, "\n".join(st.fails)


def energy_ok(e_gpu, ev, st: Stats, what=""):
    d = abs(e_gpu - ev.e_total)
    st.energy(d, ev.e_total)
    st.straddles += ev.n_straddle
    base = max(E_ABS, E_REL * abs(ev.e_total))
    tol = base + ev.e_slack
    if not (d <= tol) or not math.isfinite(e_gpu):
        st.fail(f"{what}: E gpu {e_gpu!r} oracle {ev.e_total!r}")
    elif d > base:
        st.e_allow += 1


def block_ok(g_gpu, g_ref, slack, st: Stats, what="", rnd=0.0):
    """Norm-wise gradient block check: |g - g_ref| <= G_REL max(|g_ref|, G_FLOOR) + slack (the
    straddling pairs' jumps) + rnd (the float32 rounding allowance); checks that need either
    allowance are counted."""
    g_gpu = np.asarray(g_gpu, dtype=np.float64)
    g_ref = np.asarray(g_ref, dtype=np.float64)
    if g_ref.size == 0:
        return
    num = np.linalg.norm(g_gpu - g_ref)
    den = max(np.linalg.norm(g_ref), G_FLOOR)
    base = G_REL * den
    st.n_grad += 1
    st.grad(num / den, f"{what}: |dg| {num:.2e}, |g| {np.linalg.norm(g_ref):.2e}, allowed {base + slack + rnd:.2e}")
    if not (num <= base + slack + rnd):
        st.fail(f"{what}: |dg| {num:.3e} |g| {np.linalg.norm(g_ref):.3e} slack {slack:.2e} rounding {rnd:.2e}")
    elif num > base + rnd:
        st.g_straddle += 1
    elif num > base:
        st.g_round += 1


EPS32 = 2.0 ** -24


def t_slack(ev):
    # dE/dt is the sum of the ligand atoms' forces: a jump J of one pair's dE/dr moves it by
    # at most J (an intra pair's jumps cancel in the sum), with no lever arm
    return ev.g_slack


def grad_slack(ev):
    # a force jump J on one atom moves a rotation or torsion gradient by at most J times
    # the lever arm (< 40 A inside a pocket)
    return 40.0 * ev.g_slack


def xyz_slack(ev):
    # the per-atom force block: a straddling pair's jump J moves the force of each of its (one
    # or two) ligand atoms by J, no lever arm: |dg| <= sqrt(2) x the summed jumps
    return 2.0 * ev.g_slack


def round_slack(ev, lo, hi):
    """float32 rounding allowance for DOF components [lo, hi) (see module docstring)."""
    return 4.0 * EPS32 * float(np.linalg.norm(np.array(ev.g_mag[lo:hi])))


def quat_angle(a, b):
    a = np.asarray(a, dtype=np.float64) / np.linalg.norm(a)
    b = np.asarray(b, dtype=np.float64) / np.linalg.norm(b)
    return 2.0 * math.acos(min(1.0, abs(float(np.dot(a, b)))))


def state_err(d_gpu, d_ref, T):
    d_gpu = np.asarray(d_gpu, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    e = float(np.abs(d_gpu[:3] - d_ref[:3]).max())
    e = max(e, quat_angle(d_gpu[3:7], d_ref[3:7]))
    if T:
        dt = (d_gpu[7:7 + T] - d_ref[7:7 + T] + math.pi) % (2 * math.pi) - math.pi
        e = max(e, float(np.abs(dt).max()))
    return e


def check_trace(trace, poses_g, P, ligs_or, pxyz, ptype, op, cfg_or, S, Lmc, seed, dof_final, e_final,
                lig_base=0, st: Stats | None = None, mds=None, mp=None) -> Stats:
    """Per-evaluation parity of a sampler trace.

    trace [S, n_trace, rec] (GPU float32), poses_g = global pose ids (l * P + p) of the slots.
    For every traced pose and evaluation: the oracle re-scores the GPU's state in FP64 and
    compares energy and gradient; the Monte-Carlo helper ``McPose`` (the statement of the
    loop that the oracle's own sampler is pinned to) then applies the method's next action
    (update, or Metropolis decision + perturbation at a loop boundary) in FP64 to the GPU's
    state, energy and gradient, and the result is compared with the GPU's next state;
    finally the returned state and energy are checked.  A Metropolis decision that the
    oracle marks as a near tie may go either way: the other branch is followed when the
    GPU's next state matches it.  mds: per-ligand residue-level E_MDN inputs (term set 2);
    mp: the grid-map domain when the GPU scored with maps.
    """
    from mc_replay import McPose
    st = st or Stats()
    trace = np.asarray(trace, dtype=np.float64)
    D = (trace.shape[2] - 14) // 2 + 7
    for slot, g in enumerate(poses_g):
        l, p = divmod(int(g), P)
        lg = ligs_or[l]
        T = lg.n_tor
        mc = McPose(cfg_or, T, lig_base + l, p, S, Lmc, seed)
        init = mc.start()
        e0 = state_err(trace[0, slot, :7 + T], init, T)
        st.state(e0)
        if e0 > S_TOL:
            st.fail(f"pose {g}: initial state differs by {e0:.2e}")
        for s in range(S):
            rec = trace[s, slot]
            dof = rec[:7 + T]
            E = rec[D]
            gt, tau, gth = rec[D + 1:D + 4], rec[D + 4:D + 7], rec[D + 7:D + 7 + T]
            stt, ev = oracle.score(op, pxyz, ptype, lg, dof, None if mds is None else mds[l], mp)
            st.n += 1
            energy_ok(E, ev, st, f"pose {g} step {s}")
            sl = grad_slack(ev)
            block_ok(gt, ev.g_dof[:3], t_slack(ev), st, f"pose {g} step {s} dE/dt", rnd=round_slack(ev, 0, 3))
            block_ok(tau, ev.tau[:], sl, st, f"pose {g} step {s} torque", rnd=round_slack(ev, 3, 7))
            block_ok(gth, ev.g_dof[7:7 + T], sl, st, f"pose {g} step {s} dE/dtheta", rnd=round_slack(ev, 7, 7 + T))
            nxt = mc.step(dof, E, np.concatenate([gt, tau, gth]))
            if mc.near:
                got = trace[s + 1, slot, :7 + T] if nxt is not None else dof_final[l, p, :7 + T]
                if state_err(got, mc.alternative(), T) <= S_TOL:
                    st.near_ties += 1
                    nxt = mc.alternative()
                    mc.take_alternative()
            if nxt is not None:
                es = state_err(trace[s + 1, slot, :7 + T], nxt, T)
                st.state(es)
                if es > S_TOL:
                    st.fail(f"pose {g} step {s}->{s + 1}: state differs by {es:.2e}")
        ef = state_err(dof_final[l, p, :7 + T], mc.final, T)
        st.state(ef)
        if ef > S_TOL:
            st.fail(f"pose {g}: final state differs by {ef:.2e}")
        if float(e_final[l, p]) != float(np.float32(mc.e_cur)):
            st.fail(f"pose {g}: final energy {float(e_final[l, p])} vs {mc.e_cur}")
    return st
