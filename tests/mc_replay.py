"""One statement of the Monte-Carlo loop (Sec. 2 "Conformation sampling", Fig. 2), shared by
the oracle's pins and the GPU trace checker.

``McPose`` is the loop's control flow for one pose, built only from the oracle's separately
pinned pieces (init_pose, opt_step, perturb, metropolis_u / metropolis_accept, loop_steps).
It is fed each evaluation's state, energy and gradient and answers with the next state to
evaluate, so it can be driven either by its own outputs (a whole FP64 trajectory) or by a
GPU trace (the next action applied to the GPU's state, evaluation by evaluation).

Order of one loop l (loops with no evaluations are skipped; they only occur at the end):
  l > 0: save (state, loop-end energy), then resample one of the 6+T variables (perturb);
  the optimiser moments restart;
  n_l evaluations; each but the last is followed by an update from its gradient, the
  last one gives the loop-end energy E_l;
  l > 0: accept iff u < exp(-beta (E_l - E_saved)); a rejection restores the saved state
  and energy.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

NEAR_TIE = 1e-5   # |u - exp(-beta dE)| below which a float32 and an FP64 decision may differ


class McPose:
    """Monte-Carlo control flow of one pose; see the module docstring."""

    def __init__(self, cfg, T, lig, pose, S, Lmc, seed):
        self.cfg, self.T, self.lig, self.pose, self.seed = cfg, T, lig, pose, seed
        self.S = S
        self.sched = [(l, j, oracle.loop_steps(S, Lmc, l)) for l in range(Lmc)
                      for j in range(oracle.loop_steps(S, Lmc, l))]
        self.s = 0
        self.m = self.v = None
        self.e_cur = math.nan
        self.e_saved = math.nan
        self.saved = None
        self.final = None
        self.near = False        # the last Metropolis decision was a near tie
        self._alt = None         # (state, energy) of the other decision
        self._alt_next = None
        self.accepted = []       # (loop, accepted) of every decision
        self.perturbed = []      # (loop, variable) of every perturbation

    def start(self):
        """The initial state (A1)."""
        return oracle.init_pose(self.cfg, self.T, self.lig, self.pose)

    def _perturb_into_next_loop(self, base, loop):
        c, nxt = oracle.perturb(self.cfg, self.T, self.lig, self.pose, loop, base)
        return c, nxt

    def step(self, dof, E, grad):
        """Feed evaluation s (state dof, energy E, gradient (dE/dt, tau, dE/dtheta)); returns
        the state of evaluation s + 1, or None after the last one (then ``final`` and
        ``e_cur`` hold the returned state and energy)."""
        loop, j, n = self.sched[self.s]
        T = self.T
        dof = np.asarray(dof, dtype=np.float64)
        self.near = False
        self._alt = self._alt_next = None
        if j == 0:                                    # moments restart with every loop
            self.m, self.v = np.zeros(6 + T), np.zeros(6 + T)
        self.s += 1
        if j < n - 1:                                 # update from this evaluation's gradient
            nxt = dof.copy()
            oracle.opt_step(self.cfg, T, j + 1, np.asarray(grad, dtype=np.float64), self.m, self.v, nxt,
                            pose=self.pose)
            return nxt
        e_new = float(E)                              # loop end
        if loop == 0:
            base, self.e_cur = dof.copy(), e_new
        else:
            u = oracle.metropolis_u(self.seed, self.lig, self.pose, loop)
            acc = oracle.metropolis_accept(e_new, self.e_saved, self.cfg.beta, u)
            thr = math.exp(min(50.0, -self.cfg.beta * (e_new - self.e_saved)))
            self.near = abs(u - thr) < NEAR_TIE
            self.accepted.append((loop, acc))
            base = dof.copy() if acc else self.saved.copy()
            other = (self.saved.copy(), self.e_saved) if acc else (dof.copy(), e_new)
            self.e_cur = e_new if acc else self.e_saved
            self._alt = other
        if self.s < self.S:                           # save, then perturb for the next loop
            l2 = self.sched[self.s][0]
            self.saved, self.e_saved = base.copy(), self.e_cur
            c, nxt = self._perturb_into_next_loop(base, l2)
            self.perturbed.append((l2, c))
            if self._alt is not None:
                self._alt_next = self._perturb_into_next_loop(self._alt[0], l2)[1]
            return nxt
        self.final = base
        return None

    def alternative(self):
        """After a Metropolis decision: what step() would have returned under the other
        decision (the next state, or the final state after the last evaluation)."""
        if self._alt is None:
            return None
        return self._alt_next if self._alt_next is not None else self._alt[0]

    def take_alternative(self):
        """Follow the other decision of the last Metropolis test (a near tie that the
        float32 run decided the other way)."""
        st, e = self._alt
        self.e_cur = e
        if self.final is not None:
            self.final = st.copy()
        else:
            self.saved, self.e_saved = st.copy(), e
        loop, acc = self.accepted[-1]
        self.accepted[-1] = (loop, not acc)
        self._alt = self._alt_next = None


def replay(cfg, op, pxyz, ptype, lg, lig, pose, S, Lmc, seed, md=None, mp=None, record=None):
    """Whole FP64 trajectory of one pose driven by the oracle's score; returns (McPose, final
    state, final energy).  record (a list, optional) gets every evaluated (state, energy)."""
    T = lg.n_tor
    mc = McPose(cfg, T, lig, pose, S, Lmc, seed)
    dof = mc.start()
    while dof is not None:
        stt, ev = oracle.score(op, pxyz, ptype, lg, dof, md, mp)
        assert stt == 0
        if record is not None:
            record.append((dof.copy(), ev.e_total))
        grad = np.concatenate([np.array(ev.g_dof[:3]), np.array(ev.tau[:]), np.array(ev.g_dof[7:7 + T])])
        dof = mc.step(dof, ev.e_total, grad)
    return mc, mc.final, mc.e_cur
