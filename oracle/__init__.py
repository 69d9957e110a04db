"""ctypes front end of the FP64 CPU oracle (``trids_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package, and this package never imports the product library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "trids_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

LMAX, TMAX, NT, KMAX = 70, 20, 16, 4
PMAX = LMAX * (LMAX - 1) // 2


class Params(C.Structure):
    _fields_ = [("term_set", C.c_int32), ("n_types", C.c_int32), ("w", C.c_double * 5),
                ("radius", C.c_double * NT), ("flags", C.c_int32 * NT), ("cutoff", C.c_double),
                ("w_tor", C.c_double), ("gmm_k", C.c_int32), ("gmm", C.c_double * (NT * NT * KMAX * 3))]


class Ligand(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("n_tor", C.c_int32), ("n_pairs", C.c_int32),
                ("perm", C.c_int32 * LMAX), ("frag", C.c_int32 * LMAX), ("type", C.c_int32 * LMAX),
                ("y", (C.c_double * 3) * LMAX), ("c", C.c_double * 3),
                ("tp", C.c_int32 * TMAX), ("th", C.c_int32 * TMAX), ("tpar", C.c_int32 * TMAX),
                ("sb", C.c_int32 * TMAX), ("se", C.c_int32 * TMAX),
                ("pi", C.c_int32 * PMAX), ("pj", C.c_int32 * PMAX)]


class Eval(C.Structure):
    _fields_ = [("e_total", C.c_double), ("e_inter", C.c_double), ("e_intra", C.c_double),
                ("g_dof", C.c_double * (7 + TMAX)), ("tau", C.c_double * 3),
                ("g_x", (C.c_double * 3) * LMAX), ("x", (C.c_double * 3) * LMAX),
                ("g_w", C.c_double * 5), ("g_R", C.c_double * NT),
                ("n_inter", C.c_int64), ("n_intra", C.c_int64), ("n_straddle", C.c_int32),
                ("e_slack", C.c_double), ("g_slack", C.c_double), ("e_mag", C.c_double),
                ("g_mag", C.c_double * (7 + TMAX)), ("n_res_pairs", C.c_int64), ("n_map_atoms", C.c_int64)]


class Mdn(C.Structure):
    _fields_ = [("n_res", C.c_int32), ("K", C.c_int32), ("res", C.POINTER(C.c_int32)),
                ("prm", C.POINTER(C.c_double))]


def mdn(res, prm):
    """Residue-level E_MDN inputs: res [M] residue of each pocket atom, prm [L_input, n_res, K, 3]
    of (pi, mu, sigma).  The arrays are kept alive on the returned object."""
    res = np.ascontiguousarray(res, dtype=np.int32)
    prm = np.ascontiguousarray(prm, dtype=np.float64)
    m = Mdn()
    m.n_res, m.K = prm.shape[1], prm.shape[2]
    m.res = res.ctypes.data_as(C.POINTER(C.c_int32))
    m.prm = prm.ctypes.data_as(C.POINTER(C.c_double))
    m._keep = (res, prm)
    return m


class Maps(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("h", C.c_double), ("n", C.c_int32 * 3)]


def maps(lo, h, n):
    """Grid-map domain: points lo + h * (a, b, c), 0 <= (a, b, c) < n."""
    m = Maps()
    for d in range(3):
        m.lo[d] = float(lo[d])
        m.n[d] = int(n[d])
    m.h = float(h)
    return m


MAX_BOXES = 8


class SampleCfg(C.Structure):
    _fields_ = [("steps", C.c_int32), ("mc_loops", C.c_int32), ("lr", C.c_double), ("b1", C.c_double),
                ("b2", C.c_double), ("eps", C.c_double), ("beta", C.c_double), ("seed", C.c_uint64),
                ("n_boxes", C.c_int32), ("box_lo", (C.c_double * 3) * MAX_BOXES),
                ("box_hi", (C.c_double * 3) * MAX_BOXES), ("optimizer", C.c_int32),
                ("weight_decay", C.c_double), ("momentum", C.c_double), ("alpha", C.c_double)]


OPTIMIZERS = {"adam": 0, "adamw": 1, "rmsprop": 2, "adagrad": 3, "sgd": 4}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + pthreads, FP64, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", SRC, "-o", LIB, "-lm", "-lpthread"])
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        L.or_philox.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.or_rand_word.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_rand_word.restype = C.c_uint32
        L.or_rot.argtypes = [P(C.c_double), C.c_double, P(C.c_double)]
        L.or_quat_mat.argtypes = [P(C.c_double), P(C.c_double)]
        L.or_pack.argtypes = [C.c_int, P(C.c_double), P(C.c_int32), C.c_int, C.c_int, P(C.c_int32),
                              P(C.c_uint8), P(Ligand)]
        L.or_topology.argtypes = [P(Ligand), P(C.c_int32), C.c_int]
        L.or_fk.argtypes = [P(Ligand), P(C.c_double), P(C.c_double)]
        L.or_fk_brute.argtypes = [P(Ligand), P(C.c_double), P(C.c_double)]
        L.or_pair.argtypes = [P(Params), C.c_int, C.c_int, C.c_double, C.c_int, P(C.c_double),
                              P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]
        L.or_score.argtypes = [P(Params), C.c_int, P(C.c_double), P(C.c_int32), P(Ligand),
                               P(C.c_double), P(Eval)]
        L.or_score_mdn.argtypes = [P(Params), C.c_int, P(C.c_double), P(C.c_int32), P(Mdn), P(Ligand),
                                   P(C.c_double), P(Eval)]
        L.or_score_full.argtypes = [P(Params), C.c_int, P(C.c_double), P(C.c_int32), P(Mdn), P(Maps), P(Ligand),
                                    P(C.c_double), P(Eval)]
        L.or_loop_steps.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_init_pose.argtypes = [P(SampleCfg), C.c_int, C.c_uint32, C.c_uint32, P(C.c_double)]
        L.or_perturb.argtypes = [P(SampleCfg), C.c_int, C.c_uint32, C.c_uint32, C.c_uint32, P(C.c_double)]
        L.or_metropolis_u.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_metropolis_u.restype = C.c_double
        L.or_metropolis_accept.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_screen_energy.argtypes = [C.c_double, C.c_double, C.c_int]
        L.or_screen_energy.restype = C.c_double
        L.or_opt_step.argtypes = [P(SampleCfg), C.c_int, C.c_int, C.c_uint32, P(C.c_double), P(C.c_double),
                                  P(C.c_double), P(C.c_double)]
        L.or_sample_pose.argtypes = [P(SampleCfg), P(Params), C.c_int, P(C.c_double), P(C.c_int32),
                                     P(Mdn), P(Maps), P(Ligand), C.c_uint32, C.c_uint32, P(C.c_double),
                                     P(C.c_int64)]
        L.or_sample_pose.restype = C.c_double
        L.or_sample_ligand.argtypes = [P(SampleCfg), P(Params), C.c_int, P(C.c_double), P(C.c_int32),
                                       P(Mdn), P(Maps), P(Ligand), C.c_uint32, C.c_int, C.c_int, P(C.c_double),
                                       P(C.c_double), C.c_int]
        L.or_sample_ligand.restype = C.c_int64
        L.or_topk.argtypes = [C.c_int, P(C.c_double), P(C.c_double), C.c_int, C.c_int, C.c_double,
                              P(C.c_int32), P(C.c_int32)]
        for fn in ("or_sizeof_ligand", "or_sizeof_eval", "or_sizeof_params"):
            getattr(L, fn).restype = C.c_size_t
        assert L.or_sizeof_ligand() == C.sizeof(Ligand)
        assert L.or_sizeof_eval() == C.sizeof(Eval)
        assert L.or_sizeof_params() == C.sizeof(Params)
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_params(term_set=0, radius=None, flags=None, w=None, cutoff=8.0, w_tor=0.01, gmm=None):
    """Oracle parameter block.  gmm: array [n_types, n_types, K, 3] of (pi, mu, sigma)."""
    p = Params()
    p.term_set = term_set
    radius = list(radius)
    p.n_types = len(radius)
    for i, r in enumerate(radius):
        p.radius[i] = float(r)
    for i, f in enumerate(flags):
        p.flags[i] = int(f)
    for i, x in enumerate(w):
        p.w[i] = float(x)
    p.cutoff = float(cutoff)
    p.w_tor = float(w_tor)
    if gmm is not None:
        g = np.asarray(gmm, dtype=np.float64)
        n, K = g.shape[0], g.shape[2]
        p.gmm_k = K
        full = np.zeros((NT, NT, KMAX, 3))
        full[:n, :n, :K] = g
        C.memmove(p.gmm, full.ctypes.data, full.nbytes)
    return p


def pack(xyz, types, bonds, rot, n_types=8):
    """Pack one ligand; returns (status, Ligand)."""
    lg = Ligand()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    types = np.ascontiguousarray(types, dtype=np.int32)
    bonds = np.ascontiguousarray(np.asarray(bonds).reshape(-1, 2), dtype=np.int32)
    rot = np.ascontiguousarray(rot, dtype=np.uint8)
    st = lib().or_pack(len(types), _dp(xyz), _ip(types), n_types, len(bonds), _ip(bonds),
                       rot.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(lg))
    return st, lg


def topology(lg) -> np.ndarray:
    out = np.zeros(3 + 2 * LMAX + 5 * TMAX + 2 * PMAX, dtype=np.int32)
    n = lib().or_topology(C.byref(lg), _ip(out), len(out))
    return out[:n]


def fk(lg, dof, brute=False):
    dof = np.ascontiguousarray(dof, dtype=np.float64)
    x = np.zeros((lg.n_atoms, 3))
    (lib().or_fk_brute if brute else lib().or_fk)(C.byref(lg), _dp(dof), _dp(x))
    return x


def score(p, pxyz, ptype, lg, dof, md=None, mp=None):
    """Returns (status, Eval) in FP64.  md: residue-level E_MDN inputs (term_set 2), see mdn();
    mp: grid-map domain (the map form of the ligand-pocket atom-pair terms), see maps()."""
    ev = Eval()
    pxyz = np.ascontiguousarray(pxyz, dtype=np.float64)
    ptype = np.ascontiguousarray(ptype, dtype=np.int32)
    dof = np.ascontiguousarray(dof, dtype=np.float64)
    st = lib().or_score_full(C.byref(p), len(ptype), _dp(pxyz), _ip(ptype), None if md is None else C.byref(md),
                             None if mp is None else C.byref(mp), C.byref(lg), _dp(dof), C.byref(ev))
    return st, ev


def pair(p, ti, tj, r, inter=True):
    e = np.zeros(5)
    dr = np.zeros(5)
    dR = np.zeros(5)
    vj = C.c_double()
    gj = C.c_double()
    lib().or_pair(C.byref(p), ti, tj, float(r), int(inter), _dp(e), _dp(dr), _dp(dR), C.byref(vj), C.byref(gj))
    return e, dr, dR


def rot(u, th):
    R = np.zeros(9)
    lib().or_rot(_dp(np.ascontiguousarray(u, dtype=np.float64)), float(th), _dp(R))
    return R.reshape(3, 3)


def quat_mat(q):
    R = np.zeros(9)
    lib().or_quat_mat(_dp(np.ascontiguousarray(q, dtype=np.float64)), _dp(R))
    return R.reshape(3, 3)


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox(c, k, o)
    return list(o)


def sample_cfg(steps=30, mc_loops=8, lr=0.1, b1=0.9, b2=0.999, eps=1e-8, beta=0.069, seed=0,
               box_lo=(-11.25,) * 3, box_hi=(11.25,) * 3, optimizer="adam", weight_decay=0.01, momentum=0.0,
               alpha=0.99):
    """box_lo / box_hi: one box (3 values) or several ([n][3]); pose p uses box p mod n.
    optimizer: adam, adamw, rmsprop, adagrad or sgd (eps is the caller's, as in torch)."""
    c = SampleCfg()
    c.steps, c.mc_loops, c.lr, c.b1, c.b2, c.eps, c.beta, c.seed = steps, mc_loops, lr, b1, b2, eps, beta, seed
    c.optimizer = OPTIMIZERS[optimizer] if isinstance(optimizer, str) else int(optimizer)
    c.weight_decay, c.momentum, c.alpha = weight_decay, momentum, alpha
    lo = np.atleast_2d(np.asarray(box_lo, dtype=np.float64))
    hi = np.atleast_2d(np.asarray(box_hi, dtype=np.float64))
    c.n_boxes = len(lo)
    for b in range(len(lo)):
        for d in range(3):
            c.box_lo[b][d] = lo[b, d]
            c.box_hi[b][d] = hi[b, d]
    return c


def init_pose(cfg, T, lig, pose):
    dof = np.zeros(7 + T)
    lib().or_init_pose(C.byref(cfg), T, lig, pose, _dp(dof))
    return dof


def perturb(cfg, T, lig, pose, loop, dof):
    d = np.ascontiguousarray(dof, dtype=np.float64).copy()
    c = lib().or_perturb(C.byref(cfg), T, lig, pose, loop, _dp(d))
    return c, d


def metropolis_u(seed, lig, pose, loop):
    return lib().or_metropolis_u(seed, lig, pose, loop)


def metropolis_accept(e_new, e_old, beta, u):
    return bool(lib().or_metropolis_accept(e_new, e_old, beta, u))


def opt_step(cfg, T, ta, g, m, v, dof, pose=0):
    """In-place FP64 update of (m, v, dof) with cfg's optimizer; g = (dE/dt, tau, dE/dtheta)."""
    lib().or_opt_step(C.byref(cfg), T, ta, pose, _dp(g), _dp(m), _dp(v), _dp(dof))


adam_step = opt_step


def loop_steps(S, Lmc, l):
    return lib().or_loop_steps(S, Lmc, l)


def sample_ligand(cfg, p, pxyz, ptype, lg, lig, P, n_threads=1, md=None, mp=None):
    """FP64 trajectories of P poses; returns (dof [P, 7+T], energy [P], in-cutoff pair count)."""
    T = lg.n_tor
    dof = np.zeros((P, 7 + T))
    e = np.zeros(P)
    pxyz = np.ascontiguousarray(pxyz, dtype=np.float64)
    ptype = np.ascontiguousarray(ptype, dtype=np.int32)
    pairs = lib().or_sample_ligand(C.byref(cfg), C.byref(p), len(ptype), _dp(pxyz), _ip(ptype),
                                   None if md is None else C.byref(md), None if mp is None else C.byref(mp),
                                   C.byref(lg), lig, P, 7 + T, _dp(dof), _dp(e), n_threads)
    return dof, e, pairs


def screen_energy(e_inter, w_tor, n_tor):
    """E_screen = E_inter / (1 + w_tor N_tor) (FP64)."""
    return lib().or_screen_energy(float(e_inter), float(w_tor), int(n_tor))


def topk(E, X, k, rho):
    E = np.ascontiguousarray(E, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    P, L = X.shape[0], X.shape[1]
    idx = np.zeros(k, dtype=np.int32)
    near = C.c_int32()
    lib().or_topk(P, _dp(E), _dp(X), L, k, float(rho), _ip(idx), C.byref(near))
    return idx, near.value
