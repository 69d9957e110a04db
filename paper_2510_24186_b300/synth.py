"""Seeded synthetic inputs: ligand trees, pockets, random poses and workloads.

This module only draws inputs. It holds none of the scoring, kinematics or
sampling arithmetic, so both the CUDA path and the FP64 oracle can be fed from
it without sharing any of the method's code.

The paper's datasets (PDBbind, DEKOIS 2.0, PoseBusters) are not available, so
every workload is a seeded stand-in with the shapes the paper's sampler sees:
a pocket of atoms around a cavity, a translation box around it (Sec. 2,
"Conformation sampling": translation in [box_min, box_max], rotation and
torsions in [-pi, pi)), and ligands with a few to twenty rotatable bonds.

Recipes (all distances in Angstrom):
  * ligand: random bonded tree. Each new atom bonds to a random atom of degree
    < 4 at 1.5 A; bond angles to the parent's other neighbours ~109.5 +- 5 deg;
    the dihedral is random. A placement closer than 2.0 A to any non-bonded atom
    is retried (100 tries) and then the parent is re-drawn. T rotatable bonds are
    drawn uniformly among the internal edges (both ends of degree >= 2); T is
    clamped to the number of internal edges.
  * pocket: random sequential addition in a shell 4 A <= r <= R_out around a
    cavity centre (or a union of such shells), atoms >= 3 A apart. R_out starts
    at 12 A and grows by 0.5 A after 10,000 consecutive rejections.
  * 8 Vina-style atom types with project-chosen radii and flags (below).
  * residues (for the residue-level E_MDN): greedy spatial groups of pocket
    atoms. Seed = the lowest-index unassigned atom; the group takes the seed's
    nearest unassigned atoms within 6 A, up to a size drawn from U{4..14}.
  * per-(ligand atom, residue) Gaussian kernels (what the paper's network would
    predict): pi ~ U(0.05, 1) / K, mu ~ U(2.0, 5.5), sigma ~ U(0.3, 1.5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial import cKDTree

# Eight Vina-style atom types.  flags: bit0 hydrophobic, bit1 donor, bit2 acceptor.
TYPE_NAMES = ("C_H", "C_P", "N_P", "N_D", "N_A", "O_A", "O_DA", "Cl_H")
TYPE_RADIUS = (1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 1.8)
TYPE_FLAGS = (1, 0, 0, 2, 4, 4, 6, 1)
N_TYPES = len(TYPE_NAMES)
UNIFORM_MIX = tuple([1.0 / N_TYPES] * N_TYPES)
DRUGLIKE_MIX = (0.40, 0.20, 0.06, 0.06, 0.08, 0.10, 0.06, 0.04)

# Published AutoDock Vina weights (Trott & Olson, J. Comput. Chem. 2010):
# gauss1, gauss2, repulsion, hydrophobic, hydrogen bond.
VINA_WEIGHTS = (-0.0356, -0.00516, 0.840, -0.0351, -0.587)
# TRIDS weights for (E_MDN, E_long, E_clash, E_Hbond) (Sec. 2, "Scoring functions").
TRIDS_WEIGHTS = (1.0, 0.2, 10.0, 0.6, 0.0)

BOND = 1.5
TETRA = math.radians(109.5)


@dataclasses.dataclass
class Ligand:
    xyz: np.ndarray        # [L, 3] float64 input geometry
    type: np.ndarray       # [L] int32
    bonds: np.ndarray      # [nb, 2] int32 (a < b)
    rotatable: np.ndarray  # [nb] uint8
    n_tor: int             # realised number of rotatable bonds


@dataclasses.dataclass
class Pocket:
    xyz: np.ndarray        # [M, 3] float64
    type: np.ndarray       # [M] int32
    centers: np.ndarray    # [n_cav, 3]
    r_out: float           # realised outer radius of the shell
    density: float         # atoms per A^3 inside the shell


def _norm3(v):
    return math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])


def _unit(v):
    n = _norm3(v)
    return (v[0] / n, v[1] / n, v[2] / n)


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _lin(a, sa, b, sb):
    return (a[0] * sa + b[0] * sb, a[1] * sa + b[1] * sb, a[2] * sa + b[2] * sb)


def _rand_unit(rng):
    while True:
        v = tuple(rng.normal(size=3).tolist())
        n = _norm3(v)
        if n > 1e-6:
            return (v[0] / n, v[1] / n, v[2] / n)


def _rotate(v, axis, ang):
    """Rotate v about unit axis by ang (used only to scatter generated geometry)."""
    c, s = math.cos(ang), math.sin(ang)
    cr = _cross(axis, v)
    ad = _dot(axis, v) * (1.0 - c)
    return (v[0] * c + cr[0] * s + axis[0] * ad, v[1] * c + cr[1] * s + axis[1] * ad,
            v[2] * c + cr[2] * s + axis[2] * ad)


def _perp(u, rng):
    w = _rand_unit(rng)
    return _unit(_lin(w, 1.0, u, -_dot(u, w)))


def _bond_direction(rng, nbr_dirs):
    """Direction for a new bond given unit vectors to the parent's neighbours."""
    k = len(nbr_dirs)
    if k == 0:
        return _rand_unit(rng)
    if k == 1:
        u = nbr_dirs[0]
        ang = TETRA + math.radians(rng.uniform(-5.0, 5.0))
        p = _perp(u, rng)  # random dihedral
        return _unit(_lin(u, math.cos(ang), p, math.sin(ang)))
    if k == 2:
        u1, u2 = nbr_dirs
        bis = _unit(_lin(u1, -1.0, u2, -1.0))
        n = _cross(u1, u2)
        nn = _norm3(n)
        n = _perp(bis, rng) if nn < 1e-6 else (n[0] / nn, n[1] / nn, n[2] / nn)
        half = 0.5 * TETRA
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        d = _unit(_lin(bis, math.cos(half), n, sgn * math.sin(half)))
    else:
        s = _lin(_lin(nbr_dirs[0], 1.0, nbr_dirs[1], 1.0), 1.0, nbr_dirs[2], 1.0)
        d = _unit((-s[0], -s[1], -s[2]))
    # scatter by up to 5 degrees about a random perpendicular axis
    return _unit(_rotate(d, _perp(d, rng), math.radians(rng.uniform(-5.0, 5.0))))


def _units(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _rand_units(rng, n):
    v = rng.normal(size=(n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    return v / np.where(nrm > 1e-6, nrm, 1.0)


def _perps(u, rng, n):
    """n random unit vectors perpendicular to the unit vector(s) u ([3] or [n, 3])."""
    w = _rand_units(rng, n)
    return _units(w - u * np.sum(u * w, axis=-1, keepdims=True))


def _bond_directions(rng, nbr_dirs, n):
    """n candidate directions for a new bond, each drawn as _bond_direction draws one."""
    k = len(nbr_dirs)
    if k == 0:
        return _rand_units(rng, n)
    if k == 1:
        u = np.asarray(nbr_dirs[0])
        ang = TETRA + np.radians(rng.uniform(-5.0, 5.0, n))[:, None]
        return _units(u * np.cos(ang) + _perps(u, rng, n) * np.sin(ang))
    if k == 2:
        u1, u2 = np.asarray(nbr_dirs[0]), np.asarray(nbr_dirs[1])
        bis = _units(-u1 - u2)
        nc = np.cross(u1, u2)
        nn = np.linalg.norm(nc)
        nv = _perps(bis, rng, n) if nn < 1e-6 else np.broadcast_to(nc / nn, (n, 3))
        sgn = np.where(rng.random(n) < 0.5, 1.0, -1.0)[:, None]
        half = 0.5 * TETRA
        d = _units(bis * math.cos(half) + nv * sgn * math.sin(half))
    else:
        d = np.broadcast_to(_units(-(np.asarray(nbr_dirs[0]) + nbr_dirs[1] + nbr_dirs[2])), (n, 3))
    # scatter by up to 5 degrees about a random perpendicular axis (Rodrigues)
    ax = _perps(d, rng, n)
    ang = np.radians(rng.uniform(-5.0, 5.0, n))[:, None]
    c, s_ = np.cos(ang), np.sin(ang)
    return _units(d * c + np.cross(ax, d) * s_ + ax * np.sum(ax * d, axis=1, keepdims=True) * (1.0 - c))


def gen_ligand(rng: np.random.Generator, n_atoms: int, n_tor: int,
               type_probs=UNIFORM_MIX, center=(0.0, 0.0, 0.0), vector_tries: bool = False) -> Ligand:
    """Random bonded tree ligand (see module docstring for the recipe).  vector_tries draws
    a parent's 100 candidate placements at once and keeps the first that clears the 2 A
    test: the same distribution as trying them one by one, with the random stream
    consumed in another order (several times faster; used for the 100,000-ligand set)."""
    assert n_atoms >= 1
    xyz = np.zeros((n_atoms, 3))
    pos_l = [(0.0, 0.0, 0.0)]
    nbrs: list[list[int]] = [[] for _ in range(n_atoms)]
    bonds = []
    for a in range(1, n_atoms):
        placed = False
        while not placed:
            cand = [i for i in range(a) if len(nbrs[i]) < 4]
            par = cand[rng.integers(len(cand))]
            pp = pos_l[par]
            dirs = [_unit(_lin(pos_l[n], 1.0, pp, -1.0)) for n in nbrs[par]]
            if vector_tries:
                pts = np.asarray(pp) + BOND * _bond_directions(rng, dirs, 100)
                d2 = np.sum((pts[:, None, :] - xyz[None, :a, :]) ** 2, axis=2)
                d2[:, par] = 1e9
                ok = np.nonzero(d2.min(axis=1) >= 4.0)[0]
                if len(ok):
                    pos = tuple(pts[ok[0]].tolist())
                    placed = True
                continue
            for _ in range(100):
                pos = _lin(pp, 1.0, _bond_direction(rng, dirs), BOND)
                d2 = np.sum((xyz[:a] - np.asarray(pos)) ** 2, axis=1)
                d2[par] = 1e9
                if d2.min(initial=1e9) >= 4.0:
                    placed = True
                    break
        xyz[a] = pos
        pos_l.append(pos)
        nbrs[par].append(a)
        nbrs[a].append(par)
        bonds.append((par, a))
    bonds = np.array(bonds, dtype=np.int32).reshape(-1, 2)
    bonds.sort(axis=1)
    rot = np.zeros(len(bonds), dtype=np.uint8)
    if len(bonds):
        deg = np.array([len(n) for n in nbrs])
        internal = np.nonzero((deg[bonds[:, 0]] >= 2) & (deg[bonds[:, 1]] >= 2))[0]
        t = min(n_tor, len(internal))
        if t > 0:
            rot[rng.choice(internal, size=t, replace=False)] = 1
    types = rng.choice(N_TYPES, size=n_atoms, p=np.asarray(type_probs)).astype(np.int32)
    xyz = xyz - xyz.mean(axis=0) + np.asarray(center, dtype=np.float64)
    return Ligand(xyz=xyz, type=types, bonds=bonds, rotatable=rot, n_tor=int(rot.sum()))


def gen_pocket(rng: np.random.Generator, n_atoms: int, centers, r_in=4.0, r_out=12.0,
               min_sep=3.0, type_probs=UNIFORM_MIX, grow_after=10000, grow_by=0.5) -> Pocket:
    """Random sequential addition in the union of shells around `centers`."""
    centers = np.atleast_2d(np.asarray(centers, dtype=np.float64))
    pts = np.zeros((0, 3))
    tree = None
    fails = 0
    batch = 2048
    while len(pts) < n_atoms:
        ci = rng.integers(len(centers), size=batch)
        u = rng.random(batch)
        r = np.cbrt(r_in ** 3 + u * (r_out ** 3 - r_in ** 3))
        dirs = rng.normal(size=(batch, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        cand = centers[ci] + dirs * r[:, None]
        dc = np.linalg.norm(cand[:, None, :] - centers[None, :, :], axis=2).min(axis=1)
        ok = dc >= r_in
        if tree is not None:
            dmin, _ = tree.query(cand, k=1, distance_upper_bound=min_sep)
            ok &= ~np.isfinite(dmin) | (dmin >= min_sep)
        new = []
        grew = False
        for i in range(batch):
            good = ok[i]
            if good and new:
                good = np.min(np.sum((np.asarray(new) - cand[i]) ** 2, axis=1)) >= min_sep ** 2
            if good:
                new.append(cand[i])
                fails = 0
                if len(pts) + len(new) >= n_atoms:
                    break
            else:
                fails += 1
                if fails >= grow_after:
                    r_out += grow_by
                    fails = 0
                    grew = True
                    break
        if new:
            pts = np.vstack([pts, np.asarray(new)])
            tree = cKDTree(pts)
        del grew
    pts = pts[:n_atoms]
    types = rng.choice(N_TYPES, size=n_atoms, p=np.asarray(type_probs)).astype(np.int32)
    vol = len(centers) * 4.0 / 3.0 * math.pi * (r_out ** 3 - r_in ** 3)
    return Pocket(xyz=pts, type=types, centers=centers, r_out=float(r_out),
                  density=float(n_atoms / vol))


def gen_residues(rng: np.random.Generator, xyz: np.ndarray, size_range=(4, 14), reach=6.0) -> np.ndarray:
    """Residue index of each pocket atom (greedy spatial groups, see the module notes)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = len(xyz)
    res = np.full(n, -1, dtype=np.int32)
    tree = cKDTree(xyz)
    r = 0
    for seed in range(n):
        if res[seed] >= 0:
            continue
        size = int(rng.integers(size_range[0], size_range[1] + 1))
        near = tree.query_ball_point(xyz[seed], reach)
        near = [j for j in near if res[j] < 0]
        near.sort(key=lambda j: (float(np.sum((xyz[j] - xyz[seed]) ** 2)), j))
        for j in near[:size]:
            res[j] = r
        r += 1
    return res


def gen_mdn(rng: np.random.Generator, n_lig_atoms: int, n_res: int, K: int) -> np.ndarray:
    """Kernels [n_lig_atoms, n_res, K, 3] of (pi, mu, sigma), float32."""
    out = np.empty((n_lig_atoms, n_res, K, 3), dtype=np.float32)
    out[..., 0] = rng.uniform(0.05, 1.0, (n_lig_atoms, n_res, K)) / K
    out[..., 1] = rng.uniform(2.0, 5.5, (n_lig_atoms, n_res, K))
    out[..., 2] = rng.uniform(0.3, 1.5, (n_lig_atoms, n_res, K))
    return out


def random_dofs(rng: np.random.Generator, n_tor: np.ndarray, poses: int, box_min, box_max,
                dof_stride: int) -> np.ndarray:
    """Random (not optimised) poses: t ~ U(box), q ~ uniform unit, theta ~ U[-pi, pi)."""
    n_lig = len(n_tor)
    out = np.zeros((n_lig, poses, dof_stride), dtype=np.float32)
    lo = np.asarray(box_min, dtype=np.float64)
    hi = np.asarray(box_max, dtype=np.float64)
    out[:, :, 0:3] = lo + rng.random((n_lig, poses, 3)) * (hi - lo)
    q = rng.normal(size=(n_lig, poses, 4))
    q /= np.linalg.norm(q, axis=2, keepdims=True)
    out[:, :, 3:7] = q
    th = rng.uniform(-math.pi, math.pi, size=(n_lig, poses, dof_stride - 7))
    for l in range(n_lig):
        out[l, :, 7:7 + n_tor[l]] = th[l, :, :n_tor[l]]
    return out


@dataclasses.dataclass
class Workload:
    name: str
    pocket: Pocket
    ligands: list
    box_center: np.ndarray
    box_size: np.ndarray
    poses: int
    steps: int
    mc_loops: int
    cutoff: float
    topk: int
    seed: int
    cell: float = 0.0
    box_centers: np.ndarray | None = None   # several docking boxes: pose p uses box p mod n
    box_sizes: np.ndarray | None = None


def concat_ligands(ligs):
    """Flatten a ligand list into the concatenated arrays the C-ABI takes."""
    n_atoms = np.array([len(l.type) for l in ligs], dtype=np.int32)
    n_bonds = np.array([len(l.bonds) for l in ligs], dtype=np.int32)
    xyz = np.concatenate([l.xyz for l in ligs]).astype(np.float32)
    types = np.concatenate([l.type for l in ligs]).astype(np.int32)
    bonds = (np.concatenate([l.bonds for l in ligs]) if n_bonds.sum() else
             np.zeros((0, 2))).astype(np.int32)
    rot = (np.concatenate([l.rotatable for l in ligs]) if n_bonds.sum() else
           np.zeros(0)).astype(np.uint8)
    return n_atoms, xyz, types, n_bonds, bonds, rot


def _ligand_set(rng, n_lig, l_range, t_range, mix, center):
    out = []
    for _ in range(n_lig):
        L = int(rng.integers(l_range[0], l_range[1] + 1))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        out.append(gen_ligand(rng, L, T, mix, center))
    return out


def _indexed_chunk(args):
    seed, lo, hi, l_range, t_range, mix, center = args
    out = []
    for i in range(lo, hi):
        rng = np.random.default_rng([seed, i])
        L = int(rng.integers(l_range[0], l_range[1] + 1))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        out.append(gen_ligand(rng, L, T, mix, center, vector_tries=True))
    return out


def _ligand_set_indexed(seed, n_lig, l_range, t_range, mix, center, workers=None, min_parallel=2000):
    """Ligand i drawn from its own generator, seeded (seed, i): the set does not depend on
    how it is split, so large sets are generated on worker processes (spawned, so that a
    process that already uses CUDA is never forked)."""
    import os
    workers = workers or len(os.sched_getaffinity(0))
    if n_lig < min_parallel or workers <= 1:
        return _indexed_chunk((seed, 0, n_lig, l_range, t_range, mix, center))
    import concurrent.futures as cf
    import multiprocessing as mp
    step = -(-n_lig // (4 * workers))
    jobs = [(seed, lo, min(n_lig, lo + step), l_range, t_range, mix, center) for lo in range(0, n_lig, step)]
    out = []
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for part in ex.map(_indexed_chunk, jobs):
            out.extend(part)
    return out


# Named seeded workloads and their seeds.
WORKLOAD_SEEDS = {
    "single_ligand": 1001,
    "batched_screening": 1002,
    "adjoint_check": 1003,
    "screening_stream": 1004,
    "blind_docking": 1005,
}


def workload(name: str, n_lig: int | None = None) -> Workload:
    """The five seeded workloads, by name.  `n_lig` truncates the ligand set.

    single_ligand:     1 ligand, L=24, T=4, M=300, P=64, S=30.
    batched_screening: 1,024 ligands, L~U{10..60}, T~U{0..15}, M=1,500, P=128, S=50, top-9.
    adjoint_check:     256 ligands, L~U{10..40}, T~U{0..10}, M=1,500, P=64 random poses.
    screening_stream:  100,000 ligands, L~U{10..70}, T~U{0..20}, drug-like mix, M=2,000, P=64, S=40;
                       ligand i from its own generator seeded (1004, i), built on worker processes.
    blind_docking:     6,000 atoms around 3 cavities, 4,096 ligands, L~U{20..60}, T<=15, P=512, S=100.
    """
    if name not in WORKLOAD_SEEDS:
        raise ValueError(f"unknown workload {name!r}; one of {sorted(WORKLOAD_SEEDS)}")
    seed = WORKLOAD_SEEDS[name]
    rng = np.random.default_rng(seed)
    c0 = np.zeros(3)
    box = np.full(3, 22.5)
    if name == "single_ligand":
        pk = gen_pocket(rng, 300, c0)
        ligs = [gen_ligand(rng, 24, 4, UNIFORM_MIX, c0)]
        return Workload("single ligand (L=24, T=4), 300-atom pocket, 64 poses x 30 steps",
                        pk, ligs, c0, box, 64, 30, 8, 8.0, 9, seed)
    if name == "batched_screening":
        pk = gen_pocket(rng, 1500, c0)
        ligs = _ligand_set(rng, n_lig or 1024, (10, 60), (0, 15), UNIFORM_MIX, c0)
        return Workload("batched screening: 1,024 ligands (L 10-60, T 0-15) x 128 poses x 50 steps, "
                        "1,500-atom pocket, top-9", pk, ligs, c0, box, 128, 50, 8, 8.0, 9, seed)
    if name == "adjoint_check":
        pk = gen_pocket(rng, 1500, c0)
        ligs = _ligand_set(rng, n_lig or 256, (10, 40), (0, 10), UNIFORM_MIX, c0)
        return Workload("adjoint check: 256 ligands (L 10-40, T 0-10) x 64 random poses",
                        pk, ligs, c0, box, 64, 0, 8, 8.0, 9, seed)
    if name == "screening_stream":
        pk = gen_pocket(rng, 2000, c0, type_probs=DRUGLIKE_MIX)
        ligs = _ligand_set_indexed(seed, n_lig or 100000, (10, 70), (0, 20), DRUGLIKE_MIX, c0)
        return Workload("screening stream: 100,000 ligands (L 10-70, T 0-20) x 64 poses x 40 steps, "
                        "2,000-atom pocket", pk, ligs, c0, box, 64, 40, 8, 8.0, 9, seed)
    if name == "blind_docking":
        side = 18.0
        cav = np.array([[0.0, 0.0, 0.0], [side, 0.0, 0.0], [side / 2, side * math.sqrt(3) / 2, 0.0]])
        cav -= cav.mean(axis=0)
        pk = gen_pocket(rng, 6000, cav)
        ligs = _ligand_set(rng, n_lig or 4096, (20, 60), (0, 15), UNIFORM_MIX, c0)
        return Workload("blind-docking scale: 6,000-atom region, 3 cavities, 4,096 ligands x 512 poses "
                        "x 100 steps", pk, ligs, c0, np.full(3, 22.5), 512, 100, 8, 8.0, 9,
                        seed, cell=1.0, box_centers=cav, box_sizes=np.full((3, 3), 22.5))
    raise AssertionError(name)
