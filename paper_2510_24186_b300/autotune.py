"""Launch-shape autotuner for the persistent sampler.

Two shapes decide the sampler's speed on a given GPU, pocket and ligand mix:
  * warps per block (= poses per block: one warp owns one pose); it sets the
    granularity of work stealing and, with the shared memory per warp, how many
    blocks fit on an SM;
  * the candidate-grid cell edge of the pocket (tile of the ligand-pocket culling):
    smaller cells test fewer pairs outside the cutoff but make longer lists.
The tuner times a sampling pass over a subset of the ligands for every combination,
keeps the fastest, and caches the choice in a JSON file keyed by the GPU, the pocket
size, the ligand-size profile, the pose count and the schedule.  Given the workload's
schedule (steps, mc_loops) the probe runs it in full: poses that start at random in the
box and poses that have settled into the pocket meet different candidate-list lengths,
so a few evaluations from random starts can favour another cell size than the whole run.  The warp count
does not change results (one warp owns a pose whatever the block shape); the cell edge changes which
out-of-cutoff candidates are tested (they add exact zeros) and the order of the pair sums, so only the
last bits of a result.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os
import time
from typing import Optional, Sequence

import numpy as np
import torch

from . import api

CELLS = (0.5, 0.75, 1.0)
WARPS = (20, 24, 28)   # the library caps each at the kernel's compiled maximum


@dataclasses.dataclass
class Choice:
    cell: float
    warps_per_block: int
    ms: float
    table: dict


def _key(pocket_n, n_atoms, n_tor, poses, steps, mc_loops, device_name):
    la = np.asarray(n_atoms)
    lt = np.asarray(n_tor)
    prof = (int(pocket_n), int(la.max()), int(round(la.mean())), int(lt.max()), int(round(lt.mean())), int(poses),
            int(steps), int(mc_loops))
    return hashlib.sha1(f"{device_name}|{prof}".encode()).hexdigest()[:16]


def autotune(pocket_xyz, pocket_type, box_center, box_size, params: api.ScoreParams, lig_arrays,
             poses: int, steps: Optional[int] = None, mc_loops: int = 8, probe_ligands: int = 128,
             cells: Sequence[float] = CELLS, warps: Sequence[int] = WARPS, cache_path: Optional[str] = None,
             repeats: int = 2) -> Choice:
    """lig_arrays = (n_atoms, xyz, type, n_bonds, bonds, rotatable) as for api.Batch.  steps and
    mc_loops: the workload's schedule, run in full by the probe (steps=None: 6 evaluations in
    2 loops, a quick probe from random starts)."""
    probe_steps, probe_loops = (steps, mc_loops) if steps else (6, 2)
    n_atoms, xyz, types, n_bonds, bonds, rot = lig_arrays
    dev = torch.cuda.get_device_name()
    # probe subset: the first ligands, whole
    k = min(probe_ligands, len(n_atoms))
    na = np.asarray(n_atoms)[:k]
    nb = np.asarray(n_bonds)[:k]
    sub = (na, np.asarray(xyz)[:na.sum()], np.asarray(types)[:na.sum()], nb, np.asarray(bonds)[:nb.sum()],
           np.asarray(rot)[:nb.sum()])
    key = None
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    table = {}
    best = None
    stream = torch.cuda.Stream()
    for cell in cells:
        pk = api.Pocket(pocket_xyz, pocket_type, box_center, box_size, params, cell=cell)
        b = api.Batch(pk, *sub)
        if key is None:
            key = _key(len(pocket_type), n_atoms, b.n_tor, poses, probe_steps, probe_loops, dev)
            if key in cache:
                c = cache[key]
                return Choice(c["cell"], c["warps_per_block"], c["ms"], c.get("table", {}))
        for wpb in warps:
            ts = []
            with torch.cuda.stream(stream):
                for r in range(repeats + 1):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    api.sample(pk, b, poses, probe_steps, mc_loops=probe_loops, seed=17 + r, warps_per_block=wpb,
                               stream=stream)
                    e1.record(stream)
                    stream.synchronize()
                    if r > 0:
                        ts.append(e0.elapsed_time(e1))
            ms = min(ts)
            table[f"{cell}/{wpb}"] = ms
            if best is None or ms < best[2]:
                best = (cell, wpb, ms)
        b.close()
        pk.close()
    choice = Choice(best[0], best[1], best[2], table)
    if cache_path:
        cache[key] = dataclasses.asdict(choice)
        try:
            os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return choice
