"""Benchmark: poses x evaluations per second of the persistent fused sampler on one B300.

One benchmark step = one full sampling pass over the batched-screening workload
(1,024 seeded ligands, 10-60 heavy atoms, 0-15 rotatable bonds, 128 poses each,
50 score+gradient evaluations in 8 Monte-Carlo loops, 1,500-atom pocket) followed by
the top-9 rank+cluster, with every input resident in HBM.  The plain form (one launch
per ligand and evaluation, same device code) is timed beside it, the FP64 CPU oracle
on a bounded sample, and an end-to-end pass that packs host ligand arrays, samples,
ranks and copies the results back.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {trids,reference}]
Multi-GPU (torchrun): the ligand set is split over the ranks by longest-processing-time
on each ligand's cost.  For the batched-screening workload the job on N GPUs is N times the
one-GPU set (its first 1,024 ligands are that set, the rest drawn from the same seeded
generator), so every GPU gets about 1,024 ligands (weak scaling); the larger workloads
split their one fixed set (strong scaling).  Every rank samples its shard with the
ligands' global indices as random-stream ids, so the results do not depend on the split.  No collective touches the data path; the timed
region is bracketed by barriers, the slowest rank's time is used, and the shards' top-k
are gathered on rank 0 on the host after it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import select
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_24186_b300 import synth  # noqa: E402

METRIC = "poses×steps/sec (score + DOF gradient) at 1 B300 vs plain per-ligand launch"
UNIT = "pose-steps/s"
# Algorithmic FP32 FLOPs (FMA = 2; rsqrt, exp and log counted apart as transcendentals),
# counted from the evaluations' expressions, per unit of work the counting run reports:
F_PAIR_VINA = 53            # an in-cutoff pair of the Vina-form terms (5 terms, + 3 transcendentals)
F_PAIR_TRIDS = 27           # an in-cutoff pair of the TRIDS atom-pair terms: distance, E_long, force
F_CLASH = 5                 # + a pair inside the E_clash range
F_HBOND = 8                 # + a donor-acceptor pair inside the E_Hbond range
F_MDN_PAIR = 20             # an atom-pair E_MDN pair inside 5 A (term set 1): distance, mask, force ...
F_MDN_KERNEL = 8            # ... + per Gaussian kernel
F_RES_SCAN = 8              # a residue atom scanned for the residue minimum (term set 2)
F_RES_PAIR = 13             # a (ligand atom, residue) pair inside 5 A: distance, force, + 8 per kernel
FP32_LANES_PER_SM = 128


def pair_flops(term_set, pairs, work, K):
    """Algorithmic FLOPs of the pairwise-energy phase of one sampling pass from its counts
    (work: the counting run's TRIDS_WORK_* counts)."""
    if term_set == 0:
        return pairs * F_PAIR_VINA
    f = pairs * F_PAIR_TRIDS + work["clash"] * F_CLASH + work["hbond"] * F_HBOND
    if term_set == 1:
        f += work["mdn_pairs"] * (F_MDN_PAIR + F_MDN_KERNEL * K)
    else:
        f += work["res_scan"] * F_RES_SCAN + work["res_pairs"] * (F_RES_PAIR + F_MDN_KERNEL * K)
    return f
TERMS = {"vina5": 0, "trids": 1, "trids_res": 2}
GMM_K = 4                   # Gaussian kernels per type pair (term set 1) / per atom-residue pair (2)


def score_setup(terms, w):
    """Scoring parameters of a term set; residues of the pocket for term set 2."""
    from paper_2510_24186_b300 import api
    ts = TERMS[terms]
    if ts == 0:
        return api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff), None
    rng = np.random.default_rng(w.seed + 71)
    gmm = None
    if ts == 1:
        gmm = np.empty((synth.N_TYPES, synth.N_TYPES, GMM_K, 3))
        gmm[..., 0] = rng.uniform(0.05, 1.0, gmm.shape[:3]) / GMM_K
        gmm[..., 1] = rng.uniform(2.0, 5.5, gmm.shape[:3])
        gmm[..., 2] = rng.uniform(0.3, 1.5, gmm.shape[:3])
    sp = api.ScoreParams(ts, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0, gmm=gmm)
    res = synth.gen_residues(rng, w.pocket.xyz) if ts == 2 else None
    return sp, res


def mdn_kernels(w, n_atoms_total, res):
    return synth.gen_mdn(np.random.default_rng(w.seed + 72), n_atoms_total, int(res.max()) + 1, GMM_K)


def kernel_source_hash():
    """Hash of the files that define the sampler kernels' code (not the host code around them)."""
    h = hashlib.sha256()
    for f in ("trids_internal.h", "device_core.cuh", "device_passes.cuh", "device_kernels.cuh"):
        f = os.path.join("paper_2510_24186_b300", "csrc", f)
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def sm_max_mhz():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]), "measured"
    except Exception:
        pass
    try:
        out = subprocess.check_output(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                      text=True)
        return float(out.split()[0]), "nvidia-smi"
    except Exception:
        return 2032.0, "fallback"


class ClockSampler:
    """nvidia-smi clock + throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(self.index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            # wait for the first sample (taken before the timed region; dropped), so that the
            # sampler is running when the region starts
            if select.select([self.p.stdout], [], [], 10.0)[0]:
                self.p.stdout.readline()
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                mhz.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(mhz)}


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample_rate(w, budget_s=12.0, max_ligs=64, n_threads=None, first=0, terms="vina5", optimizer="adam"):
    """FP64 oracle sampler on whole ligands of the workload until ~budget_s of wall time."""
    import oracle
    n_threads = n_threads or cpu_threads()
    f32 = lambda v: [float(np.float32(x)) for x in v]
    sp, res = score_setup(terms, w)
    op = oracle.make_params(sp.term_set, f32(sp.radius), sp.flags, f32(sp.w), float(np.float32(sp.cutoff)),
                            gmm=None if sp.gmm is None else np.asarray(sp.gmm, dtype=np.float32).astype(np.float64))
    mdn = offs = None
    if res is not None:
        n_atoms = np.array([len(l.type) for l in w.ligands])
        offs = np.concatenate([[0], np.cumsum(n_atoms)])
        mdn = mdn_kernels(w, int(n_atoms.sum()), res)
    if w.box_centers is not None:   # several docking boxes: pose p in box p mod n
        lo = w.box_centers - w.box_sizes / 2
        hi = w.box_centers + w.box_sizes / 2
    else:
        lo = w.box_center - w.box_size / 2
        hi = w.box_center + w.box_size / 2
    cfg = oracle.sample_cfg(steps=w.steps, mc_loops=w.mc_loops, seed=7, box_lo=lo, box_hi=hi, optimizer=optimizer)
    pxyz = w.pocket.xyz.astype(np.float32).astype(np.float64)
    ptype = w.pocket.type.astype(np.int32)
    t0 = time.perf_counter()
    n, units = 0, 0
    for l in range(first, min(len(w.ligands), first + max_ligs)):
        lg = w.ligands[l]
        st, ol = oracle.pack(lg.xyz.astype(np.float32).astype(np.float64), lg.type, lg.bonds, lg.rotatable)
        md = None if mdn is None else oracle.mdn(res, mdn[offs[l]:offs[l + 1]].astype(np.float64))
        oracle.sample_ligand(cfg, op, pxyz, ptype, ol, l, w.poses, n_threads, md=md)
        n += 1
        units += w.poses * w.steps
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return units / dt, n_threads, n, dt


# Workloads whose job grows with the GPU count (weak scaling), with their one-GPU ligand
# count; the others split one fixed ligand set over the GPUs (strong scaling).
WEAK_LIGANDS = {"batched_screening": 1024}


def job_ligands(args, world):
    """Ligands of the whole job (None: the workload's own set): N times the one-GPU set for a
    weakly scaled workload on N GPUs."""
    if args.workload in WEAK_LIGANDS and world > 1:
        return world * (args.n_lig or WEAK_LIGANDS[args.workload])
    return args.n_lig or None


def scaling_of(args):
    return "weak" if args.workload in WEAK_LIGANDS else "strong"


def workload_config(w, args, world):
    """The workload a bench line measures (the same dict for both arms of the comparison)."""
    name = w.name
    if world > 1:
        name += (f"; on {world} GPUs {len(w.ligands)} ligands ({world} x the one-GPU set) in {world} "
                 "longest-processing-time shards" if scaling_of(args) == "weak" else
                 f"; split over {world} GPUs in longest-processing-time shards")
    return {"workload": name, "n_lig": len(w.ligands), "poses": w.poses, "steps": w.steps,
            "mc_loops": w.mc_loops, "pocket_atoms": len(w.pocket.type), "top_k": w.topk, "term_set": args.terms,
            "optimizer": args.optimizer, "maps_spacing": args.maps or None,
            "l2": "flushed between steps (256 MB write)", "parallelism": f"ligand shards x{world}"}


def run_reference(args, rank):
    if rank != 0:
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = synth.workload(args.workload, n_lig=job_ligands(args, world))
    rates = []
    for k in range(args.warmup + args.steps):
        r, cores, n, dt = oracle_sample_rate(w, budget_s=0.0, max_ligs=1, first=k % len(w.ligands), terms=args.terms,
                                             optimizer=args.optimizer)
        if k >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * w.poses * w.steps / value,
            "higher_is_better": True, "scaling": scaling_of(args), "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one ligand x {w.poses} poses x {w.steps} evaluations per step, FP64 "
                                       "all-pairs oracle on all host threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="trids", choices=["trids", "reference"])
    ap.add_argument("--per-ligand-steps", type=int, default=None,
                    help="timed steps of the plain per-ligand form (default 1 for batched_screening, else 0)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--n-lig", type=int, default=0, help="first N ligands only (small profiling case)")
    ap.add_argument("--workload", default="batched_screening",
                    choices=["batched_screening", "screening_stream", "blind_docking"],
                    help="batched_screening (the headline); screening_stream: 100,000 ligands end to end "
                         "over uneven batches; blind_docking: 6,000-atom region, three cavities")
    ap.add_argument("--cell", type=float, default=0.0, help="candidate-grid cell edge in A (0 = library default)")
    ap.add_argument("--terms", default="vina5", choices=sorted(TERMS),
                    help="term set: vina5 (default), trids (atom-pair E_MDN), trids_res (residue-level E_MDN)")
    ap.add_argument("--optimizer", default="adam", choices=["adam", "adamw", "rmsprop", "adagrad", "sgd"])
    ap.add_argument("--maps", type=float, default=0.0,
                    help="grid-map spacing in A (0 = direct pair sums, the paper's form); margin 8 A")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    from paper_2510_24186_b300 import api, parallel
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = synth.workload(args.workload, n_lig=job_ligands(args, world))
    if w.cell and not args.cell:
        args.cell = w.cell
    if args.per_ligand_steps is None:
        args.per_ligand_steps = 1 if args.workload == "batched_screening" and world == 1 else 0
    sp, res = score_setup(args.terms, w)
    all_arrays = synth.concat_ligands(w.ligands)
    # this rank's shard of the ligand set (all of it on one GPU)
    mine = parallel.shard_lpt(parallel.ligand_cost([len(l.type) for l in w.ligands],
                                                   [l.n_tor for l in w.ligands]), world)[rank]
    arrays = synth.concat_ligands([w.ligands[i] for i in mine]) if world > 1 else all_arrays
    tuned = None
    if sp.term_set != 0:
        args.cell, args.warps = args.cell or 0.5, args.warps or 24
    if not args.cell and not args.warps:
        shape = [None]
        if rank == 0:
            from paper_2510_24186_b300 import autotune
            tuned = autotune.autotune(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp, all_arrays,
                                      w.poses, steps=w.steps, mc_loops=w.mc_loops)
            shape = [(tuned.cell, tuned.warps_per_block)]
        if dist:
            dist.broadcast_object_list(shape, src=0)   # every rank runs rank 0's tuned shape
        args.cell, args.warps = shape[0]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()               # so the job's tensors are not served from the tuner's cached blocks
    free0 = torch.cuda.mem_get_info()[0]   # device memory of the job: pocket, batch, state, work lists, graph
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp, cell=args.cell)
    if w.box_centers is not None:
        pk.set_boxes(w.box_centers, w.box_sizes)
    maps = None
    if args.maps > 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pk.build_maps(args.maps, 8.0)
        torch.cuda.synchronize()
        lo, hm, dims = pk.maps_info()
        maps = {"spacing": hm, "margin": 8.0, "points": list(dims), "build_ms": 1000 * (time.perf_counter() - t0),
                "bytes": int(np.prod(dims)) * synth.N_TYPES * 4}
    mdn = None
    if res is not None:
        pk.set_residues(res)
        rows = mdn_kernels(w, int(all_arrays[0].sum()), res)
        offs = np.concatenate([[0], np.cumsum(all_arrays[0])])
        rows = np.concatenate([rows[offs[i]:offs[i + 1]] for i in mine]) if world > 1 else rows
        mdn = torch.from_numpy(rows).cuda()
    b = api.Batch(pk, *arrays)
    b.set_stream_ids(mine)          # global ligand ids: the samples do not depend on the split
    if mdn is not None:
        b.set_mdn(mdn)
    P, S, Lm = w.poses, w.steps, w.mc_loops
    n_lig = b.n_lig
    units = n_lig * P * S                   # this rank's pose-evaluations per step
    units_all = len(w.ligands) * P * S      # the whole job's
    lig_base = 0
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2
    dof = torch.zeros(n_lig, P, b.dof_stride, device="cuda")
    state = torch.zeros(b.state_floats(P), device="cuda")
    energy = torch.empty(n_lig, P, device="cuda")

    def one_step(seed, **kw):
        o = api.sample(pk, b, P, S, mc_loops=Lm, seed=seed, lig_base=lig_base, dof=dof, state=state, energy=energy,
                       warps_per_block=args.warps, stream=stream, optimizer=args.optimizer, **kw)
        return o

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            one_step(100 + k)
            api.topk(b, energy, dof, w.topk, 1.0, stream=stream)
    stream.synchronize()
    job_mb = (free0 - torch.cuda.mem_get_info()[0] - flush.numel()) / 2 ** 20
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    seeds = [1000 + k for k in range(args.steps)]
    energies = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    g0 = pk.graph_stats()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xff)                       # evict the previous step from L2 (untimed)
                ev[k][0].record(stream)
                one_step(seeds[k])
                ev[k][1].record(stream)
                idx, etop = api.topk(b, energy, dof, w.topk, 1.0, stream=stream)
                ev[k][2].record(stream)
                energies.append(energy.clone())
        stream.synchronize()
    if dist:
        dist.barrier()
    g1 = pk.graph_stats()
    graph_timed = {k: g1[k] - g0[k] for k in g1}
    t_sample = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_step = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    total_ms = parallel.max_over_ranks(sum(t_step), device="cuda")
    rc = api.sync(b, P, state, timeout_ms=60000)
    # the last step's top-k of every shard, gathered on rank 0 in global ligand order (host)
    gathered = parallel.gather_topk(mine, idx.cpu().numpy(), etop.cpu().numpy())

    # in-cutoff pair counts of the same trajectories (untimed counting variant; the
    # energies must come out bit-identical to the timed runs)
    # and the SM cycles the warps spent in each phase of an evaluation (the same counting
    # variant times its phases; their shares apportion the timed kernel's duration)
    pairs, works = [], []
    cycles = np.zeros(len(api.PHASES))
    identical = True
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            o = one_step(seeds[k], count_pairs=True)
            stream.synchronize()
            pairs.append(int(o["pair_count"].item()))
            works.append(dict(zip(api.WORK, o["work_count"].cpu().numpy().tolist())))
            cycles += o["phase_cycles"].cpu().numpy().astype(np.float64)
            identical &= bool(torch.equal(energy, energies[k]))
    phase_share = {n: float(c / cycles.sum()) for n, c in zip(api.PHASES, cycles)}

    # plain per-ligand form, same device code
    pl_ms = None
    if args.per_ligand_steps > 0:
        with torch.cuda.stream(stream):
            one_step(7, mode=1)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.per_ligand_steps):
                one_step(8 + k, mode=1)
            e1.record(stream)
            stream.synchronize()
            pl_ms = e0.elapsed_time(e1) / args.per_ligand_steps

    # end to end through the public API: the screening stream packs each batch's host arrays
    # (on a host thread, while the previous batch samples), uploads them, samples, ranks and
    # copies the top-k back to pinned host memory; every step is one whole batch
    # (screening_stream: one pass over the whole ligand set in seeded uneven batches of 500-5,000
    # ligands, the first batch untimed)
    stats = {}
    torch.cuda.synchronize()
    marks = []
    prep = (lambda bb: bb.set_mdn(mdn, stream=stream)) if mdn is not None else None
    if args.workload == "screening_stream" and mdn is None:
        rng4 = np.random.default_rng(w.seed + 4)
        cuts = [0]
        while cuts[-1] < len(w.ligands):
            cuts.append(min(len(w.ligands), cuts[-1] + int(rng4.integers(500, 5001))))
        spans = list(zip(cuts[:-1], cuts[1:]))[rank::world]      # every world-th batch on this rank
        batches = [synth.concat_ligands(w.ligands[a:b]) for a, b in spans]
        e2e_units = sum(b - a for a, b in spans[1:]) * P * S
        e2e_note = (f"one pass over {len(w.ligands)} ligands in {len(cuts) - 1} uneven batches (500-5,000), "
                    f"every {world}th on each rank, each rank's first untimed")
    else:
        batches = [arrays] * (args.warmup + args.steps)
        e2e_units = units * args.steps
        e2e_note = "every step is the whole batch"
    for _ in api.screen_stream(pk, batches, P, S, w.topk, 1.0, seed=5000, mc_loops=Lm, warps_per_block=args.warps,
                               stream=stream, stats=stats, prepare=prep, optimizer=args.optimizer):
        marks.append(time.perf_counter())
    n_untimed = 1 if len(batches) != args.warmup + args.steps else args.warmup
    e2e_s = marks[-1] - marks[n_untimed - 1]
    e2e_ms = 1000 * e2e_s / (len(marks) - n_untimed)
    # the whole job: every rank's pose-evaluations over the slowest rank's time
    e2e_s_max = parallel.max_over_ranks(e2e_s, device="cuda")
    e2e_units_all = e2e_units
    if dist:
        t = torch.tensor([float(e2e_units)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t)
        e2e_units_all = float(t.item())
    e2e_value = e2e_units_all / e2e_s_max
    h2d, d2h = stats["h2d_bytes"], stats["d2h_bytes"]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = units_all / (total_ms / 1000.0 / args.steps)
    mhz, mhz_src = sm_max_mhz()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    flops = [pair_flops(sp.term_set, p, wk, GMM_K) for p, wk in zip(pairs, works)]
    achieved = sum(flops) / (sum(t_sample) / 1000.0) / 1e12
    # the pairwise-energy phase: the pair loop plus, for the TRIDS terms, the E_MDN passes
    pair_ms = statistics.mean(t_sample) * (phase_share["pairs"] + phase_share["passes"])
    achieved_pair = sum(flops) / len(flops) / (pair_ms / 1000.0) / 1e12
    clocks = clk.summary()
    traffic = None
    prof = os.path.join(ROOT, "profiles", "sample_persistent_vina5_batched_screening.json")
    if os.path.exists(prof) and sp.term_set == 0 and args.optimizer == "adam" and maps is None and args.workload == "batched_screening":
        pj = json.load(open(prof))
        if pj.get("source_hash") == kernel_source_hash() and (pj.get("cell"), pj.get("warps")) == (args.cell, args.warps):
            traffic = pj.get("dram_bytes_per_launch")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": scaling_of(args), "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, args, world),
        "launch": {"graph": {"timed_region": graph_timed, "total": g1,
                             "note": "one CUDA graph per launch shape, built in the warm-up; each timed step "
                                     "replays it after updating its nodes with that step's seed"},
                   "cell": args.cell or 0.5, "warps_per_block": args.warps, "maps": maps,
                   "autotuned": None if tuned is None else {"table_ms": tuned.table, "probe": f"first 128 ligands x "
                                                            f"{P} poses x {S} evaluations per shape"},
                   "shards": {"split": "longest-processing-time on ligand cost, global ligand ids as stream ids",
                              "rank0_ligands": len(mine), "topk_gathered_ligands": len(gathered[0])}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "note": ("in-cutoff atom pairs x 53 FP32 FLOP" if sp.term_set == 0 else
                              f"counted work x FLOPs per unit: pairs x {F_PAIR_TRIDS} + E_clash pairs x {F_CLASH} + "
                              f"E_Hbond pairs x {F_HBOND} + "
                              + (f"E_MDN pairs x ({F_MDN_PAIR} + {F_MDN_KERNEL} K)" if sp.term_set == 1 else
                                 f"residue atoms scanned x {F_RES_SCAN} + residue pairs x ({F_RES_PAIR} + "
                                 f"{F_MDN_KERNEL} K)") + f", K = {GMM_K}")
                             + f" / persistent-sampler time; peak = {n_sm} SM x 128 lanes x 2 x {mhz:.0f} MHz "
                               f"({mhz_src})"
                             + ("" if maps is None else "; with maps only the atoms outside the map grid sum "
                                "pairs, so this counts the direct pairs alone")},
        "kernel": {"sample_ms": statistics.mean(t_sample), "phase_share": phase_share,
            "phase_share_note": "share of the warps' SM clock cycles per phase, from the counting variant of the "
                                "sampler (same trajectories); pairs = per-atom candidate set-up, pair sums and "
                                "lane-order combine",
            "topk_ms": statistics.mean(
            [t_step[k] - t_sample[k] for k in range(args.steps)]), "pairs_per_step": statistics.mean(pairs),
            "pairs_per_pose_step": statistics.mean(pairs) / units, "count_run_bit_identical": identical,
            "work_per_pose_step": {k: statistics.mean(wk[k] for wk in works) / units for k in api.WORK},
            "flops_per_pose_step": statistics.mean(flops) / units,
            "status": rc},
        "per_ligand": None if pl_ms is None else {
            "value": units / (pl_ms / 1000.0), "ms_per_step": pl_ms, "launches_per_step": n_lig * S,
            "speedup_persistent": (pl_ms / (sum(t_sample) / args.steps))},
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "includes": "api.screen_stream: host pack (overlapped with the previous batch's sampling) + "
                            "upload, sample, top-k, D2H of top-k to pinned memory; " + e2e_note},
        "gpu_launches": 2 * args.steps,
        "device_memory_mb": {"job": round(job_mb, 1),
                             "what": "device memory taken from before the pocket is built to after the warm-up "
                                     "(pocket grids, packed batch, DOF / sampler state / energies, work lists, "
                                     "CUDA graph), less the L2-flush buffer"},
        "clocks": clocks,
    }
    # the pair phase alone: its FLOPs over its share of the timed kernel's duration
    line["roofline"]["achieved_pair"] = achieved_pair
    line["roofline"]["frac_pair"] = achieved_pair / peak
    line["roofline"]["pair_ms"] = pair_ms
    if clocks["sm_mhz"]:
        line["roofline"]["frac_at_load_clock"] = achieved / (peak * clocks["sm_mhz"] / mhz)
    if not args.no_cpu and world == 1:
        r, cores, n, dt = oracle_sample_rate(w, budget_s=12.0, terms=args.terms)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {n} ligands x {P} poses x {S} evaluations, FP64 all-pairs "
                                          f"oracle, {dt:.1f} s"}
        if args.terms == "vina5":
            w1 = synth.workload("single_ligand")
            r1, c1, n1, dt1 = oracle_sample_rate(w1, budget_s=0.0, max_ligs=1, n_threads=1)
            line["cpu_baseline_single_ligand"] = {"value": r1, "unit": UNIT, "cores": c1, "kind": "oracle",
                                            "sample": f"the single-ligand workload in full ({w1.poses} poses x "
                                                      f"{w1.steps} evaluations, 300-atom pocket), one thread, "
                                                      f"{dt1:.2f} s"}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
