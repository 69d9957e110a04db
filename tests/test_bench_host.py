"""Host logic of bench.py that needs no GPU: the size of the job on N GPUs."""
import argparse

import numpy as np

import bench
from paper_2510_24186_b300 import parallel, synth


def _args(workload, n_lig=0):
    return argparse.Namespace(workload=workload, n_lig=n_lig, terms="vina5", optimizer="adam", maps=0.0)


def test_batched_screening_scales_weakly_and_keeps_the_one_gpu_set_first():
    """On N GPUs the batched-screening job is N times the one-GPU ligand set, whose ligands
    come first; longest-processing-time shards give every GPU about one set's work."""
    a = _args("batched_screening", n_lig=16)
    assert bench.scaling_of(a) == "weak"
    assert bench.job_ligands(a, 1) == 16 and bench.job_ligands(a, 3) == 48
    assert bench.job_ligands(_args("batched_screening"), 1) is None
    assert bench.job_ligands(_args("batched_screening"), 2) == 2048
    one = synth.workload("batched_screening", n_lig=16).ligands
    job = synth.workload("batched_screening", n_lig=bench.job_ligands(a, 3)).ligands
    assert len(job) == 48
    for x, y in zip(one, job[:16]):
        assert np.array_equal(x.xyz, y.xyz) and np.array_equal(x.type, y.type)
    cost = parallel.ligand_cost([len(l.type) for l in job], [l.n_tor for l in job])
    shards = parallel.shard_lpt(cost, 3)
    assert sorted(i for s in shards for i in s) == list(range(48))
    per = [sum(cost[i] for i in s) for s in shards]
    assert max(per) <= 1.2 * min(per)
    cfg = bench.workload_config(synth.workload("batched_screening", n_lig=48), a, 3)
    assert cfg["n_lig"] == 48 and "3 x the one-GPU set" in cfg["workload"]


def test_the_larger_workloads_split_one_fixed_set():
    for name in ("screening_stream", "blind_docking"):
        a = _args(name)
        assert bench.scaling_of(a) == "strong"
        assert bench.job_ligands(a, 4) is None
