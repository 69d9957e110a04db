"""The culling lists of the library's pocket grids hold every pair the kernels must see.

Builds tests/grid_reach_check.cpp against the library's host grid builders (pack.cpp) with
g++ and runs it on the batched-screening pocket with seeded residues: for seeded points
(a quarter of them on cell corners and faces) the list prefix of the point's reach level,
chosen with the kernels' float arithmetic, must contain every pocket atom within the cutoff
(candidate lists), within the near cutoff (near lists of the atom-pair E_MDN) and every
residue with an atom within 5 A (residue lists), and each level table must be monotone and
end at the whole list.  No GPU.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_2510_24186_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_24186_b300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("grid")
    exe = str(d / "grid_reach_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           "-I", CUDA_INC, os.path.join(ROOT, "tests", "grid_reach_check.cpp"),
                           os.path.join(CSRC, "pack.cpp"), "-o", exe])
    w = synth.workload("batched_screening")
    xyz = w.pocket.xyz.astype(np.float32)
    res = np.asarray(synth.gen_residues(np.random.default_rng(7), w.pocket.xyz), dtype=np.int32)
    inp = str(d / "pocket.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("i", len(xyz)) + xyz.tobytes() + res.tobytes())
    return exe, inp


@pytest.mark.parametrize("cutoff,cell", [(8.0, 0.5), (10.0, 1.0)])
def test_reach_level_prefixes_hold_every_pair_in_range(checker, cutoff, cell):
    exe, inp = checker
    r = subprocess.run([exe, inp, str(cutoff), "5.0", str(cell), "3000"], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    ok, pts, used, whole = r.stdout.split()
    assert ok == "ok" and int(pts) > 1000
    assert float(used) <= float(whole)
