"""The C-ABI driven from a C program on the GPU: tests/capi_sample.c builds the pocket and
the batch, allocates device buffers with the CUDA runtime, samples and ranks; its energies,
DOFs and top-k indices must equal the Python path's bit for bit (the same kernels and launch
shapes on the same inputs)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2510_24186_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_c_program_matches_python_path_bit_for_bit(tmp_path):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    if shutil.which("gcc") is None:
        pytest.skip("gcc not installed")
    from paper_2510_24186_b300 import api, build
    lib = build.build()
    exe = tmp_path / "capi_sample"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "capi_sample.c"),
                           "-L" + os.path.dirname(lib), "-ltrids", "-L" + os.path.join(CUDA, "lib64"), "-lcudart",
                           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + os.path.join(CUDA, "lib64"),
                           "-o", str(exe)])
    w = synth.workload("adjoint_check", n_lig=6)
    P, S, Lmc, k, seed = 32, 12, 3, 4, 77
    n_atoms, xyz, types, n_bonds, bonds, rot = synth.concat_ligands(w.ligands)
    radius = np.asarray(synth.TYPE_RADIUS, dtype=np.float32)
    flags = np.asarray(synth.TYPE_FLAGS, dtype=np.uint8)
    blob = b"".join([
        np.array([len(w.pocket.type), len(n_atoms), int(n_atoms.sum()), int(n_bonds.sum()), P, S, Lmc, k],
                 dtype=np.int32).tobytes(),
        np.array([seed], dtype=np.uint64).tobytes(),
        np.asarray(w.box_center, dtype=np.float32).tobytes(), np.asarray(w.box_size, dtype=np.float32).tobytes(),
        np.asarray(w.pocket.xyz, dtype=np.float32).tobytes(), np.asarray(w.pocket.type, dtype=np.int32).tobytes(),
        np.array([len(radius)], dtype=np.int32).tobytes(), radius.tobytes(), flags.tobytes(),
        np.asarray(synth.VINA_WEIGHTS, dtype=np.float32).tobytes(), np.array([w.cutoff], dtype=np.float32).tobytes(),
        n_atoms.tobytes(), xyz.tobytes(), types.tobytes(), n_bonds.tobytes(), bonds.tobytes(), rot.tobytes()])
    (tmp_path / "in.bin").write_bytes(blob)
    run = subprocess.run([str(exe), str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], capture_output=True,
                         text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    out = np.frombuffer((tmp_path / "out.bin").read_bytes(), dtype=np.uint8)
    stride = int(out[:4].view(np.int32)[0])
    n_lig = len(n_atoms)
    o = 4
    e_c = out[o:o + 4 * n_lig * P].view(np.float32).reshape(n_lig, P)
    o += 4 * n_lig * P
    dof_c = out[o:o + 4 * n_lig * P * stride].view(np.float32).reshape(n_lig, P, stride)
    o += 4 * n_lig * P * stride
    idx_c = out[o:o + 4 * n_lig * k].view(np.int32).reshape(n_lig, k)

    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, w.cutoff)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    assert b.dof_stride == stride
    r = api.sample(pk, b, P, S, mc_loops=Lmc, seed=seed)
    idx, _ = api.topk(b, r["energy"], r["dof"], k, 1.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(r["energy"].cpu().numpy().view(np.uint32), e_c.view(np.uint32))
    np.testing.assert_array_equal(r["dof"].cpu().numpy().view(np.uint32), dof_c.view(np.uint32))
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_c)
