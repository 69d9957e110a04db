"""The allocation-free scoring entry point against the regular one, through the C-ABI.

trids_score_grad_noalloc serves callers that cannot let a library allocate device
memory during their work (own memory pools or fixed arenas, latency-bound loops); its
scratch is a fixed array inside the library.  This file is collected last so that a
stop-at-first-failure run has already run everything else; it also passes on its own.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("term_set", [0, 1])
def test_noalloc_matches_regular_entry_point_twice(term_set):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2510_24186_b300 import _lib, api, synth
    w = synth.workload("adjoint_check", n_lig=24)
    rng = np.random.default_rng(17)
    if term_set == 0:
        sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    else:
        g = np.zeros((8, 8, 2, 3))
        g[..., 0] = rng.uniform(0.2, 1.0, (8, 8, 2))
        g[..., 1] = rng.uniform(2.0, 4.5, (8, 8, 2))
        g[..., 2] = rng.uniform(0.4, 1.2, (8, 8, 2))
        sp = api.ScoreParams(1, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.TRIDS_WEIGHTS, 10.0, gmm=g)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    L = _lib.lib()
    stream = torch.cuda.current_stream()
    for call in range(2):
        P = 45 if call == 0 else 70
        dof = torch.from_numpy(synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2,
                                                 w.box_center + w.box_size / 2, b.dof_stride)).cuda()
        ebar = torch.from_numpy(rng.uniform(-1, 1, (b.n_lig, P)).astype(np.float32)).cuda()
        outs = []
        for fn in (L.trids_score_grad, L.trids_score_grad_noalloc):
            o = {"energy": torch.empty(b.n_lig, P, device="cuda"), "e_inter": torch.empty(b.n_lig, P, device="cuda"),
                 "g_dof": torch.empty_like(dof), "g_xyz": torch.empty(b.n_lig, P, b.max_atoms, 3, device="cuda"),
                 "g_w": torch.empty(5, device="cuda"), "g_r": torch.empty(8, device="cuda")}
            rc = fn(pk.handle, b.handle, P, _p(dof), _p(o["energy"]), _p(o["e_inter"]), _p(o["g_dof"]),
                    _p(o["g_xyz"]), _p(ebar), _p(o["g_w"]), _p(o["g_r"]), C.c_void_p(stream.cuda_stream))
            assert rc == 0, L.trids_last_error().decode()
            torch.cuda.synchronize()
            outs.append({k: v.cpu().numpy().astype(np.float64) for k, v in o.items()})
        ref, got = outs
        for k in ("energy", "e_inter", "g_dof", "g_xyz"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)   # same per-pose arithmetic
        for k in ("g_w", "g_r"):                                        # sums in another order
            num = np.linalg.norm(got[k] - ref[k])
            assert num <= 1e-3 * max(np.linalg.norm(ref[k]), 1e-3), (k, got[k], ref[k])


def test_noalloc_rejects_requests_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2510_24186_b300 import _lib, api, synth
    w = synth.workload("single_ligand")
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    P = 32 * 20000                         # 20,000 items x 92 bytes > 1 MiB
    L = _lib.lib()
    dof = torch.zeros(1, 1, b.dof_stride, device="cuda")
    e = torch.empty(1, device="cuda")
    gw = torch.empty(5, device="cuda")
    rc = L.trids_score_grad_noalloc(pk.handle, b.handle, P, _p(dof), _p(e), None, None, None, None, _p(gw), None,
                                    None)
    assert rc == _lib.EINVAL
    assert "static scratch" in L.trids_last_error().decode()
