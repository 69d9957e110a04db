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


def _case(term_set=0, n_lig=12, maps=False):
    from paper_2510_24186_b300 import api, synth
    w = synth.workload("adjoint_check", n_lig=n_lig)
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    if maps:
        pk.build_maps(0.5, 8.0)
    return w, pk, api.Batch.from_ligands(pk, w.ligands)


def _outputs(b, P, params):
    o = {"energy": torch.empty(b.n_lig, P, device="cuda"), "e_inter": torch.empty(b.n_lig, P, device="cuda"),
         "g_dof": torch.empty(b.n_lig, P, b.dof_stride, device="cuda"),
         "g_xyz": torch.empty(b.n_lig, P, b.max_atoms, 3, device="cuda")}
    if params:
        o["g_w"], o["g_r"] = torch.empty(5, device="cuda"), torch.empty(8, device="cuda")
    return o


def _call(fn, pk, b, P, dof, o, ebar=None):
    from paper_2510_24186_b300 import _lib
    rc = fn(pk.handle, b.handle, P, _p(dof), _p(o["energy"]), _p(o["e_inter"]), _p(o["g_dof"]), _p(o["g_xyz"]),
            _p(ebar), _p(o.get("g_w")), _p(o.get("g_r")), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.lib().trids_last_error().decode()


@pytest.mark.parametrize("maps", [False, True], ids=["direct", "grid_maps"])
def test_noalloc_without_parameter_gradients_on_a_fresh_batch(maps):
    """The items-only scratch layout (no parameter partials), called first on a batch that
    the regular entry point has not prepared, with and without grid maps: per-pose outputs
    equal the regular entry point's bit for bit on two calls in a row."""
    from paper_2510_24186_b300 import _lib, synth
    w, pk, b = _case(maps=maps)
    L = _lib.lib()
    rng = np.random.default_rng(4)
    for P in (33, 96):
        dof = torch.from_numpy(synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2,
                                                 w.box_center + w.box_size / 2, b.dof_stride)).cuda()
        got, ref = _outputs(b, P, False), _outputs(b, P, False)
        _call(L.trids_score_grad_noalloc, pk, b, P, dof, got)
        _call(L.trids_score_grad, pk, b, P, dof, ref)
        torch.cuda.synchronize()
        for k in got:
            assert torch.equal(got[k], ref[k]), k


def test_noalloc_allocates_no_device_memory():
    """After one warm-up call (which may load the library's module), further calls with
    other pose counts leave the device's free memory unchanged."""
    from paper_2510_24186_b300 import _lib, synth
    w, pk, b = _case()
    L = _lib.lib()
    rng = np.random.default_rng(6)
    Pmax = 160
    dof = torch.from_numpy(synth.random_dofs(rng, b.n_tor, Pmax, w.box_center - w.box_size / 2,
                                             w.box_center + w.box_size / 2, b.dof_stride)).cuda()
    o = _outputs(b, Pmax, True)
    ebar = torch.ones(b.n_lig, Pmax, device="cuda")
    _call(L.trids_score_grad_noalloc, pk, b, Pmax, dof, o, ebar)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for P in (1, 31, 64, 97, Pmax):
        _call(L.trids_score_grad_noalloc, pk, b, P, dof, o, ebar)   # first P rows of every buffer
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def _need(n_items, params):
    """Scratch bytes of n_items work items, as the header states them: 256 B + 8 B per item,
    plus (5 + 16) floats per item, 256-aligned, with parameter gradients."""
    items_end = 256 + 8 * n_items
    return (items_end + 255) // 256 * 256 + 84 * n_items if params else items_end


def test_noalloc_accepts_the_largest_request_and_rejects_one_more_item():
    from paper_2510_24186_b300 import _lib, api, synth
    w = synth.workload("single_ligand")
    sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)
    pk = api.Pocket(w.pocket.xyz, w.pocket.type, w.box_center, w.box_size, sp)
    b = api.Batch.from_ligands(pk, w.ligands)
    L = _lib.lib()
    n_max = max(n for n in range(1, 20000) if _need(n, True) <= 1 << 20)
    P = 32 * n_max                                     # one ligand: one item per 32 poses
    rng = np.random.default_rng(8)
    dof = torch.from_numpy(synth.random_dofs(rng, b.n_tor, P, w.box_center - w.box_size / 2,
                                             w.box_center + w.box_size / 2, b.dof_stride)).cuda()
    ebar = torch.from_numpy(rng.uniform(-1, 1, (1, P)).astype(np.float32)).cuda()
    got, ref = _outputs(b, P, True), _outputs(b, P, True)
    _call(L.trids_score_grad_noalloc, pk, b, P, dof, got, ebar)
    _call(L.trids_score_grad, pk, b, P, dof, ref, ebar)
    torch.cuda.synchronize()
    for k in ("energy", "e_inter", "g_dof", "g_xyz"):
        assert torch.equal(got[k], ref[k]), k
    for k in ("g_w", "g_r"):
        g, r = got[k].double().cpu().numpy(), ref[k].double().cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-3 * max(np.linalg.norm(r), 1e-3), k
    rc = L.trids_score_grad_noalloc(pk.handle, b.handle, P + 32, _p(dof), _p(got["energy"]), None, None, None,
                                    None, _p(got["g_w"]), None, None)
    assert rc == _lib.EINVAL and "static scratch" in L.trids_last_error().decode()


def _other_context_child(q):
    """In a fresh process that never touches torch's CUDA: score through the allocation-free
    entry point in the device's primary context, then in a context this process creates
    and makes current (another context, so the scratch array has another address), and
    compare each with the regular entry point."""
    try:
        import ctypes as C
        import numpy as np
        from paper_2510_24186_b300 import _lib, api, synth
        cu = C.CDLL("libcuda.so.1")
        rt = C.CDLL("/usr/local/cuda/lib64/libcudart.so.13")
        L = _lib.lib(build_if_missing=False)
        w = synth.workload("adjoint_check", n_lig=6)
        rng = np.random.default_rng(9)
        P = 40
        arrays = synth.concat_ligands(w.ligands)
        sp = api.ScoreParams(0, synth.TYPE_RADIUS, synth.TYPE_FLAGS, synth.VINA_WEIGHTS, 8.0)

        def score():
            cp = sp.to_c()
            pk, b = C.c_void_p(), C.c_void_p()
            bc = (C.c_float * 3)(*[float(x) for x in w.box_center])
            bs = (C.c_float * 3)(*[float(x) for x in w.box_size])
            xyz = np.ascontiguousarray(w.pocket.xyz, dtype=np.float32)
            ty = np.ascontiguousarray(w.pocket.type, dtype=np.int32)
            assert L.trids_make_pocket(xyz.ctypes.data, ty.ctypes.data, len(ty), C.byref(bc), C.byref(bs), 0.0,
                                       C.byref(cp), C.byref(pk)) == 0, L.trids_last_error()
            na, lx, lt, nb, bo, ro = [np.ascontiguousarray(a) for a in arrays]
            assert L.trids_pack_ligands(pk, len(na), na.ctypes.data, lx.ctypes.data, lt.ctypes.data, nb.ctypes.data,
                                        bo.ctypes.data, ro.ctypes.data, C.byref(b)) == 0, L.trids_last_error()
            d = _lib.BatchDims()
            L.trids_batch_info(b, C.byref(d))
            n_tor = np.zeros(d.n_lig, dtype=np.int32)
            L.trids_batch_query(b, n_tor.ctypes.data, None, 0, None, 0)
            dof = np.ascontiguousarray(synth.random_dofs(np.random.default_rng(9), n_tor, P,
                                                         w.box_center - w.box_size / 2,
                                                         w.box_center + w.box_size / 2, d.dof_stride),
                                       dtype=np.float32)
            out = []
            bufs = []

            def dev(nbytes):
                p = C.c_void_p()
                assert rt.cudaMalloc(C.byref(p), C.c_size_t(nbytes)) == 0
                bufs.append(p)
                return p

            ddof = dev(dof.nbytes)
            assert rt.cudaMemcpy(ddof, dof.ctypes.data, C.c_size_t(dof.nbytes), 1) == 0
            for fn in (L.trids_score_grad_noalloc, L.trids_score_grad, L.trids_score_grad_noalloc):
                e, g = dev(4 * d.n_lig * P), dev(dof.nbytes)
                assert fn(pk, b, P, ddof, e, None, g, None, None, None, None, None) == 0, L.trids_last_error()
                assert rt.cudaDeviceSynchronize() == 0
                he, hg = np.empty(d.n_lig * P, np.float32), np.empty_like(dof)
                rt.cudaMemcpy(he.ctypes.data, e, C.c_size_t(he.nbytes), 2)
                rt.cudaMemcpy(hg.ctypes.data, g, C.c_size_t(hg.nbytes), 2)
                out.append((he, hg))
            L.trids_free_batch(b)
            L.trids_free_pocket(pk)
            for p in bufs:
                rt.cudaFree(p)
            return out

        first = score()                                     # primary context
        assert cu.cuInit(0) == 0
        devh, ctx = C.c_int(), C.c_void_p()
        assert cu.cuDeviceGet(C.byref(devh), 0) == 0
        assert cu.cuCtxCreate_v4(C.byref(ctx), None, 0, devh) == 0   # current on this thread
        try:
            second = score()
        finally:
            cu.cuCtxDestroy_v2(ctx)
        ok = all(np.array_equal(a[0], r[0]) and np.array_equal(a[1], r[1])
                 for run in (first, second) for a, r in ((run[0], run[1]), (run[2], run[1])))
        same = np.array_equal(first[1][0], second[1][0])
        q.put(("ok", ok, same))
    except Exception as ex:   # report, do not hang the parent
        q.put(("error", repr(ex), False))


def test_noalloc_follows_a_change_of_context():
    """The scratch array's address is looked up again when the calling thread's context
    changes (a context of the caller's own here; a reset device gets a new context too)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_other_context_child, args=(q,))
    p.start()
    p.join(300)
    assert p.exitcode == 0
    status, ok, same = q.get(timeout=5)
    assert status == "ok", ok
    assert ok and same
