"""Python API over libtrids: pockets, ligand batches and the hot calls on torch CUDA tensors.

PyTorch supplies device memory and streams; every step of the path runs in libtrids'
kernels.  There is no CPU fallback: the calls raise if CUDA or the library is missing.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libtrids needs a CUDA device; there is no CPU path")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclasses.dataclass
class ScoreParams:
    """Scoring parameters (include/trids.h, trids_params)."""
    term_set: int = _lib.TERMS_VINA5
    radius: Sequence[float] = ()
    flags: Sequence[int] = ()
    w: Sequence[float] = (-0.0356, -0.00516, 0.840, -0.0351, -0.587)
    cutoff: float = 8.0
    w_tor: float = 0.01
    gmm: Optional[np.ndarray] = None     # [n_types, n_types, K, 3] (pi, mu, sigma)

    def to_c(self) -> _lib.Params:
        p = _lib.Params()
        p.term_set = int(self.term_set)
        p.n_types = len(self.radius)
        for i, r in enumerate(self.radius):
            p.radius[i] = float(r)
        for i, f in enumerate(self.flags):
            p.flags[i] = int(f)
        for i, x in enumerate(self.w):
            p.w[i] = float(x)
        p.cutoff = float(self.cutoff)
        p.w_tor = float(self.w_tor)
        if self.gmm is not None:
            g = np.asarray(self.gmm, dtype=np.float32)
            n, K = g.shape[0], g.shape[2]
            p.gmm_k = K
            full = np.zeros((_lib.MAX_TYPES, _lib.MAX_TYPES, _lib.MAX_GMM, 3), dtype=np.float32)
            full[:n, :n, :K] = g
            C.memmove(p.gmm, full.ctypes.data, full.nbytes)
        return p


class Pocket:
    """Receptor pocket atoms, translation box and scoring parameters (trids_make_pocket)."""

    def __init__(self, xyz, types, box_center, box_size, params: ScoreParams, cell: float = 0.0):
        _require_cuda()
        L = _lib.lib()
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        types = np.ascontiguousarray(types, dtype=np.int32)
        self.params = params
        self.n_atoms = len(types)
        self.box_center = np.asarray(box_center, dtype=np.float32)
        self.box_size = np.asarray(box_size, dtype=np.float32)
        h = C.c_void_p()
        bc = (C.c_float * 3)(*self.box_center.tolist())
        bs = (C.c_float * 3)(*self.box_size.tolist())
        cp = params.to_c()
        check(L.trids_make_pocket(xyz.ctypes.data, types.ctypes.data, len(types), C.byref(bc), C.byref(bs),
                                  float(cell), C.byref(cp), C.byref(h)))
        self.handle = h

    def set_params(self, params: ScoreParams, stream=None):
        cp = params.to_c()
        check(_lib.lib().trids_set_params(self.handle, C.byref(cp), _stream(stream)))
        self.params = params

    def set_boxes(self, centers, sizes):
        """Several docking boxes: pose p samples in box p mod len(centers) (trids_set_boxes)."""
        c = np.ascontiguousarray(np.atleast_2d(centers), dtype=np.float32)
        s = np.ascontiguousarray(np.atleast_2d(sizes), dtype=np.float32)
        check(_lib.lib().trids_set_boxes(self.handle, len(c), c.ctypes.data, s.ctypes.data))
        self.box_center, self.box_size = c, s

    def set_residues(self, residue):
        """Residue index of each pocket atom, for the residue-level E_MDN (trids_set_residues)."""
        r = np.ascontiguousarray(residue, dtype=np.int32)
        if len(r) != self.n_atoms:
            raise ValueError(f"need {self.n_atoms} residue indices, got {len(r)}")
        self.n_res = int(r.max()) + 1
        check(_lib.lib().trids_set_residues(self.handle, self.n_res, r.ctypes.data))

    def build_maps(self, spacing: float = 0.375, margin: float = 8.0, stream=None):
        """Grid maps of the ligand-pocket terms (trids_build_maps); spacing 0 frees them."""
        check(_lib.lib().trids_build_maps(self.handle, float(spacing), float(margin), _stream(stream)))

    def maps_info(self):
        """(origin [3], spacing, points per axis [3]) of the maps in use (zeros without maps)."""
        lo = (C.c_float * 3)()
        h = C.c_float()
        n = (C.c_int32 * 3)()
        check(_lib.lib().trids_maps_info(self.handle, C.byref(lo), C.byref(h), C.byref(n)))
        return np.array(lo[:], dtype=np.float32), float(h.value), tuple(n[:])

    def graph_stats(self) -> dict:
        """Counters of the pocket's sampler CUDA graph (trids_graph_stats): instantiations,
        in-place node updates and launches."""
        v = [C.c_int64(0) for _ in range(3)]
        check(_lib.lib().trids_graph_stats(self.handle, *[C.byref(x) for x in v]))
        return {"instantiations": v[0].value, "updates": v[1].value, "launches": v[2].value}

    def close(self):
        if getattr(self, "handle", None):
            _lib.lib().trids_free_pocket(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Packed ligands (trids_pack_ligands).  Arrays as in include/trids.h."""

    def __init__(self, pocket: Pocket, n_atoms, xyz, types, n_bonds, bonds, rotatable):
        L = _lib.lib()
        n_atoms = np.ascontiguousarray(n_atoms, dtype=np.int32)
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        types = np.ascontiguousarray(types, dtype=np.int32)
        n_bonds = np.ascontiguousarray(n_bonds, dtype=np.int32)
        bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
        rotatable = np.ascontiguousarray(rotatable, dtype=np.uint8)
        h = C.c_void_p()
        check(L.trids_pack_ligands(pocket.handle, len(n_atoms), n_atoms.ctypes.data, xyz.ctypes.data,
                                   types.ctypes.data, n_bonds.ctypes.data,
                                   bonds.ctypes.data if len(bonds) else None,
                                   rotatable.ctypes.data if len(rotatable) else None, C.byref(h)))
        self.handle = h
        self.pocket = pocket
        d = _lib.BatchDims()
        check(L.trids_batch_info(h, C.byref(d)))
        self.n_lig, self.max_atoms, self.max_tor = d.n_lig, d.max_atoms, d.max_tor
        self.dof_stride, self.state_fields, self.n_intra = d.dof_stride, d.state_fields, d.n_intra
        self.upload_bytes = d.upload_bytes
        self.n_tor = np.zeros(self.n_lig, dtype=np.int32)
        self.n_atoms = np.zeros(self.n_lig, dtype=np.int32)
        check(L.trids_batch_query(h, self.n_tor.ctypes.data, self.n_atoms.ctypes.data, 0, None, 0))

    @classmethod
    def from_ligands(cls, pocket: Pocket, ligands):
        from .synth import concat_ligands
        return cls(pocket, *concat_ligands(ligands))

    def topology(self, lig: int) -> np.ndarray:
        cap = 3 + 2 * _lib.MAX_ATOMS + 5 * _lib.MAX_TOR + _lib.MAX_ATOMS * (_lib.MAX_ATOMS - 1)
        out = np.zeros(cap, dtype=np.int32)
        check(_lib.lib().trids_batch_query(self.handle, None, None, lig, out.ctypes.data, cap))
        L, T, P = out[0], out[1], out[2]
        return out[:3 + 2 * L + 5 * T + 2 * P].copy()

    def set_stream_ids(self, ids):
        """Random-stream ids of the ligands (trids_set_stream_ids): ligand l samples as ligand
        lig_base + ids[l], e.g. its index in a larger set this batch is a shard of."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        if ids.shape != (self.n_lig,):
            raise ValueError(f"need {self.n_lig} stream ids, got shape {ids.shape}")
        check(_lib.lib().trids_set_stream_ids(self.handle, ids.ctypes.data))

    def state_floats(self, poses: int) -> int:
        return int(_lib.lib().trids_state_floats(self.handle, poses))

    def set_mdn(self, mdn: torch.Tensor, stream=None):
        """Residue-level E_MDN kernels (trids_set_mdn): a CUDA float32 tensor
        [n_atoms_total, n_res, K, 3] of (pi, mu, sigma) in input atom order."""
        if not (mdn.is_cuda and mdn.dtype == torch.float32 and mdn.dim() == 4 and mdn.shape[3] == 3):
            raise ValueError("mdn must be a CUDA float32 tensor [n_atoms_total, n_res, K, 3]")
        if mdn.shape[0] != int(self.n_atoms.sum()):
            raise ValueError(f"mdn has {mdn.shape[0]} rows, the batch has {int(self.n_atoms.sum())} atoms")
        m = mdn.contiguous()
        check(_lib.lib().trids_set_mdn(self.handle, int(m.shape[1]), int(m.shape[2]), _ptr(m), _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            _lib.lib().trids_free_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_topology(xyz, types, bonds, rotatable, n_types=8) -> np.ndarray:
    """Host-only packing of one ligand (no GPU): flat topology as in trids_batch_query."""
    L = _lib.lib()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    types = np.ascontiguousarray(types, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    rot = np.ascontiguousarray(rotatable, dtype=np.uint8)
    cap = 3 + 2 * _lib.MAX_ATOMS + 5 * _lib.MAX_TOR + _lib.MAX_ATOMS * (_lib.MAX_ATOMS - 1)
    out = np.zeros(cap, dtype=np.int32)
    n = C.c_int32()
    check(L.trids_pack_topology(len(types), xyz.ctypes.data, types.ctypes.data, n_types, len(bonds),
                                bonds.ctypes.data if len(bonds) else None,
                                rot.ctypes.data if len(rot) else None, out.ctypes.data, cap, C.byref(n)))
    return out[:n.value].copy()


def _check_dev(t: torch.Tensor, name: str, dtype=torch.float32):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor")


def score_grad(pocket: Pocket, batch: Batch, dof: torch.Tensor, grad: bool = True, xyz_grad: bool = False,
               e_bar: Optional[torch.Tensor] = None, param_grad: bool = False, stream=None) -> dict:
    """Energies and analytic gradients of poses dof [n_lig, P, dof_stride] (trids_score_grad)."""
    _require_cuda()
    _check_dev(dof, "dof")
    n_lig, P, D = dof.shape
    if n_lig != batch.n_lig or D != batch.dof_stride:
        raise ValueError("dof must have shape [n_lig, poses, dof_stride]")
    dev = dof.device
    out = {"energy": torch.empty(n_lig, P, device=dev), "e_inter": torch.empty(n_lig, P, device=dev)}
    if grad:
        out["g_dof"] = torch.empty_like(dof)
    if xyz_grad:
        out["g_xyz"] = torch.empty(n_lig, P, batch.max_atoms, 3, device=dev)
    if param_grad:
        out["g_w"] = torch.empty(5, device=dev)
        out["g_radius"] = torch.empty(len(pocket.params.radius), device=dev)
    if e_bar is not None:
        _check_dev(e_bar, "e_bar")
    check(_lib.lib().trids_score_grad(pocket.handle, batch.handle, P, _ptr(dof), _ptr(out["energy"]),
                                      _ptr(out["e_inter"]), _ptr(out.get("g_dof")), _ptr(out.get("g_xyz")),
                                      _ptr(e_bar), _ptr(out.get("g_w")), _ptr(out.get("g_radius")),
                                      _stream(stream)))
    return out


PHASES = _lib.PHASES
WORK = _lib.WORK


def sample(pocket: Pocket, batch: Batch, poses: int, steps: int, mc_loops: int = 8, lr: float = 0.1,
           beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, beta: float = 0.069, seed: int = 0,
           lig_base: int = 0, mode: int = _lib.MODE_PERSISTENT, warps_per_block: int = 0, use_graph: bool = True,
           trace_poses: Optional[Sequence[int]] = None, count_pairs: bool = False,
           dof: Optional[torch.Tensor] = None, state: Optional[torch.Tensor] = None,
           energy: Optional[torch.Tensor] = None, step_begin: int = 0, step_end: Optional[int] = None,
           stream=None, optimizer: str = "adam", weight_decay: float = 0.01, momentum: float = 0.0,
           alpha: float = 0.99) -> dict:
    """Monte-Carlo + gradient sampling of every ligand's poses (trids_sample).  optimizer:
    adam (the paper's), adamw, rmsprop, adagrad or sgd; eps is passed as given (torch's
    defaults are 1e-8, except Adagrad's 1e-10).  count_pairs runs the counting form of the
    sampler (same trajectories): out["pair_count"] gets the in-cutoff pairs evaluated,
    out["phase_cycles"] the warps' SM clock cycles per phase (names in PHASES) and
    out["work_count"] the other work counts (names in WORK)."""
    _require_cuda()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_lig, D = batch.n_lig, batch.dof_stride
    if dof is None:
        dof = torch.zeros(n_lig, poses, D, device=dev)
    if state is None:
        state = torch.zeros(batch.state_floats(poses), device=dev)
    if energy is None:
        energy = torch.empty(n_lig, poses, device=dev)
    for t, n in ((dof, "dof"), (state, "state"), (energy, "energy")):
        _check_dev(t, n)
    step_end = steps if step_end is None else step_end
    cfg = _lib.SampleCfg()
    cfg.poses, cfg.steps, cfg.step_begin, cfg.step_end, cfg.mc_loops = poses, steps, step_begin, step_end, mc_loops
    cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, cfg.beta = lr, beta1, beta2, eps, beta
    cfg.seed, cfg.lig_base, cfg.mode = seed, lig_base, mode
    cfg.warps_per_block, cfg.use_graph = warps_per_block, int(use_graph)
    cfg.optimizer = _lib.OPTIMIZERS[optimizer]
    cfg.weight_decay, cfg.momentum, cfg.alpha = weight_decay, momentum, alpha
    out = {"dof": dof, "state": state, "energy": energy}
    if trace_poses is not None:
        tp = np.asarray(trace_poses, dtype=np.int64)
        slot = torch.full((n_lig * poses,), -1, dtype=torch.int32)
        slot[torch.as_tensor(tp)] = torch.arange(len(tp), dtype=torch.int32)
        slot = slot.to(dev)
        rec = 2 * batch.max_tor + 14
        trace = torch.full(((step_end - step_begin), len(tp), rec), float("nan"), device=dev)
        cfg.trace, cfg.trace_slot, cfg.n_trace = trace.data_ptr(), slot.data_ptr(), len(tp)
        out["trace"], out["trace_slot"] = trace, slot
    if count_pairs:
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        cfg.pair_count = cnt.data_ptr()
        out["pair_count"] = cnt
        cyc = torch.zeros(len(_lib.PHASES), dtype=torch.int64, device=dev)
        cfg.phase_cycles = cyc.data_ptr()
        out["phase_cycles"] = cyc
        wk = torch.zeros(len(_lib.WORK), dtype=torch.int64, device=dev)
        cfg.work_count = wk.data_ptr()
        out["work_count"] = wk
    check(_lib.lib().trids_sample(pocket.handle, batch.handle, C.byref(cfg), _ptr(dof), _ptr(state),
                                  _ptr(energy), _stream(stream)))
    return out


def topk(batch: Batch, energy: torch.Tensor, dof: torch.Tensor, k: int, rmsd: float = 1.0, stream=None):
    """Rank + cluster + cut (trids_topk).  Returns (idx [n_lig, k] int32, energies [n_lig, k])."""
    _require_cuda()
    _check_dev(energy, "energy")
    _check_dev(dof, "dof")
    n_lig, P = energy.shape
    idx = torch.empty(n_lig, k, dtype=torch.int32, device=energy.device)
    e = torch.empty(n_lig, k, device=energy.device)
    check(_lib.lib().trids_topk(batch.handle, P, _ptr(energy), _ptr(dof), k, float(rmsd), _ptr(idx), _ptr(e),
                                _stream(stream)))
    return idx, e


def screen_energy(pocket: Pocket, batch: Batch, idx: torch.Tensor, e_inter: torch.Tensor, stream=None):
    """E_screen = E_inter / (1 + w_tor N_tor) of the kept poses (trids_screen_energy).
    idx [n_lig, k] int32 from topk(); e_inter [n_lig, poses] from score_grad().  Returns
    [n_lig, k] float32, NaN in empty slots."""
    _require_cuda()
    _check_dev(idx, "idx", torch.int32)
    _check_dev(e_inter, "e_inter")
    n_lig, k = idx.shape
    P = e_inter.shape[1]
    out = torch.empty(n_lig, k, device=idx.device)
    check(_lib.lib().trids_screen_energy(pocket.handle, batch.handle, P, k, _ptr(idx), _ptr(e_inter), _ptr(out),
                                         _stream(stream)))
    return out


def sync(batch: Batch, poses: int, state: Optional[torch.Tensor] = None, timeout_ms: float = 0.0, stream=None) -> int:
    """Wait for the stream (bounded) and check per-pose status words (trids_sync).  Returns the code."""
    return _lib.lib().trids_sync(batch.handle, poses, _ptr(state), _stream(stream), float(timeout_ms))


def screen_stream(pocket: Pocket, batches, poses: int, steps: int, k: int, rmsd: float = 1.0, seed: int = 0,
                  mc_loops: int = 8, warps_per_block: int = 0, stream=None, stats: Optional[dict] = None,
                  prepare=None, lookahead: int = 2, **sample_kw):
    """Screen an iterable of ligand batches (each a tuple of arrays as for Batch) through one
    pocket.  A host thread packs the next `lookahead` batches while the current one samples (so
    a small batch's short pass does not leave the GPU waiting for a large batch's packing), and
    each batch's sampling is queued on the stream before the previous batch's results are
    waited for (so the GPU does not idle while the host takes them); the DOF, state and energy
    buffers stay on the device and are reused in stream order.  Yields (first ligand id, top-k
    indices [n, k], top-k energies [n, k]) per batch, in order, as numpy arrays.  Ligand ids
    (the random-stream ids) run on across batches; each batch is freed on the packing thread
    once its results are back (its device block then serves a later batch).  stats (optional
    dict) receives the host-to-device and device-to-host bytes of the last batch;
    prepare(batch), if given, runs on each packed batch before it samples (e.g. Batch.set_mdn);
    sample_kw go to sample()."""
    stats = {} if stats is None else stats
    import collections
    import concurrent.futures as cf
    _require_cuda()
    if lookahead < 1:
        raise ValueError("lookahead must be >= 1")
    st = stream or torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = {"dof": torch.empty(0, device=dev), "state": torch.empty(0, device=dev),
            "energy": torch.empty(0, device=dev)}

    def view(name, n):
        if bufs[name].numel() < n:
            bufs[name] = torch.empty(int(n * 1.25) + 1024, device=dev)
        return bufs[name][:n]

    it = iter(batches)
    base = 0
    # pinned result buffers, one pair per batch in flight: batch n's copies land in slot n % 2,
    # which batch n + 2 reuses only after batch n's results have been taken
    slots = [None, None]
    # one packing thread: packs (and frees) run in submission order, so only this thread
    # touches the pocket's list of batches
    with cf.ThreadPoolExecutor(max_workers=1) as ex:
        pending = collections.deque()

        def submit_next():
            nxt = next(it, None)
            if nxt is not None:
                pending.append(ex.submit(Batch, pocket, *nxt))

        def finish(q):
            q_base, q_batch, idx_h, e_h, done = q
            done.synchronize()
            stats["h2d_bytes"] = q_batch.upload_bytes
            stats["d2h_bytes"] = idx_h.numel() * idx_h.element_size() + e_h.numel() * e_h.element_size()
            out = (q_base, idx_h.numpy().copy(), e_h.numpy().copy())
            ex.submit(q_batch.close)   # on the packing thread, after the packing already queued
            return out

        for _ in range(lookahead):
            submit_next()
        prev = None
        n = 0
        while pending:
            b = pending.popleft().result()
            if prepare is not None:
                prepare(b)
            submit_next()
            D = b.dof_stride
            with torch.cuda.stream(st):
                # allocated on the sampling stream: a buffer replaced here while the previous
                # batch still uses it goes back to the allocator in that stream's order
                dof = view("dof", b.n_lig * poses * D).view(b.n_lig, poses, D)
                state = view("state", b.state_floats(poses))
                energy = view("energy", b.n_lig * poses).view(b.n_lig, poses)
                sample(pocket, b, poses, steps, mc_loops=mc_loops, seed=seed, lig_base=base, dof=dof, state=state,
                       energy=energy, warps_per_block=warps_per_block, stream=st, **sample_kw)
                idx, e = topk(b, energy, dof, k, rmsd, stream=st)
                s = n & 1
                if slots[s] is None or slots[s][0].shape != idx.shape:
                    slots[s] = (torch.empty(idx.shape, dtype=idx.dtype, pin_memory=True),
                                torch.empty(e.shape, dtype=e.dtype, pin_memory=True))
                idx_h, e_h = slots[s]
                idx_h.copy_(idx, non_blocking=True)
                e_h.copy_(e, non_blocking=True)
                done = torch.cuda.Event()
                done.record(st)
            cur = (base, b, idx_h, e_h, done)
            base += b.n_lig
            n += 1
            if prev is not None:
                yield finish(prev)       # the previous batch, while this one samples
            prev = cur
        if prev is not None:
            yield finish(prev)


def screen_sharded(pocket: Pocket, ligands, poses: int, steps: int, k: int, rmsd: float = 1.0, seed: int = 0,
                   mc_loops: int = 8, rank: Optional[int] = None, world: Optional[int] = None, gather: bool = True,
                   stream=None, **sample_kw):
    """Screen a ligand set split over GPUs, one process per GPU (torch.distributed supplies
    rank and world size unless given).  The set is split by longest-processing-time on each
    ligand's cost; this rank packs its shard, gives every ligand its global index as its
    random-stream id (so the results do not depend on the split), samples, ranks, and copies
    the top-k back; rank 0 then gathers every shard's top-k on the host in global ligand order
    (ids [n], pose indices [n, k], energies [n, k]; other ranks get None).  gather=False
    returns each rank's own shard instead.  ligands: objects with xyz, type, bonds, rotatable
    (as synth.Ligand)."""
    from . import parallel
    from .synth import concat_ligands
    _require_cuda()
    n_atoms = [len(l.type) for l in ligands]
    n_tor = [int(np.asarray(l.rotatable).sum()) for l in ligands]
    st = stream or torch.cuda.current_stream()

    def run_shard(ids):
        b = Batch(pocket, *concat_ligands([ligands[i] for i in ids]))
        try:
            b.set_stream_ids(ids)
            with torch.cuda.stream(st):
                out = sample(pocket, b, poses, steps, mc_loops=mc_loops, seed=seed, lig_base=0, stream=st,
                             **sample_kw)
                idx, e = topk(b, out["energy"], out["dof"], k, rmsd, stream=st)
            st.synchronize()
            return idx.cpu().numpy(), e.cpu().numpy()
        finally:
            b.close()

    return parallel.screen_shards(n_atoms, n_tor, run_shard, rank, world, gather)
