"""ctypes binding of libtrids (include/trids.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

MAX_TYPES, MAX_GMM, MAX_ATOMS, MAX_TOR = 16, 4, 70, 20
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE = 0, -1, -2, -3, -4, -5
TERMS_VINA5, TERMS_TRIDS, TERMS_TRIDS_RES = 0, 1, 2
MAX_MDN_K, MAX_RESIDUES = 16, 8191
MODE_PERSISTENT, MODE_PER_LIGAND = 0, 1
PHASES = ("fk", "pairs", "passes", "adjoint", "update", "other")
WORK = ("clash", "hbond", "mdn_pairs", "res_scan", "res_pairs")

EXPORTS = ("trids_last_error", "trids_version", "trids_make_pocket", "trids_set_params", "trids_set_boxes",
           "trids_free_pocket", "trids_set_residues", "trids_build_maps", "trids_maps_info",
           "trids_pack_ligands", "trids_free_batch", "trids_set_mdn", "trids_batch_info", "trids_batch_query",
           "trids_pack_topology", "trids_score_grad", "trids_score_grad_noalloc", "trids_state_floats",
           "trids_sample", "trids_topk", "trids_screen_energy", "trids_sync", "trids_graph_stats", "trids_set_stream_ids")


class Params(C.Structure):
    _fields_ = [("term_set", C.c_int32), ("n_types", C.c_int32), ("w", C.c_float * 5),
                ("radius", C.c_float * MAX_TYPES), ("flags", C.c_uint8 * MAX_TYPES), ("cutoff", C.c_float),
                ("w_tor", C.c_float), ("gmm_k", C.c_int32),
                ("gmm", C.c_float * (MAX_TYPES * MAX_TYPES * MAX_GMM * 3))]


class BatchDims(C.Structure):
    _fields_ = [("n_lig", C.c_int32), ("max_atoms", C.c_int32), ("max_tor", C.c_int32),
                ("dof_stride", C.c_int32), ("state_fields", C.c_int32), ("n_intra", C.c_int64),
                ("upload_bytes", C.c_int64)]


class SampleCfg(C.Structure):
    _fields_ = [("poses", C.c_int32), ("steps", C.c_int32), ("step_begin", C.c_int32), ("step_end", C.c_int32),
                ("mc_loops", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("beta", C.c_float), ("seed", C.c_uint64), ("lig_base", C.c_int32),
                ("mode", C.c_int32), ("warps_per_block", C.c_int32), ("use_graph", C.c_int32),
                ("trace", C.c_void_p), ("trace_slot", C.c_void_p), ("n_trace", C.c_int32),
                ("pair_count", C.c_void_p), ("optimizer", C.c_int32), ("weight_decay", C.c_float),
                ("momentum", C.c_float), ("alpha", C.c_float), ("phase_cycles", C.c_void_p),
                ("work_count", C.c_void_p)]


OPTIMIZERS = {"adam": 0, "adamw": 1, "rmsprop": 2, "adagrad": 3, "sgd": 4}


class TridsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtrids error {code}: {msg}")
        self.code = code


_lib = None


def lib(build_if_missing: bool = True):
    """Load libtrids.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libtrids.so not found at {_build.LIB}; run paper_2510_24186_b300.build")
    L = C.CDLL(_build.LIB)
    vp, i32, i64, fp = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    P = C.POINTER
    L.trids_last_error.restype = C.c_char_p
    L.trids_version.restype = C.c_int
    L.trids_make_pocket.argtypes = [vp, vp, i32, P(C.c_float * 3), P(C.c_float * 3), fp, P(Params), P(vp)]
    L.trids_set_params.argtypes = [vp, P(Params), vp]
    L.trids_set_boxes.argtypes = [vp, i32, vp, vp]
    L.trids_free_pocket.argtypes = [vp]
    L.trids_pack_ligands.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, P(vp)]
    L.trids_free_batch.argtypes = [vp]
    L.trids_set_residues.argtypes = [vp, i32, vp]
    L.trids_build_maps.argtypes = [vp, fp, fp, vp]
    L.trids_maps_info.argtypes = [vp, P(C.c_float * 3), P(C.c_float), P(C.c_int32 * 3)]
    L.trids_set_mdn.argtypes = [vp, i32, i32, vp, vp]
    L.trids_batch_info.argtypes = [vp, P(BatchDims)]
    L.trids_batch_query.argtypes = [vp, vp, vp, i32, vp, i32]
    L.trids_pack_topology.argtypes = [i32, vp, vp, i32, i32, vp, vp, vp, i32, P(i32)]
    L.trids_score_grad.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.trids_score_grad_noalloc.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.trids_state_floats.argtypes = [vp, i32]
    L.trids_state_floats.restype = i64
    L.trids_sample.argtypes = [vp, vp, P(SampleCfg), vp, vp, vp, vp]
    L.trids_topk.argtypes = [vp, i32, vp, vp, i32, fp, vp, vp, vp]
    L.trids_screen_energy.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
    L.trids_sync.argtypes = [vp, i32, vp, vp, C.c_double]
    L.trids_graph_stats.argtypes = [vp, P(i64), P(i64), P(i64)]
    L.trids_set_stream_ids.argtypes = [vp, vp]
    for name in EXPORTS:
        if name not in ("trids_last_error", "trids_version", "trids_state_floats"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(code: int):
    if code != OK:
        raise TridsError(code, lib().trids_last_error().decode())
    return code
