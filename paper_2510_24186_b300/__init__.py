"""B300-native gradient-guided ligand pose sampling (TRIDS hot path, arXiv 2510.24186).

Layout: ``csrc/`` holds the CUDA kernels and the C-ABI (declared in include/trids.h),
``_lib`` the ctypes binding, ``api`` the torch-facing calls, ``autograd`` the
torch.autograd.Function, ``autotune`` the launch-shape tuner and ``synth`` the seeded
synthetic inputs.  Importing the package loads nothing; the library is loaded on the
first call that needs it.
"""
import importlib

__all__ = ["api", "autograd", "autotune", "synth", "ScoreParams", "Pocket", "Batch", "score_grad", "sample",
           "topk", "sync", "pack_topology", "TridsScore"]

_API = {"ScoreParams", "Pocket", "Batch", "score_grad", "sample", "topk", "sync", "pack_topology"}


def __getattr__(name):
    if name in ("api", "autograd", "autotune", "synth", "build", "parallel"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in _API:
        return getattr(importlib.import_module(f"{__name__}.api"), name)
    if name == "TridsScore":
        return importlib.import_module(f"{__name__}.autograd").TridsScore
    raise AttributeError(name)
