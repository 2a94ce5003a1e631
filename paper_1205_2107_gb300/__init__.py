"""GB300-native MRRR eigensolver for real symmetric tridiagonal matrices (FP64).

The compute path is the CUDA shared library built from ``csrc/`` (C ABI in
``include/mrrr.h``); this package only marshals arguments to it.  Submodules
load lazily so that ``paper_1205_2107_gb300.inputs`` imports without torch.
"""
import importlib

__all__ = ["Plan", "BatchLayout", "eigh_tridiagonal", "eigh_tridiagonal_batched", "build", "inputs",
           "EighTridiagonal", "eigh_tridiagonal_autograd", "EighTridiagonalBatched",
           "eigh_tridiagonal_batched_autograd", "eigh_tridiagonal_backward", "autotune_batched"]

_LAZY = {"Plan": "api", "BatchLayout": "api", "eigh_tridiagonal": "api", "eigh_tridiagonal_batched": "api",
         "default_plan": "api", "eigh_tridiagonal_backward": "api", "autotune_batched": "api", "EighTridiagonal": "autograd",
         "eigh_tridiagonal_autograd": "autograd", "EighTridiagonalBatched": "autograd",
         "eigh_tridiagonal_batched_autograd": "autograd"}


def __getattr__(name):
    if name in _LAZY:
        mod = importlib.import_module(f".{_LAZY[name]}", __name__)
        return getattr(mod, name)
    if name in ("build", "inputs", "api", "autograd"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
