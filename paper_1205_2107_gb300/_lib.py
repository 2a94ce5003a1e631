"""ctypes binding of the C ABI in include/mrrr.h (argument marshalling only).

The shared library libmrrr.so is built in-tree by ``build.build()``.  Loading
fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_double, c_int, c_int64, c_size_t, c_void_p = (ctypes.c_double, ctypes.c_int, ctypes.c_int64,
                                               ctypes.c_size_t, ctypes.c_void_p)

STATUS = {0: "MRRR_OK", 1: "MRRR_ERR_ARG", 2: "MRRR_ERR_WORKSPACE", 3: "MRRR_ERR_NONFINITE",
          4: "MRRR_ERR_NOCONV", 5: "MRRR_ERR_QUEUE", 6: "MRRR_ERR_TIMEOUT", 7: "MRRR_ERR_CUDA",
          8: "MRRR_ERR_NOTIMPL", 9: "MRRR_ERR_MARGIN", 10: "MRRR_ERR_NOTSPD"}
(OK, ERR_ARG, ERR_WORKSPACE, ERR_NONFINITE, ERR_NOCONV, ERR_QUEUE, ERR_TIMEOUT, ERR_CUDA, ERR_NOTIMPL,
 ERR_MARGIN, ERR_NOTSPD) = range(11)

# every function include/mrrr.h declares
EXPORTS = ["mrrr_options_default", "mrrr_plan_create", "mrrr_plan_destroy", "mrrr_workspace_size",
           "mrrr_stein", "mrrr_stein_batched", "mrrr_backward", "mrrr_backward_workspace_size",
           "mrrr_get_status", "mrrr_status_string", "mrrr_version", "mrrr_set_timing", "mrrr_get_profile",
           "mrrr_eigenvalues_static", "mrrr_autotune_batched", "mrrr_probe_peak", "mrrr_slice_range",
           "mrrr_stein_slice", "mrrr_dense_workspace_size", "mrrr_sytrd", "mrrr_ormtr", "mrrr_dense_eigh",
           "mrrr_dense_status", "mrrr_gen_workspace_size", "mrrr_potrf", "mrrr_sygst", "mrrr_trsm_lt",
           "mrrr_gen_eigh", "mrrr_gen_status"]
STATIC_MAX_N = 8192  # MRRR_STATIC_MAX_N


class Options(ctypes.Structure):
    _fields_ = [("gap_tol", c_double), ("classify_rtol", c_double), ("max_depth", c_int),
                ("max_bisect_steps", c_int), ("engine_blocks_per_sm", c_int), ("threads_per_block", c_int),
                ("vec_blocks_per_sm", c_int), ("use_graph", c_int), ("max_nodes", c_int64),
                ("pool_rows", c_int64), ("cluster_rtol", c_double), ("root_perturb", c_double),
                ("width_scale", c_double), ("prebisect_rtol", c_double), ("multisection_width", c_int), ("root_side", c_int),
                ("vector_precision", c_int), ("singleton_rq", c_int),
                ("reserved_", c_int * 4)]


class Info(ctypes.Structure):
    _fields_ = [("status", c_int), ("depth", c_int), ("nodes", c_int64), ("pool_rows_used", c_int64),
                ("fallbacks", c_int64), ("twisted_solves", c_int64), ("levels", c_int64), ("diag", c_int64 * 12),
                ("sturm_counts", c_int64 * 4), ("sturm_rows", c_int64 * 4), ("warp_passes", c_int64 * 4)]

    def as_dict(self) -> dict:
        arrays = ("diag", "sturm_counts", "sturm_rows", "warp_passes")
        out = {f: getattr(self, f) for f, _ in self._fields_ if f not in arrays}
        for f in arrays:
            out[f] = list(getattr(self, f))
        return out


class Tuning(ctypes.Structure):
    _fields_ = [("engine_blocks_per_sm", c_int), ("configs", c_int), ("width_scale", c_double),
                ("best_ms", c_double), ("default_ms", c_double), ("singleton_rq", c_int), ("pad_", c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("nstages", c_int), ("pad_", c_int), ("name", (ctypes.c_char * 24) * 32),
                ("ms", c_double * 32)]

    def stages(self) -> dict:
        return {bytes(self.name[i]).split(b"\0")[0].decode(): float(self.ms[i]) for i in range(self.nstages)}


class MrrrError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(self.code, self.code)}")


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmrrr.so (optionally building it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (call build())")
        lib = ctypes.CDLL(path)
        P = c_void_p
        dp = c_void_p
        lib.mrrr_options_default.argtypes = [ctypes.POINTER(Options)]
        lib.mrrr_plan_create.argtypes = [ctypes.POINTER(c_void_p), ctypes.POINTER(Options)]
        lib.mrrr_plan_destroy.argtypes = [P]
        lib.mrrr_workspace_size.argtypes = [P, c_int, c_int64, c_int64, c_int, ctypes.POINTER(c_size_t)]
        lib.mrrr_stein.argtypes = [P, c_int, dp, dp, c_int, c_int, dp, dp, c_int64, dp, c_size_t, P]
        lib.mrrr_stein_batched.argtypes = [P, c_int, dp, dp, dp, dp, dp, dp, dp, dp, dp, c_int64, c_int64,
                                           c_int, dp, c_size_t, P]
        lib.mrrr_backward.argtypes = [P, c_int, dp, dp, dp, dp, dp, c_double, c_int, c_int64, dp, dp, dp, c_size_t, P]
        lib.mrrr_backward_workspace_size.argtypes = [P, c_int, c_int64, ctypes.POINTER(c_size_t)]
        lib.mrrr_get_status.argtypes = [P, P, ctypes.POINTER(Info)]
        lib.mrrr_status_string.argtypes = [c_int]
        lib.mrrr_status_string.restype = ctypes.c_char_p
        lib.mrrr_version.argtypes = []
        lib.mrrr_set_timing.argtypes = [P, c_int]
        lib.mrrr_get_profile.argtypes = [P, ctypes.POINTER(Profile)]
        lib.mrrr_eigenvalues_static.argtypes = [c_int, dp, dp, c_int, c_int, dp, P]
        lib.mrrr_autotune_batched.argtypes = [P, c_int, dp, dp, dp, dp, dp, dp, dp, dp, dp, c_int64, c_int64,
                                              c_int, dp, c_size_t, P, ctypes.POINTER(Tuning)]
        lib.mrrr_probe_peak.argtypes = [c_int, ctypes.POINTER(c_double)]
        lib.mrrr_slice_range.argtypes = [c_int, c_int, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.mrrr_stein_slice.argtypes = [P, c_int, dp, dp, c_int, c_int, c_int, c_int, c_int, dp, dp, c_int64, dp,
                                         c_size_t, P]
        lib.mrrr_dense_workspace_size.argtypes = [P, c_int, c_int, ctypes.POINTER(c_size_t)]
        lib.mrrr_sytrd.argtypes = [P, c_int, dp, c_int64, dp, dp, dp, dp, c_size_t, P]
        lib.mrrr_ormtr.argtypes = [P, c_int, c_int, dp, c_int64, dp, dp, c_int64, dp, c_size_t, P]
        lib.mrrr_dense_eigh.argtypes = [P, c_int, dp, c_int64, c_int, c_int, dp, dp, c_int64, dp, c_size_t, P]
        lib.mrrr_dense_status.argtypes = [dp, P]
        lib.mrrr_gen_workspace_size.argtypes = [P, c_int, c_int, ctypes.POINTER(c_size_t)]
        lib.mrrr_potrf.argtypes = [P, c_int, dp, c_int64, dp, c_size_t, P]
        lib.mrrr_sygst.argtypes = [P, c_int, dp, c_int64, dp, c_int64, dp, c_size_t, P]
        lib.mrrr_trsm_lt.argtypes = [P, c_int, c_int, dp, c_int64, dp, c_int64, dp, c_size_t, P]
        lib.mrrr_gen_eigh.argtypes = [P, c_int, dp, c_int64, dp, c_int64, c_int, c_int, dp, dp, c_int64, dp,
                                      c_size_t, P]
        lib.mrrr_gen_status.argtypes = [P, c_int, c_int, dp, P]
        for name in EXPORTS:
            if name not in ("mrrr_status_string", "mrrr_version"):
                getattr(lib, name).restype = c_int
        lib.mrrr_version.restype = c_int
        _lib = lib
        return lib


def check(rc: int, where: str) -> None:
    if rc != OK:
        raise MrrrError(rc, where)
