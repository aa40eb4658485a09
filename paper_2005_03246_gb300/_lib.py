"""ctypes loader for libfastecdf.so (the C ABI of include/fastecdf.h).

Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfastecdf.so")

FK_F32, FK_F64 = 0, 1
FK_PATH_MIXED, FK_PATH_FP64 = 0, 1
FK_LOO = 1
FK_BATCH_ECDF, FK_BATCH_KDE = 1, 2


class Dataset(ctypes.Structure):
    """fk_dataset of include/fastecdf.h."""
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("N", ctypes.c_int64), ("d", ctypes.c_int),
                ("reserved", ctypes.c_int)]

class BatchConfig(ctypes.Structure):
    """fk_batch_config of include/fastecdf.h."""
    _fields_ = [("streams", ctypes.c_int), ("coarsen", ctypes.c_int), ("kernel_tile", ctypes.c_int),
                ("count_tile", ctypes.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


STATUS = {0: "FK_OK", -1: "FK_ERR_INVALID_ARG", -2: "FK_ERR_UNSUPPORTED", -3: "FK_ERR_WORKSPACE",
          -4: "FK_ERR_NONFINITE", -5: "FK_ERR_CUDA", -6: "FK_ERR_TIMEOUT"}

# Every symbol the header declares, with its ctypes signature.
P, I64, I, U, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t
SIGNATURES = {
    "fk_last_error": (ctypes.c_char_p, []),
    "fk_version": (ctypes.c_char_p, []),
    "fk_device_status": (I, [P]),
    "fk_debug_lookback_timeout": (I, [I64, P]),
    "fk_ecdf_grid_workspace": (SZ, [I64, I, P, I, I]),
    "fk_ecdf_grid": (I, [P, I, I64, I, P, P, P, P, P, I, P, SZ, P]),
    "fk_kde_grid_workspace": (SZ, [I64, I, P, I]),
    "fk_kde_grid": (I, [P, I, I64, I, P, P, P, P, P, I, P, SZ, P]),
    "fk_grid_interp_workspace": (SZ, []),
    "fk_grid_interp": (I, [P, I, P, P, P, I, I64, P, P, SZ, P]),
    "fk_ecdf_points_workspace": (SZ, [I64, I, I64, I, I, I]),
    "fk_ecdf_points": (I, [P, I, I64, I, P, P, I64, P, P, I, P, SZ, P]),
    "fk_esf_points": (I, [P, I, I64, I, P, P, I64, P, I, P, SZ, P]),
    "fk_kde_laplace_workspace": (SZ, [I64, I, I64, I, I, I]),
    "fk_kde_laplace": (I, [P, I, I64, I, P, P, I64, P, U, P, P, I, P, SZ, P]),
    "fk_kreg_laplace_workspace": (SZ, [I64, I, I64, I, I]),
    "fk_kreg_laplace": (I, [P, I, I64, I, P, P, I64, P, U, P, I, P, SZ, P]),
    "fk_kde_laplace_backward_workspace": (SZ, [I64, I, I64, I, I]),
    "fk_kde_laplace_backward": (I, [P, I, I64, I, P, P, I64, P, U, P, P, P, P, I, P, SZ, P]),
    "fk_loo_laplace_workspace": (SZ, [I64, I, I]),
    "fk_loo_laplace": (I, [P, I, I64, I, P, P, P, P, I, P, SZ, P]),
    "fk_batched_workspace": (SZ, [P, I, I, U, I]),
    "fk_batched": (I, [P, I, I, U, ctypes.c_double, P, P, I, P, SZ, P]),
    "fk_batched_config_default": (None, [P]),
    "fk_batched_workspace_ex": (SZ, [P, I, I, U, I, P]),
    "fk_batched_ex": (I, [P, I, I, U, ctypes.c_double, P, P, I, P, P, SZ, P]),
    "fk_batched_autotune_workspace": (SZ, [P, I, I, U, I]),
    "fk_batched_autotune": (I, [P, I, I, U, ctypes.c_double, P, P, I, P, SZ, P, P, P]),
    "fk_kde_uniform_workspace": (SZ, [I64, I, I64, I, I, I]),
    "fk_kde_uniform": (I, [P, I, I64, I, P, P, I64, P, U, P, I, P, SZ, P]),
    "fk_kde_matern32_workspace": (SZ, [I64, I, I64, I, I, I]),
    "fk_kde_matern32": (I, [P, I, I64, I, P, P, I64, P, U, P, I, P, SZ, P]),
    "fk_kde_laplace_hmatrix_workspace": (SZ, [I64, I, I64, I, I]),
    "fk_kde_laplace_hmatrix": (I, [P, I, I64, I, P, P, I64, P, U, P, I, P, SZ, P]),
    "fk_hmatrix_factor": (I, [P, I, P, P]),
    "fk_kreg_loclin_laplace_workspace": (SZ, [I64, I, I64, I, I]),
    "fk_kreg_loclin_laplace": (I, [P, I, I64, I, P, P, I64, P, U, P, I, P, SZ, P]),
    "fk_ecdf_grid_counts_noalloc": (I, [P, I, I64, I, P, P, P, P, P]),
    "fk_release_cached_memory": (I, []),
    "fk_kernel_launches": (ctypes.c_uint64, []),
    "fk_profile_enable": (None, [I]),
    "fk_profile_reset": (None, []),
    "fk_profile_read": (I, [I, P, P, P]),
    "fk_profile_busy": (I, [I, P]),
    "fk_profile_read_bytes": (I, [I, P]),
}

PROFILE_FAMILIES = {"merge_sweep": 0, "merge_totals": 1, "merge_plain": 2, "grid_pass": 3,
                    "grid_hist": 4, "radix": 5, "gather": 6, "local_sweep": 7, "kernel_local": 8}

_lib = None


class FastEcdfError(RuntimeError):
    pass


def load():
    """Load the library (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int, what: str):
    if rc != 0:
        msg = load().fk_last_error().decode(errors="replace")
        raise FastEcdfError("%s failed: %s (%s)" % (what, STATUS.get(rc, rc), msg))
