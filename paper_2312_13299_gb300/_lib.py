"""ctypes declarations of the C ABI in ``include/plas.h``.

Loading fails loudly (RuntimeError) when the CUDA library has not been built:
there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int, c_uint32, c_uint64, c_ll, c_double, c_float, c_size_t, c_void_p = (
    ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_longlong, ctypes.c_double,
    ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p)

PLAS_OK = 0
PLAS_ERR_INVALID_ARG = -1
PLAS_ERR_OOM = -2
PLAS_ERR_CUDA = -3
PLAS_ERR_TIMEOUT = -4
PLAS_ERR_NONFINITE = -5
PLAS_ERR_BUDGET = -6
PLAS_ERR_INTERNAL = -7
PLAS_ERR_NOT_PERMUTATION = -8

K_PREP, K_BLUR_ROWS, K_BLUR_COLS, K_GROUPS, K_ASSIGN, K_GATHER, K_COUNT = range(7)
KERNEL_NAMES = ["prep", "blur_rows", "blur_cols", "groups", "assign", "gather"]


class plas_schedule(ctypes.Structure):
    _fields_ = [("phi0", c_double), ("shrink", c_double), ("phi_min", c_double),
                ("tol", c_double), ("sigma_ratio", c_double), ("min_block", c_int),
                ("shuffle_init", c_int), ("normalize", c_int), ("iters_per_poll", c_int),
                ("max_iters", c_ll), ("profile", c_int), ("graphs", c_int), ("target_mode", c_int),
                ("persistent", c_int), ("whole_blocks", c_int), ("checked", c_int),
                ("trace_S", c_void_p), ("trace_level", c_void_p), ("trace_cap", c_ll)]


class plas_state(ctypes.Structure):
    _fields_ = [("it", c_ll), ("epoch", c_ll), ("redraws", c_ll), ("level", c_int),
                ("stall", c_int), ("has_prev", c_int), ("done", c_int), ("d_prev", c_double),
                ("d_last", c_double), ("scale_exp", c_int), ("status", c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class plas_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", c_ll), ("ms", c_double), ("bytes", c_double), ("flops", c_double)]


class plas_stats(ctypes.Structure):
    _fields_ = [("iterations", c_ll), ("redraws", c_ll), ("grouped_cells", c_ll),
                ("levels", c_int), ("status", c_int), ("final_l2_to_target", c_double),
                ("neighbour_l2", c_double), ("ms_total", c_double), ("launches", c_ll),
                ("kernel", plas_kernel_stat * K_COUNT), ("graph_launches", c_ll),
                ("graph_captures", c_ll)]


class plas_job(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("H", c_int), ("W", c_int), ("carried", c_void_p),
                ("C", c_int), ("seed", c_uint64), ("perm_out", c_void_p),
                ("carried_out", c_void_p), ("state_out", ctypes.POINTER(plas_state))]


TUNE_MAX_RADII = 16
TUNE_ASSIGN_CANDIDATES = 4


class plas_tuning(ctypes.Structure):
    _fields_ = [("fir_small_below", c_int), ("fir_medium_below", c_int),
                ("assign_ctas_per_sm", c_int), ("n_radii", c_int),
                ("radius", c_int * TUNE_MAX_RADII), ("fir_small_us", c_float * TUNE_MAX_RADII),
                ("fir_medium_us", c_float * TUNE_MAX_RADII),
                ("fir_large_us", c_float * TUNE_MAX_RADII),
                ("assign_per_sm", c_int * TUNE_ASSIGN_CANDIDATES),
                ("assign_us", c_float * TUNE_ASSIGN_CANDIDATES), ("large_tma", c_int),
                ("fir_large_ring_us", c_float * TUNE_MAX_RADII),
                ("fir_large_tma_us", c_float * TUNE_MAX_RADII), ("small_fused", c_int)]


P = ctypes.POINTER

# name -> (restype, argtypes); every symbol declared in include/plas.h
SIGNATURES = {
    "plas_default_schedule": (c_int, [P(plas_schedule)]),
    "plas_num_levels": (c_int, [c_int, c_int, P(plas_schedule)]),
    "plas_sort_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "plas_sort_workspace_bytes_ex": (c_size_t, [c_int, c_int, c_int, P(plas_schedule)]),
    "plas_sort": (c_int, [c_void_p, c_int, c_int, c_int, P(c_float), c_void_p, c_int, c_uint64,
                          P(plas_schedule), c_void_p, P(plas_state), c_void_p, c_void_p,
                          c_void_p, c_void_p, c_size_t, P(plas_stats), c_void_p]),
    "plas_select_rows": (c_int, [c_void_p, c_ll, c_int, c_void_p, c_ll, c_void_p, c_void_p]),
    "plas_gather_rows": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "plas_target": (c_int, [c_void_p, c_int, c_int, c_int, P(c_float), c_int, c_void_p,
                            c_double, c_double, c_void_p, c_void_p]),
    "plas_target_box": (c_int, [c_void_p, c_int, c_int, c_int, P(c_float), c_int, c_void_p,
                                c_double, c_void_p, c_void_p]),
    "plas_group_permutation": (c_int, [c_uint64, c_uint32, c_uint64, c_uint32, c_void_p,
                                       c_void_p]),
    "plas_philox": (c_int, [c_void_p, c_uint32, c_uint32, c_int, c_void_p, c_void_p]),
    "plas_grid_metrics": (c_int, [c_void_p, c_int, c_int, c_int, c_double, P(c_double),
                                  c_void_p]),
    "plas_check_permutation": (c_int, [c_void_p, c_int, P(c_int), c_void_p]),
    "plas_smooth_loss_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "plas_smooth_loss_fwd": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_int, c_void_p,
                                     c_void_p, c_void_p, c_size_t, c_void_p]),
    "plas_smooth_loss_bwd": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_int, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "plas_smooth_loss_fwd_ex": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_int, c_void_p,
                                        c_float, c_void_p, c_void_p, c_size_t, c_void_p]),
    "plas_smooth_loss_bwd_ex": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_int, c_void_p,
                                        c_float, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "plas_smooth_loss_fwd_noalloc": (c_int, [c_void_p, c_int, c_int, c_int, c_float, c_int,
                                             c_void_p, c_void_p, c_void_p]),
    "plas_activate_3dgs": (c_int, [c_void_p, c_ll, c_int, c_void_p, c_void_p]),
    "plas_grid_select_workspace_bytes": (c_size_t, [c_ll]),
    "plas_grid_select": (c_int, [c_void_p, c_ll, c_int, c_void_p, P(c_int), c_void_p, c_size_t,
                                 c_void_p]),
    "plas_quantize": (c_int, [c_void_p, c_ll, c_int, P(c_float), P(c_float), P(c_int), c_void_p,
                              c_void_p]),
    "plas_dequantize": (c_int, [c_void_p, c_ll, c_int, P(c_float), P(c_float), P(c_int),
                                c_void_p, c_void_p]),
    "plas_batch_workspace_bytes": (c_size_t, [c_int, P(plas_job), c_int]),
    "plas_batch_sort": (c_int, [c_int, P(plas_job), c_int, P(c_float), P(plas_schedule),
                                c_void_p, c_size_t, c_void_p]),
    "plas_autotune": (c_int, [c_int, c_int, c_int, c_void_p, P(plas_tuning)]),
    "plas_set_tuning": (c_int, [c_int, c_int, c_int, P(plas_tuning)]),
    "plas_get_tuning": (c_int, [c_int, c_int, c_int, P(plas_tuning)]),
    "plas_server_create": (c_int, [c_int, P(c_float), P(plas_schedule), c_size_t, c_void_p,
                                   P(c_void_p)]),
    "plas_server_set_policy": (c_int, [c_void_p, c_int]),
    "plas_server_submit": (c_int, [c_void_p, P(plas_job), P(c_ll)]),
    "plas_server_step": (c_int, [c_void_p, c_int, P(c_ll), c_int, P(c_int)]),
    "plas_server_status": (c_int, [c_void_p, P(c_int), P(c_int), P(c_size_t)]),
    "plas_server_cancel": (c_int, [c_void_p, c_ll]),
    "plas_server_destroy": (c_int, [c_void_p]),
    "plas_status_string": (ctypes.c_char_p, [c_int]),
    "plas_last_error": (ctypes.c_char_p, []),
    "plas_version": (c_int, []),
    "plas_debug_inject": (c_int, [c_int, c_ll]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libplas.so (the CUDA path).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(
                f"PLAS CUDA library not found at {path}; build it first "
                "(python -c 'import __graft_entry__ as g; g.build()').  There is no CPU fallback.")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class PlasError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.plas_last_error().decode() or lib.plas_status_string(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != PLAS_OK:
        raise PlasError(code, where)
