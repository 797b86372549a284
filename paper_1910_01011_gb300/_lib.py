"""ctypes binding of the C ABI in include/bem.h (argument marshalling only).

The shared library is built in-tree by build.py.  Nothing here computes any
part of the method; if the library is missing or fails to load, every call
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbem.so")

BEM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "MESH_INVALID", -3: "OUT_OF_BUDGET", -4: "NOT_CONVERGED", -5: "TIMEOUT",
          -6: "CUDA", -7: "STATE"}
PREC_FP64, PREC_FP32, PREC_BF16X3, PREC_FP64_ASSEMBLED = 0, 1, 2, 3
OP_AHAT, OP_PREC, OP_PREC_AHAT = 0, 1, 2
ERR_OUT_OF_BUDGET, ERR_NOT_CONVERGED, ERR_TIMEOUT = -3, -4, -5


class bem_z(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class bem_opts(ctypes.Structure):
    _fields_ = [("n_gauss_singular", ctypes.c_int32), ("chunk_tiles", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("n_pade", ctypes.c_int32), ("pade_theta", ctypes.c_double),
                ("r_eps", ctypes.c_double), ("eps_exponent", ctypes.c_double), ("osrc_tol", ctypes.c_double),
                ("osrc_solver", ctypes.c_int32), ("osrc_wavenumber", ctypes.c_int32),
                ("fp64_far", ctypes.c_int32)]


class bem_solve_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("precision", ctypes.c_int32), ("precondition", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int32), ("operator_mode", ctypes.c_int32), ("batch_rhs", ctypes.c_int32),
                ("flexible", ctypes.c_int32), ("prec_tol", ctypes.c_double), ("block_gmres", ctypes.c_int32),
                ("recycle", ctypes.c_int32)]


class bem_solve_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("residual", ctypes.c_double),
                ("seconds", ctypes.c_double)]


class bem_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch_rhs", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("solve", bem_solve_opts), ("join", ctypes.c_int32)]


class bem_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("excitations", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch_exc", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("p50_wait_ms", ctypes.c_double), ("requests_per_s", ctypes.c_double),
                ("excitations_per_s", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("peak_device_bytes", ctypes.c_int64), ("evictions", ctypes.c_int64), ("joined", ctypes.c_int64)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bem error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "bem_default_opts": [ctypes.POINTER(bem_opts)],
    "bem_create": [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.POINTER(bem_opts)],
    "bem_destroy": [_P],
    "bem_set_exterior": [_P, bem_z, ctypes.c_double],
    "bem_add_domain": [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, bem_z, ctypes.c_double,
                       ctypes.POINTER(ctypes.c_int32)],
    "bem_set_material": [_P, ctypes.c_int32, bem_z, ctypes.c_double],
    "bem_num_dofs": [_P, ctypes.POINTER(ctypes.c_int64)],
    "bem_interaction_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "bem_apply": [_P, ctypes.c_int, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int],
    "bem_apply_noalloc": [_P, _P, _P],
    "bem_apply_group": [_P, ctypes.c_int32, _P, _P],
    "bem_zgemm_bf16x3": [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P, _P],
    "bem_apply_block": [_P, ctypes.c_int32, ctypes.c_int32, bem_z, _P, _P, ctypes.c_int, ctypes.c_int],
    "bem_set_plane_wave": [_P, ctypes.POINTER(ctypes.c_double), bem_z],
    "bem_set_transducer": [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_double],
    "bem_set_excitations": [_P, _P, ctypes.c_int64],
    "bem_rhs": [_P, _P, ctypes.c_int],
    "bem_default_solve_opts": [ctypes.POINTER(bem_solve_opts)],
    "bem_solve": [_P, ctypes.POINTER(bem_solve_opts), ctypes.POINTER(bem_solve_report)],
    "bem_get_traces": [_P, ctypes.c_int32, ctypes.c_int64, _P, _P, ctypes.c_int],
    "bem_get_solution": [_P, ctypes.c_int64, _P, ctypes.c_int],
    "bem_solve_basis": [_P, ctypes.POINTER(bem_solve_opts), ctypes.POINTER(bem_solve_report)],
    "bem_superpose": [_P, _P, ctypes.c_int64, _P, ctypes.c_int],
    "bem_server_default_opts": [ctypes.POINTER(bem_server_opts)],
    "bem_server_create": [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(bem_server_opts)],
    "bem_server_destroy": [_P],
    "bem_server_add_scene": [_P, _P, ctypes.POINTER(ctypes.c_int32)],
    "bem_server_scene_info": [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int64)],
    "bem_server_estimate": [_P, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
    "bem_server_submit": [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
    "bem_server_poll": [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)],
    "bem_server_wait": [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int32)],
    "bem_server_result": [_P, ctypes.c_int64, _P, ctypes.POINTER(bem_solve_report), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int],
    "bem_server_error": [_P, ctypes.c_int64],
    "bem_server_get_stats": [_P, ctypes.POINTER(bem_server_stats)],
    "bem_field": [_P, ctypes.c_int64, _P, _P, ctypes.c_int64, _P, ctypes.c_int],
    "bem_last_error": [_P],
    "bem_memory_info": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "bem_estimate_solve_bytes": [_P, ctypes.c_int64, ctypes.POINTER(bem_solve_opts), ctypes.POINTER(ctypes.c_int64)],
    "bem_autotune": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)],
    "bem_profile_enable": [_P, ctypes.c_int],
    "bem_profile_read": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int],
    "bem_peak_probe": [ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)],
    "bem_quadrature_table": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int)],
}


def load(build_if_missing: bool = True):
    """Load libgbem.so (building it in-tree first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise ImportError(f"CUDA library not built: {LIB_PATH}")
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name in ("bem_last_error", "bem_server_error") else ctypes.c_int
    _lib = lib
    return lib


def check(rc, ctx=None):
    if rc != BEM_OK:
        msg = load().bem_last_error(ctx).decode() if ctx else ""
        raise BemError(rc, msg)
    return rc
