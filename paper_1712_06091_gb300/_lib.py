"""ctypes declarations of the C ABI in include/adr.h (argument marshalling only).

Loading fails loudly when libadr.so has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadr.so")

ADR_OK = 0
ADR_ERR_ARG = -1
ADR_ERR_CUDA = -2
ADR_ERR_OOM = -3
ADR_ERR_NOT_CONVERGED = -4
ADR_ERR_NAN = -5
ADR_ERR_STATE = -6

ADR_F64 = 0
ADR_F32 = 1
SCHEMES = {"2up": 0, "1up": 1, "cen": 2, "prec": 3}
CYCLES = {"V": 0, "K": 1}
RELAX = {"jacobi": 0, "mr": 1}
COARSE_SOLVERS = {"auto": 0, "kernels": 1, "cta": 2, "cluster": 3, "grid": 4}
MAX_LEVELS = 8
TRAVELTIME_STATIC_MAX_SWEEPS = 8192

# The exported entry points, in the order include/adr.h declares them.
EXPORTS = (
    "adr_params_default", "adr_operator_create", "adr_operator_create_tau", "adr_operator_update", "adr_batch_create",
    "adr_batch_create_grids", "adr_batch_update",
    "adr_operator_destroy", "adr_operator_info",
    "adr_coefficients", "adr_apply", "adr_level_stencil", "adr_vcycle", "adr_point_source_rhs",
    "adr_solve", "adr_solve_two_stage", "adr_reconstruct", "adr_solve_host", "adr_adjoint_solve", "adr_apply_adjoint", "adr_vcycle_adjoint",
    "adr_receivers", "adr_kappa_gradient", "adr_traveltime", "adr_traveltime_order", "adr_traveltime_static",
    "adr_profile_kernel",
    "adr_profile_read",
    "adr_kernel_launches", "adr_last_error", "adr_version",
)
PROFILE_CLASSES = {"none": 0, "level1_relax": 1, "fine_relax": 2, "outer_apply": 3, "coarsest": 4, "cycle": 5}


class Params(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("cycle", ctypes.c_int),
        ("relax", ctypes.c_int),
        ("pre_sweeps", ctypes.c_int * MAX_LEVELS),
        ("post_sweeps", ctypes.c_int * MAX_LEVELS),
        ("jacobi_weight", ctypes.c_double * MAX_LEVELS),
        ("coarse_iterations", ctypes.c_int),
        ("kcycle_iterations", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("precond_precision", ctypes.c_int),
        ("near_source", ctypes.c_int),
        ("reorth_eta", ctypes.c_double),
        ("adjoint", ctypes.c_int),
        ("relax_blocks", ctypes.c_int),
        ("coarse_solver", ctypes.c_int),
        ("tma", ctypes.c_int),
        ("shift", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("prec_scheme", ctypes.c_int),
        ("rescale", ctypes.c_int),
        ("kcycle_threshold", ctypes.c_double),
        ("outer_df", ctypes.c_int),
    ]


class LevelInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nodes", ctypes.c_int64), ("stencil_points", ctypes.c_int)]


class OpInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("levels", ctypes.c_int), ("level", LevelInfo * MAX_LEVELS),
                ("arena_bytes", ctypes.c_int64), ("problems", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_estimate", ctypes.c_double), ("status", ctypes.c_int)]


class ADRError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"libadr error {code}: {message}")
        self.code = code


_lib = None


def load():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(python -m paper_1712_06091_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    sig = {
        "adr_params_default": [ctypes.POINTER(Params)],
        "adr_operator_create": [i, ip, dp, ip, d, vp, vp, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)],
        "adr_operator_create_tau": [i, ip, dp, ip, d, vp, vp, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)],
        "adr_operator_update": [vp, ip, d, vp, vp, vp],
        "adr_batch_create": [i, ip, dp, i, ip, dp, vp, vp, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)],
        "adr_batch_create_grids": [i, i, ip, dp, ip, dp, vp, vp, vp, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)],
        "adr_batch_update": [vp, ip, dp, vp, vp, vp],
        "adr_operator_destroy": [vp],
        "adr_operator_info": [vp, ctypes.POINTER(OpInfo)],
        "adr_coefficients": [vp, vp],
        "adr_apply": [vp, i, i, vp, vp],
        "adr_level_stencil": [vp, i, vp],
        "adr_vcycle": [vp, vp, vp],
        "adr_point_source_rhs": [vp, vp],
        "adr_solve": [vp, vp, vp, i, d, i, ctypes.POINTER(SolveInfo)],
        "adr_solve_two_stage": [vp, vp, vp, vp, d, i, d, i, ctypes.POINTER(SolveInfo)],
        "adr_reconstruct": [vp, vp, vp],
        "adr_solve_host": [i, ip, dp, ip, d, vp, vp, vp, ctypes.POINTER(Params), d, i, vp, vp, vp,
                           ctypes.POINTER(SolveInfo)],
        "adr_adjoint_solve": [vp, vp, vp, i, d, i, ctypes.POINTER(SolveInfo)],
        "adr_apply_adjoint": [vp, vp, vp],
        "adr_vcycle_adjoint": [vp, vp, vp],
        "adr_receivers": [vp, i, vp, vp, vp, vp, vp, dp],
        "adr_kappa_gradient": [vp, vp, vp, vp, vp, vp],
        "adr_traveltime": [i, ip, dp, ip, vp, vp, i, vp, ip],
        "adr_traveltime_order": [i, ip, dp, ip, vp, vp, i, i, vp, ip],
        "adr_traveltime_static": [i, ip, dp, ip, vp, vp, i, vp, ip],
        "adr_profile_kernel": [vp, i],
        "adr_profile_read": [vp, ctypes.POINTER(ctypes.c_longlong), dp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.adr_kernel_launches.argtypes = []
    lib.adr_kernel_launches.restype = ctypes.c_longlong
    lib.adr_last_error.argtypes = []
    lib.adr_last_error.restype = ctypes.c_char_p
    lib.adr_version.argtypes = []
    lib.adr_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(rc, allow=()):
    if rc != ADR_OK and rc not in allow:
        raise ADRError(rc, load().adr_last_error().decode())
    return rc
