"""ctypes declarations of the C ABI in include/mbs.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmbs.so")

MBS_OK = 0
STATUS = {
    0: "MBS_OK", 1: "MBS_ERR_ARG", 2: "MBS_ERR_GEOMETRY", 3: "MBS_ERR_NOMEM", 4: "MBS_ERR_CUDA",
    5: "MBS_ERR_NOCONV", 6: "MBS_ERR_TIMEOUT", 7: "MBS_ERR_NEAR_TARGET", 8: "MBS_ERR_STATE",
    9: "MBS_ERR_UNSUPPORTED",
}
PREC_FP64, PREC_MIXED, PREC_FP32 = 0, 1, 2


class mbs_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("tol", C.c_double), ("inner_tol", C.c_double),
        ("restart", C.c_int), ("max_iter", C.c_int), ("max_sweeps", C.c_int),
        ("ls_rcond", C.c_double), ("stream", C.c_void_p), ("hbm_budget", C.c_size_t),
        ("tile_override", C.c_int), ("block_krylov", C.c_int), ("mac_path", C.c_int),
        ("autotune", C.c_int), ("cuda_graphs", C.c_int), ("fp64_kernel", C.c_int),
        ("sbuild_threads", C.c_int), ("id_sketch", C.c_int), ("id_seed", C.c_uint),
    ]


class mbs_shape(C.Structure):
    _fields_ = [
        ("m", C.c_int), ("n", C.c_int), ("p", C.c_int),
        ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)), ("z", C.POINTER(C.c_double)),
        ("k", C.c_int), ("eps", C.c_double), ("proxy_radius", C.c_double),
    ]


class mbs_body(C.Structure):
    _fields_ = [("shape", C.c_int), ("c", C.c_double * 3), ("R", C.c_double * 9)]


class mbs_solve_info(C.Structure):
    _fields_ = [
        ("inner_iterations", C.c_int), ("sweeps", C.c_int), ("matvecs_fp32", C.c_int),
        ("matvecs_fp64", C.c_int), ("converged", C.c_int), ("fp64_finish", C.c_int),
        ("rel_residual", C.c_double),
        ("seconds", C.c_double),
        ("fp64_kernel", C.c_int),
    ]


class mbs_request(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("kappa", C.c_double), ("nshapes", C.c_int),
        ("shapes", C.POINTER(mbs_shape)), ("nbodies", C.c_int), ("bodies", C.POINTER(mbs_body)),
        ("nrhs", C.c_int), ("v", C.POINTER(C.c_double)), ("tol", C.c_double),
        ("fp64", C.c_int), ("max_iter", C.c_int),
    ]


class mbs_request_result(C.Structure):
    _fields_ = [
        ("done", C.c_int), ("status", C.c_int), ("N", C.c_int64), ("rel_residual", C.c_double),
        ("inner_iterations", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
        ("t_end", C.c_double), ("converged", C.c_int), ("dev_start", C.c_double),
        ("dev_end", C.c_double), ("g_busy_ms", C.c_double),
    ]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "mbs_default_options": (None, [C.POINTER(mbs_options)]),
    "mbs_create": (C.c_int, [C.c_int, C.c_double, C.POINTER(mbs_options), C.POINTER(_P)]),
    "mbs_destroy": (None, [_P]),
    "mbs_set_options": (C.c_int, [_P, C.POINTER(mbs_options)]),
    "mbs_last_error": (C.c_char_p, [_P]),
    "mbs_build_scattering_matrices": (C.c_int, [_P, C.c_int, C.POINTER(mbs_shape), C.c_int,
                                                C.POINTER(mbs_body)]),
    "mbs_get_layout": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P]),
    "mbs_get_shape": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _P, _D]),
    "mbs_get_shape_stats": (C.c_int, [_P, C.c_int] + [C.POINTER(C.c_int)] * 4 + [_D]),
    "mbs_rhs": (C.c_int, [_P, C.c_int, _P, _P]),
    "mbs_apply_operator": (C.c_int, [_P, C.c_int, _P, _P]),
    "mbs_apply_G": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "mbs_solve": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(mbs_solve_info)]),
    "mbs_evaluate_field": (C.c_int, [_P, C.c_int, C.c_int64, _P, _P, _P]),
    "mbs_reconstruct": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mbs_evaluate_field_near": (C.c_int, [_P, C.c_int, C.c_int64, _P, _P, _P, _P]),
    "mbs_inject_scattering": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int), _P, _P]),
    "mbs_measure_peaks": (C.c_int, [_D]),
    "mbs_apply_G_noalloc": (C.c_int, [C.c_int, C.c_double, C.c_int64, C.c_int, _P, _P, _P,
                                      C.c_int, _P, _P, _P]),
    "mbs_launch_count": (C.c_int64, []),
    "mbs_profile": (C.c_int, [_P, C.c_int]),
    "mbs_kernel_times": (C.c_int, [_P, _D]),
    "mbs_serve_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(_P)]),
    "mbs_serve_submit": (C.c_int, [_P, C.POINTER(mbs_request), C.POINTER(C.c_int64)]),
    "mbs_serve_poll": (C.c_int, [_P, C.c_int64, C.POINTER(mbs_request_result), _P]),
    "mbs_serve_drain": (C.c_int, [_P]),
    "mbs_serve_set_policy": (C.c_int, [_P, C.c_int]),
    "mbs_serve_destroy": (None, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libmbs.so and declare every entry point.  Raises if it is missing:
    there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2603_19113_gb300.build.build() "
                          "(nvcc, sm_103a); the library has no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
