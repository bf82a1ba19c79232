"""ctypes declarations of the C ABI in include/gofd.h (argument marshalling only).

Loading fails loudly when libgofd.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgofd.so")

STATUS = {
    0: "GOFD_OK", 1: "GOFD_E_ARG", 2: "GOFD_E_DEGENERATE_SIMPLEX", 3: "GOFD_E_OUTSIDE_BOX",
    4: "GOFD_E_GRID", 5: "GOFD_E_TOO_FEW_GRID_NODES", 6: "GOFD_E_ZERO_COLSUM", 7: "GOFD_E_PRECOND",
    8: "GOFD_E_NOT_CONVERGED", 9: "GOFD_E_TIMEOUT", 10: "GOFD_E_CUDA", 11: "GOFD_E_NOMEM",
}

FP64, FP32, FP64_DF = 0, 1, 2
SOLVE_FP64, SOLVE_MIXED = 0, 1
OP_STIFFNESS, OP_FRACLAP = 0, 1
RHS_GRID, RHS_VERTEX = 0, 1


class Options(C.Structure):
    _fields_ = [("precond", C.c_int), ("ic_level", C.c_int), ("filon_M", C.c_int64),
                ("richardson_levels", C.c_int), ("wait_budget_cycles", C.c_uint64),
                ("inner_tol", C.c_double), ("check_every", C.c_int), ("ordering", C.c_int),
                ("chunk_planes", C.c_int), ("fp64_residual", C.c_int),
                ("ic_solve", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters", C.c_int), ("rel_res_fp64", C.c_double),
                ("ic_shift", C.c_double), ("a_h", C.c_double), ("min_colsum", C.c_double),
                ("h_within_strict_bound", C.c_int), ("h_within_practical_bound", C.c_int),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double), ("device_loop", C.c_int)]


class Info(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int * 3), ("P", C.c_int), ("n_v", C.c_int64), ("n_e", C.c_int64),
                ("n_interior", C.c_int64), ("n_grid", C.c_int64), ("n_loc", C.c_int64), ("nnz_t", C.c_int64),
                ("n_runs", C.c_int64), ("filon_M", C.c_int64), ("richardson_levels", C.c_int),
                ("alpha", C.c_double), ("s", C.c_double), ("h", C.c_double), ("a_h", C.c_double),
                ("min_colsum", C.c_double), ("precond_nnz", C.c_int64), ("precond_levels", C.c_int), ("ic_shift", C.c_double),
                ("t_setup_ms", C.c_double), ("tune_lines_per_cta", C.c_int), ("tune_cols_per_cta", C.c_int),
                ("tune_scatter_lanes", C.c_int), ("tune_col_elems", C.c_int),
                ("tune_batch_chunk", C.c_int), ("tune_row_elems", C.c_int), ("warp_fft_path", C.c_int)]


_P = C.c_void_p
EXPORTS = {
    "gofd_build": (C.c_int, [C.c_int, _P, C.c_int64, _P, C.c_int64, C.c_double, C.c_double, _P, _P,
                             C.POINTER(Options), C.POINTER(_P)]),
    "gofd_apply": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "gofd_apply_host": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "gofd_apply_interior": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "gofd_precond_apply": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "gofd_apply_interior_batch": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int64, _P, _P]),
    "gofd_apply_interior_profiled": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(C.c_float),
                                               C.POINTER(C.c_char_p), C.c_int, C.POINTER(C.c_int)]),
    "gofd_solve": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_double, C.c_int, C.c_int, _P,
                             C.POINTER(SolveInfo), _P]),
    "gofd_adjoint": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_double, C.c_int, _P, _P, C.POINTER(SolveInfo), _P]),
    "gofd_solve_batch": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, C.c_int64, C.c_double, C.c_int, _P,
                                   _P, _P]),
    "gofd_autotune": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_double)]),
    "gofd_group_create": (C.c_int, [C.c_int, _P, C.c_int, C.POINTER(_P)]),
    "gofd_group_autotune": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
    "gofd_group_solve": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_double, C.c_int, _P, _P, _P]),
    "gofd_group_destroy": (None, [_P]),
    "gofd_set_launch_shapes": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "gofd_get_info": (C.c_int, [_P, C.POINTER(Info)]),
    "gofd_export_transfer": (C.c_int, [_P, _P, _P, _P]),
    "gofd_export_vertex_data": (C.c_int, [_P, _P, _P]),
    "gofd_get_coefficients": (C.c_int, [_P, _P]),
    "gofd_export_precond": (C.c_int, [_P, _P, _P, _P, _P]),
    "gofd_export_diagonal": (C.c_int, [_P, _P]),
    "gofd_get_symbol": (C.c_int, [_P, _P]),
    "gofd_afd_apply": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "gofd_afd_apply_noalloc": (C.c_int, [C.c_int, C.c_int, _P, _P, _P, _P]),
    "gofd_destroy": (None, [_P]),
    "gofd_fma_rates": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "gofd_last_error": (C.c_char_p, [_P]),
}

_lib = None


def load() -> C.CDLL:
    """Load libgofd.so (built by paper_2307_14437_gb300.build_native)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2307_14437_gb300.build_native.build() "
                          "(the GoFD path has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
