"""ctypes declarations of the C ABI in include/sbm.h (argument marshalling only).

The library is the in-tree ``libsbm.so`` built by ``paper_2212_02362_gb300.build``.
Importing this module fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsbm.so")

SBM_OK, SBM_ERR_ARG, SBM_ERR_STATE, SBM_ERR_CUDA, SBM_ERR_OOM, SBM_ERR_NOCONV, SBM_ERR_DIVERGED = range(7)
SBM_FP64, SBM_MIXED = 0, 1
SBM_JACOBI, SBM_MCGS = 0, 1
SBM_CUBIC, SBM_ISO_LAME, SBM_ISO_ENU = 0, 1, 2
SBM_FREE, SBM_DIRICHLET, SBM_DIRICHLET_FROM_U = 0, 1, 2
SBM_K_RESIDUAL64, SBM_K_JACOBI, SBM_K_RESIDUAL, SBM_K_SOURCE, SBM_K_TOPOPT, SBM_K_FMA64, SBM_K_FMA32, SBM_K_GS = range(8)
SBM_NOALLOC_MAX_BLOCKS = 16384


class sbm_grid_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double), ("precision", C.c_int),
                ("stream", C.c_void_p), ("device", C.c_int)]


class sbm_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("omega", C.c_double), ("smoother", C.c_int), ("inner_cycles", C.c_int),
                ("use_graph", C.c_int), ("inner_rtol", C.c_double)]


class sbm_box(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3)]


class sbm_info(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("vcycles", C.c_int), ("levels", C.c_int),
                ("r0", C.c_double), ("relres", C.c_double), ("history", C.POINTER(C.c_double)),
                ("history_capacity", C.c_int), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("launches", C.c_longlong)]


class sbm_topopt_params(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("alpha", "beta", "zeta", "lambda_", "lambda_rate", "V0", "mobility", "dt",
                                          "psi_min")]


class sbm_topopt_info(C.Structure):
    _fields_ = [("steps", C.c_int), ("capacity", C.c_int), ("compliance", C.POINTER(C.c_double)),
                ("volume", C.POINTER(C.c_double)), ("cycles", C.POINTER(C.c_int)), ("ms", C.c_double)]


_grid = C.c_void_p
_dptr = C.c_void_p          # device pointers are passed as plain addresses

_SIGS = {
    "sbm_default_opts": (None, [C.POINTER(sbm_opts)]),
    "sbm_status_string": (C.c_char_p, [C.c_int]),
    "sbm_last_error": (C.c_char_p, [_grid]),
    "sbm_grid_create": (C.c_int, [C.POINTER(sbm_grid_desc), C.POINTER(_grid)]),
    "sbm_grid_destroy": (C.c_int, [_grid]),
    "sbm_grid_levels": (C.c_int, [_grid, C.POINTER(C.c_int)]),
    "sbm_grid_level_shape": (C.c_int, [_grid, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "sbm_set_psi": (C.c_int, [_grid, C.c_int, _dptr, C.c_double]),
    "sbm_set_density": (C.c_int, [_grid, C.c_int, _dptr, C.c_double, C.c_double]),
    "sbm_set_moduli": (C.c_int, [_grid, C.c_int, C.POINTER(C.c_double)]),
    "sbm_set_bc": (C.c_int, [_grid, C.c_int, C.c_int, C.c_int, C.c_double]),
    "sbm_set_source": (C.c_int, [_grid, C.c_int, _dptr]),
    "sbm_solve": (C.c_int, [_grid, _dptr, C.POINTER(sbm_opts), C.POINTER(sbm_info)]),
    "sbm_adjoint": (C.c_int, [_grid, _dptr, _dptr, _dptr, _dptr, _dptr, C.POINTER(sbm_opts),
                              C.POINTER(sbm_info)]),
    "sbm_apply": (C.c_int, [_grid, C.c_int, C.c_int, _dptr, _dptr]),
    "sbm_residual": (C.c_int, [_grid, C.c_int, C.c_int, _dptr, _dptr, _dptr, C.POINTER(C.c_double)]),
    "sbm_smooth": (C.c_int, [_grid, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, _dptr, _dptr]),
    "sbm_restrict": (C.c_int, [_grid, C.c_int, C.c_int, _dptr, _dptr]),
    "sbm_prolong_add": (C.c_int, [_grid, C.c_int, C.c_int, _dptr, _dptr]),
    "sbm_get_psi": (C.c_int, [_grid, C.c_int, _dptr]),
    "sbm_bottom_correct": (C.c_int, [_grid, C.c_int, _dptr, _dptr]),
    "sbm_dJdpsi": (C.c_int, [_grid, _dptr, _dptr, _dptr]),
    "sbm_set_alloc_limit": (None, [C.c_size_t]),
    "sbm_set_wait_limit": (C.c_int, [_grid, C.c_longlong]),
    "sbm_source_terms": (C.c_int, [_grid, C.c_int, _dptr, _dptr, _dptr, _dptr, _dptr]),
    "sbm_topopt_step": (C.c_int, [_grid, C.POINTER(sbm_topopt_params), C.c_int, _dptr, _dptr, _dptr,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sbm_topopt_run": (C.c_int, [_grid, C.POINTER(sbm_topopt_params), C.c_int, _dptr, _dptr, C.POINTER(sbm_opts),
                                 C.POINTER(sbm_topopt_info)]),
    "sbm_apply_product": (C.c_int, [_grid, C.c_int, _dptr, _dptr, _dptr]),
    "sbm_jacobi_product": (C.c_int, [_grid, C.c_int, _dptr, _dptr, _dptr, C.c_double, C.c_int]),
    "sbm_time_kernel": (C.c_int, [_grid, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    "sbm_amr_add_level": (C.c_int, [_grid, C.POINTER(sbm_box)]),
    "sbm_amr_add_box": (C.c_int, [_grid, C.c_int, C.POINTER(sbm_box), C.POINTER(C.c_int)]),
    "sbm_amr_regrid": (C.c_int, [_grid, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "sbm_amr_get_box": (C.c_int, [_grid, C.c_int, C.POINTER(sbm_box), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sbm_amr_remove_levels": (C.c_int, [_grid, C.c_int]),
    "sbm_amr_set_psi": (C.c_int, [_grid, C.c_int, _dptr, C.c_double]),
    "sbm_amr_set_source": (C.c_int, [_grid, C.c_int, _dptr]),
    "sbm_amr_solve": (C.c_int, [_grid, C.POINTER(C.c_void_p), C.POINTER(sbm_opts), C.POINTER(sbm_info)]),
    "sbm_amr_residual": (C.c_int, [_grid, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_double)]),
    "sbm_amr_adjoint": (C.c_int, [_grid, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(sbm_opts), C.POINTER(sbm_info)]),
    "sbm_residual_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_double, C.POINTER(C.c_double),
                                       C.POINTER(C.c_uint), _dptr, _dptr, _dptr, _dptr, C.POINTER(C.c_double),
                                       C.c_void_p]),
}

EXPORTED = tuple(_SIGS)

SBM_OP_PRODUCT_NODE, SBM_OP_PRODUCT_CELL = 1, 2

_lib = None


def load(path: str = LIB_PATH):
    """Load libsbm.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2212_02362_gb300.build` "
                          "(the solver has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


def status_string(status: int) -> str:
    return load().sbm_status_string(status).decode()


def check(status: int, grid=None, allow=(SBM_OK,)):
    if status not in allow:
        raise SBMError(status, load().sbm_last_error(grid).decode())
    return status
