"""ctypes view of include/to.h (argument marshalling only; all work runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfbto.so")

TO_OK, TO_ERR_ARG, TO_ERR_CUDA, TO_ERR_NONFINITE, TO_ERR_INFEASIBLE, TO_ERR_TIMEOUT, TO_ERR_SINGULAR, TO_ERR_STATE = range(8)
TO_FP64, TO_FP32_MIXED = 0, 1
TO_PRECOND_JACOBI, TO_PRECOND_MG, TO_PRECOND_NONE, TO_PRECOND_KRYLOV = 0, 1, 2, 3
TO_INNER_SD, TO_INNER_RICHARDSON, TO_INNER_PFBTO, TO_INNER_PCG = 0, 1, 2, 3

ERROR_NAMES = {0: "TO_OK", 1: "TO_ERR_ARG", 2: "TO_ERR_CUDA", 3: "TO_ERR_NONFINITE", 4: "TO_ERR_INFEASIBLE",
               5: "TO_ERR_TIMEOUT", 6: "TO_ERR_SINGULAR", 7: "TO_ERR_STATE"}


class to_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double)]


class to_material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E0", "Emin", "nu", "p", "volfrac", "rmin", "rho_min", "rho_max")]


class to_loads(C.Structure):
    _fields_ = [("n", C.c_int64), ("dof", C.POINTER(C.c_int64)), ("val", C.POINTER(C.c_double))]


class to_bcs(C.Structure):
    _fields_ = [("n", C.c_int64), ("dof", C.POINTER(C.c_int64))]


class to_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("precond", C.c_int32), ("inner_mode", C.c_int32), ("n_inner", C.c_int32),
                ("beta", C.c_double), ("alpha0", C.c_double), ("alpha_scale", C.c_double), ("m", C.c_double),
                ("mean_proj", C.c_int32), ("mg_levels", C.c_int32), ("mg_nu_pre", C.c_int32), ("mg_nu_post", C.c_int32),
                ("mg_omega", C.c_double),
                ("tile_x", C.c_int32), ("tile_y", C.c_int32), ("tile_z", C.c_int32), ("no_graph", C.c_int32),
                ("krylov_dim", C.c_int32), ("proj_sort", C.c_int32), ("adj_stride", C.c_int32),
                ("op_kernel", C.c_int32), ("mg_legs", C.c_int32), ("mg_cluster", C.c_int32)]


class to_stats(C.Structure):
    _fields_ = [("k", C.c_int64), ("J", C.c_double), ("res_inf", C.c_double), ("res2", C.c_double),
                ("drho_inf", C.c_double), ("volume", C.c_double), ("lambda_", C.c_double), ("alpha", C.c_double),
                ("gmax", C.c_double), ("beta_first", C.c_double), ("beta_last", C.c_double),
                ("proj_iters", C.c_int32), ("status", C.c_int32)]

    def as_dict(self):
        return {("lambda" if n == "lambda_" else n): getattr(self, n) for n, _ in self._fields_}


P = C.c_void_p
# name -> (restype, argtypes); every symbol declared in include/to.h
SIGNATURES = {
    "to_default_params": (None, [C.POINTER(to_params)]),
    "to_create": (C.c_int, [C.POINTER(to_grid), C.POINTER(to_material), C.POINTER(to_loads), C.POINTER(to_bcs),
                            C.POINTER(to_params), C.c_int, C.POINTER(C.c_void_p)]),
    "to_destroy": (None, [P]),
    "to_sizes": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "to_set_design": (C.c_int, [P, P, P]),
    "to_apply_K": (C.c_int, [P, P, P, P]),
    "to_residual": (C.c_int, [P, P, P, P, P, C.POINTER(C.c_double), P]),
    "to_smooth": (C.c_int, [P, P, P, P, C.c_double, P]),
    "to_inner_solve": (C.c_int, [P, P, C.c_int32, C.POINTER(C.c_double), P]),
    "to_sensitivity": (C.c_int, [P, P, P, P]),
    "to_filter": (C.c_int, [P, P, P, C.c_int32, P]),
    "to_project": (C.c_int, [P, P, P, C.POINTER(C.c_double), P]),
    "to_step": (C.c_int, [P, C.c_int32, C.POINTER(to_stats), P]),
    "to_get_stats": (C.c_int, [P, C.c_int32, P, P]),
    "to_step_host": (C.c_int, [P, P, P, P, P]),
    "to_get_state": (C.c_int, [P, P, P, C.POINTER(C.c_int64), C.POINTER(C.c_double), P]),
    "to_set_state": (C.c_int, [P, P, P, C.c_int64, C.c_double, P]),
    "to_check": (C.c_int, [P, P]),
    "to_barrier_selftest": (C.c_int, [P, C.c_int32, C.c_int64, P]),
    "to_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "to_batch_destroy": (None, [P]),
    "to_batch_step": (C.c_int, [P, C.c_int32, C.POINTER(to_stats), P]),
    "to_batch_tile": (C.c_int, [P, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "to_compliance_truncated": (C.c_int, [P, P, C.c_int32, C.c_double, C.POINTER(C.c_double), P]),
    "to_compliance_truncated_grad": (C.c_int, [P, C.c_double, P, P]),
    "to_compliance_truncated_id": (C.c_int, [P, C.POINTER(C.c_int64)]),
    "to_project_noalloc": (C.c_int, [P, P, C.c_int64, C.c_int32, C.c_double, C.c_double, C.c_double,
                                     C.POINTER(C.c_double), P]),
    "to_last_error": (C.c_char_p, []),
}

_lib = None


class ToError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load the CUDA library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != TO_OK:
        msg = load().to_last_error()
        raise ToError(rc, msg.decode() if msg else "")
