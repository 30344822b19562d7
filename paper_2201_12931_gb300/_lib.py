"""ctypes binding of libtopo_gb300.so (the C-ABI declared in include/topo.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtopo_gb300.so")

TOPO_OK, TOPO_BADARG, TOPO_OOM, TOPO_MAXITER, TOPO_BREAKDOWN, TOPO_CUDA = range(6)
STATUS_NAMES = {0: "TOPO_OK", 1: "TOPO_BADARG", 2: "TOPO_OOM", 3: "TOPO_MAXITER", 4: "TOPO_BREAKDOWN",
                5: "TOPO_CUDA"}
TOPO_FP64, TOPO_MIXED, TOPO_MIXED_BF16, TOPO_DF32, TOPO_FP32_TC = 0, 1, 2, 3, 4


class TopoParams(C.Structure):
    _fields_ = [("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double), ("penal", C.c_double),
                ("levels", C.c_int), ("pre", C.c_int), ("post", C.c_int), ("omega", C.c_double),
                ("precision", C.c_int), ("inner_tol", C.c_double), ("inner_max_it", C.c_int),
                ("max_refine", C.c_int), ("homogenize", C.c_int), ("graphs", C.c_int),
                ("outer_residual", C.c_int), ("tensor_cores", C.c_int),
                ("cg_check", C.c_int)]


class TopoSolveStats(C.Structure):
    _fields_ = [("outer_steps", C.c_int), ("inner_iters", C.c_int), ("relres", C.c_double),
                ("solve_ms", C.c_double), ("status", C.c_int), ("graph_replays", C.c_int)]


H = C.c_void_p
P = C.c_void_p   # device pointer
_SIGS = {
    "topo_default_params": ([C.POINTER(TopoParams)], C.c_int),
    "topo_create_grid": ([C.c_int, C.c_int, C.c_int, C.POINTER(TopoParams), C.c_void_p, C.POINTER(H)], C.c_int),
    "topo_destroy_grid": ([H], C.c_int),
    "topo_set_density": ([H, P], C.c_int),
    "topo_set_bc_loads": ([H, P, P], C.c_int),
    "topo_solve_state": ([H, C.c_double, C.c_int, P, C.POINTER(C.c_int), C.POINTER(C.c_double)], C.c_int),
    "topo_compliance_and_sensitivity": ([H, C.POINTER(C.c_double), P], C.c_int),
    "topo_state_step_host": ([H, P, C.c_double, C.c_int, C.POINTER(C.c_double), P, C.POINTER(C.c_int),
                              C.POINTER(C.c_double)], C.c_int),
    "topo_filter": ([H, C.c_double, P, P, C.c_int], C.c_int),
    "topo_oc_update": ([H, C.c_double, C.c_double, C.c_double, P, P, C.POINTER(C.c_double)], C.c_int),
    "topo_sensitivity_filter": ([H, C.c_double, C.c_double, P, P, P], C.c_int),
    "topo_oc_update_unfiltered": ([H, C.c_double, C.c_double, P, P, P, C.POINTER(C.c_double)], C.c_int),
    "topo_gravity_load": ([H, C.c_double, P, P, P], C.c_int),
    "topo_gravity_sensitivity": ([H, C.c_double, P], C.c_int),
    "topo_last_error": ([H], C.c_char_p),
    "topo_level_dims": ([H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "topo_apply_operator": ([H, C.c_int, C.c_int, P, P], C.c_int),
    "topo_jacobi_sweep": ([H, C.c_int, C.c_int, P, P, P], C.c_int),
    "topo_residual": ([H, C.c_int, C.c_int, P, P, P], C.c_int),
    "topo_restrict": ([H, C.c_int, P, P], C.c_int),
    "topo_prolong_add": ([H, C.c_int, P, P], C.c_int),
    "topo_level_density": ([H, C.c_int, P], C.c_int),
    "topo_vcycle": ([H, C.c_int, P, P], C.c_int),
    "topo_get_stats": ([H, C.POINTER(TopoSolveStats)], C.c_int),
    "topo_launch_count": ([H, C.POINTER(C.c_longlong)], C.c_int),
    "topo_measure_peak": ([C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "topo_reset_solution": ([H], C.c_int),
    "topo_profile_enable": ([H, C.c_int], C.c_int),
    "topo_profile_read": ([H, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double)], C.c_int),
    "topo_filter_noalloc": ([C.c_int, C.c_int, C.c_int, C.c_double, P, P, C.c_int, C.c_void_p], C.c_int),
}

_lib = None


def load(path: str | None = None):
    """Load (once) and return the CDLL; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(
            f"{path} not found: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()' or python paper_2201_12931_gb300/build.py)")
    lib = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_names():
    return list(_SIGS)
