"""ctypes declarations of include/weno3.h (same names, argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import _build

WENO_OK, WENO_EINVAL, WENO_EMESH, WENO_EPERIODIC, WENO_ENOMEM, WENO_ECUDA, WENO_ENONPHYS, WENO_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
WENO_BC_PERIODIC, WENO_BC_OUTFLOW = 0, 1
WENO_EQN_SCALAR, WENO_EQN_EULER = 0, 1
WENO_FP64, WENO_FP32C = 0, 1

STATUS_NAMES = {0: "WENO_OK", -1: "WENO_EINVAL", -2: "WENO_EMESH", -3: "WENO_EPERIODIC", -4: "WENO_ENOMEM",
                -5: "WENO_ECUDA", -6: "WENO_ENONPHYS", -7: "WENO_ETIMEOUT"}


class weno_mesh_opts(C.Structure):
    _fields_ = [("bc", C.c_int32), ("origin", C.c_double * 2), ("extent", C.c_double * 2), ("walls", C.c_int32),
                ("wall_from", C.c_double * 4), ("inflow", C.c_int32)]


class weno_params(C.Structure):
    _fields_ = [("eqn", C.c_int32), ("precision", C.c_int32), ("gas_gamma", C.c_double), ("adv", C.c_double * 2),
                ("eps", C.c_double), ("theta", C.c_double), ("rcond", C.c_double), ("optimize", C.c_int32),
                ("linear", C.c_int32), ("n_threads", C.c_int32), ("characteristic", C.c_int32),
                ("inflow_a", C.c_double * 4), ("inflow_b", C.c_double * 4), ("inflow_line", C.c_double * 4)]


class weno_mesh_info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_quads", C.c_int64), ("n_tris", C.c_int64), ("n_faces", C.c_int64),
                ("n_boundary", C.c_int64), ("n_instances", C.c_int32), ("n_inflow", C.c_int32)]


# exported symbols with (restype, argtypes)
P = C.c_void_p
SIGNATURES = {
    "weno_params_default": (None, [C.POINTER(weno_params)]),
    "weno_mesh_create": (C.c_int, [P, C.c_int64, P, P, C.c_int64, C.POINTER(weno_mesh_opts), C.POINTER(P)]),
    "weno_mesh_concat": (C.c_int, [P, C.c_int32, C.POINTER(P)]),
    "weno_mesh_get_info": (C.c_int, [P, C.POINTER(weno_mesh_info)]),
    "weno_mesh_cell_permutation": (C.c_int, [P, P]),
    "weno_mesh_cell_instance": (C.c_int, [P, P]),
    "weno_mesh_weight_stats": (C.c_int, [P, C.POINTER(weno_params), P, P]),
    "weno_mesh_cell_tables": (C.c_int, [P, C.POINTER(weno_params), C.c_int64, P, P, P, P, P]),
    "weno_mesh_destroy": (None, [P]),
    "weno_solver_create": (C.c_int, [P, C.POINTER(weno_params), P, C.POINTER(P)]),
    "weno_solver_get_info": (C.c_int, [P, C.POINTER(weno_mesh_info)]),
    "weno_residual": (C.c_int, [P, P, P, P, P]),
    "weno_residual_static": (C.c_int, [P, P, P, P, P]),
    "weno_set_time": (C.c_int, [P, C.c_double, P]),
    "weno_get_time": (C.c_int, [P, P, P]),
    "weno_step": (C.c_int, [P, P, P, C.c_double, P]),
    "weno_step_instances": (C.c_int, [P, P, P, P, P]),
    "weno_max_dt": (C.c_int, [P, P, P, C.c_double, P, P]),
    "weno_conservation": (C.c_int, [P, P, P, P, P]),
    "weno_check": (C.c_int, [P, P]),
    "weno_check_instances": (C.c_int, [P, P, P]),
    "weno_pass": (C.c_int, [P, C.c_int32, P, P, P]),
    "weno_autotune": (C.c_int, [P, P, P, P]),
    "weno_solver_launch_config": (C.c_int, [P, P]),
    "weno_solver_debug_stall": (C.c_int, [P, C.c_int32]),
    "weno_probe_peak": (C.c_int, [C.c_int32, C.c_int32, P, P, P]),
    "weno_solver_destroy": (None, [P]),
    "weno_last_error": (C.c_char_p, []),
}

_lib = None


class WenoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libweno3.so (building it first if it is missing); raise if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing; run paper_1712_08317_gb300._build.build()")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int):
    if code != WENO_OK:
        raise WenoError(code, load().weno_last_error().decode())
