"""ctypes binding of ``libunocg.so`` (the C ABI declared in ``include/unocg.h``).

Only argument marshalling happens here: every step of the solve runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libunocg.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_NOT_SPD = -3
ERR_NOT_CONVERGED = -4
ERR_BREAKDOWN = -5
ERR_DEVICE_TIMEOUT = -6
ERR_CUDA = -7
ERR_STATE = -8
STATUS_NAMES = {OK: "OK", ERR_INVALID_ARG: "INVALID_ARG", ERR_OOM: "OOM", ERR_NOT_SPD: "NOT_SPD",
                ERR_NOT_CONVERGED: "NOT_CONVERGED", ERR_BREAKDOWN: "BREAKDOWN",
                ERR_DEVICE_TIMEOUT: "DEVICE_TIMEOUT", ERR_CUDA: "CUDA", ERR_STATE: "STATE"}

THERMAL = 1
ELASTIC = 3
PRECOND_NONE = 0
PRECOND_JACOBI = 1
PRECOND_UNO = 2
FP64 = 0
MIXED = 1
W_REFERENCE_MEDIUM = 0
W_BLOCKS = 1
W_THETA = 2
W_MODES = 3
DTYPE_F64 = 0
DTYPE_F32 = 1


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("replace_every", C.c_int), ("flexible", C.c_int),
                ("use_graph", C.c_int), ("replace_drop", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("max_iters", C.c_int), ("iters", C.POINTER(C.c_int)),
                ("rel_res", C.POINTER(C.c_double)), ("true_rel_res", C.POINTER(C.c_double)),
                ("load_status", C.POINTER(C.c_int)), ("checks", C.c_int), ("replacements", C.c_int)]


_vp = C.c_void_p
_i = C.c_int
_d = C.c_double

# name -> (restype, argtypes); names equal the C entry points
SIGNATURES = {
    "unocg_create": (_i, [C.POINTER(_vp), _i, _i, _i, _i, _i, _d]),
    "unocg_destroy": (None, [_vp]),
    "unocg_last_error": (C.c_char_p, [_vp]),
    "unocg_set_stream": (_i, [_vp, _vp]),
    "unocg_set_wait_limit": (_i, [_vp, _d]),
    "unocg_set_microstructure": (_i, [_vp, _vp, _i]),
    "unocg_set_microstructure_dev": (_i, [_vp, _vp, _i, _vp]),
    "unocg_set_phase_properties": (_i, [_vp, _vp]),
    "unocg_set_macro_load": (_i, [_vp, _i, _vp]),
    "unocg_set_uno_weights": (_i, [_vp, _i, _vp, _i, _d]),
    "unocg_set_uno_modes": (_i, [_vp, _i, _vp, _i, _d]),
    "unocg_get_uno_weights": (_i, [_vp, _i, _vp]),
    "unocg_solve": (_i, [_vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "unocg_solve_async": (_i, [_vp, C.POINTER(SolveOpts)]),
    "unocg_solve_wait": (_i, [_vp, C.POINTER(SolveInfo)]),
    "unocg_get_fluctuation": (_i, [_vp, _i, _i, _vp]),
    "unocg_get_fluctuation_dev": (_i, [_vp, _i, _i, _vp, _vp]),
    "unocg_get_effective_tensor": (_i, [_vp, _vp]),
    "unocg_get_sensitivity": (_i, [_vp, _vp]),
    "unocg_batch_solve": (_i, [_i, C.POINTER(_vp), C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "unocg_profile_iteration": (_i, [_vp, C.POINTER(SolveOpts), _i, _vp, _i]),
    "unocg_set_tuning": (_i, [_vp, _i, _i]),
    "unocg_autotune": (_i, [_vp, C.POINTER(SolveOpts), _i, _vp]),
    "unocg_uno_create": (_i, [C.POINTER(_vp), _i, _i, _i, _i]),
    "unocg_uno_destroy": (None, [_vp]),
    "unocg_uno_last_error": (C.c_char_p, [_vp]),
    "unocg_uno_set_theta_dev": (_i, [_vp, _vp, _vp]),
    "unocg_uno_set_modes_dev": (_i, [_vp, _i, _vp, _vp]),
    "unocg_uno_features_dev": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp]),
    "unocg_uno_apply_dev": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_uno_backward_dev": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "unocg_apply_K_dev": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_apply_K32_dev": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_newton_create": (_i, [_vp, _i, _i]),
    "unocg_newton_destroy": (None, [_vp]),
    "unocg_newton_last_error": (C.c_char_p, [_vp]),
    "unocg_newton_set_features": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "unocg_newton_run": (_i, [_vp, _vp, _i, C.c_double, _vp, _vp, _vp]),
    "unocg_set_ku_tile": (_i, [_vp, _i]),
    "unocg_get_ku_tile": (_i, [_vp, _vp]),
    "unocg_autotune_ku": (_i, [_vp, _i, _vp, _vp]),
    "unocg_apply_uno_dev": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_apply_uno_dev_noalloc": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_rhs_dev": (_i, [_vp, _i, _i, _vp, _vp]),
    # Dirichlet boundary conditions (sine transform)
    "unocg_dir_create": (_i, [C.POINTER(_vp), _i, _i, _i, _i, _i, _d]),
    "unocg_dir_create_bc": (_i, [C.POINTER(_vp), _i, _i, _i, _i, _i, _d, _vp]),
    "unocg_dir_destroy": (None, [_vp]),
    "unocg_dir_last_error": (C.c_char_p, [_vp]),
    "unocg_dir_set_stream": (_i, [_vp, _vp]),
    "unocg_dir_set_microstructure": (_i, [_vp, _vp, _i]),
    "unocg_dir_set_phase_properties": (_i, [_vp, _vp]),
    "unocg_dir_set_macro_load": (_i, [_vp, _i, _vp]),
    "unocg_dir_set_uno_weights": (_i, [_vp, _i, _vp, _i, _d]),
    "unocg_dir_set_uno_modes": (_i, [_vp, _i, _vp, _i, _d]),
    "unocg_dir_get_uno_weights": (_i, [_vp, _i, _vp]),
    "unocg_dir_solve": (_i, [_vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "unocg_dir_solve_async": (_i, [_vp, C.POINTER(SolveOpts)]),
    "unocg_dir_solve_wait": (_i, [_vp, C.POINTER(SolveInfo)]),
    "unocg_dir_get_fluctuation": (_i, [_vp, _i, _i, _vp]),
    "unocg_dir_get_fluctuation_dev": (_i, [_vp, _i, _i, _vp, _vp]),
    "unocg_dir_get_effective_tensor": (_i, [_vp, _vp]),
    "unocg_dir_apply_K_dev": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_dir_apply_uno_dev": (_i, [_vp, _i, _vp, _vp, _vp]),
    "unocg_dir_set_tuning": (_i, [_vp, _i, _i, _i]),
    "unocg_dir_autotune": (_i, [_vp, C.POINTER(SolveOpts), _i, _vp]),
}

_LIB = None


def load(path: str | None = None) -> C.CDLL:
    """Load the library once; raises ``OSError`` if it is missing (build it first)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libunocg.so not found at {p}: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class UnocgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
