"""ctypes view of the liblbm C-ABI (include/lbm.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_STATE = range(6)
LBM_F64, LBM_F32, LBM_F32_STORE_F16, LBM_F32_FRAMED = 0, 1, 2, 3
LBM_BC_SIDE_HEATED, LBM_BC_COOLED = 0, 1
LBM_MRT, LBM_LBGK = 0, 1

ERROR_NAMES = {1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_DIVERGED", 4: "LBM_ERR_TIMEOUT",
               5: "LBM_ERR_STATE"}


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("Ra", C.c_double), ("Da", C.c_double), ("Pr", C.c_double), ("J", C.c_double),
                ("phi", C.c_double), ("Ma", C.c_double), ("sigma", C.c_double), ("varpi", C.c_double),
                ("Th", C.c_double), ("Tc", C.c_double), ("Qppp", C.c_double),
                ("precision", C.c_int), ("use_phi_field", C.c_int), ("forchheimer", C.c_int),
                ("thermal_bc", C.c_int), ("adiabatic_order", C.c_int), ("collision", C.c_int),
                ("block_x", C.c_int), ("block_y", C.c_int), ("nodes_per_thread", C.c_int),
                ("RaI", C.c_double)]


class Obs(C.Structure):
    _fields_ = [("t", C.c_long), ("nu_hot", C.c_double), ("nu_cold", C.c_double),
                ("residual", C.c_double), ("umax", C.c_double), ("mass", C.c_double),
                ("heat", C.c_double), ("status", C.c_int)]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/lbm.h
SIGNATURES = [
    ("lbm_params_default", None, [C.POINTER(Params), C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
    ("lbm_init", C.c_int, [C.POINTER(Params), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("lbm_set_porous_field", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("lbm_step", C.c_int, [C.c_void_p, C.c_long]),
    ("lbm_reset", C.c_int, [C.c_void_p]),
    ("lbm_bounds_check", C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_long)]),
    ("lbm_tune", C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("lbm_observables", C.c_int, [C.c_void_p, C.POINTER(Obs), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_adjoint_step", C.c_int, [C.c_void_p, C.c_long, C.c_long, C.POINTER(C.c_double), C.c_void_p]),
    ("lbm_run_steady", C.c_int, [C.c_void_p, C.c_double, C.c_long, C.c_long, C.POINTER(C.c_long),
                                 C.POINTER(C.c_double)]),
    ("lbm_field_extrema", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    ("lbm_nusselt_async", C.c_int, [C.c_void_p, C.c_void_p]),
    ("lbm_step_nusselt", C.c_int, [C.c_void_p, C.c_long, C.c_void_p]),
    ("lbm_nusselt", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("lbm_read_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_checkpoint_size", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("lbm_save", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("lbm_load", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("lbm_observables_noalloc", C.c_int, [C.POINTER(Params), C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(Obs),
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_batch_init", C.c_int, [C.POINTER(Params), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("lbm_batch_step", C.c_int, [C.c_void_p, C.c_long]),
    ("lbm_batch_nusselt", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lbm_batch_status", C.c_int, [C.c_void_p, C.c_void_p]),
    ("lbm_batch_read_state", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("lbm_batch_set_wait_limit", C.c_int, [C.c_void_p, C.c_longlong]),
    ("lbm_batch_tune", C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)]),
    ("lbm_batch_set_tiles", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    ("lbm_batch_query", C.c_int, [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("lbm_batch_destroy", C.c_int, [C.c_void_p]),
    ("lbm_batch_last_error", C.c_char_p, [C.c_void_p]),
    ("lbm_query", C.c_int, [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_int)]),
    ("lbm_destroy", C.c_int, [C.c_void_p]),
    ("lbm_last_error", C.c_char_p, [C.c_void_p]),
]


def load(path: str | None = None):
    """Loads liblbm.so; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"liblbm.so is missing at {p}: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(p)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int, handle=None, batch=None):
    if rc != LBM_OK:
        msg = load().lbm_batch_last_error(batch) if batch is not None else load().lbm_last_error(handle)
        raise LbmError(rc, msg.decode() if msg else "")
