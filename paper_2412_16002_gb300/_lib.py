"""ctypes declarations of the C ABI in include/crkdg.h (argument marshalling only).

Loading fails loudly when libcrkdg.so has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcrkdg.so")

OK, E_ARG, E_CUDA, E_OOM, E_BOUNDS, E_TIMEOUT, E_UNSUPPORTED = range(7)
STATUS = {0: "OK", 1: "E_ARG", 2: "E_CUDA", 3: "E_OOM", 4: "E_BOUNDS", 5: "E_TIMEOUT", 6: "E_UNSUPPORTED"}
BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3}
FLUX = {"advection": 0, "burgers": 1, "euler": 2}
PREC = {"fp64": 0, "mixed": 1}
INDICATOR = {"off": 0, "tvb": 1, "mlp": 2}
SCHEME = {"compact": 0, "standard": 1}
THETA2 = {"ratio": 0, "exact": 1}
SOURCE = {None: 0, "scenario1": 1}
BASIS = {"Q": 0, "P": 1}
OPS = {"G": 0, "F": 1, "limit": 2}


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("bc", C.c_int * 4), ("bc_state", (C.c_double * 4) * 4)]


class Flux(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double), ("velocity", C.c_double * 2)]


class Bounds(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("eps", C.c_double)]


class Tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("A", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_halvings", C.c_int), ("indicator", C.c_int),
                ("tvb_M", C.c_double), ("cuda_stream", C.c_void_p), ("scheme", C.c_int),
                ("theta2", C.c_int), ("source", C.c_int), ("basis", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("dt_taken", C.c_double), ("restarts", C.c_int), ("cells_limited", C.c_longlong),
                ("theta_min", C.c_double), ("troubled", C.c_longlong), ("mass_drift", C.c_double)]


class EnsProblem(C.Structure):
    _fields_ = [("mesh", Mesh), ("k", C.c_int), ("tableau", C.POINTER(Tableau)), ("cfl", C.c_double),
                ("t_end", C.c_double)]


class EnsInfo(C.Structure):
    _fields_ = [("t", C.c_double), ("steps", C.c_longlong), ("restarts", C.c_longlong), ("done", C.c_int),
                ("status", C.c_int), ("last", StepInfo)]


class CrkdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_dp = C.POINTER(C.c_double)
_H = C.c_void_p

# entry points declared in include/crkdg.h
SYMBOLS = {
    "crkdg_options_default": (None, [C.POINTER(Options)]),
    "crkdg_create": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.POINTER(Flux), C.POINTER(Bounds),
                               C.POINTER(Options), C.POINTER(_H)]),
    "crkdg_destroy": (C.c_int, [_H]),
    "crkdg_set_state": (C.c_int, [_H, C.c_void_p, C.c_size_t, C.c_int]),
    "crkdg_get_state": (C.c_int, [_H, C.c_void_p, C.c_size_t, C.c_int]),
    "crkdg_max_dt": (C.c_int, [_H, C.c_double, _dp]),
    "crkdg_set_time": (C.c_int, [_H, C.c_double]),
    "crkdg_get_time": (C.c_int, [_H, _dp]),
    "crkdg_step": (C.c_int, [_H, C.c_double, C.POINTER(Tableau), C.POINTER(StepInfo)]),
    "crkdg_advance": (C.c_int, [_H, C.c_int, C.c_double, C.c_double, C.POINTER(Tableau), _dp,
                                C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "crkdg_advance_fixed": (C.c_int, [_H, C.c_int, C.c_double, C.c_double, C.POINTER(Tableau), _dp,
                                      C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "crkdg_apply_operator": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_void_p]),
    "crkdg_troubled_flags": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "crkdg_cell_averages": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "crkdg_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "crkdg_mlp_fault": (C.c_int, [C.POINTER(C.c_int)]),
    "crkdg_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "crkdg_mlp_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_void_p]),
    "crkdg_set_mlp": (C.c_int, [_H, C.c_void_p]),
    "crkdg_set_harvest": (C.c_int, [_H, C.c_int]),
    "crkdg_last_features": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "crkdg_bound_margins": (C.c_int, [_H, _dp]),
    "crkdg_total_mass": (C.c_int, [_H, C.c_int, _dp]),
    "crkdg_set_profiling": (C.c_int, [_H, C.c_int]),
    "crkdg_set_barrier_test": (C.c_int, [_H, C.c_int]),
    "crkdg_set_run1d_chunk": (C.c_int, [_H, C.c_int]),
    "crkdg_set_tensor_cores": (C.c_int, [_H, C.c_int]),
    "crkdg_kernel_times": (C.c_int, [_H, _dp, C.POINTER(C.c_longlong)]),
    "crkdg_state_size": (C.c_size_t, [_H]),
    "crkdg_step_attempt": (C.c_int, [_H, C.c_double, C.POINTER(Tableau), C.POINTER(C.c_int)]),
    "crkdg_step_accept": (C.c_int, [_H, C.POINTER(StepInfo)]),
    "crkdg_set_subdomain": (C.c_int, [_H, C.POINTER(Mesh), C.c_int, C.c_int, C.c_int, C.c_int]),
    "crkdg_set_geometry": (C.c_int, [_H, C.POINTER(C.c_uint), _dp, _dp, C.c_double, C.c_double]),
    "crkdg_cells_bytes": (C.c_size_t, [_H, C.c_longlong]),
    "crkdg_pack_cells": (C.c_int, [_H, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "crkdg_unpack_cells": (C.c_int, [_H, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "crkdg_last_error": (C.c_char_p, [_H]),
    "crkdg_apply_F_noalloc": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.POINTER(Flux), C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "crkdg_ensemble_create": (C.c_int, [C.c_int, C.POINTER(EnsProblem), C.c_int, C.POINTER(Flux), C.POINTER(Bounds),
                                        C.POINTER(Options), C.POINTER(_H)]),
    "crkdg_ensemble_destroy": (C.c_int, [_H]),
    "crkdg_ensemble_set_state": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "crkdg_ensemble_get_state": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "crkdg_ensemble_state_size": (C.c_size_t, [_H, C.c_int]),
    "crkdg_ensemble_step": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "crkdg_ensemble_info": (C.c_int, [_H, C.c_int, C.POINTER(EnsInfo)]),
    "crkdg_ensemble_set_mlp": (C.c_int, [_H, C.c_void_p]),
    "crkdg_ensemble_set_harvest": (C.c_int, [_H, C.c_int]),
    "crkdg_ensemble_last_features": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_int]),
    "crkdg_ensemble_troubled_flags": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_int]),
    "crkdg_ensemble_autotune": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int)]),
    "crkdg_ensemble_plan": (C.c_int, [C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.c_int,
                                      C.POINTER(C.c_int), C.c_int]),
    "crkdg_ensemble_set_profiling": (C.c_int, [_H, C.c_int]),
    "crkdg_ensemble_times": (C.c_int, [_H, _dp, C.POINTER(C.c_longlong)]),
    "crkdg_ensemble_last_error": (C.c_char_p, [_H]),
}


def load(path: str = LIB_PATH):
    """Load libcrkdg.so (raises if it is missing: build it with paper_2412_16002_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2412_16002_gb300.build.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(lib, h, status):
    if status != OK:
        msg = lib.crkdg_last_error(h)
        raise CrkdgError(status, msg.decode() if msg else "")


def check_ens(lib, e, status):
    if status != OK:
        msg = lib.crkdg_ensemble_last_error(e)
        raise CrkdgError(status, msg.decode() if msg else "")
