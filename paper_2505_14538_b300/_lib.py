"""ctypes declarations of the C ABI in ``include/swift_gpu.h`` and ``include/swift_gpu_time.h``.

Loading fails loudly (ImportError) when ``libswift_gpu.so`` has not been
built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswift_gpu.so")

OK = 0
ERR_ARG = -1
ERR_ORDER = -2
ERR_CUDA = -3
ERR_H_NOT_CONVERGED = -4
ERR_H_EXCEEDS_CELL = -5
ERR_TIMEOUT = -6
ERR_NOMEM = -7
ERR_CAPACITY = -8

ERR_NAMES = {OK: "OK", ERR_ARG: "ERR_ARG", ERR_ORDER: "ERR_ORDER", ERR_CUDA: "ERR_CUDA",
             ERR_H_NOT_CONVERGED: "ERR_H_NOT_CONVERGED", ERR_H_EXCEEDS_CELL: "ERR_H_EXCEEDS_CELL",
             ERR_TIMEOUT: "ERR_TIMEOUT", ERR_NOMEM: "ERR_NOMEM", ERR_CAPACITY: "ERR_CAPACITY"}

FLAG_PLAIN = 1
FLAG_NO_H_ITER = 2
FLAG_NO_COMPENSATION = 4
FLAG_ADAPTIVE = 8

KERNEL_CUBIC = 0
KERNEL_WENDLAND_C2 = 1
KERNEL_WENDLAND_C4 = 2
# H/h of each shape from the second-moment definition (sqrt(30)/3, sqrt(15)/2, sqrt(78)/4)
COLLECT_ROWS = 0  # swift_gpu_tuning.group_collect
COLLECT_WINDOWS = 1
KERNEL_GAMMAS = {KERNEL_CUBIC: 1.825742, KERNEL_WENDLAND_C2: 1.936492, KERNEL_WENDLAND_C4: 2.207940}

EXPORTED = ("swift_gpu_default_params", "swift_gpu_create", "swift_gpu_destroy", "swift_gpu_set_params",
            "swift_gpu_build_cells", "swift_gpu_density", "swift_gpu_gradient", "swift_gpu_force",
            "swift_gpu_force_backward", "swift_gpu_sync_status", "swift_gpu_get_info", "swift_gpu_get_cells",
            "swift_gpu_get_tuning", "swift_gpu_set_tuning", "swift_gpu_autotune", "swift_gpu_density_static",
            "swift_gpu_get_leaves", "swift_gpu_gradient_force", "swift_gpu_default_time_params",
            "swift_gpu_kick_drift", "swift_gpu_viscosity_switch", "swift_gpu_kick_finish",
            "swift_gpu_set_inactive")

STATIC_MAX_PARTICLES = 32768


class Params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_float * 3),
        ("gamma_eos", ctypes.c_float),
        ("eta", ctypes.c_float),
        ("kernel_gamma", ctypes.c_float),
        ("alpha_v", ctypes.c_float),
        ("beta_v", ctypes.c_float),
        ("alpha_c", ctypes.c_float),
        ("h_tol", ctypes.c_float),
        ("max_iter", ctypes.c_int),
        ("h_max", ctypes.c_float),
        ("cell_margin", ctypes.c_float),
        ("flags", ctypes.c_int),
        ("leaf_max", ctypes.c_int),
        ("leaf_margin", ctypes.c_float),
        ("kernel", ctypes.c_int),
    ]


class Tuning(ctypes.Structure):
    _fields_ = [
        ("threads_per_block", ctypes.c_int),
        ("max_lanes_per_particle", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("wait_limit_us", ctypes.c_int),
        ("group_collect", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nc", ctypes.c_int32 * 3),
        ("cell_width", ctypes.c_float * 3),
        ("h_cap", ctypes.c_float),
        ("n_cells", ctypes.c_int64),
        ("n_items", ctypes.c_int64),
        ("density_passes", ctypes.c_int32),
        ("interactions", ctypes.c_uint64 * 3),
        ("candidates", ctypes.c_uint64 * 3),
        ("launches", ctypes.c_uint64),
        ("h_iteration_pairs", ctypes.c_uint64),
        ("n_leaves", ctypes.c_int64),
        ("leaf_pairs", ctypes.c_int64),
        ("tree_depth", ctypes.c_int32),
    ]


class TimeParams(ctypes.Structure):
    _fields_ = [
        ("cfl", ctypes.c_float),
        ("dt_max", ctypes.c_float),
        ("alpha_v_max", ctypes.c_float),
        ("alpha_v_min", ctypes.c_float),
        ("visc_length", ctypes.c_float),
        ("alpha_c_max", ctypes.c_float),
        ("alpha_c_min", ctypes.c_float),
        ("beta_c", ctypes.c_float),
        ("u_min_frac", ctypes.c_float),
    ]


class Clock(ctypes.Structure):
    """Host image of swift_gpu_clock (32 bytes; the library reads and writes a device copy)."""
    _fields_ = [
        ("t", ctypes.c_double),
        ("t_end", ctypes.c_double),
        ("dt", ctypes.c_float),
        ("dt_next", ctypes.c_float),
        ("step", ctypes.c_int64),
    ]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64

_SIGS = {
    "swift_gpu_default_params": (None, [ctypes.POINTER(Params)]),
    "swift_gpu_create": (_I, [ctypes.POINTER(_VP), ctypes.POINTER(Params), _I64]),
    "swift_gpu_destroy": (_I, [_VP]),
    "swift_gpu_set_params": (_I, [_VP, ctypes.POINTER(Params)]),
    "swift_gpu_build_cells": (_I, [_VP, _VP, _I64, ctypes.c_float, _VP]),
    "swift_gpu_density": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "swift_gpu_gradient": (_I, [_VP, _VP, _VP, _VP]),
    "swift_gpu_force": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "swift_gpu_force_backward": (_I, [_VP, _VP, _VP, _VP, _VP, _I, _VP]),
    "swift_gpu_sync_status": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I64)]),
    "swift_gpu_get_info": (_I, [_VP, ctypes.POINTER(Info)]),
    "swift_gpu_get_cells": (_I, [_VP, _VP, _VP, _VP]),
    "swift_gpu_get_tuning": (_I, [_VP, ctypes.POINTER(Tuning)]),
    "swift_gpu_set_tuning": (_I, [_VP, ctypes.POINTER(Tuning)]),
    "swift_gpu_autotune": (_I, [_VP, _I, _VP]),
    "swift_gpu_density_static": (_I, [ctypes.POINTER(Params), _VP, _VP, _I64, ctypes.c_float, _VP, _VP, _VP, _VP,
                                      _VP, _VP]),
    "swift_gpu_get_leaves": (_I, [_VP, _VP, _VP, _VP, _I64, _VP]),
    "swift_gpu_gradient_force": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "swift_gpu_set_inactive": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "swift_gpu_default_time_params": (None, [ctypes.POINTER(TimeParams)]),
    "swift_gpu_kick_drift": (_I, [_VP, ctypes.POINTER(TimeParams), _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                  _VP]),
    "swift_gpu_viscosity_switch": (_I, [_VP, ctypes.POINTER(TimeParams), _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP,
                                        _VP]),
    "swift_gpu_kick_finish": (_I, [_VP, ctypes.POINTER(TimeParams), _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                   _VP, _VP]),
}

_lib = None


def load():
    """Load the shared library (ImportError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2505_14538_b300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_params() -> Params:
    p = Params()
    load().swift_gpu_default_params(ctypes.byref(p))
    return p


def default_time_params() -> TimeParams:
    tp = TimeParams()
    load().swift_gpu_default_time_params(ctypes.byref(tp))
    return tp
