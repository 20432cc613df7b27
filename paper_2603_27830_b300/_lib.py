"""ctypes binding of ``libsgp4_b300.so`` (the C ABI declared in include/sgp4.h).

This module only loads the library and declares the entry points.  It raises if
the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsgp4_b300.so")

SGP4_OK = 0
SGP4_ERR_ARG = -1
SGP4_ERR_CUDA = -2
SGP4_ERR_OOM = -3
SGP4_ERR_TIMEOUT = -4
SGP4_FP64 = 0
SGP4_FP32 = 1

RESULT_NAMES = {0: "SGP4_OK", -1: "SGP4_ERR_ARG", -2: "SGP4_ERR_CUDA", -3: "SGP4_ERR_OOM",
                -4: "SGP4_ERR_TIMEOUT"}

# Every symbol include/sgp4.h declares (checked by the CPU tests).
EXPORTS = (
    "sgp4_version", "sgp4_wgs72", "sgp4_records_bytes", "sgp4_records_bind", "sgp4_init",
    "sgp4_propagate", "sgp4_propagate_jd", "sgp4_batch_workspace_bytes", "sgp4_batch_plan_init",
    "sgp4_propagate_batched", "sgp4_batch_graph_create", "sgp4_batch_graph_launch",
    "sgp4_batch_graph_destroy", "sgp4_propagate_batched_static", "sgp4_adjoint_workspace_bytes",
    "sgp4_adjoint", "sgp4_fit_workspace_bytes", "sgp4_fit_step", "sgp4_tle_parse",
    "sgp4_tle_parse_text", "sgp4_tle_format", "sgp4_jacobian_workspace_bytes", "sgp4_jacobian",
    "sgp4_omm_parse_text", "sgp4_omm_format",
)
STATIC_MAX_REQUESTS = 1024


class Sgp4Consts(ctypes.Structure):
    _fields_ = [("mu_km3s2", ctypes.c_double), ("radius_km", ctypes.c_double),
                ("j2", ctypes.c_double), ("j3", ctypes.c_double), ("j4", ctypes.c_double)]


class Sgp4Records(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("consts", Sgp4Consts)]


class Sgp4Request(ctypes.Structure):
    _fields_ = [("sat_offset", ctypes.c_int64), ("n", ctypes.c_int64),
                ("t_offset", ctypes.c_int64), ("t_count", ctypes.c_int64),
                ("out_offset", ctypes.c_int64)]


class Sgp4BatchPlan(ctypes.Structure):
    _fields_ = [("workspace", ctypes.c_void_p), ("n_requests", ctypes.c_int32),
                ("tile_states", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("total_tiles", ctypes.c_int64),
                ("total_states", ctypes.c_int64), ("sats_needed", ctypes.c_int64),
                ("tsince_needed", ctypes.c_int64), ("out_needed", ctypes.c_int64)]


class Sgp4Error(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {RESULT_NAMES.get(code, code)}")
        self.code = code


_lock = threading.Lock()
_lib = None


def _declare(lib):
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    R = ctypes.POINTER(Sgp4Records)
    lib.sgp4_version.restype = I32
    lib.sgp4_wgs72.restype = Sgp4Consts
    lib.sgp4_records_bytes.argtypes = [I64]
    lib.sgp4_records_bytes.restype = ctypes.c_size_t
    lib.sgp4_records_bind.argtypes = [P, ctypes.c_size_t, I64, ctypes.POINTER(Sgp4Consts), R]
    lib.sgp4_records_bind.restype = I32
    lib.sgp4_init.argtypes = [P, P, P, I64, R, P, P]
    lib.sgp4_init.restype = I32
    lib.sgp4_propagate.argtypes = [R, P, I64, I32, I32, P, P, P, P, P]
    lib.sgp4_propagate.restype = I32
    lib.sgp4_propagate_jd.argtypes = [R, P, P, I64, I32, P, P, P, P, P]
    lib.sgp4_propagate_jd.restype = I32
    BP = ctypes.POINTER(Sgp4BatchPlan)
    lib.sgp4_batch_workspace_bytes.argtypes = [ctypes.c_int32]
    lib.sgp4_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.sgp4_batch_plan_init.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                         ctypes.c_size_t, BP, P]
    lib.sgp4_batch_plan_init.restype = I32
    lib.sgp4_propagate_batched.argtypes = [BP, R, P, I64, I32, P, P, P, I64, P, P]
    lib.sgp4_propagate_batched.restype = I32
    lib.sgp4_batch_graph_create.argtypes = [BP, R, P, I64, I32, P, P, P, I64, P, P,
                                            ctypes.POINTER(ctypes.c_void_p)]
    lib.sgp4_batch_graph_create.restype = I32
    lib.sgp4_batch_graph_launch.argtypes = [P, P]
    lib.sgp4_batch_graph_launch.restype = I32
    lib.sgp4_batch_graph_destroy.argtypes = [P]
    lib.sgp4_batch_graph_destroy.restype = I32
    lib.sgp4_propagate_batched_static.argtypes = [P, ctypes.c_int32, ctypes.c_int32, R, P, I64,
                                                  I32, P, P, P, I64, P]
    lib.sgp4_propagate_batched_static.restype = I32
    lib.sgp4_adjoint_workspace_bytes.argtypes = [I64]
    lib.sgp4_adjoint_workspace_bytes.restype = ctypes.c_size_t
    lib.sgp4_adjoint.argtypes = [P, R, P, I64, I32, I32, P, P, P, P, ctypes.c_size_t, P]
    lib.sgp4_adjoint.restype = I32
    lib.sgp4_fit_workspace_bytes.argtypes = [I64]
    lib.sgp4_fit_workspace_bytes.restype = ctypes.c_size_t
    lib.sgp4_fit_step.argtypes = [P, R, P, I64, I32, I32, P, P, P, P, P, ctypes.c_size_t, P]
    lib.sgp4_fit_step.restype = I32
    lib.sgp4_jacobian_workspace_bytes.argtypes = [I64]
    lib.sgp4_jacobian_workspace_bytes.restype = ctypes.c_size_t
    lib.sgp4_jacobian.argtypes = [P, R, P, I64, I32, I32, P, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.sgp4_jacobian.restype = I32
    CP = ctypes.c_char_p
    lib.sgp4_tle_parse.argtypes = [CP, CP, P, P, P, P]
    lib.sgp4_tle_parse.restype = I32
    lib.sgp4_tle_parse_text.argtypes = [CP, ctypes.c_size_t, I64, P, P, P, P, P]
    lib.sgp4_tle_parse_text.restype = I64
    lib.sgp4_tle_format.argtypes = [P, I32, ctypes.c_double, I32, P, P]
    lib.sgp4_tle_format.restype = I32
    lib.sgp4_omm_parse_text.argtypes = [CP, ctypes.c_size_t, I64, P, P, P, P, P]
    lib.sgp4_omm_parse_text.restype = I64
    lib.sgp4_omm_format.argtypes = [P, I32, ctypes.c_double, I32, CP, P, ctypes.c_size_t]
    lib.sgp4_omm_format.restype = I32
    return lib


def load(path: str | None = None):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None or path is not None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"{p} is missing: build it with "
                                   "`python -m paper_2603_27830_b300.build`")
            lib = _declare(ctypes.CDLL(p))
            if path is not None:
                return lib
            _lib = lib
        return _lib


def check(fn: str, code: int) -> None:
    if code != SGP4_OK:
        raise Sgp4Error(fn, code)
