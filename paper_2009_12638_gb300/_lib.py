"""ctypes binding of libms (include/ms.h): argument marshalling only.

Every computation happens in the CUDA library.  If libms.so is missing or
cannot be loaded this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libms.so")

MS_OK = 0
MS_ERR_ARG = 1
MS_ERR_CUDA = 2
MS_ERR_OOM = 3
MS_ERR_NOT_CONVERGED = 4
MS_ERR_TIMEOUT = 5
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_CONVERGED", 5: "ERR_TIMEOUT"}

MODE = {"sync": 0, "async": 1}
PRECISION = {"fp64": 0, "mixed": 1}

# Symbols declared in include/ms.h (checked by the CPU tests).
EXPORTS = ("ms_boundary_size", "ms_default_opts", "ms_create_grid", "ms_partition", "ms_get_cuts", "ms_solve",
           "ms_solve_host", "ms_residual", "ms_face_gather", "ms_destroy", "ms_last_error",
           "ms_residual_noalloc", "ms_resident_variant", "ms_gcg_solve", "ms_norms", "ms_sweep")
NOALLOC_MAX_RHS = 1024


class TraceRec(ctypes.Structure):
    _fields_ = [
        ("sweep", ctypes.c_int),
        ("block", ctypes.c_int),
        ("rhs", ctypes.c_int),
        ("inner_its", ctypes.c_int),
        ("block_rr", ctypes.c_double),
        ("t_ns", ctypes.c_ulonglong),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("inner_rtol", ctypes.c_double),
        ("inner_maxit", ctypes.c_int),
        ("outer_tol", ctypes.c_double),
        ("outer_maxit", ctypes.c_int),
        ("time_limit_ms", ctypes.c_double),
        ("cluster", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("slots", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("slow_block", ctypes.c_int),
        ("slow_ns", ctypes.c_int),
        ("res_hist", ctypes.POINTER(ctypes.c_double)),
        ("profile", ctypes.c_int),
        ("persistent", ctypes.c_int),
        ("engine", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("inner_adapt", ctypes.c_int),
        ("overlap", ctypes.c_int),
        ("inner_method", ctypes.c_int),
        ("gmres_restart", ctypes.c_int),
        ("time_hist", ctypes.POINTER(ctypes.c_double)),
        ("wait_polls", ctypes.c_int),
        ("trace_cap", ctypes.c_int),
        ("trace", ctypes.POINTER(TraceRec)),
        ("sum_polls", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("outer_its", ctypes.c_int),
        ("inner_its", ctypes.c_longlong),
        ("lups", ctypes.c_longlong),
        ("rel_residual", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("launches", ctypes.c_int),
        ("cluster", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("slots", ctypes.c_int),
        ("per_rhs_outer_its", ctypes.POINTER(ctypes.c_int)),
        ("per_rhs_rel", ctypes.POINTER(ctypes.c_double)),
        ("sweep_ms", ctypes.c_double),
        ("sweep_launches", ctypes.c_int),
        ("engine", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("inner_rtol_final", ctypes.c_double),
        ("trace_count", ctypes.c_longlong),
    ]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libms.so (built by __graft_entry__.build() or paper_2009_12638_gb300._build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libms.so not found at {path}: build it first (python -m paper_2009_12638_gb300._build)")
        lib = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        c_int = ctypes.c_int
        lib.ms_boundary_size.argtypes = [c_int, c_int, c_int]
        lib.ms_boundary_size.restype = ctypes.c_longlong
        lib.ms_default_opts.argtypes = [ctypes.POINTER(Opts)]
        lib.ms_default_opts.restype = None
        lib.ms_create_grid.argtypes = [c_int, c_int, c_int, c_int, ctypes.POINTER(vp)]
        lib.ms_partition.argtypes = [vp, c_int, c_int, c_int, ip, ip, ip]
        lib.ms_get_cuts.argtypes = [vp, ip, ip, ip]
        lib.ms_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
        lib.ms_solve_host.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
        lib.ms_gcg_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
        lib.ms_residual.argtypes = [vp, vp, vp, vp, dp, vp]
        lib.ms_face_gather.argtypes = [vp, vp, vp, vp]
        lib.ms_norms.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.ms_sweep.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
        lib.ms_residual_noalloc.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.ms_resident_variant.argtypes = [c_int, ip, ip, ip, ip, ip, ip, ip]
        lib.ms_destroy.argtypes = [vp]
        lib.ms_last_error.argtypes = [vp]
        lib.ms_last_error.restype = ctypes.c_char_p
        for name in ("ms_create_grid", "ms_partition", "ms_get_cuts", "ms_solve", "ms_solve_host", "ms_residual",
                     "ms_face_gather", "ms_destroy", "ms_residual_noalloc", "ms_norms", "ms_sweep", "ms_gcg_solve"):
            getattr(lib, name).restype = c_int
        _lib = lib
        return lib


class MsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
