"""ctypes view of libroots (include/rootdensity.h): structs, signatures, errors.

Argument marshalling only. Loading fails loudly when the library has not been
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

RD_OK, RD_EINVAL, RD_ECUDA, RD_EUNSUPPORTED = 0, -1, -2, -3
STATUS_OK, STATUS_NOT_CONVERGED, STATUS_REJECTED, STATUS_DEGENERATE = 0, 1, 2, 3
C64, C128 = 0, 1
PLAIN_FP64, MIXED = 0, 1
SHIFT_WILKINSON, SHIFT_RAYLEIGH = 0, 1
POLISH_FP64, POLISH_DF = 0, 1
L2_FP64, L2_DF = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int32), ("shift", ctypes.c_int32),
                ("exc_period", ctypes.c_int32), ("polish_steps", ctypes.c_int32),
                ("residual_tol", ctypes.c_double), ("collapse_tol", ctypes.c_double),
                ("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("polish_extra", ctypes.c_int32), ("fixed_sweeps", ctypes.c_int32),
                ("polish_mode", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("polish_warps", ctypes.c_int32), ("ring_slots", ctypes.c_int32)]


class Window(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double)]


class Clip(ctypes.Structure):
    _fields_ = [("centres", ctypes.c_void_p), ("radius", ctypes.c_double), ("tile_index", ctypes.c_void_p),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tiles", Window)]


class UnevenTuning(ctypes.Structure):
    # indexed by degree (1..12 used)
    _fields_ = [("block", ctypes.c_int32 * 16), ("ctas_per_sm", ctypes.c_int32 * 16), ("lanes", ctypes.c_int32 * 16),
                ("polish_warps", ctypes.c_int32 * 16)]


class FieldSpec(ctypes.Structure):
    _fields_ = [("tiles", Window), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("radius", ctypes.c_double),
                ("nr", ctypes.c_int32), ("degree", ctypes.c_int32), ("poly_degree", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("poly", ctypes.c_double * 26)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("polish_warps", ctypes.c_int32), ("ms", ctypes.c_float)]


class Tuning(ctypes.Structure):
    _fields_ = [("best", TuneEntry), ("one_role", TuneEntry), ("n_candidates", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


ABI_VERSION = 2
PEAK_FP32, PEAK_FP64 = 0, 1
F_SIN_CUBE, F_POLY = 0, 1
SPLAT_FP64, SPLAT_FP32 = 0, 1

STATS_FIELDS = ("polys", "status_ok", "status_not_converged", "status_rejected", "status_degenerate",
                "sweeps", "pair_updates", "rotations", "newton_steps", "binned", "out_of_window", "clipped",
                "flops_fp32", "flops_fp64", "wait_timeouts")
STATS_WORDS = len(STATS_FIELDS)  # uint64 words of rd_stats
STATIC_SCRATCH_BYTES = 32 * 1024 * 1024  # RD_STATIC_SCRATCH_BYTES

# entry point -> (restype, argtypes); every name here is declared in include/rootdensity.h
P, I32, I64, F64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "rd_ws_selftest_timeout": (I32, [P, I64, P, P, P]),
    "rd_abi_version": (I32, []),
    "rd_pointer_is_device_accessible": (I32, [P]),
    "rd_last_error": (ctypes.c_char_p, []),
    "rd_device_sm_count": (I32, []),
    "rd_default_params": (None, [I32, ctypes.POINTER(Params)]),
    "rd_roots_batched": (I32, [P, I32, I32, I64, I32, ctypes.POINTER(Params), P, P, P, P]),
    "rd_roots_density": (I32, [P, I32, I32, I64, I32, ctypes.POINTER(Params), ctypes.POINTER(Clip), Window,
                               I32, I32, P, P, P, P, P]),
    "rd_density_accumulate": (I32, [P, P, I64, I64, Window, I32, I32, ctypes.POINTER(Clip), P, P, P]),
    "rd_hist_clear": (I32, [P, I64, P]),
    "rd_roots_backward": (I32, [P, I32, I32, I64, P, P, P, P, P]),
    "rd_roots_backward_uneven": (I32, [P, I32, P, P, I64, I64, P, P, P, P, P]),
    "rd_autotune": (I32, [I32, I32, I32, I32, I64, I32, ctypes.POINTER(Tuning), ctypes.POINTER(TuneEntry), I32,
                          ctypes.POINTER(ctypes.c_int)]),
    "rd_alu_peak": (I32, [I32, I64, I32, P, ctypes.POINTER(ctypes.c_uint64), P]),
    "rd_uneven_workspace_bytes": (SZ, [I64, I64, I32]),
    "rd_roots_uneven": (I32, [P, I32, P, P, I64, I64, I32, ctypes.POINTER(Params), ctypes.POINTER(UnevenTuning),
                              ctypes.POINTER(Window), I32, I32, P, P, P, P, P, SZ, P]),
    "rd_roots_uneven_static": (I32, [P, I32, P, P, I64, I64, I32, ctypes.POINTER(Params),
                                     ctypes.POINTER(UnevenTuning), ctypes.POINTER(Window), I32, I32, P, P, P, P, P]),
    "rd_l2_nodes": (I32, [I32, I32, P, P, P]),
    "rd_l2_approx": (I32, [P, I64, I32, I32, I32, I32, P, F64, P, ctypes.POINTER(Clip), P]),
    "rd_splat": (I32, [P, I64, Window, I32, I32, F64, F64, I32, P, P]),
    "rd_splat_backward": (I32, [P, I64, Window, I32, I32, F64, F64, I32, P, P, P]),
    "rd_field_density": (I32, [I32, ctypes.POINTER(FieldSpec), I32, ctypes.POINTER(Params), Window, I32, I32, P, P,
                               P, P, P, P]),
}

_lock = threading.Lock()
_lib = None


class RootDensityError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed ({code}): {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libroots.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if build_if_missing and _build.stale():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libroots.so not found at {path}: run paper_2507_02164_gb300.build.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            if L.rd_abi_version() != ABI_VERSION:
                raise RuntimeError(f"libroots ABI version {L.rd_abi_version()}, binding expects {ABI_VERSION}")
            _lib = L
    return _lib


def call(name: str, *args) -> int:
    L = load()
    rc = getattr(L, name)(*args)
    if rc is not None and rc != RD_OK:
        msg = L.rd_last_error()
        raise RootDensityError(name, rc, msg.decode() if msg else "")
    return rc


def default_params(mode: int) -> Params:
    p = Params()
    load().rd_default_params(mode, ctypes.byref(p))
    return p
