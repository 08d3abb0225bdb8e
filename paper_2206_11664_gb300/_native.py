"""ctypes declarations of the C ABI in include/sd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsd.so")

c_int, c_i64, c_dbl, c_vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P_u64 = ctypes.POINTER(ctypes.c_uint64)
P_i64 = ctypes.POINTER(ctypes.c_int64)
P_dbl = ctypes.POINTER(ctypes.c_double)
P_i32 = ctypes.POINTER(ctypes.c_int32)
P_u8 = ctypes.POINTER(ctypes.c_uint8)

SD_OK, SD_EINVAL, SD_ENOMEM, SD_ECUDA, SD_ENOPLAN, SD_ETIMEOUT, SD_EINTERNAL = range(7)
SD_C64, SD_C128 = 0, 1
STATUS_NAMES = {0: "SD_OK", 1: "SD_EINVAL", 2: "SD_ENOMEM", 3: "SD_ECUDA", 4: "SD_ENOPLAN",
                5: "SD_ETIMEOUT", 6: "SD_EINTERNAL"}


class PlanOpts(ctypes.Structure):
    _fields_ = [("skip_rule", c_int), ("tile_bits", c_int), ("jit", c_int), ("grouping", c_int),
                ("layout", c_int), ("prefetch", c_int), ("reserved", c_int * 2)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best_k", c_int), ("best_layout", c_int), ("best_prefetch", c_int), ("ms", (c_dbl * 5) * 4)]


class PlanView(ctypes.Structure):
    _fields_ = [("n", c_int), ("m", c_i64), ("n_groups", c_i64),
                ("group_offsets", P_i64), ("group_terms", P_i64), ("masks", P_u64),
                ("signs", P_u8), ("gate_offsets", P_i64), ("gates", P_i32),
                ("cnot_cols", P_u64), ("cnot_inv_cols", P_u64)]


class ScheduleStats(ctypes.Structure):
    _fields_ = [("tile_bits", c_int), ("passes_per_step", c_i64), ("rounds_per_step", c_i64),
                ("diag_passes", c_i64), ("onchip", c_int)]


# name -> (restype, argtypes); every symbol here is declared in include/sd.h
SIGNATURES = {
    "sd_create": (c_int, [c_int, c_i64, P_u64, P_u64, P_dbl, ctypes.POINTER(c_vp)]),
    "sd_create_str": (c_int, [c_int, c_i64, ctypes.POINTER(ctypes.c_char_p), P_dbl,
                              ctypes.POINTER(c_vp)]),
    "sd_set_coeffs": (c_int, [c_vp, P_dbl]),
    "sd_plan": (c_int, [c_vp, ctypes.POINTER(PlanOpts)]),
    "sd_get_plan": (c_int, [c_vp, ctypes.POINTER(PlanView)]),
    "sd_get_schedule": (c_int, [c_vp, c_int, c_int, ctypes.POINTER(ScheduleStats)]),
    "sd_prepare": (c_int, [c_vp, c_int, c_dbl, c_i64, c_int]),
    "sd_autotune": (c_int, [c_vp, c_int, c_dbl, c_i64, c_int, c_int, c_int, ctypes.POINTER(c_int), P_dbl]),
    "sd_autotune_shape": (c_int, [c_vp, c_int, c_dbl, c_i64, c_int, c_int, c_int, ctypes.POINTER(TuneResult)]),
    "sd_evolve_host": (c_int, [c_vp, c_vp, c_vp, c_int, c_dbl, c_i64, c_int, c_vp]),
    "sd_precompile": (c_int, [c_vp, c_int, c_i64, c_int, ctypes.POINTER(c_i64)]),
    "sd_count_passes": (c_int, [c_vp, c_int, c_int, c_i64, ctypes.POINTER(c_i64)]),
    "sd_evolve": (c_int, [c_vp, c_vp, c_int, c_dbl, c_i64, c_int, c_vp]),
    "sd_evolve_observe": (c_int, [c_vp, c_vp, c_int, c_dbl, c_i64, c_int, c_i64, P_u64, P_u64,
                                  P_dbl, c_vp, c_vp]),
    "sd_evolve_pauli": (c_int, [c_vp, c_vp, c_int, c_dbl, c_i64, c_int, c_vp]),
    "sd_expect": (c_int, [c_vp, c_vp, c_int, c_i64, P_u64, P_u64, P_dbl, P_dbl, c_vp]),
    "sd_grad": (c_int, [c_vp, c_vp, c_int, c_dbl, c_i64, c_int, c_i64, P_u64, P_u64, P_dbl,
                        P_dbl, P_dbl, c_vp]),
    "sd_evolve_batch": (c_int, [ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_i64, c_int, c_dbl,
                                c_i64, c_int, c_vp]),
    "sd_prepare_batch": (c_int, [ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), c_i64, c_int, c_dbl,
                                 c_i64, c_int]),
    "sd_expect_noalloc": (c_int, [c_int, c_vp, c_int, c_i64, P_u64, P_u64, P_dbl, P_dbl, c_vp]),
    "sd_last_error": (ctypes.c_char_p, [c_vp]),
    "sd_destroy": (None, [c_vp]),
}

_lib = None


def load():
    """Load libsd.so; raises if the native library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"native library {LIB_PATH} is missing: build it with "
                "`python -m paper_2206_11664_gb300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
