"""ctypes declarations of the libbrr C ABI (include/brr.h).

Argument marshalling only: every step of every call runs in the CUDA
library.  There is no fallback: if ``libbrr.so`` has not been built, loading
fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbrr.so")
SCHED_KMAX = 8

u64, u32, i32, vp = C.c_uint64, C.c_uint32, C.c_int, C.c_void_p

BRR_OK, BRR_EINVAL, BRR_ENOMEM, BRR_ECUDA, BRR_ERETRY, BRR_ETIMEOUT, BRR_ENODEV = range(7)


class Schedule(C.Structure):
    _fields_ = [("n_k", u64 * (SCHED_KMAX + 1)), ("k_max", u32)]


class Segment(C.Structure):
    _fields_ = [("g0", u64), ("count", u64), ("u", u64), ("i0", u32), ("k", u32)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "brr_schedule_paper": (None, [C.POINTER(Schedule)]),
    "brr_shuffle_plan": (i32, [u64, u64, C.POINTER(Schedule), C.POINTER(Segment), u32,
                               C.POINTER(u32), C.POINTER(u64)]),
    "brr_status_str": (C.c_char_p, [i32]),
    "brr_version": (C.c_char_p, []),
    "brr_create": (i32, [C.POINTER(vp)]),
    "brr_destroy": (i32, [vp]),
    "brr_last_device_error": (i32, [vp, vp]),
    "brr_reserve": (i32, [vp, u64, u64]),
    "brr_dice": (i32, [vp, vp, vp, u64, u64, u64, vp, vp]),
    "brr_dice_fixed": (i32, [vp, u64, u32, u64, u64, vp, vp]),
    "brr_shuffle": (i32, [vp, vp, u64, u32, u64, C.POINTER(Schedule), vp, vp]),
    "brr_shuffle_batched": (i32, [vp, vp, vp, u32, u32, vp, u64, C.POINTER(Schedule), vp]),
    "brr_set_swap_method": (i32, [vp, u32]),
    "brr_tune": (i32, [vp, u32, u64]),
    "brr_tune_get": (i32, [vp, u32, C.POINTER(u64)]),
    "brr_calibrate": (i32, [vp, C.POINTER(C.c_double), vp]),
    "brr_shuffle_naive": (i32, [vp, vp, u64, u32, u64, C.POINTER(Schedule), vp, vp]),
    "brr_schedule_naive2": (None, [C.POINTER(Schedule)]),
    "brr_schedule_l32": (None, [C.POINTER(Schedule)]),
    "brr_shuffle_words": (i32, [vp, u32, vp, u64, u32, u64, C.POINTER(Schedule), vp, vp]),
    "brr_dice_fixed_words": (i32, [vp, u32, u64, u32, u64, u64, vp, vp]),
    "brr_dice_words": (i32, [vp, u32, vp, vp, u64, u64, u64, vp, vp]),
    "brr_shuffle_batched_words": (i32, [vp, u32, vp, vp, u32, u32, vp, u64, C.POINTER(Schedule), vp]),
    "brr_sample": (i32, [vp, u64, u32, u64, C.POINTER(Schedule), vp, vp]),
    "brr_sample_batched": (i32, [vp, vp, vp, vp, vp, u32, u32, C.POINTER(Schedule), vp, vp]),
    "brr_selftest_threshold": (i32, [vp, vp, u64, vp]),
    "brr_selftest_barrier_timeout": (i32, [vp, u64, vp]),
    "brr_selftest_attempt_limit": (i32, [vp, u32]),
    "brr_shuffle_noalloc": (i32, [vp, u64, u32, u64, C.POINTER(Schedule), vp, vp, vp]),
}


def lib():
    """Load libbrr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)
