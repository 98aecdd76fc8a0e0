"""ctypes binding of the C ABI in include/radix_gb300.h (argument marshalling only).

Every step of a sort runs in the CUDA library; there is no CPU fallback: if the library
cannot be built or loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

RS_STATUS = {
    0: "RS_OK", 1: "RS_ERR_INVALID_ARG", 2: "RS_ERR_MISALIGNED", 3: "RS_ERR_OVERLAP", 4: "RS_ERR_TOO_LARGE",
    5: "RS_ERR_NO_MEMORY", 6: "RS_ERR_CUDA", 7: "RS_ERR_DEVICE_TIMEOUT", 8: "RS_ERR_QUEUE_OVERFLOW",
    9: "RS_ERR_UNSUPPORTED", 10: "RS_ERR_INTERNAL",
}

# name -> (restype, argtypes) for every entry point of include/radix_gb300.h
_vp, _u64, _u32, _i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int


class RsPlan(ctypes.Structure):
    _fields_ = [("digit_bits_max", ctypes.c_uint32), ("tile_records", ctypes.c_uint32),
                ("chunk_records", ctypes.c_uint32), ("sm_limit", ctypes.c_uint32),
                ("watchdog_polls", ctypes.c_uint32), ("tiny_records", ctypes.c_uint32),
                ("enum_records", ctypes.c_uint32)]


class RsKernelTime(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_uint32), ("level", ctypes.c_uint32), ("ms", ctypes.c_float)]


KERNEL_NAMES = {0: "init", 1: "hist", 2: "hist_redo", 3: "scatter", 4: "classify", 5: "chunk", 6: "copy", 7: "tiny"}

SIGNATURES = {
    "radix_sort": (_i32, [_vp, _vp, _u64, _u32, _u32, _vp]),
    "radix_sort_host": (_i32, [_vp, _vp, _vp, _vp, _u64, _u32, _u32, _vp]),
    "radix_sort_segmented": (_i32, [_vp, _vp, _vp, _u64, _u64, _u32, _u32, _vp]),
    "radix_partition": (_i32, [_vp, _vp, _u64, _u32, _u32, _u32, _u32, _vp]),
    "radix_histogram": (_i32, [_vp, _u64, _u32, _u32, _u32, _u32, _vp, _vp]),
    "radix_count_runs": (_i32, [_vp, _u64, _u32, _u32, _vp, _vp, _vp, _vp]),
    "radix_sort_status": (_i32, [_vp]),
    "radix_sort_strerror": (ctypes.c_char_p, [_i32]),
    "radix_sort_release": (_i32, []),
    "radix_sort_set_plan": (_i32, [ctypes.POINTER(RsPlan)]),
    "radix_sort_get_plan": (_i32, [ctypes.POINTER(RsPlan)]),
    "radix_sort_launch_count": (_u64, []),
    "radix_sort_chunk_records": (_u32, [_u32]),
    "radix_sort_workspace_bytes": (_u64, [_u64, _u32, _u32, _u64]),
    "radix_sort_reserve": (_i32, [_u64, _u32, _u32, _u64, _vp]),
    "radix_sort_test_inject": (_i32, [_u32]),
    "radix_sort_noalloc": (_i32, [_vp, _vp, _u64, _u32, _u32, _vp, _vp]),
    "radix_sort_profile": (_i32, [_i32]),
    "radix_sort_profile_kernels": (_i32, [ctypes.c_uint32]),
    "radix_sort_profile_read": (ctypes.c_int64, [ctypes.POINTER(RsKernelTime), ctypes.c_int64]),
}

_lock = threading.Lock()
_L = None


class RadixSortError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        self.name = RS_STATUS.get(code, f"status {code}")
        msg = f"{where}: {self.name}" if where else self.name
        try:
            msg += f" ({lib().radix_sort_strerror(code).decode()})"
        except Exception:
            pass
        super().__init__(msg)


def lib(build_if_missing: bool = True):
    """The loaded shared library (built in-tree with nvcc if missing or stale)."""
    global _L
    with _lock:
        if _L is None:
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is missing; build it with paper_1703_00687_gb300.build.build()")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _L = L
        return _L


def check(code: int, where: str = "") -> None:
    if code != 0:
        raise RadixSortError(code, where)
