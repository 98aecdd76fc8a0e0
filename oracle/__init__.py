"""ORACLE — test infrastructure only (see oracle.c for what it computes and why).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It is independent of the GPU sorter: it shares no code with it and never
imports it.

Inputs and outputs are numpy uint8 arrays of shape (n, rec_size).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_OUT))
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.oracle_partition_bits.restype = i32
        L.oracle_partition_bits.argtypes = [vp, vp, u64, u32, u32, u32, u32]
        L.oracle_histogram_bits.restype = i32
        L.oracle_histogram_bits.argtypes = [vp, u64, u32, u32, u32, u32, vp]
        L.oracle_lsd_sort.restype = i32
        L.oracle_lsd_sort.argtypes = [vp, vp, u64, u32, u32]
        L.oracle_sort_segmented.restype = i32
        L.oracle_sort_segmented.argtypes = [vp, vp, vp, u64, u32, u32]
        L.oracle_count_runs.restype = i32
        L.oracle_count_runs.argtypes = [vp, u64, u32, u32, vp, vp, vp]
        _lib = L
    return _lib


def _records(a: np.ndarray) -> np.ndarray:
    assert a.dtype == np.uint8 and a.ndim == 2, "records are a (n, rec_size) uint8 array"
    return np.ascontiguousarray(a)


def sort(records: np.ndarray, key_size: int) -> np.ndarray:
    """Stable LSD radix sort by the little-endian key in bytes [0, key_size)."""
    buf = _records(records).copy()
    n, r = buf.shape
    tmp = np.empty_like(buf)
    if lib().oracle_lsd_sort(buf.ctypes.data, tmp.ctypes.data, n, r, key_size) != 0:
        raise ValueError("bad oracle_lsd_sort arguments")
    return buf


def partition(records: np.ndarray, key_size: int, lo: int, width: int) -> np.ndarray:
    """One stable counting-sort phase on the digit made of key bits [lo, lo + width)."""
    src = _records(records)
    n, r = src.shape
    dst = np.empty_like(src)
    if lib().oracle_partition_bits(src.ctypes.data, dst.ctypes.data, n, r, key_size, lo, width) != 0:
        raise ValueError("bad oracle_partition_bits arguments")
    return dst


def histogram(records: np.ndarray, key_size: int, lo: int, width: int) -> np.ndarray:
    src = _records(records)
    n, r = src.shape
    counts = np.zeros(1 << width, dtype=np.uint64)
    if lib().oracle_histogram_bits(src.ctypes.data, n, r, key_size, lo, width, counts.ctypes.data) != 0:
        raise ValueError("bad oracle_histogram_bits arguments")
    return counts


def sort_segmented(records: np.ndarray, offsets: np.ndarray, key_size: int) -> np.ndarray:
    buf = _records(records).copy()
    n, r = buf.shape
    tmp = np.empty_like(buf)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    if lib().oracle_sort_segmented(buf.ctypes.data, tmp.ctypes.data, off.ctypes.data, len(off) - 1, r, key_size) != 0:
        raise ValueError("bad oracle_sort_segmented arguments")
    return buf


def sort_inplace_raw(ptr: int, tmp_ptr: int, n: int, rec_size: int, key_size: int) -> None:
    """Sort n records at host address ptr (tmp_ptr: scratch of the same size)."""
    if lib().oracle_lsd_sort(ptr, tmp_ptr, n, rec_size, key_size) != 0:
        raise ValueError("bad oracle_lsd_sort arguments")


def count_runs(records: np.ndarray, key_size: int):
    """Runs of equal keys in consecutive records: (first record of each run, run lengths)."""
    src = _records(records)
    n, r = src.shape
    first = np.empty((max(n, 1), r), dtype=np.uint8)
    counts = np.zeros(max(n, 1), dtype=np.uint64)
    nruns = np.zeros(1, dtype=np.uint64)
    if lib().oracle_count_runs(src.ctypes.data, n, r, key_size, first.ctypes.data, counts.ctypes.data,
                               nruns.ctypes.data) != 0:
        raise ValueError("bad oracle_count_runs arguments")
    m = int(nruns[0])
    return first[:m], counts[:m]
