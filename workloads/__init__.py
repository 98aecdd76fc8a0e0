"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

Holds no sorting arithmetic: it only draws records (see gen.c for the generators and
their published definitions).  Records are ``rec_size``-byte rows of 8-byte
little-endian words; the key is the first ``key_size`` bytes.

The C library is compiled on first use (gcc) into ``workloads/_build``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_OUT = os.path.join(_HERE, "_build", "libworkloads.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (atomic rename, safe under parallel pytest)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_OUT))
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread", "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u8p, u64, u32, i32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
        L.wl_u64.restype = u64
        L.wl_u64.argtypes = [u64, u64, u64]
        L.wl_fill_uniform.restype = i32
        L.wl_fill_uniform.argtypes = [u8p, u64, u32, u32, u64, u64, i32]
        L.wl_fill_zipf.restype = i32
        L.wl_fill_zipf.argtypes = [u8p, u64, u32, u64, dbl, u64, u64, i32]
        L.wl_zipf_rank.restype = u64
        L.wl_zipf_rank.argtypes = [u64, u64, dbl, u64]
        L.wl_zipf_key_of_rank.restype = u64
        L.wl_zipf_key_of_rank.argtypes = [u64, u64]
        L.wl_kmer_table.restype = i32
        L.wl_kmer_table.argtypes = [u64, u32, ctypes.c_void_p]
        L.wl_fill_kmer.restype = i32
        L.wl_fill_kmer.argtypes = [u8p, u64, u32, u64, u32, u64, i32, ctypes.c_void_p]
        L.wl_log_uniform.restype = i32
        L.wl_log_uniform.argtypes = [ctypes.c_void_p, u64, u64, u64, u64]
        L.wl_exponential.restype = i32
        L.wl_exponential.argtypes = [ctypes.c_void_p, u64, dbl, u64]
        L.wl_uniform_below.restype = i32
        L.wl_uniform_below.argtypes = [ctypes.c_void_p, u64, u64, u64, u64]
        _lib = L
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _target(n: int, rec_size: int, out):
    """Return (array-or-None, address) of an n x rec_size byte destination."""
    if out is None:
        arr = np.empty((n, rec_size), dtype=np.uint8)
        return arr, arr.ctypes.data
    if isinstance(out, int):
        return None, out
    if hasattr(out, "data_ptr"):            # a torch tensor (e.g. pinned host memory)
        assert out.numel() * out.element_size() >= n * rec_size
        return out, out.data_ptr()
    assert out.nbytes >= n * rec_size and out.flags["C_CONTIGUOUS"]
    return out, out.ctypes.data


def uniform(n, rec_size, key_size, seed, first=0, out=None):
    arr, ptr = _target(n, rec_size, out)
    if lib().wl_fill_uniform(ptr, n, rec_size, key_size, seed, first, _threads()) != 0:
        raise ValueError("bad uniform workload arguments")
    return arr


def zipf(n, rec_size, seed, s=1.0, n_ranks=2 ** 32, first=0, out=None):
    arr, ptr = _target(n, rec_size, out)
    if lib().wl_fill_zipf(ptr, n, rec_size, seed, s, n_ranks, first, _threads()) != 0:
        raise ValueError("bad zipf workload arguments")
    return arr


def zipf_ranks(seed, idx, s=1.0, n_ranks=2 ** 32):
    L = lib()
    return np.array([L.wl_zipf_rank(seed, int(i), s, n_ranks) for i in idx], dtype=np.uint64)


def zipf_key_of_rank(seed, rank):
    return int(lib().wl_zipf_key_of_rank(seed, rank))


def kmer_table(seed, prefixes=1024):
    t = np.empty(prefixes, dtype=np.uint64)
    lib().wl_kmer_table(seed, prefixes, t.ctypes.data)
    return t


def kmer(n, rec_size, seed, prefixes=1024, first=0, out=None):
    arr, ptr = _target(n, rec_size, out)
    scratch = np.empty(prefixes, dtype=np.uint64)
    if lib().wl_fill_kmer(ptr, n, rec_size, seed, prefixes, first, _threads(), scratch.ctypes.data) != 0:
        raise ValueError("bad kmer workload arguments")
    return arr


def log_uniform(m, lo, hi, seed):
    out = np.empty(m, dtype=np.uint64)
    if lib().wl_log_uniform(out.ctypes.data, m, lo, hi, seed) != 0:
        raise ValueError("bad log-uniform arguments")
    return out


def exponential(m, rate, seed):
    out = np.empty(m, dtype=np.float64)
    if lib().wl_exponential(out.ctypes.data, m, rate, seed) != 0:
        raise ValueError("bad exponential arguments")
    return out


def uniform_below(m, bound, seed, stream=7):
    out = np.empty(m, dtype=np.uint64)
    if lib().wl_uniform_below(out.ctypes.data, m, bound, seed, stream) != 0:
        raise ValueError("bad bound")
    return out


def batched_sizes(n_segs=100_000, lo=1, hi=1_000_000, cap=2_000_000_000, seed=5):
    """Segment sizes of the batched workload.

    Sizes are log-uniform in [lo, hi].  If their sum exceeds ``cap``, every size is scaled
    by cap/sum (floor, at least 1), which keeps the instance count and the log-uniform
    shape.
    """
    s = log_uniform(n_segs, lo, hi, seed)
    total = int(s.sum(dtype=np.uint64))
    if total > cap:
        f = cap / total
        s = np.maximum(1, np.floor(s.astype(np.float64) * f)).astype(np.uint64)
    return s


# --------------------------------------------------------------------------- configs
# The synthetic workloads, shaped like the paper's experiments (16-byte records with an
# 8-byte key and 8-byte data, uniform and Zipf keys; 16-byte keys as in the k-mer use).
CONFIGS = {
    "uniform_1e6_r8": dict(n=1_000_000, rec_size=8, key_size=8, kind="uniform", seed=1),
    "uniform_1e9_r16": dict(n=1_000_000_000, rec_size=16, key_size=8, kind="uniform", seed=2),
    "zipf_1e9_r16": dict(n=1_000_000_000, rec_size=16, key_size=8, kind="zipf", seed=3),
    "kmer_5e8_r24": dict(n=500_000_000, rec_size=24, key_size=16, kind="kmer", seed=4),
}


def make(kind, n, rec_size, key_size, seed, first=0, out=None):
    if kind == "uniform":
        return uniform(n, rec_size, key_size, seed, first=first, out=out)
    if kind == "zipf":
        assert key_size == 8
        return zipf(n, rec_size, seed, first=first, out=out)
    if kind == "kmer":
        assert key_size == 16
        return kmer(n, rec_size, seed, first=first, out=out)
    raise ValueError(kind)


def harmonic(n: int, s: float = 1.0) -> float:
    """Generalised harmonic number H_{n,s} (Euler-Maclaurin for large n)."""
    if n < 100000:
        return float(sum(k ** -s for k in range(1, n + 1)))
    m = 10000
    head = sum(k ** -s for k in range(1, m))
    if s == 1.0:
        tail = math.log(n / m) + 0.5 / m + 0.5 / n - 1.0 / (12 * m * m) + 1.0 / (12 * n * n)
    else:
        tail = (n ** (1 - s) - m ** (1 - s)) / (1 - s) + 0.5 * (m ** -s + n ** -s)
    return head + tail
