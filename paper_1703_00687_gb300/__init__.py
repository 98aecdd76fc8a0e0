"""GB300-native MSD radix sorting of fixed-size records.

The method is RADULS2 (Kokot, Deorowicz, Dlugosz, "Even faster sorting of (not only)
integers"): an MSD radix sort that distributes records by key digits and sorts small bins
on chip.  Everything runs in the CUDA library ``libradix_gb300.so`` (C ABI in
``include/radix_gb300.h``); this module only marshals arguments.  PyTorch provides device
memory and streams.

Records are rows of a contiguous tensor: a 2-D tensor of shape (n, k) holds n records of
k * element_size bytes; a 1-D 8-byte tensor holds n records of 8 bytes.  The key is the
first ``key_size`` bytes of a record, read as a little-endian unsigned integer.
"""
from __future__ import annotations

import ctypes

from ._lib import KERNEL_NAMES, RadixSortError, RsKernelTime, RsPlan, check, lib

__all__ = ["sort", "sort_host", "sort_segmented", "partition", "histogram", "count_runs", "status", "release", "set_plan",
           "get_plan", "launch_count", "chunk_records", "workspace_bytes", "reserve",
           "profile", "RadixSortError", "lib", "SortGraph"]


def _torch():
    import torch
    return torch


def _rec_size(t) -> int:
    if t.dim() == 1:
        return t.element_size()
    if t.dim() != 2:
        raise ValueError("records must be a 1-D or 2-D tensor")
    return t.shape[1] * t.element_size()


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t, what):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor")


def sort(records, key_size: int, tmp=None, stream=None):
    """Sort records by key (stable), in place; returns ``records``.

    CUDA tensor: sorted on its device, asynchronously on ``stream`` (default: the current
    stream).  CPU tensor: copied to the current CUDA device, sorted there, and copied back
    (synchronously); pinned memory makes the copies faster.
    ``tmp``: optional scratch of the same size on the same device.
    """
    torch = _torch()
    if records.device.type == "cpu":
        return sort_host(records, key_size, d_tmp=tmp, stream=stream)
    _need_cuda(records, "records")
    n = records.shape[0]
    if tmp is None:
        tmp = torch.empty_like(records)
    _need_cuda(tmp, "tmp")
    check(lib().radix_sort(records.data_ptr(), tmp.data_ptr(), n, _rec_size(records), key_size, _stream(stream)),
          "radix_sort")
    return records


def sort_host(h_in, key_size: int, h_out=None, d_buf=None, d_tmp=None, stream=None):
    """Sort host records through the GPU with one ``radix_sort_host`` call: copy ``h_in`` to
    the device, sort, copy back, all on ``stream``.

    The result goes to ``h_out`` (default: ``h_in`` itself).  ``d_buf``/``d_tmp``: optional
    device buffers of the same shape, reused across calls.  Pinned host tensors make the
    copies asynchronous.  Returns after the result is on the host.
    """
    torch = _torch()
    if h_in.is_cuda or (h_out is not None and h_out.is_cuda):
        raise ValueError("sort_host takes host tensors")
    if not h_in.is_contiguous() or (h_out is not None and (not h_out.is_contiguous() or h_out.shape != h_in.shape)):
        raise ValueError("host tensors must be contiguous and of the same shape")
    if d_buf is None:
        d_buf = torch.empty_like(h_in, device="cuda")
    if d_tmp is None:
        d_tmp = torch.empty_like(d_buf)
    _need_cuda(d_buf, "d_buf")
    _need_cuda(d_tmp, "d_tmp")
    nbytes = h_in.numel() * h_in.element_size()
    if d_buf.numel() * d_buf.element_size() < nbytes or d_tmp.numel() * d_tmp.element_size() < nbytes:
        raise ValueError("d_buf and d_tmp must hold the records")
    out = h_in if h_out is None else h_out
    s = torch.cuda.current_stream() if stream is None else stream
    n = h_in.shape[0] if h_in.dim() > 0 else 0
    check(lib().radix_sort_host(h_in.data_ptr(), out.data_ptr(), d_buf.data_ptr(), d_tmp.data_ptr(), n,
                                _rec_size(h_in), key_size, _stream(s)), "radix_sort_host")
    s.synchronize()
    return out


def sort_segmented(records, offsets, key_size: int, tmp=None, stream=None, total: int | None = None):
    """Sort each segment [offsets[s], offsets[s+1]) of ``records`` on its own, in place.

    ``offsets``: CUDA int64/uint64 tensor of n_segs + 1 non-decreasing record offsets,
    offsets[0] = 0, offsets[-1] = number of records.  ``total`` (= offsets[-1]) avoids a
    device read when given.
    """
    torch = _torch()
    _need_cuda(records, "records")
    _need_cuda(offsets, "offsets")
    if offsets.element_size() != 8:
        raise ValueError("offsets must be 64-bit")
    n_segs = offsets.numel() - 1
    if total is None:
        total = int(offsets[-1].item()) if n_segs >= 0 else 0
    if tmp is None:
        tmp = torch.empty_like(records)
    check(lib().radix_sort_segmented(records.data_ptr(), tmp.data_ptr(), offsets.data_ptr(), max(n_segs, 0), total,
                                     _rec_size(records), key_size, _stream(stream)), "radix_sort_segmented")
    return records


def partition(src, dst, key_size: int, bit_lo: int, width: int, stream=None):
    """One stable counting-sort pass: ``dst`` = ``src`` ordered by key bits [bit_lo, bit_lo+width)."""
    _need_cuda(src, "src")
    _need_cuda(dst, "dst")
    check(lib().radix_partition(src.data_ptr(), dst.data_ptr(), src.shape[0], _rec_size(src), key_size, bit_lo, width,
                                _stream(stream)), "radix_partition")
    return dst


def histogram(src, key_size: int, bit_lo: int, width: int, stream=None):
    """Counts of key bits [bit_lo, bit_lo+width) over the records (CUDA int64 tensor, 2^width)."""
    torch = _torch()
    _need_cuda(src, "src")
    out = torch.empty(1 << width, dtype=torch.int64, device=src.device)
    check(lib().radix_histogram(src.data_ptr(), src.shape[0], _rec_size(src), key_size, bit_lo, width, out.data_ptr(),
                                _stream(stream)), "radix_histogram")
    return out


def count_runs(records, key_size: int, stream=None):
    """Run-length count of equal keys in records already sorted by key (k-mer counting).

    Returns (first, counts): the first record of every run (CUDA tensor, runs x rec_size
    bytes) and the number of records in each run (CUDA int64 tensor).  Reads the number of
    runs back to the host (synchronises the stream)."""
    torch = _torch()
    _need_cuda(records, "records")
    n, R = records.shape[0], _rec_size(records)
    out = torch.empty((max(n, 1), R), dtype=torch.uint8, device=records.device)
    counts = torch.empty(max(n, 1), dtype=torch.int64, device=records.device)
    nruns = torch.zeros(1, dtype=torch.int64, device=records.device)
    check(lib().radix_count_runs(records.data_ptr(), n, R, key_size, out.data_ptr(), counts.data_ptr(),
                                 nruns.data_ptr(), _stream(stream)), "radix_count_runs")
    m = int(nruns.item())
    return out[:m], counts[:m]


def status(stream=None) -> int:
    """Drains the stream and returns the device-side status code of its calls (0 = ok)."""
    return lib().radix_sort_status(_stream(stream))


def check_status(stream=None) -> None:
    check(status(stream), "device status")


def release() -> None:
    check(lib().radix_sort_release(), "radix_sort_release")


def set_plan(digit_bits_max=0, tile_records=0, chunk_records=0, sm_limit=0, watchdog_polls=0, tiny_records=0,
             enum_records=0) -> None:
    """Sets the process-wide plan (speed only; 0 = automatic).  See ``rs_plan`` in the header."""
    p = RsPlan(digit_bits_max, tile_records, chunk_records, sm_limit, watchdog_polls, tiny_records, enum_records)
    check(lib().radix_sort_set_plan(ctypes.byref(p)), "radix_sort_set_plan")


def get_plan() -> dict:
    p = RsPlan()
    check(lib().radix_sort_get_plan(ctypes.byref(p)), "radix_sort_get_plan")
    return {f: getattr(p, f) for f, _ in RsPlan._fields_}


def launch_count() -> int:
    return int(lib().radix_sort_launch_count())


def workspace_bytes(n: int, rec_size: int, key_size: int, n_segs: int = 0) -> int:
    """Library workspace bytes a call of n records (n_segs segments) needs under the plan."""
    return int(lib().radix_sort_workspace_bytes(n, rec_size, key_size, n_segs))


def reserve(n: int, rec_size: int, key_size: int, n_segs: int = 0, stream=None) -> None:
    """Pre-allocates the workspace of ``stream`` for calls of up to n records / n_segs segments."""
    check(lib().radix_sort_reserve(n, rec_size, key_size, n_segs, _stream(stream)), "radix_sort_reserve")


def chunk_records(rec_size: int) -> int:
    """Largest bin (records) the current plan sorts in one on-chip pass."""
    return int(lib().radix_sort_chunk_records(rec_size))


class profile:
    """Context manager: per-kernel CUDA-event timings of the library's launches.

    ``with profile() as p: ...`` then ``p.records`` = [(kernel_name, level, ms), ...].
    ``kernels``: names (``KERNEL_NAMES`` values) to time; default all.
    """

    def __init__(self, kernels=None):
        ids = {v: k for k, v in KERNEL_NAMES.items()}
        self.mask = 0xFFFFFFFF if kernels is None else sum(1 << ids[k] for k in kernels)

    def __enter__(self):
        check(lib().radix_sort_profile_kernels(self.mask), "radix_sort_profile_kernels")
        check(lib().radix_sort_profile(1), "radix_sort_profile")
        self.records = []
        return self

    def __exit__(self, *exc):
        L = lib()
        L.radix_sort_profile(0)
        L.radix_sort_profile_kernels(0xFFFFFFFF)
        n = L.radix_sort_profile_read(None, 0)
        buf = (RsKernelTime * max(1, n))()
        got = L.radix_sort_profile_read(buf, n)
        if got < 0:
            raise RadixSortError(6, "radix_sort_profile_read")
        self.records = [(KERNEL_NAMES.get(buf[i].kernel, str(buf[i].kernel)), buf[i].level, buf[i].ms)
                        for i in range(got)]
        return False


from .graph import SortGraph  # noqa: E402
