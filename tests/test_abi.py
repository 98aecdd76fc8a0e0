"""The C ABI library builds, loads, exports every declared symbol, and rejects bad arguments
on the host before touching the GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1703_00687_gb300 as rg
from paper_1703_00687_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "radix_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(radix_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("radix_sort", "radix_sort_segmented", "radix_partition", "radix_histogram", "radix_sort_status",
                 "radix_sort_strerror", "radix_sort_release", "radix_sort_set_plan", "radix_sort_get_plan",
                 "radix_sort_launch_count", "radix_sort_test_inject"):
        assert want in names


def test_library_exports_every_declared_symbol():
    L = rg.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_strerror_names_every_status():
    L = rg.lib()
    for code in range(11):
        s = L.radix_sort_strerror(code).decode()
        assert s and s != "unknown status"
    assert L.radix_sort_strerror(77).decode() == "unknown status"


A = 0x7f0000000000  # fake, 16-byte aligned addresses: validation fails before any CUDA call
B = 0x7f1000000000


@pytest.mark.parametrize("rec_size,key_size,code", [
    (0, 1, 1), (12, 8, 1), (264, 8, 1), (16, 0, 1), (8, 9, 1), (24, 17, 9), (32, 32, 9),
])
def test_layout_validation(rec_size, key_size, code):
    L = rg.lib()
    assert L.radix_sort(A, B, 100, rec_size, key_size, None) == code
    assert L.radix_partition(A, B, 100, rec_size, key_size, 0, 4, None) == code


def test_buffer_validation():
    L = rg.lib()
    assert L.radix_sort(None, B, 100, 16, 8, None) == 1           # null
    assert L.radix_sort(A + 8, B, 100, 16, 8, None) == 2          # misaligned
    assert L.radix_sort(A, A + 16 * 50, 100, 16, 8, None) == 3    # overlap
    assert L.radix_sort(A, B, 2 ** 62, 16, 8, None) == 4          # n * rec_size overflows
    # n <= 1: nothing to do, no launch, even with null pointers
    assert L.radix_sort(None, None, 0, 16, 8, None) == 0
    assert L.radix_sort(None, None, 1, 16, 8, None) == 0
    assert L.radix_sort_segmented(A, B, None, 10, 1000, 16, 8, None) == 1
    assert L.radix_sort_segmented(A, B, None, 0, 0, 16, 8, None) == 0


def test_host_entry_validation():
    L = rg.lib()
    H = ctypes.c_void_p(1 << 20)  # never dereferenced: every case below fails validation first
    assert L.radix_sort_host(None, H, A, B, 100, 16, 8, None) == 1       # null host input
    assert L.radix_sort_host(H, None, A, B, 100, 16, 8, None) == 1       # null host output
    assert L.radix_sort_host(H, H, A + 8, B, 100, 16, 8, None) == 2      # misaligned device buffer
    assert L.radix_sort_host(H, H, A, A + 16 * 50, 100, 16, 8, None) == 3  # device buffers overlap
    assert L.radix_sort_host(H, H, A, B, 100, 12, 8, None) == 1          # rec_size not a multiple of 8
    assert L.radix_sort_host(None, None, None, None, 0, 16, 8, None) == 0  # nothing to do


def test_digit_validation():
    L = rg.lib()
    assert L.radix_partition(A, B, 100, 16, 8, 0, 0, None) == 1     # width 0
    assert L.radix_partition(A, B, 100, 16, 8, 0, 11, None) == 1    # wider than supported
    assert L.radix_partition(A, B, 100, 16, 8, 60, 8, None) == 1    # past the key
    assert L.radix_histogram(A, 100, 16, 8, 0, 8, None, None) == 1  # no counts buffer


def test_plan_validation_and_roundtrip():
    old = rg.get_plan()
    with pytest.raises(rg.RadixSortError):
        rg.set_plan(digit_bits_max=12)
    with pytest.raises(rg.RadixSortError):
        rg.set_plan(tile_records=700)
    with pytest.raises(rg.RadixSortError):
        rg.set_plan(tile_records=1536)
    rg.set_plan(digit_bits_max=10, tile_records=2048, chunk_records=1000)
    assert rg.get_plan()["tile_records"] == 2048
    rg.set_plan(**old)
    assert rg.get_plan() == old


def test_launch_counter_starts_and_is_monotone():
    a = rg.launch_count()
    assert a >= 0
    assert rg.launch_count() >= a


def test_inject_flag_validation():
    L = rg.lib()
    assert L.radix_sort_test_inject(4) == 1  # bits 0 (range check) and 1 (wait) only
    for flags in (1, 2, 3):
        assert L.radix_sort_test_inject(flags) == 0
    assert L.radix_sort_test_inject(0) == 0


def test_chunk_records_follows_the_plan_and_rejects_bad_sizes():
    assert rg.chunk_records(7) == 0 and rg.chunk_records(0) == 0 and rg.chunk_records(264) == 0
    default16, default8 = rg.chunk_records(16), rg.chunk_records(8)
    assert default16 >= 1024 and default8 >= default16  # smaller records: more fit on chip
    old = rg.get_plan()
    try:
        rg.set_plan(**{**old, "chunk_records": 1000})
        assert rg.chunk_records(16) == 1000
        rg.set_plan(**{**old, "chunk_records": 10 ** 9})  # above the capacity: capped
        assert rg.chunk_records(16) == default16
    finally:
        rg.set_plan(**old)
