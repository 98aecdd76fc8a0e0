"""radix_sort_noalloc: the sort for callers that cannot let a library allocate device memory
(a framework that owns the GPU's memory through its own allocator, a latency-critical path
that cannot afford cudaMalloc's implicit synchronisation, a fixed memory budget).  It keeps
its workspace in a fixed device array declared by the library instead of allocating one.

The GPU test calls it through the C ABI twice in a row and checks each output against
radix_sort's (byte for byte: both are the same stable sort).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import paper_1703_00687_gb300 as rg

RS_OK, RS_ERR_TOO_LARGE = 0, 4
DEV_RANGE_CHECK = 4  # the status word's bit for a failed destination range check


def test_noalloc_rejects_sizes_beyond_its_array_without_launching():
    # the size check comes before any pointer check, so no GPU is needed
    L = rg.lib()
    assert L.radix_sort_noalloc(None, None, 10 ** 9, 16, 8, None, None) == RS_ERR_TOO_LARGE
    assert L.radix_sort_noalloc(None, None, 0, 16, 8, None, None) == RS_OK


@pytest.mark.gpu
def test_noalloc_matches_radix_sort_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    L = rg.lib()
    stream = torch.cuda.current_stream()
    # two sorts that distribute before sorting on chip, then one small enough for a single chunk
    cases = [(1_000_003, 16, 8), (700_001, 24, 16), (1_000, 16, 8)]
    for call, (n, rec, key) in enumerate(cases):
        rng = np.random.default_rng(100 + call)
        a = rng.integers(0, 256, size=(n, rec), dtype=np.uint8)
        want = torch.from_numpy(a).cuda()
        rg.sort(want, key)  # the allocating entry point, for reference
        got = torch.from_numpy(a).cuda()
        tmp = torch.empty_like(got)
        status = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = L.radix_sort_noalloc(got.data_ptr(), tmp.data_ptr(), n, rec, key, status.data_ptr(),
                                  ctypes.c_void_p(stream.cuda_stream))
        assert rc == RS_OK
        torch.cuda.synchronize()
        if call > 0:
            # the first call on a device may load the array's module (that reserves its memory);
            # every later call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before, f"call {call} took device memory"
        assert int(status.item()) == 0
        assert torch.equal(got, want), f"call {call}: output differs from radix_sort"


@pytest.mark.gpu
def test_noalloc_reports_a_failed_step_in_its_status_word():
    """The device-side status of a call reaches the caller's word: one scatter run is made to
    fail its range check (test hook), the word holds that bit alone, and nothing after the
    failed pass wrote `in`; the next call is correct."""
    torch = pytest.importorskip("torch")
    L = rg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, rec, key = 1_000_003, 16, 8
    a = np.random.default_rng(7).integers(0, 256, size=(n, rec), dtype=np.uint8)
    assert n > rg.chunk_records(rec)
    got = torch.from_numpy(a).cuda()
    tmp = torch.empty_like(got)
    status = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
    try:
        assert L.radix_sort_test_inject(1) == 0
        assert L.radix_sort_noalloc(got.data_ptr(), tmp.data_ptr(), n, rec, key, status.data_ptr(), stream) == RS_OK
        torch.cuda.synchronize()
    finally:
        L.radix_sort_test_inject(0)
    assert int(status.item()) == DEV_RANGE_CHECK
    np.testing.assert_array_equal(got.cpu().numpy(), a)
    want = torch.from_numpy(a).cuda()
    rg.sort(want, key)
    assert L.radix_sort_noalloc(got.data_ptr(), tmp.data_ptr(), n, rec, key, status.data_ptr(), stream) == RS_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(got, want)
