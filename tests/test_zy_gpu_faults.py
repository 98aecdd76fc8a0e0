"""Failure detection on the GPU without a fault (-m gpu).

What the device can find wrong: a destination outside its bin (corrupted counts), a list that
outgrows its bound, and a CTA's bounded wait for its own bulk copy into shared memory that
runs out.  Each is reported (RS_ERR_INTERNAL / RS_ERR_QUEUE_OVERFLOW / RS_ERR_DEVICE_TIMEOUT),
the call's later kernels do nothing, and the context stays usable.  The test entry point makes
one run fail its range check, or makes one wait run out on a shared-memory barrier that nothing
completes (with a short limit set through the plan); bad segment offsets are caught the same
way.  A sort of more records than one chunk holds distributes `in` into `tmp` first, so when
every kernel after a failed distribution pass does nothing, `in` is still the input."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1703_00687_gb300 as rg  # noqa: E402
from tests.gpu_checks import from_dev, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

RS_ERR_DEVICE_TIMEOUT, RS_ERR_INTERNAL = 7, 10


def _records(seed=21, n=200_000):
    return np.random.default_rng(seed).integers(0, 256, size=(n, 16), dtype=np.uint8)


def _next_sort_is_correct(a):
    t = to_dev(a)
    rg.sort(t, 8)
    torch.cuda.synchronize()
    assert rg.status() == 0
    np.testing.assert_array_equal(from_dev(t), oracle.sort(a, 8))


def test_failed_range_check_is_reported_and_later_kernels_stop():
    a = _records()
    assert a.shape[0] > rg.chunk_records(16)
    try:
        assert rg.lib().radix_sort_test_inject(1) == 0
        t = to_dev(a)
        rg.sort(t, 8)
        assert rg.status() == RS_ERR_INTERNAL
        assert rg.status() == 0   # reported once, then cleared
        # nothing after the failed pass ran: no on-chip sort or copy-back wrote `in`
        np.testing.assert_array_equal(from_dev(t), a)
    finally:
        rg.lib().radix_sort_test_inject(0)
    _next_sort_is_correct(a)


def test_device_wait_that_runs_out_is_reported_and_later_kernels_stop():
    a = _records(seed=22)
    old = rg.get_plan()
    try:
        rg.set_plan(**dict(old, watchdog_polls=4))
        assert rg.lib().radix_sort_test_inject(2) == 0
        t = to_dev(a)
        rg.sort(t, 8)
        assert rg.status() == RS_ERR_DEVICE_TIMEOUT
        assert rg.status() == 0
        np.testing.assert_array_equal(from_dev(t), a)
    finally:
        rg.lib().radix_sort_test_inject(0)
        rg.set_plan(**old)
    _next_sort_is_correct(a)


def test_short_wait_limit_alone_still_sorts_or_reports():
    """A limit of one poll on real copies: each wait either sees its copy or reports a timeout;
    either way the call ends, and the stream and the next call are unaffected."""
    a = _records(seed=23)
    old = rg.get_plan()
    try:
        rg.set_plan(**dict(old, watchdog_polls=1))
        t = to_dev(a)
        rg.sort(t, 8)
        st = rg.status()
        assert st in (0, RS_ERR_DEVICE_TIMEOUT)
        if st == 0:
            np.testing.assert_array_equal(from_dev(t), oracle.sort(a, 8))
    finally:
        rg.set_plan(**old)
    _next_sort_is_correct(a)


def test_invalid_segment_offsets_are_reported_not_written():
    n = 10_000
    a = np.random.default_rng(2).integers(0, 256, size=(n, 16), dtype=np.uint8)
    t = to_dev(a)
    bad = torch.tensor([0, 6000, 4000, n + 5], dtype=torch.int64, device="cuda")  # decreasing, past the end
    rg.sort_segmented(t, bad, 8, total=n)
    assert rg.status() == RS_ERR_INTERNAL
    assert rg.status() == 0
    np.testing.assert_array_equal(from_dev(t), a)

