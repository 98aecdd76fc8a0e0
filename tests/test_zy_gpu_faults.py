"""Failure detection on the GPU without a fault (-m gpu).  The path has no device-side waits;
what the device can find wrong is a destination outside its bin (corrupted counts) or a list
that outgrows its bound.  Such a run is reported (RS_ERR_INTERNAL / RS_ERR_QUEUE_OVERFLOW)
and not written, and the context stays usable.  The test entry point makes one run fail its
range check on purpose; bad segment offsets are caught the same way."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1703_00687_gb300 as rg  # noqa: E402
from tests.gpu_checks import from_dev, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def test_failed_range_check_is_reported_and_context_survives():
    rng = np.random.default_rng(21)
    a = rng.integers(0, 256, size=(200_000, 16), dtype=np.uint8)
    try:
        assert rg.lib().radix_sort_test_inject(1) == 0
        t = to_dev(a)
        rg.sort(t, 8)
        assert rg.status() == 10  # RS_ERR_INTERNAL
        assert rg.status() == 0   # reported once, then cleared
    finally:
        rg.lib().radix_sort_test_inject(0)
    # the context still works and the next call is correct
    t = to_dev(a)
    rg.sort(t, 8)
    torch.cuda.synchronize()
    assert rg.status() == 0
    np.testing.assert_array_equal(from_dev(t), oracle.sort(a, 8))


def test_invalid_segment_offsets_are_reported_not_written():
    n = 10_000
    a = np.random.default_rng(2).integers(0, 256, size=(n, 16), dtype=np.uint8)
    t = to_dev(a)
    bad = torch.tensor([0, 6000, 4000, n + 5], dtype=torch.int64, device="cuda")  # decreasing, past the end
    rg.sort_segmented(t, bad, 8, total=n)
    assert rg.status() == 10  # RS_ERR_INTERNAL
    assert rg.status() == 0
