"""The GPU tests' check helpers, on small CPU tensors: the record fingerprint does not depend on
the order of the records and changes when one byte of one record changes."""
import pytest

torch = pytest.importorskip("torch")
from tests.gpu_checks import check_sorted_same_records, record_fingerprint  # noqa: E402


def test_fingerprint_is_order_free_and_sees_one_flipped_bit():
    g = torch.Generator().manual_seed(3)
    a = torch.randint(0, 256, (5000, 24), dtype=torch.uint8, generator=g)
    assert record_fingerprint(a) == record_fingerprint(a[torch.randperm(5000, generator=g)])
    b = a.clone()
    b[4321, 17] ^= 4
    assert record_fingerprint(a) != record_fingerprint(b)


def test_sorted_same_records_accepts_a_sort_and_rejects_a_swap_or_a_loss():
    g = torch.Generator().manual_seed(4)
    a = torch.randint(0, 256, (3000, 8), dtype=torch.uint8, generator=g)
    keys = a.view(torch.int64).view(-1)
    order = torch.argsort(keys ^ (-(1 << 63)))  # unsigned order
    s = a[order].contiguous()
    check_sorted_same_records(s, a, 8)
    swapped = s.clone()
    swapped[[10, 11]] = swapped[[11, 10]]
    if not torch.equal(swapped[10], swapped[11]):
        with pytest.raises(AssertionError):
            check_sorted_same_records(swapped, a, 8)
    lost = s.clone()
    lost[7] = lost[6]
    if not torch.equal(s[7], s[6]):
        with pytest.raises(AssertionError):
            check_sorted_same_records(lost, a, 8)
