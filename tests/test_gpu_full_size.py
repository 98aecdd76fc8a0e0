"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (-m gpu).

The oracle cannot sort 10^9 records in test time, so the output is checked by properties
that prove it is the unique stable sort of the input at any size (tests/gpu_checks.py):
the index payload is a permutation, every output record equals the input record it names,
keys are non-decreasing and equal keys keep input order.  The batched form is checked the
same way per segment: every record stays inside its own segment."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
import paper_1703_00687_gb300 as rg  # noqa: E402
from tests.gpu_checks import check_sorted_same_records, check_stable_sorted  # noqa: E402

pytestmark = pytest.mark.gpu


def _device_input(kind, n, R, K, seed):
    h = torch.empty((n, R), dtype=torch.uint8, pin_memory=True)
    wl.make(kind, n, R, K, seed, out=h)
    return h.cuda()


@pytest.mark.parametrize("kind,n,R,K,seed,idx_word", [
    ("uniform", 1_000_000_000, 16, 8, 2, 1),
    ("zipf", 1_000_000_000, 16, 8, 3, 1),
    ("kmer", 500_000_000, 24, 16, 4, 2),
])
def test_full_size_sort_is_the_stable_sort(kind, n, R, K, seed, idx_word):
    pristine = _device_input(kind, n, R, K, seed)
    out = pristine.clone()
    tmp = torch.empty_like(out)
    rg.sort(out, K, tmp=tmp)
    torch.cuda.synchronize()
    assert rg.status() == 0
    del tmp
    check_stable_sorted(out, pristine, K, idx_word)


@pytest.mark.parametrize("n,R,K,seed", [
    (1_000_000_000, 16, 16, 8),   # 16-byte keys filling the record (two distribution levels of 9 bits)
    (2_000_000_000, 8, 8, 9),     # 8-byte records: two levels of 10-bit digits
])
def test_full_size_sort_of_keys_without_payload(n, R, K, seed):
    """Records that are all key: no index to follow, so the output is checked for order and
    for holding the same records as the input (a multiset fingerprint); with nothing but keys
    in a record, that is the unique sorted result."""
    pristine = _device_input("uniform", n, R, K, seed)
    out = pristine.clone()
    tmp = torch.empty_like(out)
    rg.sort(out, K, tmp=tmp)
    torch.cuda.synchronize()
    assert rg.status() == 0
    del tmp
    check_sorted_same_records(out, pristine, K)


def test_full_size_batched_segments_are_each_the_stable_sort():
    sizes = wl.batched_sizes(seed=5).astype(np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    n = int(off[-1])
    pristine = _device_input("uniform", n, 16, 8, 6)
    out = pristine.clone()
    d_off = torch.from_numpy(off).cuda()
    g = rg.SortGraph(out, 8, offsets=d_off)  # the bench's configuration: a graph replay
    out.copy_(pristine)
    g.stream.wait_stream(torch.cuda.current_stream())
    g.replay()
    g.stream.synchronize()
    assert rg.status(g.stream) == 0
    del g
    w = out.view(torch.int64).view(n, 2)
    idx, key = w[:, 1], w[:, 0]
    seen = torch.zeros(n, dtype=torch.bool, device="cuda")
    seen[idx] = True
    assert bool(seen.all()), "indices are not a permutation"
    del seen
    blk = 1 << 26
    for a in range(0, n, blk):
        b = min(n, a + blk)
        pos = torch.arange(a, b, device="cuda")
        seg_pos = torch.searchsorted(d_off, pos, right=True) - 1
        seg_idx = torch.searchsorted(d_off, idx[a:b], right=True) - 1
        assert torch.equal(seg_pos, seg_idx), "a record left its segment"
        assert torch.equal(pristine[idx[a:b]], out[a:b]), "records differ from the inputs they name"
    sign = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    for a in range(0, n - 1, blk):
        b = min(n - 1, a + blk)
        x, y = key[a:b] ^ sign, key[a + 1:b + 1] ^ sign  # unsigned order through signed compare
        same_seg = torch.searchsorted(d_off, torch.arange(a + 1, b + 1, device="cuda"), right=True) - 1 == \
            torch.searchsorted(d_off, torch.arange(a, b, device="cuda"), right=True) - 1
        ok = (x < y) | ((x == y) & (idx[a:b] < idx[a + 1:b + 1]))
        assert bool((ok | ~same_seg).all()), f"order violated in [{a},{b})"
