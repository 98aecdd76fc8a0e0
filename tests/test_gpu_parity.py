"""GPU parity: the CUDA sorter against the CPU oracle, byte for byte (-m gpu).

The sorter is stable, so its output is unique and must equal the oracle's stable LSD sort
exactly.  Sizes span several tiles and chunks with ragged tails; distributions cover the
degenerate cases of the method (all keys equal, long shared prefixes, heavy duplicates).
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
import paper_1703_00687_gb300 as rg  # noqa: E402
from tests.gpu_checks import from_dev, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def gsort(a, key_size):
    t = to_dev(a)
    rg.sort(t, key_size)
    torch.cuda.synchronize()
    rg.check_status()
    return from_dev(t)


def rand(rng, n, R, K, distinct=None):
    a = rng.integers(0, 256, size=(n, R), dtype=np.uint8)
    if distinct:
        pool = rng.integers(0, 256, size=(distinct, K), dtype=np.uint8)
        a[:, :K] = pool[rng.integers(0, distinct, size=n)]
    return a


# ------------------------------------------------------------------ one pass
@pytest.mark.parametrize("R,K,lo,w", [(8, 8, 56, 8), (16, 8, 0, 8), (16, 8, 37, 10), (24, 16, 60, 8),
                                      (24, 16, 120, 8), (32, 8, 3, 5), (40, 13, 90, 9), (64, 16, 64, 1)])
def test_partition_parity(R, K, lo, w):
    rng = np.random.default_rng(R * 7 + lo)
    for n in (2, 511, 4096 * 3 + 17, 100_003):
        a = rand(rng, n, R, K)
        src, dst = to_dev(a), torch.empty((n, R), dtype=torch.uint8, device="cuda")
        rg.partition(src, dst, K, lo, w)
        torch.cuda.synchronize()
        rg.check_status()
        np.testing.assert_array_equal(from_dev(dst), oracle.partition(a, K, lo, w))


@pytest.mark.parametrize("R,K,lo,w", [(8, 8, 56, 8), (16, 8, 11, 10), (24, 16, 64, 7)])
def test_histogram_parity(R, K, lo, w):
    rng = np.random.default_rng(3)
    for n in (0, 1, 1000, 300_001):
        a = rand(rng, n, R, K, distinct=50 if n > 1000 else None)
        h = rg.histogram(to_dev(a), K, lo, w)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(from_dev(h).astype(np.uint64), oracle.histogram(a, K, lo, w))


# ---------------------------------------------------------------------- sort
# record sizes of every write path: 8 and 16 bytes (one store per record), 24/40 (whole warps,
# 8-byte pieces), 32/48/64/256 (whole warps, 16-byte pieces; 256 bytes is the largest record)
LAYOUTS = [(8, 8), (8, 1), (8, 5), (16, 8), (16, 16), (24, 16), (32, 8), (40, 13), (48, 16), (64, 16), (256, 9)]


@pytest.mark.parametrize("R,K", LAYOUTS)
def test_sort_parity_sizes(R, K):
    rng = np.random.default_rng(R * 31 + K)
    cm = rg.chunk_records(R)  # the on-chip limit: sizes around it take different paths
    for n in (0, 1, 2, 3, 100, 4095, cm, cm + 1, 9000, 70_001, 300_007):
        a = rand(rng, n, R, K)
        np.testing.assert_array_equal(gsort(a, K), oracle.sort(a, K), err_msg=f"n={n}")


def test_sort_parity_uniform_1e6_r8():
    a = wl.uniform(1_000_000, 8, 8, seed=1)
    np.testing.assert_array_equal(gsort(a, 8), oracle.sort(a, 8))


@pytest.mark.parametrize("kind", ["all_equal", "two_keys", "sorted", "reverse", "last_byte", "small_ints",
                                  "few_distinct", "top_bit_only", "long_runs", "heavy_gaps"])
def test_sort_parity_degenerate(kind):
    rng = np.random.default_rng(11)
    n, R, K = 400_000, 16, 8
    a = rand(rng, n, R, K)
    keys = a[:, :8].copy().view("<u8").ravel()
    if kind == "all_equal":
        keys[:] = 0x0123456789abcdef
    elif kind == "two_keys":
        keys[:] = np.where(rng.random(n) < 0.5, np.uint64(5), np.uint64(1 << 63))
    elif kind == "sorted":
        keys.sort()
    elif kind == "reverse":
        keys[:] = np.sort(keys)[::-1]
    elif kind == "last_byte":
        keys[:] = 0xabcdef0000000000 | rng.integers(0, 256, n).astype(np.uint64)
    elif kind == "small_ints":
        keys[:] = rng.integers(0, 1 << 20, n).astype(np.uint64)
    elif kind == "few_distinct":
        keys[:] = rng.integers(0, 1 << 64, 37, dtype=np.uint64)[rng.integers(0, 37, n)]
    elif kind == "top_bit_only":
        keys[:] = (rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63))
    elif kind == "long_runs":
        keys[:] = np.repeat(rng.integers(0, 1 << 64, n // 5000 + 1, dtype=np.uint64), 5000)[:n]
    elif kind == "heavy_gaps":
        # 8 heavy top digits (large sub-bins, the next level) with a few hundred records spread
        # between them: the runs of small sub-bins between two heavy ones pack into tiny chunks
        top = rng.choice(512, 8, replace=False).astype(np.uint64)
        keys[:] = (top[rng.integers(0, 8, n)] << np.uint64(55)) | rng.integers(0, 1 << 55, n).astype(np.uint64)
        few = rng.random(n) < 0.001
        keys[few] = rng.integers(0, 1 << 64, int(few.sum()), dtype=np.uint64)
    a[:, :8] = keys.view(np.uint8).reshape(n, 8)
    np.testing.assert_array_equal(gsort(a, K), oracle.sort(a, K))


@pytest.mark.parametrize("R,K", [(16, 8), (8, 8), (24, 16), (32, 8), (16, 16)])
def test_sort_parity_composite_ties(R, K):
    """The on-chip sorter's first round ranks records by composite keys: the top key bits
    below the chunk's shared bits (at most 51 of them) plus the record's position.  Here keys
    share long prefixes drawn from a pool and differ only in their low 10 bits, so records
    of one prefix tie in the kept bits and must fall back to whole-key comparisons.  Single
    chunks (n <= the on-chip limit) and chunks formed after a distribution level both occur;
    a pool of few prefixes makes buckets larger than the enumeration limit (general rounds)."""
    rng = np.random.default_rng(R * 13 + K)
    cm = rg.chunk_records(R)
    for n, npref in ((cm, 400), (cm - 7, 20), (3000, 3000), (250_000, 30_000), (250_000, 40)):
        a = rand(rng, n, R, K)
        pool = rng.integers(0, 256, size=(npref, K), dtype=np.uint8)
        keys = pool[rng.integers(0, npref, n)]
        low = rng.integers(0, 1 << 10, n)
        keys[:, 0] = (low & 0xFF).astype(np.uint8)
        keys[:, 1] = (keys[:, 1] & 0xFC) | (low >> 8).astype(np.uint8)
        a[:, :K] = keys
        np.testing.assert_array_equal(gsort(a, K), oracle.sort(a, K), err_msg=f"n={n} prefixes={npref}")


@pytest.mark.parametrize("n,R,K", [(300_007, 16, 8), (4_000_000, 16, 8), (1_000_003, 24, 16)])
def test_sort_parity_sm_limit(n, R, K):
    """Grids capped to 19 SMs (the SM-count sweep): fewer lanes, so every histogram and scatter
    CTA walks more tiles and more bins, and fewer chunk CTAs take more chunks each."""
    rng = np.random.default_rng(n + R)
    a = rand(rng, n, R, K)
    old = rg.get_plan()
    try:
        rg.set_plan(sm_limit=19)
        got = gsort(a, K)
    finally:
        rg.set_plan(**old)
    np.testing.assert_array_equal(got, oracle.sort(a, K))


@pytest.mark.parametrize("n,K", [(4096 * 5 + 3, 8), (300_007, 8), (1_000_003, 5)])
def test_sort_parity_ten_bit_digits_8_byte_records(n, K):
    """8-byte records with 10-bit digit tables: the scatter's CTAs of 512 threads (16 warps,
    lanes grouped by winner bytes), over several tiles and a ragged last one."""
    rng = np.random.default_rng(n + K)
    a = rand(rng, n, 8, K)
    old = rg.get_plan()
    try:
        rg.set_plan(digit_bits_max=10)
        got = gsort(a, K)
    finally:
        rg.set_plan(**old)
    np.testing.assert_array_equal(got, oracle.sort(a, K))


@pytest.mark.parametrize("R,K,pattern", [(16, 8, "90"), (16, 8, "55"), (16, 8, "two"), (16, 8, "zero"),
                                         (16, 8, "ones"), (24, 16, "90"), (24, 16, "ones"), (16, 5, "90"),
                                         (8, 8, "97"), (64, 16, "two")])
def test_sort_parity_dominant_key(R, K, pattern):
    """Bins that one key dominates: the sample at bin formation flags them, and the next pass
    splits that key's digit in three (below / equal / above) and finishes the equal part.
    Payloads are random, so the equal keys must come out in input order."""
    rng = np.random.default_rng(R * 7 + K + len(pattern))
    n = 600_000
    a = rand(rng, n, R, K)
    keys = a[:, :K].copy()
    def put(mask, key_bytes):
        keys[mask] = key_bytes
    u = rng.random(n)
    if pattern in ("90", "55", "97"):
        frac = int(pattern) / 100
        put(u < frac, rng.integers(0, 256, K, dtype=np.uint8))
    elif pattern == "two":
        put(u < 0.45, rng.integers(0, 256, K, dtype=np.uint8))
        put((u >= 0.45) & (u < 0.9), rng.integers(0, 256, K, dtype=np.uint8))
    elif pattern == "zero":  # the smallest key: its digit is 0 at every level
        put(u < 0.8, np.zeros(K, dtype=np.uint8))
    elif pattern == "ones":  # the largest key: its digit is the last one
        put(u < 0.8, np.full(K, 255, dtype=np.uint8))
    a[:, :K] = keys
    np.testing.assert_array_equal(gsort(a, K), oracle.sort(a, K))


@pytest.mark.parametrize("R,K", [(16, 8), (24, 16), (8, 3)])
def test_segmented_small_total(R, K):
    """All segments together within the on-chip limit: the call launches no distribution level."""
    rng = np.random.default_rng(R + K)
    cm = rg.chunk_records(R)
    sizes = rng.integers(0, 150, 60).astype(np.uint64)
    sizes[0] = 70  # one segment of more than 64 records: the CTA sorter runs as well as the warps
    while sizes.sum() > cm:
        sizes[1:] //= 2
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    assert n <= cm
    a = rand(rng, n, R, K, distinct=40)
    t = to_dev(a)
    rg.sort_segmented(t, torch.from_numpy(off.astype(np.int64)).cuda(), K, total=n)
    torch.cuda.synchronize()
    rg.check_status()
    np.testing.assert_array_equal(from_dev(t), oracle.sort_segmented(a, off, K))


def test_segmented_dominant_segments():
    rng = np.random.default_rng(77)
    sizes = np.array([300_000, 50, 120_000, 7, 80_000, 0, 200_000], dtype=np.uint64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    a = rand(rng, n, 16, 8)
    for s in range(len(sizes)):  # every segment mostly one key of its own
        lo, hi = int(off[s]), int(off[s + 1])
        m = rng.random(hi - lo) < 0.85
        a[lo:hi][m, :8] = rng.integers(0, 256, 8, dtype=np.uint8)
    t = to_dev(a)
    rg.sort_segmented(t, torch.from_numpy(off.astype(np.int64)).cuda(), 8, total=n)
    torch.cuda.synchronize()
    rg.check_status()
    np.testing.assert_array_equal(from_dev(t), oracle.sort_segmented(a, off, 8))


def test_sort_parity_zipf():
    a = wl.zipf(1_500_000, 16, seed=3)
    np.testing.assert_array_equal(gsort(a, 8), oracle.sort(a, 8))


def test_sort_parity_kmer():
    a = wl.kmer(1_000_000, 24, seed=4)
    np.testing.assert_array_equal(gsort(a, 16), oracle.sort(a, 16))


def test_sort_parity_kmer_few_prefixes():
    a = wl.kmer(600_000, 24, seed=9, prefixes=3)
    np.testing.assert_array_equal(gsort(a, 16), oracle.sort(a, 16))


# ----------------------------------------------------------------- segmented
def test_segmented_parity():
    rng = np.random.default_rng(5)
    sizes = np.concatenate([[0, 1, 2, 0], rng.integers(0, 60, 200), rng.integers(1000, 6000, 20),
                            rng.integers(10_000, 200_000, 4), [0, 1]]).astype(np.uint64)
    rng.shuffle(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    a = rand(rng, n, 16, 8, distinct=n // 3)
    t = to_dev(a)
    offs = torch.from_numpy(off.astype(np.int64)).cuda()
    rg.sort_segmented(t, offs, 8, total=n)
    torch.cuda.synchronize()
    rg.check_status()
    np.testing.assert_array_equal(from_dev(t), oracle.sort_segmented(a, off, 8))


@pytest.mark.parametrize("R,K", [(8, 8), (8, 3), (16, 8), (16, 16), (24, 5), (40, 13), (64, 16), (256, 9)])
def test_segmented_tiny_parity(R, K):
    """Many segments of 0..80 records: tiny ones (2..64) are sorted by warps with sorting
    networks (several chunks of up to 32 records per warp, or one of 33..64 records with two
    per lane), 65..80 by the CTA sorter; a few large ones keep the level path busy.  Few
    distinct keys, so equal keys must keep their input order."""
    rng = np.random.default_rng(R * 13 + K)
    sizes = rng.integers(0, 81, 4000).astype(np.uint64)
    sizes[::97] = rng.integers(2000, 30_000, len(sizes[::97]))
    sizes[:80] = np.arange(80)  # every tiny size, in order
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    a = rand(rng, n, R, K, distinct=7)
    t = to_dev(a)
    rg.sort_segmented(t, torch.from_numpy(off.astype(np.int64)).cuda(), K, total=n)
    torch.cuda.synchronize()
    rg.check_status()
    np.testing.assert_array_equal(from_dev(t), oracle.sort_segmented(a, off, K))


def test_segmented_matches_plain_alone():
    rng = np.random.default_rng(6)
    sizes = wl.batched_sizes(n_segs=300, lo=1, hi=50_000, cap=10**9, seed=5)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    a = wl.uniform(n, 16, 8, seed=6)
    t = to_dev(a)
    rg.sort_segmented(t, torch.from_numpy(off.astype(np.int64)).cuda(), 8, total=n)
    got = from_dev(t)
    for s in rng.choice(len(sizes), 25, replace=False):
        lo, hi = int(off[s]), int(off[s + 1])
        np.testing.assert_array_equal(got[lo:hi], gsort(a[lo:hi], 8))


def test_tmp_and_stream_arguments():
    rng = np.random.default_rng(8)
    a = rand(rng, 123_457, 32, 16)
    t = to_dev(a)
    tmp = torch.empty_like(t)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rg.sort(t, 16, tmp=tmp, stream=s)
    s.synchronize()
    assert rg.status(s) == 0
    np.testing.assert_array_equal(from_dev(t), oracle.sort(a, 16))


def test_host_tensor_roundtrip():
    a = wl.uniform(200_000, 16, 8, seed=12)
    t = torch.from_numpy(a.copy())
    rg.sort(t, 8)
    np.testing.assert_array_equal(t.numpy(), oracle.sort(a, 8))


@pytest.mark.parametrize("n,R,K", [(300_007, 24, 16), (1000, 8, 8), (5, 16, 8)])
def test_sort_host_entry(n, R, K):
    """radix_sort_host: pinned input, a separate pinned output, caller's device buffers."""
    rng = np.random.default_rng(n)
    a = rand(rng, n, R, K, distinct=n // 2 + 1)
    h_in = torch.from_numpy(a.copy()).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_buf = torch.empty(h_in.shape, dtype=h_in.dtype, device="cuda")
    d_tmp = torch.empty_like(d_buf)
    rg.sort_host(h_in, K, h_out=h_out, d_buf=d_buf, d_tmp=d_tmp)
    np.testing.assert_array_equal(h_out.numpy(), oracle.sort(a, K))
    np.testing.assert_array_equal(h_in.numpy(), a)  # the input is only read


# ------------------------------------------------ run-length counting after the sort (k-mer counting)
@pytest.mark.parametrize("n,R,K,distinct", [(300_007, 24, 16, 5000), (200_000, 16, 8, 70_000), (9_000, 8, 3, 10),
                                            (50_000, 24, 16, 1), (4097, 16, 8, None)])
def test_count_runs_parity(n, R, K, distinct):
    rng = np.random.default_rng(n + R)
    a = rand(rng, n, R, K, distinct=distinct)
    t = to_dev(a)
    rg.sort(t, K)
    first, counts = rg.count_runs(t, K)
    torch.cuda.synchronize()
    rg.check_status()
    want_first, want_counts = oracle.count_runs(oracle.sort(a, K), K)
    np.testing.assert_array_equal(from_dev(first), want_first)
    np.testing.assert_array_equal(from_dev(counts).astype(np.uint64), want_counts)


def test_count_runs_edge_cases():
    for n in (0, 1):
        t = torch.zeros((n, 16), dtype=torch.uint8, device="cuda")
        first, counts = rg.count_runs(t, 8)
        assert first.shape[0] == n and counts.tolist() == [1] * n
    # one long run spanning many tiles, then single records
    a = np.zeros((100_000, 8), dtype=np.uint8)
    a[-3:, 0] = [1, 2, 3]
    first, counts = rg.count_runs(to_dev(a), 8)
    assert counts.tolist() == [99_997, 1, 1, 1]
