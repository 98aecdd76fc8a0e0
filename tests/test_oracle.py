"""Pins for the CPU oracle (no GPU).

The oracle is checked against things fixed by the mathematics of sorting, not against
itself: hand-worked examples, a library stable sort (the special case the definition
reduces to), brute force over all tiny inputs, closed forms, and invariants.  The last
test plants plausible mistakes in a copy of the oracle's source and shows each one fails
at least one of these pins.
"""
import itertools
import os
import random
import subprocess
import tempfile
import ctypes
import sys

import numpy as np
import pytest

import oracle
from tests._helpers import (as_records, key_ints, keys_nondecreasing, parse_golden, same_multiset,
                            stable_sort_by_key)


def rand_records(rng, n, rec_size, key_size, key_bytes_random=None, distinct_keys=None):
    a = rng.integers(0, 256, size=(n, rec_size), dtype=np.uint8)
    if distinct_keys is not None:
        pool = rng.integers(0, 256, size=(distinct_keys, key_size), dtype=np.uint8)
        a[:, :key_size] = pool[rng.integers(0, distinct_keys, size=n)]
    if key_bytes_random is not None:
        # only some key bytes vary; the others are constant (exercises digit skipping)
        mask = np.zeros(key_size, dtype=bool)
        mask[list(key_bytes_random)] = True
        a[:, :key_size][:, ~mask] = 7
    return a


# ----------------------------------------------------------------------------- golden
@pytest.mark.parametrize("ex", list(parse_golden()), ids=lambda e: e["name"])
def test_golden_examples(ex):
    inp = as_records(ex["inp"], ex["rec_size"])
    exp = as_records(ex["out"], ex["rec_size"])
    if ex["op"] == "sort":
        got = oracle.sort(inp, ex["key_size"])
    else:
        got = oracle.partition(inp, ex["key_size"], ex["lo"], ex["width"])
    np.testing.assert_array_equal(got, exp)


# ------------------------------------------------------------- library stable sort
LAYOUTS = [(8, 8), (8, 1), (8, 5), (16, 8), (16, 16), (24, 16), (32, 8), (64, 24), (16, 3), (24, 9)]


@pytest.mark.parametrize("rec_size,key_size", LAYOUTS)
def test_equals_python_stable_sort(rec_size, key_size):
    rng = np.random.default_rng(rec_size * 100 + key_size)
    for n in (0, 1, 2, 3, 17, 255, 256, 257, 1000):
        a = rand_records(rng, n, rec_size, key_size, distinct_keys=max(1, n // 3))
        got = oracle.sort(a, key_size)
        keys = key_ints(a, key_size)
        order = sorted(range(n), key=lambda i: keys[i])  # Python's sort is stable
        np.testing.assert_array_equal(got, a[order] if n else a)


@pytest.mark.parametrize("rec_size,key_size", [(16, 8), (24, 16), (8, 8), (40, 13)])
def test_equals_numpy_lexsort_large(rec_size, key_size):
    rng = np.random.default_rng(7)
    n = 200_000
    a = rand_records(rng, n, rec_size, key_size, distinct_keys=n // 4)
    np.testing.assert_array_equal(oracle.sort(a, key_size), stable_sort_by_key(a, key_size))


def test_equals_numpy_with_constant_bytes():
    rng = np.random.default_rng(11)
    a = rand_records(rng, 50_000, 16, 16, key_bytes_random=[0, 9, 15])
    np.testing.assert_array_equal(oracle.sort(a, 16), stable_sort_by_key(a, 16))


# ------------------------------------------------------------------- brute force
def _by_definition(recs, key_size):
    """The unique permutation with non-decreasing keys and, among equal keys, input order,
    found by trying every permutation."""
    n = len(recs)
    keys = key_ints(recs, key_size)
    found = []
    for p in itertools.permutations(range(n)):
        ok = all(keys[p[i]] < keys[p[i + 1]] or (keys[p[i]] == keys[p[i + 1]] and p[i] < p[i + 1])
                 for i in range(n - 1))
        if ok:
            found.append(p)
    assert len(found) == 1
    return recs[list(found[0])] if n else recs


def test_bruteforce_all_tiny_inputs():
    # three keys that differ at byte 0, byte 3 and byte 7 (digit boundaries of the LSD
    # phases), plus a key equal to one of them in all but the lowest bit
    base = np.zeros(8, dtype=np.uint8)
    ks = []
    for b in (0, 3, 7):
        k = base.copy(); k[b] = 0x80; ks.append(k)
    k = ks[2].copy(); k[0] = 1; ks.append(k)
    count = 0
    for n in range(0, 6):
        for combo in itertools.product(range(len(ks)), repeat=n):
            recs = np.zeros((n, 16), dtype=np.uint8)
            for i, c in enumerate(combo):
                recs[i, :8] = ks[c]
                recs[i, 8] = i            # payload = input position
            want = _by_definition(recs, 8)
            np.testing.assert_array_equal(oracle.sort(recs, 8), want)
            count += 1
    assert count == sum(4 ** n for n in range(6))


# -------------------------------------------------------------------- closed forms
def test_permutation_keys_sort_to_identity():
    rng = np.random.default_rng(3)
    n = 70_000
    perm = rng.permutation(n).astype("<u8")
    recs = np.stack([perm, np.arange(n, dtype="<u8")], axis=1).view(np.uint8).reshape(n, 16)
    out = oracle.sort(recs, 8).view("<u8").reshape(n, 2)
    np.testing.assert_array_equal(out[:, 0], np.arange(n))
    inv = np.empty(n, dtype=np.int64); inv[perm] = np.arange(n)
    np.testing.assert_array_equal(out[:, 1], inv)


def test_all_equal_is_identity_and_reverse_is_reversed():
    n = 5000
    recs = np.zeros((n, 16), dtype=np.uint8)
    recs[:, :8] = 0x5a
    recs[:, 8:] = np.arange(n, dtype="<u8").view(np.uint8).reshape(n, 8)
    np.testing.assert_array_equal(oracle.sort(recs, 8), recs)
    keys = np.arange(n, 0, -1, dtype="<u8")
    rev = np.stack([keys, np.arange(n, dtype="<u8")], axis=1).view(np.uint8).reshape(n, 16)
    np.testing.assert_array_equal(oracle.sort(rev, 8), rev[::-1])


def test_histogram_closed_form():
    # keys 0..n-1: digit bits [lo, lo+w) take value v for exactly
    # (n // 2^(lo+w)) * 2^lo + clamp(n mod 2^(lo+w) - v*2^lo, 0, 2^lo) keys
    for n, lo, w in [(100_000, 0, 8), (100_000, 5, 7), (70_001, 12, 4), (1 << 17, 16, 2)]:
        recs = np.arange(n, dtype="<u8").view(np.uint8).reshape(n, 8)
        got = oracle.histogram(recs, 8, lo, w)
        period = 1 << (lo + w)
        v = np.arange(1 << w)
        want = (n // period) * (1 << lo) + np.clip(n % period - v * (1 << lo), 0, 1 << lo)
        np.testing.assert_array_equal(got, want.astype(np.uint64))


def test_partition_is_stable_partition():
    rng = np.random.default_rng(5)
    for rec_size, key_size, lo, w in [(16, 8, 56, 8), (16, 8, 0, 11), (24, 16, 60, 8), (8, 3, 17, 7)]:
        a = rand_records(rng, 30_000, rec_size, key_size)
        got = oracle.partition(a, key_size, lo, w)
        kk = np.array([(k >> lo) & ((1 << w) - 1) for k in key_ints(a, key_size)])
        order = np.argsort(kk, kind="stable")
        np.testing.assert_array_equal(got, a[order])


def test_invariants_random():
    rng = np.random.default_rng(9)
    for rec_size, key_size in LAYOUTS:
        n = 20_000
        a = rand_records(rng, n, rec_size, key_size, distinct_keys=500)
        if rec_size >= key_size + 8:
            a[:, key_size:key_size + 8] = np.arange(n, dtype="<u8").view(np.uint8).reshape(n, 8)
        out = oracle.sort(a, key_size)
        assert keys_nondecreasing(out, key_size)
        assert same_multiset(out, a)
        if rec_size >= key_size + 8:
            # stability: among equal keys the input positions increase
            pos = out[:, key_size:key_size + 8].copy().view("<u8").ravel()
            k = key_ints(out, key_size)
            for i in range(n - 1):
                if k[i] == k[i + 1]:
                    assert pos[i] < pos[i + 1]


def test_segmented_equals_each_segment_alone():
    rng = np.random.default_rng(13)
    sizes = [0, 1, 5, 300, 0, 2, 1000, 64]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    a = rand_records(rng, int(off[-1]), 16, 8, distinct_keys=100)
    got = oracle.sort_segmented(a, off, 8)
    for s in range(len(sizes)):
        lo, hi = int(off[s]), int(off[s + 1])
        np.testing.assert_array_equal(got[lo:hi], stable_sort_by_key(a[lo:hi], 8))


# -------------------------------------------------------------- the pins have teeth
# Each mutant is a plausible slip in the oracle; all keep memory accesses in bounds.
MUTANTS = {
    # most significant byte first: LSD order reversed
    "msd_first": ("8 * byte, 8", "8 * (key_size - 1 - byte), 8"),
    # prefix sum taken over the digit values in the wrong direction
    "descending_scan": ("for (uint64_t v = 0; v < buckets; v++) { uint64_t c = count[v]; count[v] = run; run += c; }",
                        "for (uint64_t v = buckets; v-- > 0;) { uint64_t c = count[v]; count[v] = run; run += c; }"),
    # bits of a digit taken in reverse order
    "bit_order": ("v |= bit << j;", "v |= bit << (width - 1 - j);"),
    # a key byte dropped (the least significant one is never used as a digit)
    "dropped_byte": ("for (uint32_t byte = 0; byte < key_size; byte++)",
                     "for (uint32_t byte = 1; byte < key_size; byte++)"),
    # a key byte index off by one (the digit read from the byte above)
    "byte_off_by_one": ("uint32_t bit = (rec[b >> 3] >> (b & 7)) & 1u;",
                        "uint32_t bit = (rec[(b >> 3) + 1 < 8 ? (b >> 3) + 1 : (b >> 3)] >> (b & 7)) & 1u;"),
}

_MUTANT_CHECK = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from tests._helpers import as_records, parse_golden, stable_sort_by_key
L = ctypes.CDLL(sys.argv[1])
L.oracle_lsd_sort.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
def msort(a, k):
    buf = np.ascontiguousarray(a).copy(); tmp = np.empty_like(buf)
    L.oracle_lsd_sort(buf.ctypes.data, tmp.ctypes.data, buf.shape[0], buf.shape[1], k)
    return buf
failures = 0
for ex in parse_golden():
    if ex["op"] == "sort":
        inp = as_records(ex["inp"], ex["rec_size"]); exp = as_records(ex["out"], ex["rec_size"])
        failures += not np.array_equal(msort(inp, ex["key_size"]), exp)
rng = np.random.default_rng(1)
a = rng.integers(0, 256, size=(3000, 16), dtype=np.uint8)
failures += not np.array_equal(msort(a, 8), stable_sort_by_key(a, 8))
print("FAILURES", failures)
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_fail_a_pin(name):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, name
    build_dir = os.path.join(os.path.dirname(oracle.__file__), "_build")
    os.makedirs(build_dir, exist_ok=True)
    with tempfile.TemporaryDirectory(dir=build_dir) as d:  # (inside the repository)
        path = os.path.join(d, name + ".c")
        open(path, "w").write(src.replace(old, new))
        so = os.path.join(d, name + ".so")
        subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", so, path])
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        r = subprocess.run([sys.executable, "-c", _MUTANT_CHECK, so, root], capture_output=True, text=True, timeout=120)
        # a crash also counts as caught, but every mutant here is memory-safe
        assert r.returncode == 0, r.stderr
        n_fail = int(r.stdout.split("FAILURES")[1])
        assert n_fail > 0, f"mutant {name} passed every pin"


# ---------------------------------------------------------------- run-length counting (k-mer counting)
def test_count_runs_closed_forms():
    # all keys equal: one run of n; all distinct: n runs of 1; key v repeated m_v times: runs m_v
    a = np.zeros((7, 16), dtype=np.uint8)
    a[:, 8:] = np.arange(7, dtype=np.uint8)[:, None]  # payload differs, keys equal
    f, c = oracle.count_runs(a, 8)
    assert c.tolist() == [7] and np.array_equal(f[0], a[0])
    b = np.zeros((5, 8), dtype=np.uint8)
    b[:, 0] = np.arange(5)
    f, c = oracle.count_runs(b, 8)
    assert c.tolist() == [1] * 5 and np.array_equal(f, b)
    mult = [3, 1, 4, 1, 5]
    keys = np.repeat(np.arange(len(mult), dtype=np.uint64), mult)
    recs = keys.view(np.uint8).reshape(-1, 8)
    f, c = oracle.count_runs(recs, 8)
    assert c.tolist() == mult
    assert oracle.count_runs(np.zeros((0, 8), dtype=np.uint8), 8)[1].size == 0


def test_count_runs_equals_numpy_unique_on_sorted_keys():
    rng = np.random.default_rng(5)
    for key_size, rec in ((8, 16), (16, 24), (3, 8)):
        a = rng.integers(0, 256, size=(3000, rec), dtype=np.uint8)
        a[:, :key_size] = rng.integers(0, 4, size=(3000, key_size), dtype=np.uint8)  # many repeats
        s = oracle.sort(a, key_size)
        f, c = oracle.count_runs(s, key_size)
        keys = [bytes(r[:key_size]) for r in s]
        uniq, counts = np.unique(np.array(keys, dtype=object), return_counts=True)
        # np.unique orders bytes lexicographically, the sort orders little-endian integers:
        # compare as multisets of (key, count), and check the runs appear in sorted order
        assert sorted(zip(uniq.tolist(), counts.tolist())) == sorted(zip([bytes(r[:key_size]) for r in f], c.tolist()))
        assert int(c.sum()) == len(s)
        ints = [int.from_bytes(bytes(r[:key_size]), "little") for r in f]
        assert ints == sorted(ints) and len(set(ints)) == len(ints)
