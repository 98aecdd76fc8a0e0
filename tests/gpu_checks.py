"""GPU-side test helpers (plain torch, test code only): moving records, and a complete check
that an output is THE stable sort of an input whose payload carries the original index.

If every output record equals the input record its index names, the indices form a
permutation, keys are non-decreasing and equal keys have increasing indices, then the
output is the unique stable sort of the input: a full correctness proof at any size.
"""
from __future__ import annotations

import numpy as np
import torch

SIGN = -0x8000000000000000  # flipping the top bit maps unsigned order onto signed order


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def from_dev(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def _ukey_words(w: torch.Tensor, key_size: int):
    """Key words as order-preserving signed int64 columns, most significant first."""
    cols = []
    nk = (key_size + 7) // 8
    for k in reversed(range(nk)):
        x = w[:, k]
        bytes_in = key_size - 8 * k
        if bytes_in < 8:
            x = x & ((1 << (8 * bytes_in)) - 1)
        cols.append(x ^ SIGN)
    return cols


def check_stable_sorted(out: torch.Tensor, pristine: torch.Tensor, key_size: int, idx_word: int,
                        block: int = 1 << 25) -> None:
    n, R = out.shape
    assert R % 8 == 0
    wo = out.view(torch.int64).view(n, R // 8)
    idx = wo[:, idx_word]
    assert bool(((idx >= 0) & (idx < n)).all()), "index out of range"
    seen = torch.zeros(n, dtype=torch.bool, device=out.device)
    seen[idx] = True
    assert bool(seen.all()), "indices are not a permutation"
    del seen
    for a in range(0, n, block):
        b = min(n, a + block)
        assert torch.equal(pristine[idx[a:b]], out[a:b]), f"records [{a},{b}) differ from the inputs they name"
    # keys non-decreasing, ties in input order (compare each record with the next, blockwise)
    for a in range(0, n - 1, block):
        b = min(n - 1, a + block)
        x = _ukey_words(wo[a:b], key_size)
        y = _ukey_words(wo[a + 1:b + 1], key_size)
        lt = torch.zeros(b - a, dtype=torch.bool, device=out.device)
        eq = torch.ones(b - a, dtype=torch.bool, device=out.device)
        for cx, cy in zip(x, y):
            lt |= eq & (cx < cy)
            eq &= cx == cy
        ok = lt | (eq & (idx[a:b] < idx[a + 1:b + 1]))
        assert bool(ok.all()), f"order violated in [{a},{b})"


# ------------------------------------------------------- records without an index payload
_C1 = 0xBF58476D1CE4E5B9 - (1 << 64)  # SplitMix64 finaliser constants (Steele, Lea, Flood 2014),
_C2 = 0x94D049BB133111EB - (1 << 64)  # as signed int64 (products wrap like uint64)


def _lsr(x: torch.Tensor, s: int) -> torch.Tensor:
    return (x >> s) & ((1 << (64 - s)) - 1)


def _mix(x: torch.Tensor) -> torch.Tensor:
    x = x ^ _lsr(x, 30)
    x = x * _C1
    x = x ^ _lsr(x, 27)
    x = x * _C2
    return x ^ _lsr(x, 31)


def record_fingerprint(t: torch.Tensor, block: int = 1 << 25) -> tuple[int, int]:
    """Two sums (mod 2^64) of independent hashes of every record: equal for any two orders of
    the same records, and different, short of a 2^-64-scale accident, for different multisets."""
    n, R = t.shape
    w = t.view(torch.int64).view(n, R // 8)
    s1 = torch.zeros((), dtype=torch.int64, device=t.device)
    s2 = torch.zeros((), dtype=torch.int64, device=t.device)
    for a in range(0, n, block):
        b = min(n, a + block)
        h = torch.zeros(b - a, dtype=torch.int64, device=t.device)
        for k in range(R // 8):
            h = _mix(h + w[a:b, k])
        s1 += h.sum()
        s2 += _mix(h ^ 0x5DEECE66D).sum()
    return int(s1), int(s2)


def check_sorted_same_records(out: torch.Tensor, pristine: torch.Tensor, key_size: int,
                              block: int = 1 << 25) -> None:
    """Keys non-decreasing, and the same multiset of records as the input (by fingerprint).
    For records that are keys alone, or keys without duplicates, this is the unique sort."""
    n, R = out.shape
    wo = out.view(torch.int64).view(n, R // 8)
    for a in range(0, n - 1, block):
        b = min(n - 1, a + block)
        x = _ukey_words(wo[a:b], key_size)
        y = _ukey_words(wo[a + 1:b + 1], key_size)
        lt = torch.zeros(b - a, dtype=torch.bool, device=out.device)
        eq = torch.ones(b - a, dtype=torch.bool, device=out.device)
        for cx, cy in zip(x, y):
            lt |= eq & (cx < cy)
            eq &= cx == cy
        assert bool((lt | eq).all()), f"order violated in [{a},{b})"
    assert record_fingerprint(out) == record_fingerprint(pristine), "the output is not a permutation of the input"
