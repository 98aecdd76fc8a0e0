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
