"""Shared test helpers: key extraction, golden-file parsing and record invariants.

Everything here is plain numpy written from the problem statement (sort records by the
little-endian key in bytes [0, key_size)); it is independent of both the oracle and the
GPU sorter.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def key_ints(recs: np.ndarray, key_size: int) -> list[int]:
    """Python ints of each record's key (little-endian bytes [0, key_size))."""
    return [int.from_bytes(bytes(r[:key_size]), "little") for r in recs]


def key_columns(recs: np.ndarray, key_size: int) -> list[np.ndarray]:
    """Key as uint64 columns, least significant word first (vectorised, any n)."""
    n, r = recs.shape
    kb = np.zeros((n, ((key_size + 7) // 8) * 8), dtype=np.uint8)
    kb[:, :key_size] = recs[:, :key_size]
    words = kb.view("<u8").reshape(n, (key_size + 7) // 8)
    return [np.ascontiguousarray(words[:, j]) for j in range(words.shape[1])]


def stable_sort_by_key(recs: np.ndarray, key_size: int) -> np.ndarray:
    """Library stable sort (numpy lexsort) by key: a special case the oracle must equal."""
    cols = key_columns(recs, key_size)
    order = np.lexsort(cols) if len(cols) > 1 else np.argsort(cols[0], kind="stable")
    return recs[order]


def keys_nondecreasing(recs: np.ndarray, key_size: int) -> bool:
    cols = key_columns(recs, key_size)
    if len(recs) < 2:
        return True
    # lexicographic compare of adjacent rows, most significant word first
    lt = np.zeros(len(recs) - 1, dtype=bool)
    eq = np.ones(len(recs) - 1, dtype=bool)
    for c in reversed(cols):
        a, b = c[:-1], c[1:]
        lt |= eq & (a < b)
        eq &= a == b
    return bool(np.all(lt | eq))


def same_multiset(a: np.ndarray, b: np.ndarray) -> bool:
    """Full-record multiset equality (sort both by all bytes, compare)."""
    if a.shape != b.shape:
        return False
    va = a.view(np.dtype((np.void, a.shape[1]))).ravel()
    vb = b.view(np.dtype((np.void, b.shape[1]))).ravel()
    return bool(np.array_equal(np.sort(va), np.sort(vb)))


def multiset_hash(a: np.ndarray) -> bytes:
    """Order-independent hash of full records (sum and xor of per-record 128-bit digests)."""
    d = np.frombuffer(b"".join(hashlib.blake2b(bytes(r), digest_size=16).digest() for r in a), dtype="<u8")
    d = d.reshape(-1, 2)
    return (int(d[:, 0].sum(dtype=np.uint64)).to_bytes(8, "little") + int(np.bitwise_xor.reduce(d[:, 1])).to_bytes(8, "little"))


def parse_golden(name: str = "hand_examples.txt"):
    """Yield dicts {name, op, rec_size, key_size, lo, width, inp, out} from a golden file."""
    cur = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "example":
                if cur:
                    yield cur
                kv = dict(t.split("=") for t in tok[3:])
                cur = dict(name=tok[1], op=tok[2], rec_size=int(kv["rec_size"]), key_size=int(kv["key_size"]),
                           lo=int(kv.get("lo", 0)), width=int(kv.get("width", 0)), inp=[], out=[])
            elif tok[0] in ("in", "out"):
                words = [int(w, 16) for w in tok[1:]]
                rec = np.array(words, dtype="<u8").view(np.uint8)
                cur["inp" if tok[0] == "in" else "out"].append(rec)
    if cur:
        yield cur


def as_records(rows, rec_size):
    if not rows:
        return np.zeros((0, rec_size), dtype=np.uint8)
    return np.stack(rows).astype(np.uint8)
