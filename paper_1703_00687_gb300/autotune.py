"""Autotuner of the sort's plan: digit width, tile size, the on-chip (mid) bin limit, and the
tiny/mid thresholds inside the on-chip phase (the largest chunk sorted by a warp's sorting
network, the largest bucket finished by enumeration sort).

The knobs change speed only, never the result (the output is the unique stable sort).  For a
workload shape -- record size, key size, record count (rounded to a power of two) and key
distribution, or for a batch the segment count and size quantiles -- the tuner times each
candidate plan on a synthetic input of that shape with CUDA events and keeps the fastest.
Results are cached in a JSON file keyed by the GPU name and the shape, so a later process
applies the choice without timing again.

    from paper_1703_00687_gb300 import autotune
    plan = autotune.tune(n, rec_size, key_size)               # times the candidates (GPU)
    autotune.apply(n, rec_size, key_size)                      # sets the cached plan, if any
    autotune.tune_segmented(sizes, rec_size, key_size)         # the same for a batch of segments
    autotune.apply_segmented(sizes, rec_size, key_size)
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading

from . import chunk_records, get_plan, set_plan, sort

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "radix_gb300", "plans.json")
_lock = threading.Lock()


def shape_key(gpu: str, n: int, rec_size: int, key_size: int, kind: str = "uniform") -> str:
    """Cache key: the GPU, the layout and the count's power-of-two bucket."""
    bucket = max(0, int(math.log2(max(1, n))))
    return f"{gpu}|R{rec_size}|K{key_size}|n2^{bucket}|{kind}"


# knobs that size nothing: a server may switch them between groups on a reserved workspace
ONCHIP_KNOBS = ("tiny_records", "enum_records")


def segment_signature(sizes) -> str:
    """A batch's shape for the cache: segment count and size quantiles, rounded to powers of
    two (batches drawn from one distribution share it)."""
    import numpy as np

    s = np.sort(np.asarray(sizes, dtype=np.int64))
    if len(s) == 0:
        return "S0"
    q = [int(s[min(len(s) - 1, int(f * len(s)))]) for f in (0.1, 0.5, 0.9)] + [int(s[-1])]
    r = [1 << max(0, int(math.log2(max(1, v)))) for v in q]
    return f"S2^{int(math.log2(len(s)))}|q{r[0]}-{r[1]}-{r[2]}|max{r[3]}"


def onchip_candidates(tiny=(16, 32, 64), enum=(24, 32, 48, 64)):
    """Plans that vary the on-chip thresholds only (the default first)."""
    out = [{"tiny_records": 0, "enum_records": 0}]
    for t, e in itertools.product(tiny, enum):
        out.append({"tiny_records": t, "enum_records": e})
    return out


def candidates(rec_size: int, n: int, widths=(8, 9, 10), tiles=(1024, 2048, 4096), chunk_fracs=(1.0, 0.75, 0.5)):
    """Candidate plans for one shape.  Tiles above 64 KB of records and on-chip limits that
    would not shorten the level count are dropped; a plan of zeros is the built-in default."""
    cap = chunk_records(rec_size)
    out = [{"digit_bits_max": 0, "tile_records": 0, "chunk_records": 0}]
    for w, t, f in itertools.product(widths, tiles, chunk_fracs):
        if t * rec_size > 128 * 1024:
            continue
        c = int(cap * f) if f < 1.0 else 0
        if c and c < 64:
            continue
        if n <= cap and (w, t) != (widths[0], tiles[0]):
            continue  # the input fits on chip: only the on-chip limit matters
        out.append({"digit_bits_max": w, "tile_records": t, "chunk_records": c})
    seen, uniq = set(), []
    for p in out:
        k = tuple(sorted(p.items()))
        if k not in seen:
            seen.add(k)
            uniq.append(p)
    return uniq


def load(cache: str = DEFAULT_CACHE) -> dict:
    try:
        with open(cache) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, cache: str = DEFAULT_CACHE) -> None:
    with _lock:
        d = load(cache)
        d[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)


def _gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name().replace("|", "/")


def tune(n: int, rec_size: int, key_size: int, kind: str = "uniform", reps: int = 3, cache: str = DEFAULT_CACHE,
         plans=None, seed: int = 77, apply_best: bool = True) -> dict:
    """Times every candidate plan on n synthetic records of the shape; caches and returns the
    fastest ({"plan": ..., "ms": ..., "timings": [...]}).  The plan in force before the call
    is restored unless ``apply_best``."""
    import torch

    import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    h = torch.empty((n, rec_size), dtype=torch.uint8, pin_memory=True)
    wl.make(kind, n, rec_size, key_size, seed, out=h)
    pristine = h.to(dev)
    buf, tmp = torch.empty_like(pristine), torch.empty_like(pristine)
    stream = torch.cuda.current_stream(dev)
    before = get_plan()
    timings = []
    try:
        for p in plans or candidates(rec_size, n):
            set_plan(**{**before, **p})
            buf.copy_(pristine)
            sort(buf, key_size, tmp=tmp, stream=stream)  # warm-up (workspace, caches)
            ms = []
            for _ in range(reps):
                buf.copy_(pristine)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sort(buf, key_size, tmp=tmp, stream=stream)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            timings.append({"plan": p, "ms": sorted(ms)[len(ms) // 2]})
    finally:
        set_plan(**before)
    best = min(timings, key=lambda e: e["ms"])
    entry = {"plan": best["plan"], "ms": best["ms"], "n": n, "timings": timings}
    store(shape_key(_gpu_name(), n, rec_size, key_size, kind), entry, cache)
    if apply_best:
        set_plan(**{**before, **best["plan"]})
    return entry


def lookup(n: int, rec_size: int, key_size: int, kind: str = "uniform", cache: str = DEFAULT_CACHE, gpu=None):
    """The cached plan for the shape, or None."""
    e = load(cache).get(shape_key(gpu or _gpu_name(), n, rec_size, key_size, kind))
    return e["plan"] if e else None


def apply(n: int, rec_size: int, key_size: int, kind: str = "uniform", cache: str = DEFAULT_CACHE, gpu=None) -> bool:
    """Sets the cached plan for the shape (keeping the other knobs); False if none is cached."""
    p = lookup(n, rec_size, key_size, kind, cache, gpu)
    if p is None:
        return False
    set_plan(**{**get_plan(), **p})
    return True


def tune_segmented(sizes, rec_size: int, key_size: int, reps: int = 3, cache: str = DEFAULT_CACHE, plans=None,
                   seed: int = 78, apply_best: bool = True) -> dict:
    """Times candidate plans (by default the on-chip thresholds, ``onchip_candidates``) on one
    segmented sort of uniform records with these segment sizes; caches and returns the fastest
    ({"plan": ..., "ms": ..., "timings": [...]}), as ``tune`` does."""
    import numpy as np
    import torch

    import workloads as wl

    from . import sort_segmented

    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    n = int(off[-1])
    dev = torch.device("cuda", torch.cuda.current_device())
    h = torch.empty((n, rec_size), dtype=torch.uint8, pin_memory=True)
    wl.make("uniform", n, rec_size, key_size, seed, out=h)
    pristine = h.to(dev)
    d_off = torch.from_numpy(off).to(dev)
    buf, tmp = torch.empty_like(pristine), torch.empty_like(pristine)
    stream = torch.cuda.current_stream(dev)
    before = get_plan()
    timings = []
    try:
        for p in plans or onchip_candidates():
            set_plan(**{**before, **p})
            buf.copy_(pristine)
            sort_segmented(buf, d_off, key_size, tmp=tmp, stream=stream, total=n)
            ms = []
            for _ in range(reps):
                buf.copy_(pristine)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sort_segmented(buf, d_off, key_size, tmp=tmp, stream=stream, total=n)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            timings.append({"plan": p, "ms": sorted(ms)[len(ms) // 2]})
    finally:
        set_plan(**before)
    best = min(timings, key=lambda e: e["ms"])
    entry = {"plan": best["plan"], "ms": best["ms"], "n": n, "timings": timings}
    store(seg_key(_gpu_name(), sizes, rec_size, key_size), entry, cache)
    if apply_best:
        set_plan(**{**before, **best["plan"]})
    return entry


def seg_key(gpu: str, sizes, rec_size: int, key_size: int) -> str:
    return f"{gpu}|R{rec_size}|K{key_size}|seg|{segment_signature(sizes)}"


def apply_segmented(sizes, rec_size: int, key_size: int, cache: str = DEFAULT_CACHE, gpu=None, knobs=None) -> bool:
    """Sets the cached plan for a batch of this shape (only ``knobs`` of it, if given); False if
    none is cached."""
    e = load(cache).get(seg_key(gpu or _gpu_name(), sizes, rec_size, key_size))
    if e is None:
        return False
    p = e["plan"] if knobs is None else {k: v for k, v in e["plan"].items() if k in knobs}
    set_plan(**{**get_plan(), **p})
    return True
