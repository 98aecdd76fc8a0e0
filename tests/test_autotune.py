"""Autotuner: candidate plans, the JSON cache, and (GPU) that a tuned plan still sorts right."""
import numpy as np
import pytest

import paper_1703_00687_gb300 as rg
from paper_1703_00687_gb300 import autotune as at


def test_candidates_are_valid_plans_and_include_the_default():
    for R in (8, 16, 32):
        cs = at.candidates(R, 10 ** 9)
        assert cs[0] == {"digit_bits_max": 0, "tile_records": 0, "chunk_records": 0}
        assert len({tuple(sorted(c.items())) for c in cs}) == len(cs)
        old = rg.get_plan()
        try:
            for c in cs:  # every candidate is accepted by the library
                rg.set_plan(**{**old, **c})
                assert c["tile_records"] * R <= 128 * 1024
        finally:
            rg.set_plan(**old)


def test_small_inputs_only_vary_the_on_chip_limit():
    cs = at.candidates(16, 1000)
    assert {(c["digit_bits_max"], c["tile_records"]) for c in cs[1:]} == {(8, 1024)}


def test_cache_roundtrip_and_apply(tmp_path):
    cache = str(tmp_path / "plans.json")
    assert at.lookup(10 ** 6, 16, 8, cache=cache, gpu="G") is None
    assert not at.apply(10 ** 6, 16, 8, cache=cache, gpu="G")
    plan = {"digit_bits_max": 10, "tile_records": 2048, "chunk_records": 3000}
    at.store(at.shape_key("G", 10 ** 6, 16, 8), {"plan": plan, "ms": 1.0}, cache)
    # same power-of-two bucket hits, another bucket or GPU misses
    assert at.lookup(2 ** 19 + 5, 16, 8, cache=cache, gpu="G") == plan
    assert at.lookup(10 ** 7, 16, 8, cache=cache, gpu="G") is None
    assert at.lookup(10 ** 6, 16, 8, cache=cache, gpu="H") is None
    old = rg.get_plan()
    try:
        assert at.apply(10 ** 6, 16, 8, cache=cache, gpu="G")
        got = rg.get_plan()
        assert all(got[k] == v for k, v in plan.items())
    finally:
        rg.set_plan(**old)


@pytest.mark.gpu
def test_tuned_plan_is_cached_and_sorts_like_the_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    import oracle
    import workloads as wl

    cache = str(tmp_path / "plans.json")
    old = rg.get_plan()
    try:
        plans = [{"digit_bits_max": 0, "tile_records": 0, "chunk_records": 0},
                 {"digit_bits_max": 8, "tile_records": 1024, "chunk_records": 2000},
                 {"digit_bits_max": 10, "tile_records": 4096, "chunk_records": 0}]
        e = at.tune(400_000, 16, 8, reps=2, cache=cache, plans=plans)
        assert e["plan"] in plans and len(e["timings"]) == 3
        assert at.lookup(400_000, 16, 8, cache=cache) == e["plan"]
        for p in plans:  # every candidate sorts correctly (the knobs change speed only)
            rg.set_plan(**{**old, **p})
            a = wl.uniform(400_000, 16, 8, seed=78)
            t = torch.from_numpy(a).cuda()
            rg.sort(t, 8)
            np.testing.assert_array_equal(t.cpu().numpy(), oracle.sort(a, 8))
    finally:
        rg.set_plan(**old)
