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


def test_onchip_candidates_are_accepted_and_start_with_the_default():
    cs = at.onchip_candidates()
    assert cs[0] == {"tiny_records": 0, "enum_records": 0}
    old = rg.get_plan()
    try:
        for c in cs:
            rg.set_plan(**{**old, **c})
            assert all(rg.get_plan()[k] == v for k, v in c.items())
        for bad in ({"tiny_records": 1}, {"tiny_records": 65}, {"enum_records": 7}, {"enum_records": 65}):
            with pytest.raises(rg.RadixSortError):
                rg.set_plan(**{**old, **bad})
    finally:
        rg.set_plan(**old)


def test_segment_signature_groups_batches_of_one_distribution(tmp_path):
    rng = np.random.default_rng(5)
    a = rng.integers(1, 200, 3000)
    b = rng.integers(1, 200, 3000)
    assert at.segment_signature(a) == at.segment_signature(b)
    assert at.segment_signature(a) != at.segment_signature(a * 50)
    cache = str(tmp_path / "plans.json")
    plan = {"tiny_records": 32, "enum_records": 24}
    at.store(at.seg_key("G", a, 16, 8), {"plan": plan, "ms": 1.0}, cache)
    old = rg.get_plan()
    try:
        assert at.apply_segmented(b, 16, 8, cache=cache, gpu="G", knobs=at.ONCHIP_KNOBS)
        assert rg.get_plan()["tiny_records"] == 32 and rg.get_plan()["enum_records"] == 24
        assert not at.apply_segmented(a * 50, 16, 8, cache=cache, gpu="G")
    finally:
        rg.set_plan(**old)


@pytest.mark.gpu
def test_onchip_thresholds_tuned_on_a_batch_and_every_candidate_sorts_like_the_oracle(tmp_path):
    """Tunes the tiny-sorter and enumeration limits on a batch of small segments, then checks
    that every candidate plan (the limits at their extremes included) gives the oracle's
    result for segmented and plain sorts: the thresholds move work between the warp sorter,
    enumeration and further distribution, never the result."""
    torch = pytest.importorskip("torch")
    import oracle
    import workloads as wl

    cache = str(tmp_path / "plans.json")
    rng = np.random.default_rng(8)
    sizes = np.minimum(rng.geometric(1 / 60, 4000), 3000).astype(np.int64)
    e = at.tune_segmented(sizes, 16, 8, reps=2, cache=cache, apply_best=False)
    assert len(e["timings"]) == len(at.onchip_candidates())
    graph_plans = []
    old = rg.get_plan()
    try:
        assert at.apply_segmented(sizes, 16, 8, cache=cache)
        assert {k: rg.get_plan()[k] for k in at.ONCHIP_KNOBS} == {k: e["plan"][k] for k in at.ONCHIP_KNOBS}
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
        n = int(off[-1])
        a = wl.uniform(n, 16, 8, seed=9)
        a[::7, :8] = a[0, :8]  # equal keys: enumeration and the input-order restore
        want = oracle.sort_segmented(a, off, 8)
        plain = wl.uniform(300_000, 24, 16, seed=10)
        want_plain = oracle.sort(plain, 16)
        d_off = torch.from_numpy(off.astype(np.int64)).cuda()
        for p in at.onchip_candidates(tiny=(2, 16, 64), enum=(8, 48, 64)):
            rg.set_plan(**{**old, **p})
            t = torch.from_numpy(a).cuda()
            rg.sort_segmented(t, d_off, 8, total=n)
            np.testing.assert_array_equal(t.cpu().numpy(), want, err_msg=str(p))
            t = torch.from_numpy(plain).cuda()
            rg.sort(t, 16)
            np.testing.assert_array_equal(t.cpu().numpy(), want_plain, err_msg=str(p))
        # a graph recorded with the tuned plan sorts like the oracle too
        rg.set_plan(**old)
        t = torch.from_numpy(a).cuda()
        g = rg.SortGraph(t, 8, offsets=d_off, plan=e["plan"])
        graph_plans.append(g.plan)
        t.copy_(torch.from_numpy(a).cuda())
        g.stream.wait_stream(torch.cuda.current_stream())
        g.replay()
        g.stream.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), want)
        assert rg.get_plan() == old  # the graph restored the process-wide plan
    finally:
        rg.set_plan(**old)
    assert {k: graph_plans[0][k] for k in at.ONCHIP_KNOBS} == {k: e["plan"][k] for k in at.ONCHIP_KNOBS}
