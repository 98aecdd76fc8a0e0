"""CUDA-graph replay of the sorts, and the continuous-batching server: each result equals the
oracle's and is the same whether the request ran alone or in the mix."""
import time

import numpy as np
import pytest

import oracle
import paper_1703_00687_gb300 as rg
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_reserve_then_sort_and_workspace_query():
    s = torch.cuda.Stream()
    assert rg.workspace_bytes(10 ** 6, 16, 8) > 0
    rg.reserve(2_000_000, 16, 8, 0, stream=s)
    a = wl.uniform(1_500_000, 16, 8, seed=31)
    t = to_dev(a)
    s.wait_stream(torch.cuda.current_stream())
    rg.sort(t, 8, stream=s)
    assert rg.status(s) == 0
    np.testing.assert_array_equal(t.cpu().numpy(), oracle.sort(a, 8))


@pytest.mark.parametrize("n,R,K", [(3_000, 16, 8), (700_001, 24, 16)])
def test_graph_replay_of_a_plain_sort(n, R, K):
    a = wl.make("uniform", n, R, K, seed=32)
    b = wl.make("uniform", n, R, K, seed=33)
    t = to_dev(a)
    g = rg.SortGraph(t, K)
    g.stream.synchronize()
    np.testing.assert_array_equal(t.cpu().numpy(), oracle.sort(a, K))
    for src in (b, a):  # new contents into the captured buffer, then replay
        t.copy_(to_dev(src))
        g.stream.wait_stream(torch.cuda.current_stream())
        g.replay()
        g.stream.synchronize()
        assert rg.status(g.stream) == 0
        np.testing.assert_array_equal(t.cpu().numpy(), oracle.sort(src, K))


def test_graph_replay_of_a_segmented_sort():
    sizes = wl.batched_sizes(n_segs=2_000, lo=1, hi=40_000, cap=3_000_000, seed=34).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    a = wl.uniform(n, 16, 8, seed=35)
    t = to_dev(a)
    g = rg.SortGraph(t, 8, offsets=torch.from_numpy(off).cuda())
    for _ in range(2):
        t.copy_(to_dev(a))
        g.stream.wait_stream(torch.cuda.current_stream())
        g.replay()
        g.stream.synchronize()
        assert rg.status(g.stream) == 0
        np.testing.assert_array_equal(t.cpu().numpy(), oracle.sort_segmented(a, off.astype(np.uint64), 8))


def test_server_results_are_the_same_alone_and_in_the_mix():
    from paper_1703_00687_gb300.serve import Server

    rng = np.random.default_rng(40)
    reqs = []
    for i in range(48):
        R = int(rng.choice([8, 16, 32]))
        n = int(rng.choice([1, 2, 100, 5_000, 60_000, 250_000]))
        reqs.append(wl.make("uniform", n, R, 8, seed=1000 + i))
    # alone: each request sorted by itself (plain call); the oracle pins a few of them
    alone = []
    for a in reqs:
        t = to_dev(a)
        rg.sort(t, 8)
        alone.append(t.cpu().numpy())
    for i in (0, 5, 17):
        np.testing.assert_array_equal(alone[i], oracle.sort(reqs[i], 8))
    # in the mix: all submitted at once to a server whose cap admits only part of them at a
    # time, so groups form, wait for memory and overlap on several streams
    cap = 40 * 1024 * 1024
    with Server(cap_bytes=cap, lanes=3, max_group_records=400_000, max_group_requests=8) as srv:
        futs = [srv.submit(torch.from_numpy(a).pin_memory(), 8) for a in reqs]
        deadline = time.monotonic() + 120  # one limit for the whole batch
        outs = [f.result(timeout=max(0.1, deadline - time.monotonic())) for f in futs]
        assert srv.groups < len(reqs)  # some requests were batched together
        assert srv.peak_in_use <= cap
    for i, (o, want) in enumerate(zip(outs, alone)):
        np.testing.assert_array_equal(o.numpy(), want, err_msg=f"request {i}")


def test_server_rejects_a_request_larger_than_its_cap():
    from paper_1703_00687_gb300.serve import Server

    with Server(cap_bytes=1 << 20, lanes=1) as srv:
        f = srv.submit(torch.zeros((1 << 20, 16), dtype=torch.uint8), 8)
        with pytest.raises(ValueError):
            f.result(timeout=10)
