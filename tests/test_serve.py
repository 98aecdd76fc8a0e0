"""Host logic of the sort server: group formation under the admission cap (no GPU)."""
import collections

import pytest

from paper_1703_00687_gb300.serve import Request, form_group, percentile


def req(n, R=16, K=8, t=0.0):
    r = Request(records=None, key_size=K, arrival=t)
    r.n, r.rec_size = n, R
    return r


def foot(n, R, K, segs):  # device bytes of a group: in + tmp + 100 bytes per segment
    return 2 * n * R + 100 * segs


def test_oldest_request_heads_the_group_and_same_layout_joins():
    q = collections.deque([req(10), req(20, R=8), req(30), req(40, K=16), req(50)])
    g = form_group(q, 10 ** 9, 10 ** 6, 100, footprint=foot)
    assert [r.n for r in g] == [10, 30, 50]
    assert [r.n for r in q] == [20, 40]  # the rest keep their order
    g2 = form_group(q, 10 ** 9, 10 ** 6, 100, footprint=foot)
    assert [r.n for r in g2] == [20] and [r.n for r in q] == [40]


def test_head_that_does_not_fit_blocks_admission_so_it_cannot_starve():
    q = collections.deque([req(1000), req(1)])
    assert form_group(q, foot(999, 16, 8, 1), 10 ** 6, 100, footprint=foot) == []
    assert len(q) == 2  # nothing overtook the head
    g = form_group(q, foot(1001, 16, 8, 2), 10 ** 6, 100, footprint=foot)
    assert [r.n for r in g] == [1000, 1]


def test_group_limits_records_requests_and_memory():
    q = collections.deque([req(100) for _ in range(10)])
    assert len(form_group(collections.deque(q), 10 ** 9, 350, 100, footprint=foot)) == 3
    assert len(form_group(collections.deque(q), 10 ** 9, 10 ** 6, 4, footprint=foot)) == 4
    cap = foot(500, 16, 8, 5)
    g = form_group(collections.deque(q), cap, 10 ** 6, 100, footprint=foot)
    assert len(g) == 5 and foot(sum(r.n for r in g), 16, 8, len(g)) <= cap


def test_empty_queue_gives_empty_group():
    assert form_group(collections.deque(), 10 ** 9, 10, 10, footprint=foot) == []


def test_percentile_interpolates_order_statistics():
    xs = [5, 1, 4, 2, 3]
    assert percentile(xs, 0) == 1 and percentile(xs, 100) == 5 and percentile(xs, 50) == 3
    assert percentile([0, 10], 99) == pytest.approx(9.9)
    assert percentile([], 50) is None

