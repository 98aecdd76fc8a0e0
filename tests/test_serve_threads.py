"""The server's threads on the CPU: CUDA streams and events replaced by stand-ins whose work
"finishes" a few milliseconds after it is recorded, and the library's sort replaced by a numpy
sort, so that admission, grouping, completion and shutdown run for real without a GPU.  Every
request must come back sorted, within a time limit (a lost wake-up would leave one waiting
forever)."""
import random
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1703_00687_gb300 import serve  # noqa: E402


class _Event:
    def __init__(self, enable_timing=False):
        self.ready = 0.0

    def record(self, stream=None):
        self.ready = time.perf_counter() + random.uniform(0.0005, 0.004)

    def query(self):
        return time.perf_counter() >= self.ready

    def synchronize(self):
        while not self.query():
            time.sleep(0.0002)

    def elapsed_time(self, other):
        return 1.0


class _Stream:
    def __init__(self, device=None):
        pass

    def wait_stream(self, other):
        pass

    def wait_event(self, ev):
        pass


class _Ctx:
    def __init__(self, *a):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *e):
        return False


class _Cuda:
    Stream, Event = _Stream, _Event
    device = stream = _Ctx

    @staticmethod
    def set_device(d):
        pass

    @staticmethod
    def current_device():
        return 0


class _FakeTorch:
    cuda = _Cuda

    def __getattr__(self, name):
        return getattr(torch, name)

    @staticmethod
    def empty(*a, pin_memory=False, device=None, **kw):
        return torch.empty(*a, **kw)

    @staticmethod
    def zeros(*a, pin_memory=False, device=None, **kw):
        return torch.zeros(*a, **kw)


def _key_sort(t, key_size):  # stable sort of (n, R) uint8 records by their little-endian key
    a = t.numpy()
    k = a[:, :key_size].copy().view("<u8").ravel() if key_size == 8 else None
    t.copy_(torch.from_numpy(a[np.argsort(k, kind="stable")]))


@pytest.fixture
def cpu_server(monkeypatch):
    launched = {}
    monkeypatch.setattr(serve, "reserve", lambda *a, **k: None)
    monkeypatch.setattr(serve, "status", lambda *a, **k: 0)
    monkeypatch.setattr(serve, "workspace_bytes", lambda n, R, K, s: 1024 * s)
    monkeypatch.setattr(serve, "sort", lambda t, K, tmp=None, stream=None: _key_sort(t, K))

    def seg(t, offs, K, tmp=None, stream=None, total=None):
        o = offs.tolist()
        for i in range(len(o) - 1):
            _key_sort(t[o[i]:o[i + 1]], K)
    monkeypatch.setattr(serve, "sort_segmented", seg)
    return launched


@pytest.mark.timeout(120)
def test_every_request_comes_back_sorted(cpu_server):
    rng = np.random.default_rng(3)
    with serve.Server(cap_bytes=1 << 30, lanes=4, max_group_records=3000, device="cpu", _torch=_FakeTorch()) as srv:
        futs, inputs = [], []
        for i in range(300):
            n = int(rng.choice([3, 40, 200, 600, 900]))
            a = rng.integers(0, 256, size=(n, 8), dtype=np.uint8)
            inputs.append(a)
            futs.append(srv.submit(torch.from_numpy(a.copy()), 8))
            if rng.random() < 0.3:
                time.sleep(0.001)
        t0 = time.perf_counter()
        for f in futs:
            f.result(timeout=max(0.1, 30 - (time.perf_counter() - t0)))
    for a, f in zip(inputs, futs):
        k = a.copy().view("<u8").ravel()
        np.testing.assert_array_equal(f.result().numpy(), a[np.argsort(k, kind="stable")])
    assert srv.in_use == 0 and not srv.pending and srv.groups > 1


@pytest.mark.timeout(60)
def test_a_lone_request_is_served_without_any_other_activity(cpu_server):
    with serve.Server(cap_bytes=1 << 30, lanes=3, device="cpu", _torch=_FakeTorch()) as srv:
        for _ in range(5):  # each arrives while the server is idle: nothing else wakes it
            a = np.arange(64, dtype=np.uint64)[::-1].copy().view(np.uint8).reshape(64, 8)
            f = srv.submit(torch.from_numpy(a.copy()), 8)
            out = f.result(timeout=5)
            assert np.array_equal(out.numpy().view("<u8").ravel(), np.arange(64, dtype=np.uint64))
            time.sleep(0.01)


@pytest.mark.timeout(60)
def test_a_failing_launch_fails_its_requests_instead_of_leaving_them_waiting(cpu_server, monkeypatch):
    def boom(t, K, tmp=None, stream=None):
        raise RuntimeError("launch failed")
    monkeypatch.setattr(serve, "sort", boom)
    srv = serve.Server(cap_bytes=1 << 30, lanes=2, device="cpu", _torch=_FakeTorch())
    a = np.zeros((10, 8), dtype=np.uint8)
    f = srv.submit(torch.from_numpy(a), 8)
    with pytest.raises(RuntimeError, match="launch failed"):
        f.result(timeout=10)
    with pytest.raises(RuntimeError):
        srv.close()  # (re-raises the scheduler's error)
