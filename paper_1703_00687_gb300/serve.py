"""A sort server on one GPU with continuous batching and an HBM admission cap.

Requests (host record arrays) arrive at any time.  A scheduler thread admits them in arrival
order while the device memory they need fits under the cap, groups waiting requests with the
same record layout into one segmented sort, and runs each group on one of several CUDA
streams ("lanes"), with its copies on one copy-in and one copy-out stream shared by all
lanes, so that the copies and kernels of different groups overlap on the device.
A request's future resolves to its sorted records on the host.

The sort is stable and every segment of a segmented call is sorted on its own, so a
request's result does not depend on what it was batched or overlapped with: it is the same
bytes as sorting it alone.

Memory accounting (per admitted group): its input and scratch buffers (2 * records * rec_size
bytes) plus the library workspace the segmented call needs.  Each lane's workspace is
reserved up front for the largest group the server forms, so no call allocates or
synchronises while others run.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

from . import get_plan, reserve, set_plan, sort, sort_segmented, status, workspace_bytes


@dataclass
class Request:
    records: object          # CPU uint8 tensor (n, rec_size); pinned memory makes copies async
    key_size: int
    arrival: float           # time.perf_counter() when it arrived
    future: Future = field(default_factory=Future)
    n: int = 0
    rec_size: int = 0
    admitted: float = 0.0
    done: float = 0.0
    out: object = None       # pinned host tensor receiving the result

    @property
    def layout(self):
        return (self.rec_size, self.key_size)


def group_bytes(n_records: int, rec_size: int, key_size: int, n_segs: int) -> int:
    """Device bytes a group occupies while it runs: input + scratch + library workspace."""
    return 2 * n_records * rec_size + workspace_bytes(n_records, rec_size, key_size, n_segs)


def form_group(pending, free_bytes: int, max_records: int, max_requests: int, footprint=group_bytes):
    """Choose the next group from the waiting requests (oldest first).

    The oldest request must fit in ``free_bytes`` (else nothing is admitted: it is not
    overtaken, so it cannot starve).  Later requests with the same (rec_size, key_size) join
    while the group stays within ``max_records``, ``max_requests`` and ``free_bytes``.
    Returns the list of requests taken out of ``pending`` (a deque), possibly empty.
    """
    if not pending:
        return []
    head = pending[0]
    R, K = head.layout
    if footprint(head.n, R, K, 1) > free_bytes:
        return []
    group, total = [head], head.n
    for r in list(pending)[1:]:
        if len(group) >= max_requests:
            break
        if r.layout != (R, K) or total + r.n > max_records:
            continue
        if footprint(total + r.n, R, K, len(group) + 1) > free_bytes:
            continue
        group.append(r)
        total += r.n
    taken = {id(r) for r in group}
    kept = [r for r in pending if id(r) not in taken]
    pending.clear()
    pending.extend(kept)
    return group


class _Lane:
    def __init__(self, torch, device, timing, max_requests):
        self.stream = torch.cuda.Stream(device=device)
        # segment offsets of the lane's group, copied from pinned memory allocated once
        self.h_offs = torch.empty(max_requests + 1, dtype=torch.int64, pin_memory=True)
        self.d_offs = torch.empty(max_requests + 1, dtype=torch.int64, device=device)
        self.in_start = torch.cuda.Event(enable_timing=timing)  # the group's copy-in may start
        self.in_done = torch.cuda.Event(enable_timing=timing)   # the group's input is on the device
        self.sorted = torch.cuda.Event(enable_timing=timing)    # the group is sorted
        self.event = torch.cuda.Event(enable_timing=timing)     # the group's results are on the host
        self.launch_s = 0.0
        self.group = None
        self.hold = None        # device tensors of the running group
        self.bytes = 0


class Server:
    """``Server(cap_bytes).submit(records, key_size) -> Future`` of the sorted host records.

    ``cap_bytes``: device memory the admitted groups may hold at once.  ``lanes``: streams
    that run groups concurrently.  ``max_group_records`` / ``max_group_requests`` bound one
    group (and size the workspace reserved per lane).  ``plans``: on-chip thresholds to sort
    groups with (``autotune.ONCHIP_KNOBS``, which size no workspace) -- a dict per (rec_size,
    key_size), or "auto" for the autotuner's cached plan of each group's batch shape
    (``autotune.apply_segmented``); they are set around each group's launch on the scheduler
    thread (the plan is process-wide: other threads should not sort meanwhile).
    """

    def __init__(self, cap_bytes: int = 120 * 10 ** 9, lanes: int = 4, max_group_records: int = 128 * 10 ** 6,
                 max_group_requests: int = 256, device=None, poll_s: float = 20e-6, timing: bool = False,
                 plans=None, _torch=None):
        import torch

        torch = _torch or torch  # (tests: a CPU stand-in for the CUDA streams and events)
        self.plans = plans
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.cap = int(cap_bytes)
        self.max_records = int(max_group_records)
        self.max_requests = int(max_group_requests)
        self.poll_s = poll_s
        self.timing = timing  # per group: copy-in / sort / copy-out times from CUDA events
        self.lanes = [_Lane(torch, self.device, timing, self.max_requests) for _ in range(lanes)]
        self.copy_in = torch.cuda.Stream(device=self.device)
        self.copy_out = torch.cuda.Stream(device=self.device)
        self.pending = collections.deque()
        self.in_use = 0
        self.peak_in_use = 0
        self.completed = []      # (records, rec_size, arrival, admitted, done) per finished request
        self.group_times = []    # timing=True: (records, launch s, copy-in ms, sort ms, copy-out ms) per group
        self.groups = 0
        self._cv = threading.Condition()
        self._closing = False
        self._error = None
        self._reserved = {}
        self._launching = []
        self._thread = threading.Thread(target=self._run, name="sort-server", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------------ public
    def submit(self, records, key_size: int = 8, arrival: float | None = None, out=None) -> Future:
        """Queue one sort.  ``out``: optional CPU tensor of the same byte size (pinned memory
        makes the copy asynchronous) that receives the result; by default a pinned tensor is
        allocated for it.  The future resolves to the tensor holding the sorted records."""
        if records.dim() != 2 or records.device.type != "cpu":
            raise ValueError("records must be a 2-D CPU tensor (n, rec_size bytes)")
        req = Request(records=records, key_size=key_size, arrival=time.perf_counter() if arrival is None else arrival)
        req.n = int(records.shape[0])
        req.rec_size = int(records.shape[1] * records.element_size())
        if out is not None:
            if out.device.type != "cpu" or out.numel() * out.element_size() != req.n * req.rec_size:
                raise ValueError("out must be a CPU tensor of the same byte size as records")
            req.out = out
        if group_bytes(req.n, req.rec_size, key_size, 1) > self.cap or req.n > self.max_records:
            req.future.set_exception(ValueError("request larger than the server's admission cap"))
            return req.future
        with self._cv:
            if self._closing:
                raise RuntimeError("server is closed")
            self.pending.append(req)
            self._cv.notify()
        return req.future

    def close(self):
        with self._cv:
            self._closing = True
            self._cv.notify()
        self._thread.join()
        if self._error:
            raise self._error

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # --------------------------------------------------------------- scheduler
    def _reserve(self, lane, R, K):
        key = (id(lane), R, K)
        if key not in self._reserved:
            with self.torch.cuda.device(self.device):
                reserve(self.max_records, R, K, self.max_requests, stream=lane.stream)
            self._reserved[key] = True

    def _set_plan(self, group, R, K):
        """Sets the group's on-chip thresholds (if any); returns the plan to restore, or None."""
        if self.plans is None:
            return None
        from . import autotune

        before = get_plan()
        if self.plans == "auto":
            if not autotune.apply_segmented([r.n for r in group], R, K, knobs=autotune.ONCHIP_KNOBS):
                return None
            return before
        p = self.plans.get((R, K))
        if not p:
            return None
        set_plan(**{**before, **{k: v for k, v in p.items() if k in autotune.ONCHIP_KNOBS}})
        return before

    def _launch(self, lane, group):
        """Three stages on three kinds of stream: the group's host-to-device copies on the
        shared copy-in stream, its sort on the lane's stream, its device-to-host copies on the
        shared copy-out stream.  Copies in each direction therefore run one group at a time,
        in admission order and at the link's full rate, while the sorts of other groups (and
        the copies the other way) overlap with them."""
        torch = self.torch
        R, K = group[0].layout
        total = sum(r.n for r in group)
        self._reserve(lane, R, K)
        now = time.perf_counter()
        with torch.cuda.device(self.device):
            with torch.cuda.stream(lane.stream):
                d_in = torch.empty((total, R), dtype=torch.uint8, device=self.device)
                d_tmp = torch.empty_like(d_in)
            offs, o = [0], 0
            for r in group:
                o += r.n
                offs.append(o)
            d_offs = None
            self.copy_in.wait_stream(lane.stream)  # the buffers' allocation is ordered first
            with torch.cuda.stream(self.copy_in):
                lane.in_start.record(self.copy_in)
                o = 0
                for r in group:
                    d_in[o:o + r.n].copy_(r.records.view(torch.uint8).reshape(r.n, R), non_blocking=True)
                    o += r.n
                if len(group) > 1:
                    # (the lane's last group has finished, so its pinned offsets are free)
                    lane.h_offs[:len(offs)].copy_(torch.tensor(offs, dtype=torch.int64))
                    d_offs = lane.d_offs[:len(offs)]
                    d_offs.copy_(lane.h_offs[:len(offs)], non_blocking=True)
                lane.in_done.record(self.copy_in)
            lane.stream.wait_event(lane.in_done)
            before = self._set_plan(group, R, K)
            try:
                if len(group) == 1:
                    sort(d_in, K, tmp=d_tmp, stream=lane.stream)
                else:
                    sort_segmented(d_in, d_offs, K, tmp=d_tmp, stream=lane.stream, total=total)
            finally:
                if before is not None:
                    set_plan(**before)
            lane.sorted.record(lane.stream)
            self.copy_out.wait_event(lane.sorted)
            with torch.cuda.stream(self.copy_out):
                o = 0
                for r in group:
                    if r.out is None:
                        r.out = torch.empty((r.n, R), dtype=torch.uint8, pin_memory=True)
                    r.out.view(torch.uint8).reshape(r.n, R).copy_(d_in[o:o + r.n], non_blocking=True)
                    r.admitted = now
                    o += r.n
                lane.event.record(self.copy_out)
        lane.launch_s = time.perf_counter() - now
        lane.group = group
        lane.hold = (d_in, d_tmp, d_offs)
        lane.bytes = group_bytes(total, R, K, len(group))
        self.in_use += lane.bytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        self.groups += 1

    def _retire(self, lane):
        st = status(lane.stream)
        now = time.perf_counter()
        for r in lane.group:
            r.done = now
            out, r.out, r.records = r.out, None, None  # the server keeps no request data
            if st != 0:
                r.future.set_exception(RuntimeError(f"device status {st}"))
            else:
                r.future.set_result(out)
            self.completed.append((r.n, r.rec_size, r.arrival, r.admitted, r.done))
        if self.timing:
            self.group_times.append((sum(r.n for r in lane.group), lane.launch_s,
                                     lane.in_start.elapsed_time(lane.in_done), lane.in_done.elapsed_time(lane.sorted),
                                     lane.sorted.elapsed_time(lane.event)))
        self.in_use -= lane.bytes
        lane.group, lane.hold, lane.bytes = None, None, 0

    def _run(self):
        torch = self.torch
        try:
            torch.cuda.set_device(self.device)
            while True:
                busy = False
                for lane in self.lanes:
                    if lane.group is not None and lane.event.query():
                        self._retire(lane)
                        busy = True
                with self._cv:
                    free = [ln for ln in self.lanes if ln.group is None]
                    group = []
                    if free and self.pending:
                        group = form_group(self.pending, self.cap - self.in_use, self.max_records, self.max_requests)
                    idle = not group and not busy
                    if idle and self._closing and not self.pending and len(free) == len(self.lanes):
                        return
                    if idle and not self.pending and len(free) == len(self.lanes):
                        self._cv.wait(timeout=0.05)
                        continue
                if group:
                    self._launching = group  # (failed too if the launch raises)
                    self._launch(free[0], group)
                    self._launching = []
                elif idle:
                    time.sleep(self.poll_s)
        except BaseException as e:  # fail every waiting request rather than hang them
            self._error = e
            with self._cv:
                waiting = list(self.pending) + list(self._launching)
                self.pending.clear()
                self._closing = True  # (submit now raises: nothing would serve the request)
            for lane in self.lanes:
                waiting += lane.group or []
            for r in waiting:
                if not r.future.done():
                    r.future.set_exception(e)


def percentile(xs, q):
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    s = sorted(xs)
    if not s:
        return None
    k = (len(s) - 1) * q / 100.0
    i = int(k)
    j = min(i + 1, len(s) - 1)
    return s[i] + (s[j] - s[i]) * (k - i)
