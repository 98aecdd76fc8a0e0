"""A sort captured once in a CUDA graph and replayed.

Every launch of a sort is issued by the host in a fixed order (the number of levels depends
only on the key size, and each kernel reads the device-side bin lists to decide how much
work it has), so one host call can be recorded as a graph and replayed with one launch.
This removes the per-kernel launch cost, which dominates batches of many small sorts.

The graph holds the buffers and the offsets it was captured with: a replay sorts whatever
those buffers hold at that moment.  The library's workspace for the capture stream is
allocated by an uncaptured call first (an allocation cannot be recorded).
"""
from __future__ import annotations

from . import get_plan, set_plan, sort, sort_segmented


class SortGraph:
    """``SortGraph(records, key_size, offsets=None, tmp=None, plan=None)``; then ``replay()`` sorts.

    With ``offsets`` (CUDA 64-bit tensor of n_segs + 1 record offsets) each segment is
    sorted on its own (``sort_segmented``), else the whole tensor (``sort``).  Construction
    sorts ``records`` once (the uncaptured call), which a later replay repeats harmlessly.

    ``plan``: the plan the graph is recorded with -- a dict of ``set_plan`` knobs, or "auto"
    for the autotuner's cached plan of this shape (``autotune.apply`` / ``apply_segmented``;
    the current plan if none is cached).  The knobs are baked into the recorded launches; the
    process-wide plan is restored afterwards.
    """

    def __init__(self, records, key_size: int, offsets=None, tmp=None, stream=None, plan=None):
        import torch

        self.records = records
        self.offsets = offsets
        self.tmp = torch.empty_like(records) if tmp is None else tmp
        self.stream = torch.cuda.Stream(device=records.device) if stream is None else stream
        self.key_size = key_size
        self.total = int(offsets[-1].item()) if offsets is not None else records.shape[0]
        before = get_plan()
        try:
            self.applied = self._apply(plan)
            self.plan = get_plan()
            self.stream.wait_stream(torch.cuda.current_stream(records.device))
            self._call()  # allocates the workspace of this stream
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
                self._call()
        finally:
            set_plan(**before)

    def _apply(self, plan) -> bool:
        if plan is None:
            return False
        if isinstance(plan, dict):
            set_plan(**{**get_plan(), **plan})
            return True
        if plan != "auto":
            raise ValueError("plan must be None, a dict of plan knobs, or 'auto'")
        from . import autotune

        rec_size = self.records.shape[1] * self.records.element_size() if self.records.dim() == 2 else \
            self.records.element_size()
        if self.offsets is None:
            return autotune.apply(self.total, rec_size, self.key_size)
        off = self.offsets.cpu().numpy()
        return autotune.apply_segmented(off[1:] - off[:-1], rec_size, self.key_size)

    def _call(self):
        if self.offsets is None:
            sort(self.records, self.key_size, tmp=self.tmp, stream=self.stream)
        else:
            sort_segmented(self.records, self.offsets, self.key_size, tmp=self.tmp, stream=self.stream,
                           total=self.total)

    def replay(self):
        """Sorts the captured buffers again (asynchronously, on the capture stream: the caller
        orders it after the writes of its input with ``stream.wait_stream``)."""
        import torch

        with torch.cuda.stream(self.stream):
            self.graph.replay()
