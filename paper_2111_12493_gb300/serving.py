"""Request loop for summarization and update requests (continuous batching).

Requests arrive at any time and are admitted into a fixed number of slots as
slots and device memory free up; admitted requests run concurrently, each on
its own CUDA stream, so the work of several requests overlaps on the GPU.
Graphs stay resident between requests (a summarized graph keeps its context:
CSR, block ids and per-vertex signature state), and update requests are
applied incrementally (Section 3.2) to the graph they name. Requests on one
graph run one at a time in arrival order, so every result equals the result
of running that request's sequence alone.

Request kinds:
  summarize(graph_id, n, src, dst, edge_label, vertex_label, k, cap, keep)
      build a context, refine to k rounds (or the fixpoint), return the
      partition; with keep=True the graph stays resident for updates.
  update(graph_id, ops)
      apply a batch to a resident graph and return its partition at the
      context's k_incremental rounds.
  release(graph_id)
      drop a resident graph and return its memory to the budget.

Summarize requests whose graph is in host memory are uploaded one after the
other by the library (summarize_init_coo queues the edge arrays of one
context at a time on the host link), so one request's upload overlaps the
others' builds and rounds instead of sharing the link with them.

The scheduling logic (admission by slots and memory, per-graph ordering) is
independent of the GPU: `Scheduler` takes an executor callable, which the
tests replace by a CPU stand-in.
"""

from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Any, Callable


@dataclass
class Request:
    kind: str                      # "summarize" | "update" | "release"
    graph_id: Any
    payload: dict
    mem_bytes: int = 0             # device memory the request needs while it runs
    resident_bytes: int = 0        # memory it leaves resident afterwards (summarize with keep)
    arrival: float = field(default_factory=time.perf_counter)
    started: float = 0.0
    finished: float = 0.0
    future: Future = field(default_factory=Future)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class AdmissionError(RuntimeError):
    """A request that can never fit the memory budget (reported through its future)."""


class Scheduler:
    """Admits requests into `slots` concurrent workers under a memory budget.

    A request is admitted when a slot is free, its graph has no request in
    flight, and budget - resident - in_flight >= its memory. Requests that
    cannot be admitted yet wait; requests behind them on other graphs may be
    admitted first (no head-of-line blocking across graphs), while requests on
    one graph keep their arrival order. A request larger than the whole budget
    fails with AdmissionError.
    """

    def __init__(self, executor: Callable[[Request, int], Any], slots: int = 4,
                 mem_budget: int = 1 << 40):
        self.executor = executor
        self.slots = slots
        self.mem_budget = mem_budget
        self.resident: dict = {}                 # graph_id -> bytes kept on the device
        self.in_flight_bytes = 0
        self.busy_graphs: set = set()
        self.queue: collections.deque = collections.deque()
        self.lock = threading.Condition()
        self.free_slots = list(range(slots))
        self.threads: list = []
        self.closed = False
        self.completed: list = []
        self.max_concurrent = 0
        self._running = 0
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    # -- public API --------------------------------------------------------------------------
    def submit(self, req: Request) -> Future:
        with self.lock:
            if self.closed:
                raise RuntimeError("scheduler closed")
            if req.mem_bytes + req.resident_bytes > self.mem_budget:
                req.future.set_exception(AdmissionError(
                    f"request needs {req.mem_bytes + req.resident_bytes} bytes; budget {self.mem_budget}"))
                return req.future
            self.queue.append(req)
            self.lock.notify_all()
        return req.future

    def close(self, wait: bool = True):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        if wait:
            self._dispatcher.join()
            for t in list(self.threads):
                t.join()

    def drain(self):
        """Block until every submitted request has finished."""
        with self.lock:
            while self.queue or self._running:
                self.lock.wait()

    # -- internals ---------------------------------------------------------------------------
    def _free_bytes(self) -> int:
        return self.mem_budget - sum(self.resident.values()) - self.in_flight_bytes

    def _pick(self):
        """First queued request that can start now (per-graph order kept)."""
        blocked = set()
        for i, req in enumerate(self.queue):
            g = req.graph_id
            if g in blocked or g in self.busy_graphs:
                blocked.add(g)
                continue
            extra = req.resident_bytes - self.resident.get(g, 0) if req.kind == "summarize" else 0
            if req.mem_bytes + max(0, extra) <= self._free_bytes():
                del self.queue[i]
                return req
            blocked.add(g)      # later requests on this graph must wait behind it
        return None

    def _dispatch(self):
        with self.lock:
            while True:
                req = self._pick() if self.free_slots and self.queue else None
                if req is None:
                    if self.closed and not self.queue:
                        return
                    if self.closed and self._running == 0:
                        # nothing runs and nothing queued can start: these never will
                        for r in self.queue:
                            r.future.set_exception(AdmissionError("scheduler closed before the request fit"))
                        self.queue.clear()
                        self.lock.notify_all()
                        return
                    self.lock.wait()
                    continue
                slot = self.free_slots.pop()
                self.busy_graphs.add(req.graph_id)
                self.in_flight_bytes += req.mem_bytes
                self._running += 1
                self.max_concurrent = max(self.max_concurrent, self._running)
                t = threading.Thread(target=self._run, args=(req, slot), daemon=True)
                self.threads.append(t)
                t.start()

    def _run(self, req: Request, slot: int):
        req.started = time.perf_counter()
        try:
            result = self.executor(req, slot)
            err = None
        except BaseException as e:  # noqa: BLE001 - reported through the future
            result, err = None, e
        req.finished = time.perf_counter()
        with self.lock:
            self.in_flight_bytes -= req.mem_bytes
            if err is None:
                if req.kind == "summarize" and req.payload.get("keep"):
                    # the footprint the executor measured, when it reports one
                    measured = result.get("device_bytes") if isinstance(result, dict) else None
                    self.resident[req.graph_id] = int(measured) if measured else req.resident_bytes
                elif req.kind == "release":
                    self.resident.pop(req.graph_id, None)
            self.busy_graphs.discard(req.graph_id)
            self.free_slots.append(slot)
            self._running -= 1
            self.completed.append(req)
            self.lock.notify_all()
        if err is None:
            req.future.set_result(result)
        else:
            req.future.set_exception(err)


def estimate_bytes(n: int, m: int, k_incremental: int = 2) -> int:
    """Device footprint of a resident graph with its incremental state primed,
    before the context exists (admission). Per vertex: partition buffers, the
    round layout, the row store and the per-batch scratch (about 500 bytes with
    two levels) and about 90 bytes per further level; per edge: packed rows,
    CSR, row-store pools and signature lists (about 64 bytes); plus a fixed
    32 MB. Fitted to the contexts' own device_bytes on power-law and uniform
    graphs from 5k to 5M vertices (within a few percent), with a 10% margin;
    the scheduler replaces it by the measured footprint once the graph is
    resident."""
    levels_above_one = max(0, int(k_incremental) - 1)
    return int(1.1 * ((32 << 20) + 500 * n + 64 * m + 90 * levels_above_one * n))


class GpuExecutor:
    """Runs requests through the C-ABI binding, one CUDA stream per slot."""

    def __init__(self, slots: int, device: int = 0):
        import torch

        from . import bisim
        self.torch = torch
        self.bisim = bisim
        self.device = device
        torch.cuda.set_device(device)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.contexts: dict = {}

    def __call__(self, req: Request, slot: int):
        torch, B = self.torch, self.bisim
        torch.cuda.set_device(self.device)
        stream = self.streams[slot]
        with torch.cuda.stream(stream):
            p = req.payload
            if req.kind == "summarize":
                old = self.contexts.pop(req.graph_id, None)
                if old is not None:
                    B.summarize_destroy(old)
                opt = B.default_options(k_incremental=p.get("k_incremental", 2))
                ctx = B.summarize_init_coo(p["n"], p["src"], p["dst"], p["edge_label"], p["vertex_label"],
                                           options=opt, stream=stream)
                rounds, blocks = B.bisim_iterate(ctx, p.get("k", B.FIXPOINT), p.get("cap", 10), stream=stream)
                out = B.get_partition(ctx, stream=stream)
                footprint = 0
                if p.get("keep"):
                    # prime the incremental state so the first update is incremental
                    B.apply_updates(ctx, torch.zeros((0, 4), dtype=torch.int32, device="cuda"), stream=stream)
                    footprint = B.bisim_get_stats(ctx)["device_bytes"]
                    self.contexts[req.graph_id] = ctx
                else:
                    B.summarize_destroy(ctx)
                stream.synchronize()
                return dict(partition=out, rounds=rounds, blocks=blocks, device_bytes=footprint)
            if req.kind == "update":
                ctx = self.contexts[req.graph_id]
                B.apply_updates(ctx, p["ops"], stream=stream)
                out = B.get_partition(ctx, stream=stream)
                stream.synchronize()
                return dict(partition=out, frontier=B.bisim_get_stats(ctx)["last_frontier"])
            if req.kind == "release":
                ctx = self.contexts.pop(req.graph_id, None)
                if ctx is not None:
                    B.summarize_destroy(ctx)
                return None
            raise ValueError(f"unknown request kind {req.kind}")


class Server:
    """Scheduler + GPU executor."""

    def __init__(self, slots: int = 4, mem_budget: int | None = None, device: int = 0):
        import torch
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            mem_budget = int(free * 0.8)
        self.executor = GpuExecutor(slots, device)
        self.scheduler = Scheduler(self.executor, slots=slots, mem_budget=mem_budget)

    def summarize(self, graph_id, n, src, dst, edge_label, vertex_label, k=-1, cap=10, keep=False,
                  k_incremental=2) -> Future:
        m = src.numel()
        est = estimate_bytes(n, m, k_incremental)
        req = Request("summarize", graph_id,
                      dict(n=n, src=src, dst=dst, edge_label=edge_label, vertex_label=vertex_label, k=k,
                           cap=cap, keep=keep, k_incremental=k_incremental),
                      mem_bytes=est, resident_bytes=est if keep else 0)
        return self.scheduler.submit(req)

    def update(self, graph_id, ops, extra_bytes=0) -> Future:
        req = Request("update", graph_id, dict(ops=ops), mem_bytes=int(48 * ops.shape[0]) + extra_bytes)
        return self.scheduler.submit(req)

    def release(self, graph_id) -> Future:
        return self.scheduler.submit(Request("release", graph_id, {}))

    def close(self):
        self.scheduler.close()
        for ctx in list(self.executor.contexts.values()):
            self.executor.bisim.summarize_destroy(ctx)
        self.executor.contexts.clear()
