"""Serving loop: continuous batching of view requests over a resident
decoded-block cache (hmlfc_server_*).

Requests (stereo view pairs) arrive over time.  The loop admits waiting
requests into the next batch as long as their output buffers fit the free
part of a device output pool (memory-based admission) and the batch has
room; it keeps up to `max_inflight` batches enqueued on its CUDA stream, so
requests that arrive while others are on the GPU join the next batch without
waiting for the queue to drain, and the device never idles between batches.
Completed batches free their output memory.  A request whose output can
never fit the pool is rejected on arrival; a request may be cancelled while
queued or while its batch is on the device (its result is then dropped).
The host bookkeeping (Batcher) needs no GPU.  Latency = observed completion
time - arrival time; throughput = views / makespan.
"""
from __future__ import annotations

import ctypes as C
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import Stream, _check, _ptr, _stream_handle, _views_array, lib, render_views


class ResidentCache:
    """hmlfc_server: the decoded-block cache of one stream, resident across calls."""

    def __init__(self, stream: Stream, cache_bytes: int, cuda_stream=None):
        L = lib()
        P = C.c_void_p
        L.hmlfc_server_create.argtypes = [P, C.c_size_t, P, C.POINTER(P)]
        L.hmlfc_server_render.argtypes = [P, P, C.c_int, P, P]
        L.hmlfc_server_stats.argtypes = [P, P, P]
        L.hmlfc_server_free.argtypes = [P]
        L.hmlfc_server_free.restype = None
        h = P()
        _check(L.hmlfc_server_create(stream.handle, int(cache_bytes), _stream_handle(cuda_stream), C.byref(h)))
        self._h = h
        self.stream = stream

    def render(self, views, out, cuda_stream=None):
        va = _views_array(views)
        _check(lib().hmlfc_server_render(self._h, va, len(va), _ptr(out), _stream_handle(cuda_stream)))
        return out

    def stats(self, cuda_stream=None) -> dict:
        o = np.zeros(3, np.int64)
        _check(lib().hmlfc_server_stats(self._h, _stream_handle(cuda_stream), o.ctypes.data_as(C.c_void_p)))
        return {"blocks_decoded": int(o[0]), "decode_items": int(o[1]), "slots": int(o[2])}

    def free(self):
        if getattr(self, "_h", None) is not None:
            lib().hmlfc_server_free(self._h)
            self._h = None

    __del__ = free


class OutputPool:
    """First-fit allocator of FP32 output ranges in one device buffer."""

    def __init__(self, n_floats: int, device):
        import torch
        self.buf = torch.empty(n_floats, dtype=torch.float32, device=device)
        self.free = [(0, n_floats)]

    def alloc(self, n: int):
        for k, (o, sz) in enumerate(self.free):
            if sz >= n:
                if sz == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (o + n, sz - n)
                return o
        return None

    def release(self, o: int, n: int):
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, b in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + b)
            else:
                merged.append((a, b))
        self.free = merged


@dataclass
class Served:
    rid: int
    arrival: float
    done: float = 0.0
    offset: int = 0
    n: int = 0
    result: np.ndarray | None = None
    status: str = "pending"        # pending | queued | inflight | done | rejected | cancelled
    reason: str = ""


@dataclass
class Report:
    latencies_ms: list = field(default_factory=list)
    views: int = 0
    makespan_s: float = 0.0
    batches: int = 0
    rejected: int = 0
    cancelled: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "views_per_s": self.views / max(self.makespan_s, 1e-12),
                "requests": len(self.latencies_ms), "batches": self.batches, "rejected": self.rejected,
                "cancelled": self.cancelled}


def _pair_array(req, offset: int):
    import synthlf
    arr = synthlf.views_to_array([req.left, req.right])
    arr[0]["out_offset"] = offset
    arr[1]["out_offset"] = offset + req.left.width * req.left.height * 3
    return arr


def _pair_floats(req) -> int:
    return 3 * (req.left.width * req.left.height + req.right.width * req.right.height)


class Batcher:
    """Host side of continuous batching (no device work): memory-based
    admission of view requests into batches, cancellation, completion.

    - submit(req): a request whose output can never fit the output pool, or
      whose views alone exceed a batch, is rejected at once (status
      "rejected", with the reason) instead of waiting forever; the others
      queue in arrival order.
    - next_batch(): while fewer than max_inflight batches are on the device,
      admits queued requests in order while their outputs fit the free part
      of the pool and the batch has room; returns [(request, offset)] or [].
    - cancel(rid): a queued request leaves the queue; an in-flight one keeps
      its output range until its batch completes and its result is dropped.
      Returns False for an unknown, finished or rejected request.
    - complete(): the oldest in-flight batch is done; frees its ranges and
      returns its requests that were not cancelled.
    """

    def __init__(self, pool_floats: int, max_batch_views: int = 64, max_inflight: int = 2, pool=None):
        self.pool = pool if pool is not None else _RangePool(pool_floats)
        self.capacity = int(pool_floats)
        self.max_batch_views = int(max_batch_views)
        self.max_inflight = int(max_inflight)
        self.queue = deque()
        self.inflight = deque()
        self.served = {}

    def submit(self, req, now: float = 0.0) -> Served:
        n = _pair_floats(req)
        s = Served(req.rid, req.arrival, n=n)
        self.served[req.rid] = s
        if n > self.capacity:
            s.status, s.done = "rejected", now
            s.reason = f"output of {n} floats exceeds the output pool of {self.capacity} floats"
        elif 2 > self.max_batch_views:
            s.status, s.done = "rejected", now
            s.reason = f"2 views exceed the batch limit of {self.max_batch_views}"
        else:
            s.status = "queued"
            self.queue.append(req)
        return s

    def cancel(self, rid: int, now: float = 0.0) -> bool:
        s = self.served.get(rid)
        if s is None or s.status not in ("queued", "inflight"):
            return False
        if s.status == "queued":
            self.queue = deque(r for r in self.queue if r.rid != rid)
        s.status, s.done = "cancelled", now
        return True

    def next_batch(self) -> list:
        if not self.queue or len(self.inflight) >= self.max_inflight:
            return []
        batch = []
        while self.queue and 2 * (len(batch) + 1) <= self.max_batch_views:
            r = self.queue[0]
            s = self.served[r.rid]
            o = self.pool.alloc(s.n)
            if o is None:
                break                      # no output memory yet: wait for a batch to complete
            self.queue.popleft()
            s.offset, s.status = o, "inflight"
            batch.append((r, o))
        if batch:
            self.inflight.append([r for r, _ in batch])
        return batch

    def complete(self, now: float = 0.0) -> list:
        batch = self.inflight.popleft()
        done = []
        for r in batch:
            s = self.served[r.rid]
            self.pool.release(s.offset, s.n)
            if s.status == "inflight":
                s.status, s.done = "done", now
                done.append(r)
        return done

    def idle(self) -> bool:
        return not self.queue and not self.inflight


class _RangePool(OutputPool):
    """OutputPool bookkeeping without a device buffer."""

    def __init__(self, n_floats: int):
        self.buf = None
        self.free = [(0, int(n_floats))] if n_floats > 0 else []


def serve_continuous(cache: ResidentCache, requests, pool_floats: int, max_batch_views: int = 64,
                     max_inflight: int = 2, keep_results: bool = False, cancel_in_flight=()) -> tuple:
    """Run the request stream through the resident cache with continuous
    batching; returns (Report, {rid: Served}).  Requests whose output cannot
    fit the pool are rejected (Served.status "rejected").  Every rid in
    cancel_in_flight is cancelled right after the batch that holds it has
    been enqueued on the device (a cancellation mid-batch): its result is
    dropped, the batch's other requests are unaffected."""
    import torch
    dev = torch.device("cuda", cache.stream.device)
    pool = OutputPool(pool_floats, dev)
    sched = Batcher(pool_floats, max_batch_views, max_inflight, pool=pool)
    cancel_in_flight = set(cancel_in_flight)
    cs = torch.cuda.Stream(device=dev)
    events = deque()
    rep = Report()
    i = 0
    t0 = time.perf_counter()
    while i < len(requests) or not sched.idle():
        now = time.perf_counter() - t0
        while i < len(requests) and requests[i].arrival <= now:
            sched.submit(requests[i], now)
            i += 1
        while events and events[0].query():
            events.popleft()
            t = time.perf_counter() - t0
            with torch.cuda.nvtx.range("serve: complete batch"):
                for r in sched.complete(t):
                    s = sched.served[r.rid]
                    if keep_results:
                        s.result = pool.buf[s.offset:s.offset + s.n].cpu().numpy()
        batch = sched.next_batch()
        if batch:
            with torch.cuda.nvtx.range(f"serve: launch batch of {len(batch)} requests"):
                arr = np.concatenate([_pair_array(r, o) for r, o in batch])
                with torch.cuda.stream(cs):
                    cache.render(arr, pool.buf, cuda_stream=cs)
                    ev = torch.cuda.Event()
                    ev.record(cs)
            events.append(ev)
            rep.batches += 1
            rep.views += 2 * len(batch)
            for r, _ in batch:
                if r.rid in cancel_in_flight:
                    sched.cancel(r.rid, time.perf_counter() - t0)
    rep.makespan_s = time.perf_counter() - t0
    served = sched.served
    rep.latencies_ms = [1000.0 * (s.done - s.arrival) for s in served.values() if s.status == "done"]
    rep.rejected = sum(s.status == "rejected" for s in served.values())
    rep.cancelled = sum(s.status == "cancelled" for s in served.values())
    return rep, served


def serve_plain(stream: Stream, requests, keep_results: bool = False) -> tuple:
    """The baseline: one plain render call per request, in arrival order,
    each finished before the next starts (a queue, no batching, no resident
    cache)."""
    import torch
    dev = torch.device("cuda", stream.device)
    rep = Report()
    served = {}
    max_n = max(_pair_floats(r) for r in requests)
    out = torch.empty(max_n, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    for r in requests:
        while time.perf_counter() - t0 < r.arrival:
            pass
        arr = _pair_array(r, 0)
        render_views([stream], arr, out)
        torch.cuda.synchronize(dev)
        s = Served(r.rid, r.arrival, done=time.perf_counter() - t0, n=_pair_floats(r), status="done")
        if keep_results:
            s.result = out[:s.n].cpu().numpy()
        served[r.rid] = s
        rep.views += 2
        rep.batches += 1
    rep.makespan_s = time.perf_counter() - t0
    rep.latencies_ms = [1000.0 * (s.done - s.arrival) for s in served.values()]
    return rep, served
