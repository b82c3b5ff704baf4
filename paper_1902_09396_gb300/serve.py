"""Serving loop: continuous batching of view requests over a resident
decoded-block cache (hmlfc_server_*).

Requests (stereo view pairs) arrive over time.  The loop admits waiting
requests into the next batch as long as their output buffers fit the free
part of a device output pool (memory-based admission) and the batch has
room; it keeps up to `max_inflight` batches enqueued on its CUDA stream, so
requests that arrive while others are on the GPU join the next batch without
waiting for the queue to drain, and the device never idles between batches.
Completed batches free their output memory.  Latency = observed completion
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


@dataclass
class Report:
    latencies_ms: list = field(default_factory=list)
    views: int = 0
    makespan_s: float = 0.0
    batches: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "views_per_s": self.views / self.makespan_s,
                "requests": len(lat), "batches": self.batches}


def _pair_array(req, offset: int):
    import synthlf
    arr = synthlf.views_to_array([req.left, req.right])
    arr[0]["out_offset"] = offset
    arr[1]["out_offset"] = offset + req.left.width * req.left.height * 3
    return arr


def _pair_floats(req) -> int:
    return 3 * (req.left.width * req.left.height + req.right.width * req.right.height)


def serve_continuous(cache: ResidentCache, requests, pool_floats: int, max_batch_views: int = 64,
                     max_inflight: int = 2, keep_results: bool = False) -> tuple:
    """Run the request stream through the resident cache with continuous
    batching; returns (Report, {rid: Served})."""
    import torch
    dev = torch.device("cuda", cache.stream.device)
    pool = OutputPool(pool_floats, dev)
    cs = torch.cuda.Stream(device=dev)
    pending = deque()
    inflight = deque()
    served = {}
    rep = Report()
    i = 0
    t0 = time.perf_counter()
    while i < len(requests) or pending or inflight:
        now = time.perf_counter() - t0
        while i < len(requests) and requests[i].arrival <= now:
            pending.append(requests[i])
            i += 1
        while inflight and inflight[0][0].query():
            ev, batch = inflight.popleft()
            t = time.perf_counter() - t0
            for r in batch:
                s = served[r.rid]
                s.done = t
                if keep_results:
                    s.result = pool.buf[s.offset:s.offset + s.n].cpu().numpy()
                pool.release(s.offset, s.n)
        if pending and len(inflight) < max_inflight:
            batch, arrs = [], []
            while pending and 2 * (len(batch) + 1) <= max_batch_views:
                r = pending[0]
                n = _pair_floats(r)
                o = pool.alloc(n)
                if o is None:
                    break                      # no device memory for its output yet
                pending.popleft()
                served[r.rid] = Served(r.rid, r.arrival, offset=o, n=n)
                batch.append(r)
                arrs.append(_pair_array(r, o))
            if batch:
                arr = np.concatenate(arrs)
                with torch.cuda.stream(cs):
                    cache.render(arr, pool.buf, cuda_stream=cs)
                    ev = torch.cuda.Event()
                    ev.record(cs)
                inflight.append((ev, batch))
                rep.batches += 1
                rep.views += 2 * len(batch)
    rep.makespan_s = time.perf_counter() - t0
    rep.latencies_ms = [1000.0 * (s.done - s.arrival) for s in served.values()]
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
        s = Served(r.rid, r.arrival, done=time.perf_counter() - t0, n=_pair_floats(r))
        if keep_results:
            s.result = out[:s.n].cpu().numpy()
        served[r.rid] = s
        rep.views += 2
        rep.batches += 1
    rep.makespan_s = time.perf_counter() - t0
    rep.latencies_ms = [1000.0 * (s.done - s.arrival) for s in served.values()]
    return rep, served
