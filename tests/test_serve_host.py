"""Host logic of the serving and batched forms, on the CPU: the first-fit
output allocator (no overlap, exhaustion only when no free range fits,
releases merge back to one range) against an occupancy model, the latency
summary, and the autotuner's workload signature (order-free, size-aware)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_09396_gb300.serve import OutputPool, Report  # noqa: E402


def test_output_pool_against_occupancy_model():
    N = 1000
    pool = OutputPool(N, "cpu")
    used = np.zeros(N, bool)
    live = []
    rng = np.random.default_rng(5)
    for _ in range(3000):
        if live and rng.random() < 0.45:
            o, n = live.pop(int(rng.integers(len(live))))
            assert used[o:o + n].all()
            used[o:o + n] = False
            pool.release(o, n)
        else:
            n = int(rng.integers(1, 120))
            o = pool.alloc(n)
            if o is None:
                # first fit fails only when no free run of n slots exists
                runs, r = [], 0
                for u in used:
                    r = 0 if u else r + 1
                    runs.append(r)
                assert max(runs) < n
                continue
            assert 0 <= o and o + n <= N and not used[o:o + n].any()
            used[o:o + n] = True
            live.append((o, n))
        # the free list is sorted, disjoint, merged and covers exactly the free slots
        free = np.zeros(N, bool)
        prev_end = -1
        for a, b in pool.free:
            assert b > 0 and a > prev_end
            free[a:a + b] = True
            prev_end = a + b
        assert np.array_equal(free, ~used)
    for o, n in live:
        pool.release(o, n)
    assert pool.free == [(0, N)]


def test_report_summary():
    rep = Report(latencies_ms=[float(x) for x in range(1, 101)], views=200, makespan_s=2.0, batches=7)
    s = rep.summary()
    assert s["p50_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 99))
    assert s["views_per_s"] == 100.0 and s["requests"] == 100 and s["batches"] == 7


class _FakeStream:
    def __init__(self, shape):
        self.info = dict(zip(("nu", "nv", "width", "height", "levels", "block"), shape))


def test_autotune_signature_is_order_free_and_size_aware():
    from paper_1902_09396_gb300.autotune import signature
    import synthlf as S
    st = [_FakeStream((17, 17, 512, 512, 4, 16))]
    geo = S.lf_geometry(17, 17, 512, 512)
    a = S.views_to_array(S.random_views(1, geo, 6, [(256, 256), (512, 512)]))
    b = a[::-1].copy()
    assert signature(st, a) == signature(st, b)
    c = a.copy()
    c[0]["width"] = 300
    assert signature(st, a) != signature(st, c)
    assert signature([_FakeStream((9, 9, 512, 512, 4, 16))], a) != signature(st, a)


class _V:
    def __init__(self, w, h):
        self.width, self.height = w, h


class _Req:
    def __init__(self, rid, w, h, arrival=0.0):
        self.rid, self.arrival, self.left, self.right = rid, arrival, _V(w, h), _V(w, h)


def _drain(b, until_idle=200):
    """Alternate admission and completion (a device that finishes the oldest
    batch each round) until the batcher is idle; returns the batches."""
    batches = []
    for _ in range(until_idle):
        if b.idle():
            return batches
        got = b.next_batch()
        if got:
            batches.append(got)
        else:
            b.complete()
    raise AssertionError("batcher did not drain")


def test_batcher_rejects_requests_larger_than_the_pool():
    """Memory-based admission: a request whose output exceeds the whole pool
    is rejected with a reason at once (it could never be admitted), and the
    other requests are all served."""
    from paper_1902_09396_gb300.serve import Batcher
    pool = 3 * 2 * 64 * 64 * 3
    b = Batcher(pool, max_batch_views=8, max_inflight=2)
    reqs = [_Req(0, 64, 64), _Req(1, 512, 512), _Req(2, 32, 48), _Req(3, 64, 64)]
    for r in reqs:
        b.submit(r)
    assert b.served[1].status == "rejected" and "exceeds the output pool" in b.served[1].reason
    batches = _drain(b)
    assert sorted(r.rid for bt in batches for r, _ in bt) == [0, 2, 3]
    assert all(b.served[k].status == "done" for k in (0, 2, 3))
    assert b.pool.free == [(0, pool)]


def test_batcher_admits_by_free_memory_without_overlap():
    """Ranges of requests in flight at the same time never overlap, and a
    request waits (in order) until a completed batch frees enough memory."""
    from paper_1902_09396_gb300.serve import Batcher, _pair_floats
    rng = np.random.default_rng(3)
    pool = 4 * 2 * 96 * 96 * 3
    b = Batcher(pool, max_batch_views=6, max_inflight=3)
    reqs = [_Req(k, int(rng.integers(8, 97)), int(rng.integers(8, 97))) for k in range(60)]
    for r in reqs:
        b.submit(r)
    live = {}
    order = []
    for _ in range(1000):
        if b.idle():
            break
        got = b.next_batch()
        if got:
            for r, o in got:
                n = _pair_floats(r)
                assert 0 <= o and o + n <= pool
                for o2, n2 in live.values():
                    assert o + n <= o2 or o2 + n2 <= o
                live[r.rid] = (o, n)
                order.append(r.rid)
        else:
            for r in b.complete():
                live.pop(r.rid)
    assert b.idle() and order == list(range(60))


def test_batcher_cancellation_queued_and_in_flight():
    """A queued request that is cancelled is never admitted; one cancelled
    while its batch is on the device keeps its range until the batch
    completes, is not reported done, and its batch's other requests are."""
    from paper_1902_09396_gb300.serve import Batcher
    pool = 2 * 2 * 64 * 64 * 3
    b = Batcher(pool, max_batch_views=4, max_inflight=1)
    for k in range(6):
        b.submit(_Req(k, 64, 64))
    first = b.next_batch()
    assert [r.rid for r, _ in first] == [0, 1]
    assert b.cancel(1) and b.served[1].status == "cancelled"
    assert b.cancel(4) and b.served[4].status == "cancelled"
    assert not b.cancel(4) and not b.cancel(99)
    assert b.next_batch() == []                  # max_inflight reached
    done = b.complete()
    assert [r.rid for r in done] == [0]
    rest = _drain(b)
    assert sorted(r.rid for bt in rest for r, _ in bt) == [2, 3, 5]
    assert [b.served[k].status for k in range(6)] == ["done", "cancelled", "done", "done", "cancelled", "done"]
    assert not b.cancel(0)
    assert b.pool.free == [(0, pool)]
