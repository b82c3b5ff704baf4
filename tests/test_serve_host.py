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
