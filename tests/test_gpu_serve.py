"""Serving form: the resident decoded-block cache and the continuous-batching
loop give each request exactly the result it gets alone."""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve_setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_09396_gb300 as H
    lf = S.make_lf(61, 8, 8, 128, 128, 4, 3.0, "pink")
    data = O.encode(lf, 3, 16, 4, 4, t_ref=60, t_pred=120).stream
    geo = S.lf_geometry(8, 8, 128, 128)
    return torch, H, H.Stream(data), geo


def _alone(torch, H, st, arr):
    out = H.render_views([st], arr)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_resident_cache_equals_render_views(serve_setup):
    torch, H, st, geo = serve_setup
    from paper_1902_09396_gb300.serve import ResidentCache
    cache = ResidentCache(st, 64 << 20)
    sets = [S.views_to_array(S.random_views(s, geo, 3, [(96, 96), (64, 40)])) for s in (62, 63, 62, 64)]
    decoded = []
    for arr in sets:
        out = torch.zeros(H.out_size(arr), dtype=torch.float32, device="cuda")
        cache.render(arr, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), _alone(torch, H, st, arr))
        decoded.append(cache.stats()["blocks_decoded"])
    assert decoded[0] > 0
    assert decoded[2] == decoded[1]          # the repeated views found every block resident


def test_resident_cache_evicts_correctly(serve_setup):
    """A cache far smaller than one call's working set: evictions every call,
    misses that find no slot fall back to direct decode, results unchanged."""
    torch, H, st, geo = serve_setup
    from paper_1902_09396_gb300.serve import ResidentCache
    cache = ResidentCache(st, 40 * 16 * 16 * 4)
    for s in (65, 66, 65, 67):
        arr = S.views_to_array(S.random_views(s, geo, 2, [(80, 80)]))
        out = torch.zeros(H.out_size(arr), dtype=torch.float32, device="cuda")
        cache.render(arr, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), _alone(torch, H, st, arr))


def test_served_results_equal_alone(serve_setup):
    """Requests arriving together are admitted by output memory into several
    overlapping batches; each result equals the request rendered alone."""
    torch, H, st, geo = serve_setup
    from paper_1902_09396_gb300.serve import ResidentCache, serve_continuous
    reqs = S.stereo_requests(68, geo, 14, rate=5000.0, sizes=((64, 64), (96, 80), (128, 128)))
    cache = ResidentCache(st, 8 << 20)
    pool = 3 * 2 * 128 * 128 * 3           # room for about three of the largest pairs
    rep, served = serve_continuous(cache, reqs, pool, max_batch_views=6, max_inflight=2, keep_results=True)
    assert rep.batches >= 3 and len(served) == len(reqs)
    for r in reqs:
        arr = S.views_to_array([r.left, r.right])
        want = _alone(torch, H, st, arr)
        assert np.max(np.abs(served[r.rid].result - want)) <= 1e-3
        assert np.array_equal(served[r.rid].result, want)
