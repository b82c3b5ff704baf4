"""Serving form: the resident decoded-block cache and the continuous-batching
loop give each request exactly the result it gets alone."""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu
_stream_bytes = None


@pytest.fixture(scope="module")
def serve_setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_09396_gb300 as H
    lf = S.make_lf(61, 8, 8, 128, 128, 4, 3.0, "pink")
    global _stream_bytes
    data = O.encode(lf, 3, 16, 4, 4, t_ref=60, t_pred=120).stream
    _stream_bytes = data
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


def _oracle_check(ost, r, result, rng, n_pix=300):
    """Sampled pixels of both eyes of a served request against the FP64
    oracle render (random-access decode, Sec. 4.8.1) within 1e-3."""
    arr = S.views_to_array([r.left, r.right])
    pix = []
    for v, view in enumerate((r.left, r.right)):
        pix.append(np.stack([np.full(n_pix, v), rng.integers(0, view.width, n_pix),
                             rng.integers(0, view.height, n_pix)], -1))
    pix = np.concatenate(pix).astype(np.int32)
    want = ost.render_pixels(arr, pix)
    offs = [0, r.left.width * r.left.height * 3]
    widths = [r.left.width, r.right.width]
    got = np.stack([result[offs[v] + (py * widths[v] + px) * 3 + np.arange(3)] for v, px, py in pix])
    assert np.max(np.abs(got - want)) <= 1e-3


def test_served_results_equal_alone(serve_setup):
    """Requests arriving together are admitted by output memory into several
    overlapping batches; each result equals the request rendered alone, and
    sampled pixels of every request agree with the oracle within 1e-3.  In
    the same mix: a request larger than the whole output pool is rejected
    (the loop does not wait for it), two requests are cancelled while their
    batch is on the device (the others are unaffected), and two requests are
    grid views whose pixels are decoded samples: those match the oracle's
    full decode bit for bit."""
    torch, H, st, geo = serve_setup
    from paper_1902_09396_gb300.serve import ResidentCache, serve_continuous
    reqs = S.stereo_requests(68, geo, 14, rate=5000.0, sizes=((64, 64), (96, 80), (128, 128)))
    t_last = reqs[-1].arrival
    big = S.stereo_requests(69, geo, 1, rate=5000.0, sizes=((512, 512),))[0]
    grid = [S.StereoRequest(0, 0.0, S.grid_view(2.0, 5.0, 0.0, 0.0, 128, 128), S.grid_view(3.0, 5.0, 0.0, 0.0, 128, 128)),
            S.StereoRequest(0, 0.0, S.grid_view(7.0, 0.0, 0.0, 0.0, 128, 96), S.grid_view(6.0, 1.0, 0.0, 0.0, 96, 128))]
    extra = [big] + grid
    for k, r in enumerate(extra):
        r.rid, r.arrival = len(reqs) + k, t_last * (k + 1) / (len(extra) + 1)
    mix = sorted(reqs + extra, key=lambda r: r.arrival)
    cancelled = {reqs[3].rid, reqs[9].rid}
    cache = ResidentCache(st, 8 << 20)
    pool = 3 * 2 * 128 * 128 * 3           # room for about three of the largest pairs
    rep, served = serve_continuous(cache, mix, pool, max_batch_views=6, max_inflight=2, keep_results=True,
                                   cancel_in_flight=cancelled)
    assert served[big.rid].status == "rejected" and rep.rejected == 1
    assert rep.cancelled == 2 and all(served[k].status == "cancelled" for k in cancelled)
    assert rep.batches >= 3 and len(served) == len(mix)
    ost = O.Stream(_stream_bytes)
    rng = np.random.default_rng(70)
    dec = ost.decode_all()
    for r in mix:
        s = served[r.rid]
        if r.rid == big.rid or r.rid in cancelled:
            assert s.result is None
            continue
        assert s.status == "done"
        arr = S.views_to_array([r.left, r.right])
        want = _alone(torch, H, st, arr)
        assert np.array_equal(s.result, want)
        _oracle_check(ost, r, s.result, rng)
    for r in grid:
        res = served[r.rid].result
        o = 0
        for v in (r.left, r.right):
            i, j = int(v.H_uv[2]), int(v.H_uv[5])
            img = np.rint(res[o:o + v.width * v.height * 3].reshape(v.height, v.width, 3) * 255.0)
            assert np.array_equal(img.astype(np.uint8), dec[i, j, :v.height, :v.width])
            o += v.width * v.height * 3
