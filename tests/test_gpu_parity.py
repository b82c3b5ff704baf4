"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Decoded samples must be bit-exact; rendered FP32 views within max-abs 1e-3
(on the [0, 1] scale) of the oracle's FP64 render.  The FP32 render differs
from FP64 only by rounding of the ray setup and the 16-term blend (about
1e-6 here), so 1e-3 is the stated bound, not a loose fit.
"""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu

RENDER_TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def H(torch_cuda):
    import paper_1902_09396_gb300 as H
    H.lib()
    return H


def _all_coords(nu, nv, W, H_):
    ii, jj, xx, yy = np.meshgrid(np.arange(nu), np.arange(nv), np.arange(W), np.arange(H_), indexing="ij")
    return np.stack([ii, jj, xx, yy], -1).reshape(-1, 4).astype(np.int32)


def _decode_gpu(torch, st, coords):
    c = torch.from_numpy(np.ascontiguousarray(coords, np.int32)).cuda()
    out = st.decode_pixels(c)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("q", [1, 4])
def test_decode_all_samples_bit_exact_tiny(H, torch_cuda, tiny_streams, q):
    enc = tiny_streams[q]
    ost = O.Stream(enc.stream)
    full = ost.decode_all()
    st = H.Stream(enc.stream)
    coords = _all_coords(ost.nu, ost.nv, ost.W, ost.H)
    got = _decode_gpu(torch_cuda, st, coords)
    want = full[coords[:, 0], coords[:, 1], coords[:, 3], coords[:, 2]]
    assert np.array_equal(got, want)
    st.check_status()


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL, O.MC_ZERO, O.MC_INTEGER])
@pytest.mark.parametrize("shape", [(2, 8), (3, 16), (2, 5)])
def test_decode_ragged_bit_exact(H, torch_cuda, ragged_lf, mc, shape):
    """Odd grids, partial edge blocks, a non power-of-two block size, every
    MC mode, thresholds on."""
    L, B = shape
    data = O.encode(ragged_lf, L, B, 3, 4, t_ref=30, t_pred=60, mc=mc).stream
    ost = O.Stream(data)
    st = H.Stream(data)
    coords = _all_coords(ost.nu, ost.nv, ost.W, ost.H)
    assert np.array_equal(_decode_gpu(torch_cuda, st, coords), ost.decode_samples(coords))


def test_decode_out_of_range_sets_status(H, torch_cuda, tiny_streams):
    st = H.Stream(tiny_streams[4].stream)
    coords = np.array([[0, 0, 0, 0], [4, 0, 0, 0], [0, 0, 64, 0], [-1, 2, 3, 4], [3, 3, 63, 63]], np.int32)
    got = _decode_gpu(torch_cuda, st, coords)
    assert np.array_equal(got[1:4], np.zeros((3, 3), np.uint8))
    with pytest.raises(H.HmlfcError) as ei:
        st.check_status()
    assert ei.value.code == H.E_INVALID_ARG
    st.check_status()          # cleared by the first check
    want = O.Stream(tiny_streams[4].stream).decode_samples(coords[[0, 4]])
    assert np.array_equal(got[[0, 4]], want)


def test_decode_empty_and_odd_counts(H, torch_cuda, tiny_streams):
    st = H.Stream(tiny_streams[4].stream)
    ost = O.Stream(tiny_streams[4].stream)
    torch = torch_cuda
    empty = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    assert st.decode_pixels(empty).shape == (0, 3)
    rng = np.random.default_rng(5)
    for n in (1, 255, 257, 70001):
        coords = np.stack([rng.integers(0, 4, n), rng.integers(0, 4, n), rng.integers(0, 64, n),
                           rng.integers(0, 64, n)], -1).astype(np.int32)
        assert np.array_equal(_decode_gpu(torch, st, coords), ost.decode_samples(coords))


def _render_gpu(H, torch, streams, views):
    out = H.render_views(streams, views)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _views_mix(cfg, seed, n, sizes):
    geo = S.lf_geometry(cfg.nu, cfg.nv, cfg.width, cfg.height)
    return S.random_views(seed, geo, n, sizes)


@pytest.mark.parametrize("path", [0, 1, 2])
def test_render_tiny_within_tolerance(H, torch_cuda, tiny_streams, tiny_cfg, path):
    """The configured novel view (camera on the (u,v) plane at a random
    (u0, v0), (s,t) offset) plus random pinhole views of ragged sizes; both
    render paths."""
    c = tiny_cfg
    enc = tiny_streams[c.qstep]
    ost = O.Stream(enc.stream)
    dec = ost.decode_all()
    rng = np.random.default_rng(c.seed)
    views = [S.grid_view(rng.random() * 3, rng.random() * 3, rng.random() * 4 - 2, rng.random() * 4 - 2, 64, 64)]
    views += _views_mix(c, 31, 6, [(64, 64), (37, 23), (1, 1), (16, 17), (100, 3)])
    arr = S.views_to_array(views)
    want = O.render_dense(dec, arr)
    H.set_render_path(path)
    try:
        got = _render_gpu(H, torch_cuda, [H.Stream(enc.stream)], arr)
    finally:
        H.set_render_path(0)
    assert np.max(np.abs(got - want)) <= RENDER_TOL


def test_render_paths_identical(H, torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    """The cached, direct and per-tile paths decode the same integers and
    blend in the same order: bitwise equal outputs; so does the cached path
    when its capacity overflows and the rays of some cameras fall back to
    per-ray decode."""
    c = tiny_cfg
    cases = [(H.Stream(tiny_streams[c.qstep].stream), _views_mix(c, 32, 8, [(64, 64), (48, 40), (5, 70)]))]
    geo2 = S.lf_geometry(5, 3, 37, 29)
    d2 = O.encode(ragged_lf, 3, 8, 4, 2, t_ref=20, t_pred=30).stream
    cases.append((H.Stream(d2), S.random_views(37, geo2, 5, [(40, 31), (17, 9)])))
    for st, views in cases:
        arr = S.views_to_array(views)
        outs = []
        try:
            for path in (0, 1, 2):
                H.set_render_path(path)
                outs.append(_render_gpu(H, torch_cuda, [st], arr))
            H.set_render_path(0)
            # room for a few camera images (the other cameras' rays decode directly), for less than one, none
            for cap in (5 * st.info["width"] * st.info["height"] * 4, 4 * 8 * 8 * 4, 0):
                H.set_block_cache_bytes(cap)
                outs.append(_render_gpu(H, torch_cuda, [st], arr))
        finally:
            H.set_render_path(0)
            H.set_block_cache_bytes(H.DEFAULT_CACHE_BYTES)
        for o in outs[1:]:
            assert np.array_equal(outs[0], o)


def test_render_grid_samples_exact(H, torch_cuda, tiny_streams, tiny_cfg):
    """At a camera position with (s,t) on pixel centres the render is the
    decoded view / 255."""
    c = tiny_cfg
    enc = tiny_streams[c.qstep]
    dec = O.Stream(enc.stream).decode_all()
    st = H.Stream(enc.stream)
    for i, j in [(0, 0), (1, 3), (3, 2)]:
        arr = S.views_to_array([S.grid_view(float(i), float(j), 0.0, 0.0, 64, 64)])
        got = _render_gpu(H, torch_cuda, [st], arr).reshape(64, 64, 3)
        assert np.max(np.abs(got - dec[i, j] / 255.0)) <= 1e-6


def test_render_clamped_and_degenerate_views(H, torch_cuda, tiny_streams, tiny_cfg):
    """Rays far outside the grid and image clamp to the edges; a zero-size
    view writes nothing."""
    c = tiny_cfg
    enc = tiny_streams[c.qstep]
    dec = O.Stream(enc.stream).decode_all()
    views = [S.grid_view(-5.0, 9.0, -80.0, 200.0, 20, 20), S.grid_view(1.5, 1.5, 0.0, 0.0, 0, 0),
             S.grid_view(3.9, -0.2, 60.5, -3.25, 33, 9)]
    arr = S.views_to_array(views)
    want = O.render_dense(dec, arr)
    got = _render_gpu(H, torch_cuda, [H.Stream(enc.stream)], arr)
    assert np.max(np.abs(got - want)) <= RENDER_TOL


def _sign_change_view(width, height, x_zero):
    """A view whose projective maps share the denominator w = (X - x_zero) / 64,
    negative left of column x_zero and positive right of it (x_zero a quarter
    pixel off the pixel centres, so |w| >= 1/256 at every ray).  Numerators
    c * w + a small term keep most rays inside the light field on both sides."""
    wr = np.array([1.0 / 64.0, 0.0, -x_zero / 64.0])
    rows_uv = [1.5 * wr + np.array([0.0, 0.002, -0.048]), 2.0 * wr + np.array([0.001, 0.0, -0.02])]
    rows_st = [30.0 * wr + np.array([0.0, 0.2 / 64.0, -4.8 / 64.0]), 25.0 * wr + np.array([0.1 / 64.0, 0.0, -3.0 / 64.0])]
    H_uv = np.concatenate(rows_uv + [wr]).astype(np.float32)
    H_st = np.concatenate(rows_st + [wr]).astype(np.float32)
    return S.View(0, width, height, H_uv, H_st)


@pytest.mark.parametrize("path", [0, 1, 2])
def test_render_views_whose_w_changes_sign(H, torch_cuda, tiny_streams, tiny_cfg, path):
    """Tiles whose corner rays do not all have w > 0 are marked ray by ray;
    the views (ragged 96x40 and 37x23, w changing sign inside) render within
    the bound of the oracle's FP64 render on every path."""
    c = tiny_cfg
    enc = tiny_streams[c.qstep]
    dec = O.Stream(enc.stream).decode_all()
    views = [_sign_change_view(96, 40, 40.25), _sign_change_view(37, 23, 20.75), S.grid_view(1.2, 2.3, 3.5, 1.25, 48, 17)]
    arr = S.views_to_array(views)
    want = O.render_dense(dec, arr)
    try:
        H.set_render_path(path)
        got = _render_gpu(H, torch_cuda, [H.Stream(enc.stream)], arr)
    finally:
        H.set_render_path(0)
    assert np.max(np.abs(got - want)) <= RENDER_TOL


def test_render_multiple_streams(H, torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    """Views of different light fields in one call."""
    c = tiny_cfg
    d1 = tiny_streams[c.qstep].stream
    d2 = O.encode(ragged_lf, 2, 8, 4, 2).stream
    s1, s2 = H.Stream(d1), H.Stream(d2)
    geo2 = S.lf_geometry(5, 3, 37, 29)
    v1 = _views_mix(c, 33, 3, [(40, 40)])
    v2 = S.random_views(34, geo2, 3, [(30, 20)], lf=1)
    arr = S.views_to_array([v1[0], v2[0], v1[1], v2[1], v2[2], v1[2]])
    got = _render_gpu(H, torch_cuda, [s1, s2], arr)
    want1 = O.render_dense(O.Stream(d1).decode_all(), arr[arr["lf"] == 0])
    want2 = O.render_dense(O.Stream(d2).decode_all(), arr[arr["lf"] == 1])
    for k in range(len(arr)):
        o = int(arr[k]["out_offset"])
        n = int(arr[k]["width"]) * int(arr[k]["height"]) * 3
        ref = want1 if arr[k]["lf"] == 0 else want2
        assert np.max(np.abs(got[o:o + n] - ref[o:o + n])) <= RENDER_TOL


def test_dequant_matches_oracle(H, torch_cuda, tiny_streams, ragged_lf):
    for data in (tiny_streams[4].stream, O.encode(ragged_lf, 3, 8, 4, 2).stream):
        co, ro = H.Stream(data).dequant()
        oc, orr = O.Stream(data).dequant()
        assert np.array_equal(co.cpu().numpy().astype(np.float64), oc)
        assert np.array_equal(ro.cpu().numpy().astype(np.float64), orr)


def test_relaxed_forward_and_adjoint(H, torch_cuda, tiny_streams, tiny_cfg):
    """FP32 relaxed render vs the FP64 oracle, and the adjoint (FP32 atomics)
    vs the oracle's transpose, relative to the gradient scale."""
    torch = torch_cuda
    c = tiny_cfg
    data = tiny_streams[c.qstep].stream
    ost = O.Stream(data)
    st = H.Stream(data)
    arr = S.views_to_array(_views_mix(c, 35, 3, [(32, 32), (21, 19)]))
    rng = np.random.default_rng(36)
    co = rng.standard_normal((ost.n_nc, ost.H, ost.W))
    ro = rng.standard_normal((ost.n_roots, 3, ost.H, ost.W))
    want = ost.relax_render(co, ro, arr)
    got = H.render_views_relaxed([st], [torch.tensor(co, dtype=torch.float32, device="cuda")],
                                 [torch.tensor(ro, dtype=torch.float32, device="cuda")], arr)
    torch.cuda.synchronize()
    assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))
    g = rng.standard_normal(want.shape)
    wc, wr = ost.relax_adjoint(arr, g)
    gc = torch.zeros((ost.n_nc, ost.H, ost.W), dtype=torch.float32, device="cuda")
    gr = torch.zeros((ost.n_roots, 3, ost.H, ost.W), dtype=torch.float32, device="cuda")
    H.render_backward([st], arr, torch.tensor(g, dtype=torch.float32, device="cuda"), [gc], [gr])
    torch.cuda.synchronize()
    scale = max(np.max(np.abs(wc)), np.max(np.abs(wr)))
    assert np.max(np.abs(gc.cpu().numpy() - wc)) <= 1e-5 * scale
    assert np.max(np.abs(gr.cpu().numpy() - wr)) <= 1e-5 * scale


@pytest.mark.parametrize("mc", [O.MC_QPEL, O.MC_INTEGER, O.MC_OFF])
def test_relaxed_forward_with_bias(H, torch_cuda, tiny_lf, tiny_cfg, mc):
    """The relaxation carrying the expected rounding (HMLFC_RELAX_BIAS) vs the
    oracle's, at the stream's dequantised coefficients and at random ones;
    unknown flag bits are refused."""
    import ctypes as C
    torch = torch_cuda
    c = tiny_cfg
    data = O.encode(tiny_lf, c.levels, c.block, c.search, 4, mc=mc).stream
    ost = O.Stream(data)
    st = H.Stream(data)
    arr = S.views_to_array(_views_mix(c, 37, 3, [(32, 32), (21, 19)]))
    rng = np.random.default_rng(38)
    co0, ro0 = ost.dequant()
    for co, ro in ((co0, ro0), (rng.standard_normal(co0.shape) * 20, rng.standard_normal(ro0.shape) * 20)):
        want = ost.relax_render(co, ro, arr, bias=True)
        got = H.render_views_relaxed([st], [torch.tensor(co, dtype=torch.float32, device="cuda")],
                                     [torch.tensor(ro, dtype=torch.float32, device="cuda")], arr, bias=True)
        torch.cuda.synchronize()
        assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))
    lib = H.lib()
    va = H._views_array(arr)
    out = torch.zeros(H.out_size(arr), dtype=torch.float32, device="cuda")
    cp = (C.c_void_p * 1)(int(torch.zeros(1, device="cuda").data_ptr()))
    rc = lib.hmlfc_render_views_relaxed_ex(H._streams_array([st]), 1, cp, cp, va, len(va), 6,
                                           C.c_void_p(int(out.data_ptr())), None)
    assert rc == H.E_INVALID_ARG


def test_requantize_round_trip(H, torch_cuda, tiny_streams, tiny_cfg):
    """Re-encoding a stream's own dequantised coefficients reproduces a
    stream that decodes to the same samples."""
    data = tiny_streams[tiny_cfg.qstep].stream
    st = H.Stream(data)
    co, ro = st.dequant()
    new = H.requantize(st, co.cpu().numpy(), ro.cpu().numpy())
    a, b = O.Stream(data).decode_all(), O.Stream(new).decode_all()
    assert np.array_equal(a, b)


def test_render_batch_matches_render_views(H, torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    """The batched pass over several light fields (persistent decode and
    render, every tuning candidate shape) is bitwise equal to render_views,
    also when the decoded-block cache overflows."""
    c = tiny_cfg
    s1 = H.Stream(tiny_streams[c.qstep].stream)
    s2 = H.Stream(O.encode(ragged_lf, 3, 8, 4, 2, t_ref=20, t_pred=30).stream)
    geo1 = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    geo2 = S.lf_geometry(5, 3, 37, 29)
    views = (S.random_views(51, geo1, 5, [(64, 64), (33, 17), (1, 1)]) +
             S.random_views(52, geo2, 4, [(40, 31), (8, 70)], lf=1))
    views = [views[k] for k in (0, 5, 1, 6, 2, 7, 3, 8, 4)]
    arr = S.views_to_array(views)
    want = _render_gpu(H, torch_cuda, [s1, s2], arr)
    try:
        for tile in (0, 1, 2):
            for group in (1, 4, 8):
                H.set_batch_tuning(tile, group, 2)
                got = H.render_batch([s1, s2], arr)
                torch_cuda.cuda.synchronize()
                assert np.array_equal(got.cpu().numpy().astype(np.float64), want)
        # an image pool with room for no camera image, then for three (the other cameras' rays decode directly)
        for pool in (6 * 8 * 8 * 4, 3 * 64 * 64 * 4):
            H.set_batch_tuning(0, 4, 4, pool)
            got = H.render_batch([s1, s2], arr)
            torch_cuda.cuda.synchronize()
            assert np.array_equal(got.cpu().numpy().astype(np.float64), want)
    finally:
        H.set_batch_tuning(0, 4, 8, 2 << 30)


def test_render_batch_mixed_block_sizes_and_chroma(H, torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    """One batched pass over streams of block sizes 8 and 4 and a 4:2:0
    stream gives the bits of hmlfc_render_views, and stays within the bound
    of the oracle's FP64 render."""
    c = tiny_cfg
    datas = [tiny_streams[c.qstep].stream, O.encode(ragged_lf, 2, 4, 2, 4, mc=O.MC_INTEGER).stream,
             O.encode(ragged_lf, 3, 8, 4, 2, t_ref=20, t_pred=30, sub=1).stream]
    streams = [H.Stream(d) for d in datas]
    geo1 = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    geo2 = S.lf_geometry(5, 3, 37, 29)
    views = (S.random_views(61, geo1, 3, [(64, 64), (33, 17)]) + S.random_views(62, geo2, 3, [(40, 31)], lf=1) +
             S.random_views(63, geo2, 3, [(29, 44)], lf=2))
    arr = S.views_to_array([views[k] for k in (0, 3, 6, 1, 4, 7, 2, 5, 8)])
    want = _render_gpu(H, torch_cuda, streams, arr)
    for tile in (0, 1, 2):
        try:
            H.set_batch_tuning(tile, 2, 4)
            got = H.render_batch(streams, arr)
            torch_cuda.cuda.synchronize()
        finally:
            H.set_batch_tuning(0, 4, 8, 2 << 30)
        assert np.array_equal(got.cpu().numpy().astype(np.float64), want)
    for lf, d in enumerate(datas):
        sel = arr[arr["lf"] == lf].copy()
        sel["lf"] = 0
        ref = O.render_dense(O.Stream(d).decode_all(), sel)     # each view at its own out_offset
        for v in sel:
            o, n = int(v["out_offset"]), int(v["width"] * v["height"] * 3)
            assert np.max(np.abs(want[o:o + n] - ref[o:o + n])) <= RENDER_TOL


def test_render_batch_graph_replay(H, torch_cuda, tiny_streams, tiny_cfg):
    """A captured batched render replays to the same output (no host memory
    is read at replay)."""
    torch = torch_cuda
    c = tiny_cfg
    st = H.Stream(tiny_streams[c.qstep].stream)
    arr = S.views_to_array(_views_mix(c, 53, 6, [(64, 64), (40, 24)]))
    want = _render_gpu(H, torch, [st], arr)
    out = torch.zeros(H.out_size(arr), dtype=torch.float32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        H.render_batch([st], arr, out)                  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        H.render_batch([st], arr, out)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.float64), want)


@pytest.mark.parametrize("path", [0, 1, 2])
def test_render_views_host_equals_device_render(torch_cuda, tiny_streams, tiny_cfg, path):
    """The host-output render gives the device render's bits for every path,
    with gaps between views left untouched, also when the decoded-block cache
    overflows or is absent (per-tile fallback)."""
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    st = H.Stream(tiny_streams[c.qstep].stream)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(51, geo, 19, [(64, 64), (33, 17), (48, 80)]))
    gap = 7
    off = 0
    for v in range(len(views)):                     # leave 7 floats between views
        views[v]["out_offset"] = off
        off += int(views[v]["width"]) * int(views[v]["height"]) * 3 + gap
    H.set_render_path(path)
    try:
        for cache in (H.DEFAULT_CACHE_BYTES, 5 * c.width * c.height * 4, 3 * st.info["block"] ** 2 * 4, 0):
            H.set_block_cache_bytes(cache)
            dev = torch.full((off,), -5.0, dtype=torch.float32, device="cuda")
            H.render_views([st], views, dev)
            host = torch.full((off,), -5.0, dtype=torch.float32).pin_memory()
            H.render_views_host([st], views, host)
            torch.cuda.synchronize()
            assert torch.equal(dev.cpu(), host), (path, cache)
    finally:
        H.set_block_cache_bytes(H.DEFAULT_CACHE_BYTES)
        H.set_render_path(0)


def test_render_views_host_two_streams_and_back_to_back(torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    a = H.Stream(tiny_streams[c.qstep].stream)
    b = H.Stream(O.encode(ragged_lf, 2, 8, 4, 4).stream)
    va = S.random_views(61, S.lf_geometry(c.nu, c.nv, c.width, c.height), 5, [(40, 40)])
    vb = S.random_views(62, S.lf_geometry(5, 3, 37, 29), 6, [(30, 20)], lf=1)
    views = S.views_to_array(va + vb)
    dev = H.render_views([a, b], views)
    outs = [H.render_views_host([a, b], views) for _ in range(3)]   # three calls in flight on one stream
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(dev.cpu(), o)
