"""Chroma sub-sampled 4:2:0 streams (Sec. 4.5) through the C ABI: decoded
samples bit-exact against the oracle, rendered views within 1e-3 of its FP64
render, every render path the same bits, progressive levels, the touched-bytes
counter, the allocation-free entry point, the serving form's resident
cache, and the calls that decode full-resolution chroma only refusing the
mode."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_09396_gb300 as H
    return H


def _fields(tiny_lf, tiny_cfg, ragged_lf):
    """(stream bytes, light field, levels) of 4:2:0 streams: the tiny field,
    and odd-sized ragged fields with 8x8 and 4x4 blocks, MC modes mixed."""
    c = tiny_cfg
    return [
        (O.encode(tiny_lf, c.levels, c.block, c.search, c.qstep, sub=1).stream, tiny_lf, c.levels),
        (O.encode(ragged_lf, 3, 8, 4, 2, t_ref=20, t_pred=30, sub=1).stream, ragged_lf, 3),
        (O.encode(ragged_lf, 2, 4, 2, 4, mc=O.MC_INTEGER, sub=1).stream, ragged_lf, 2),
        (O.encode(ragged_lf, 3, 8, 4, 1, mc=O.MC_OFF, sub=1).stream, ragged_lf, 3),
    ]


def _coords(nu, nv, W, H_):
    ii, jj, xx, yy = np.meshgrid(np.arange(nu), np.arange(nv), np.arange(W), np.arange(H_), indexing="ij")
    return np.stack([ii, jj, xx, yy], -1).reshape(-1, 4).astype(np.int32)


def test_chroma_420_decode_bit_exact(H, tiny_lf, tiny_cfg, ragged_lf):
    import torch
    for data, lf, L in _fields(tiny_lf, tiny_cfg, ragged_lf):
        st, ost = H.Stream(data), O.Stream(data)
        assert st.info["chroma"] == 1
        nu, nv, Hh, W = lf.shape[:4]
        co = _coords(nu, nv, W, Hh)
        dec = ost.decode_all()
        for level in range(L + 1):
            got = st.decode_pixels(torch.from_numpy(co).cuda(), level=level).cpu().numpy()
            want = dec[co[:, 0], co[:, 1], co[:, 3], co[:, 2]] if level == 0 else ost.decode_samples(co, level=level)
            assert np.array_equal(got, want), level
        st.check_status()


def test_chroma_420_render_paths(H, tiny_lf, tiny_cfg, ragged_lf):
    """Cached (all cameras, a few camera images, none), per-ray and per-tile
    requests give the same bits, within 1e-3 of the FP64 dense render of the
    oracle's full decode; the batched form hands the call to the same path."""
    import torch
    for data, lf, L in _fields(tiny_lf, tiny_cfg, ragged_lf):
        st = H.Stream(data)
        nu, nv, Hh, W = lf.shape[:4]
        geo = S.lf_geometry(nu, nv, W, Hh)
        views = S.views_to_array(S.random_views(55, geo, 4, [(48, 40), (17, 9)]))
        outs = []
        try:
            for path in (0, 1, 2):
                H.set_render_path(path)
                outs.append(H.render_views([st], views))
            H.set_render_path(0)
            for cap in (3 * W * Hh * 4, 64):
                H.set_block_cache_bytes(cap)
                outs.append(H.render_views([st], views))
        finally:
            H.set_render_path(0)
            H.set_block_cache_bytes(H.DEFAULT_CACHE_BYTES)
        outs.append(H.render_batch([st], views))
        torch.cuda.synchronize()
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        want = O.render_dense(O.Stream(data).decode_all(), views)
        assert np.max(np.abs(outs[0].cpu().numpy().astype(np.float64) - want)) <= 1e-3


def test_chroma_420_progressive_render(H, tiny_lf, tiny_cfg, ragged_lf):
    for data, lf, L in _fields(tiny_lf, tiny_cfg, ragged_lf)[:2]:
        st, ost = H.Stream(data), O.Stream(data)
        nu, nv, Hh, W = lf.shape[:4]
        geo = S.lf_geometry(nu, nv, W, Hh)
        views = S.views_to_array(S.random_views(56, geo, 3, [(40, 36)]))
        rng = np.random.default_rng(57)
        pix = np.stack([rng.integers(0, 3, 800), rng.integers(0, 40, 800), rng.integers(0, 36, 800)], -1).astype(np.int32)
        idx = (views["out_offset"][pix[:, 0]] + (pix[:, 2] * 40 + pix[:, 1]) * 3)[:, None] + np.arange(3)[None, :]
        for level in range(1, L + 1):
            out = H.render_views([st], views, level=level).cpu().numpy().astype(np.float64)
            assert np.max(np.abs(out[idx] - ost.render_pixels(views, pix, level=level))) <= 1e-3


def test_chroma_420_touched_bytes_match_oracle(H, tiny_lf, tiny_cfg, ragged_lf):
    for data, lf, L in _fields(tiny_lf, tiny_cfg, ragged_lf):
        nu, nv, Hh, W = lf.shape[:4]
        geo = S.lf_geometry(nu, nv, W, Hh)
        views = S.views_to_array(S.random_views(58, geo, 3, [(33, 21)]))
        st = H.Stream(data)
        want = O.Stream(data).touched_bytes(views)
        assert np.allclose(H.touched_bytes([st], views), want, rtol=0, atol=1e-6)
        for level in range(1, L + 1):
            lw = O.Stream(data).touched_bytes(views[:1], level=level)[0]
            assert abs(H.touched_bytes_union([st], views[:1], level=level) - lw) < 1e-6


def test_chroma_420_noalloc_equals_render_views(H, tiny_lf, tiny_cfg):
    import torch
    lib = H.lib()
    fn = lib.hmlfc_render_views_noalloc
    fn.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    c = tiny_cfg
    st = H.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, c.qstep, sub=1).stream)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    arr = S.views_to_array(S.random_views(59, geo, 3, [(64, 64)]))
    want = H.render_views([st], arr)
    got = torch.full_like(want, -3.0)
    va = H._views_array(arr)
    rc = fn(H._streams_array([st]), 1, va, len(va), C.c_void_p(int(got.data_ptr())),
            C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    assert rc == 0, lib.hmlfc_last_error().decode()
    torch.cuda.synchronize()
    assert torch.equal(got, want)


def test_chroma_420_served_from_the_resident_cache(H, tiny_lf, tiny_cfg, ragged_lf):
    """The serving form's resident cache renders 4:2:0 streams with the bits
    of hmlfc_render_views, on consecutive calls (hits) and with a cache
    smaller than one call (evictions and direct decode)."""
    import torch
    from paper_1902_09396_gb300.serve import ResidentCache
    for data, lf, L in _fields(tiny_lf, tiny_cfg, ragged_lf)[:2]:
        st = H.Stream(data)
        nu, nv, Hh, W = lf.shape[:4]
        geo = S.lf_geometry(nu, nv, W, Hh)
        for cache_bytes in (1 << 22, 6 * 8 * 8 * 4):
            cache = ResidentCache(st, cache_bytes)
            for seed in (71, 72):
                views = S.views_to_array(S.random_views(seed, geo, 3, [(40, 36), (17, 9)]))
                want = H.render_views([st], views)
                out = torch.zeros(H.out_size(views), dtype=torch.float32, device="cuda")
                cache.render(views, out)
                torch.cuda.synchronize()
                assert torch.equal(out, want)


def test_chroma_420_refused_where_full_chroma_only(H, tiny_lf, tiny_cfg):
    """The relaxation (forward, adjoint, starting point), the re-quantiser and
    the device encoder decode or code full-resolution chroma only: each
    refuses a 4:2:0 stream with HMLFC_E_UNSUPPORTED."""
    import torch
    c = tiny_cfg
    data = O.encode(tiny_lf, c.levels, c.block, c.search, c.qstep, sub=1).stream
    st = H.Stream(data)
    lib = H.lib()
    d = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    lib.hmlfc_dequant.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.hmlfc_dequant(st.handle, C.c_void_p(int(d.data_ptr())), C.c_void_p(int(d.data_ptr())), None) \
        == H.E_UNSUPPORTED
    prm = H.EncodeParams(c.levels, c.block, c.search, c.qstep, 0, 0, 1, 0, 1)
    out, n = C.c_void_p(), C.c_size_t()
    dlf = torch.from_numpy(tiny_lf).cuda()
    rc = lib.hmlfc_encode_device(C.c_void_p(int(dlf.data_ptr())), c.nu, c.nv, c.width, c.height, C.byref(prm), None,
                                 C.byref(out), C.byref(n), None)
    assert rc == H.E_UNSUPPORTED


@pytest.mark.slow
def test_chroma_420_paper_scale(H):
    """The paper-scale field coded 4:2:0 (17x17x512², L=4, B=16, q=4,
    T=(400, 800)): every sample bit-exact, every pixel of the 64-pose path
    within 1e-3 of the FP64 dense render of the oracle's decode."""
    import torch
    c = S.CONFIGS["paper"]
    lf = S.make_lf(c.seed, c.nu, c.nv, c.width, c.height, c.n_planes, c.disp_max, c.texture)
    data = O.encode(lf, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800, sub=1).stream
    assert H.encode(lf, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800, sub=1) == data
    del lf
    st = H.Stream(data)
    dec = O.Stream(data).decode_all()
    yy, xx = np.meshgrid(np.arange(c.height), np.arange(c.width), indexing="ij")
    for i in range(c.nu):
        jj = np.repeat(np.arange(c.nv), c.width * c.height)
        co = np.stack([np.full(jj.size, i), jj, np.tile(xx.ravel(), c.nv), np.tile(yy.ravel(), c.nv)],
                      -1).astype(np.int32)
        got = st.decode_pixels(torch.from_numpy(co).cuda()).cpu().numpy().reshape(c.nv, c.height, c.width, 3)
        assert np.array_equal(got, dec[i])
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.circle_path(geo, 64, 512, 512))
    out = H.render_views([st], views)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - O.render_dense(dec, views))) <= 1e-3
