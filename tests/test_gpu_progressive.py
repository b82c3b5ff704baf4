"""Progressive decoding through the C ABI: samples and views decoded down to
a level k of the tree (the level-k node's reconstruction stands for each of
its cameras) against the oracle's progressive decode -- bit-exact samples,
views within 1e-3 of its FP64 render, every render path equal to the others
-- plus the level checks and the compulsory-byte counter at each level."""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _coords(nu, nv, W, H):
    return np.stack(np.meshgrid(np.arange(nu), np.arange(nv), np.arange(W), np.arange(H), indexing="ij"),
                    -1).reshape(-1, 4).astype(np.int32)


def test_progressive_samples_bit_exact(torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    cases = [(tiny_streams[c.qstep].stream, c.nu, c.nv, c.width, c.height, c.levels),
             (O.encode(ragged_lf, 3, 8, 4, 3).stream, 5, 3, 37, 29, 3)]
    for data, nu, nv, W, Hh, L in cases:
        st, ost = H.Stream(data), O.Stream(data)
        co = _coords(nu, nv, W, Hh)
        d = torch.from_numpy(co).cuda()
        for k in range(L + 1):
            got = st.decode_pixels(d, level=k).cpu().numpy()
            assert np.array_equal(got, ost.decode_samples(co, level=k)), k
        st.check_status()


def test_progressive_level_checks(torch_cuda, tiny_streams, tiny_cfg):
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    st = H.Stream(tiny_streams[c.qstep].stream)
    d = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(3, geo, 1, [(8, 8)]))
    for bad in (-1, c.levels + 1):
        with pytest.raises(H.HmlfcError) as e1:
            st.decode_pixels(d, level=bad)
        with pytest.raises(H.HmlfcError) as e2:
            H.render_views([st], views, level=bad)
        assert e1.value.code == e2.value.code == H.E_INVALID_ARG


@pytest.mark.parametrize("path", [0, 1, 2])
def test_progressive_views_match_oracle(torch_cuda, tiny_streams, tiny_cfg, path):
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    data = tiny_streams[c.qstep].stream
    st, ost = H.Stream(data), O.Stream(data)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(21, geo, 5, [(64, 64), (37, 23), (80, 48)]))
    pix = np.concatenate([np.stack(np.meshgrid([v], np.arange(views[v]["width"]), np.arange(views[v]["height"]),
                                               indexing="ij"), -1).reshape(-1, 3) for v in range(len(views))])
    H.set_render_path(path)
    try:
        for k in range(1, c.levels + 1):
            out = H.render_views([st], views, level=k).cpu().numpy()
            ref = ost.render_pixels(views, pix.astype(np.int32), level=k)
            offs = views["out_offset"][pix[:, 0]] + (pix[:, 2] * views["width"][pix[:, 0]] + pix[:, 1]) * 3
            got = out[offs[:, None] + np.arange(3)]
            assert np.max(np.abs(got - ref)) <= 1e-3, k
    finally:
        H.set_render_path(0)


def test_progressive_paths_bitwise_equal_and_cache_overflow(torch_cuda, tiny_streams, tiny_cfg, ragged_lf):
    """Cached, direct and per-tile paths give the same bits at every level,
    also when the decoded-block cache holds only a few blocks."""
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    for data, nu, nv, W, Hh, L in [(tiny_streams[c.qstep].stream, c.nu, c.nv, c.width, c.height, c.levels),
                                   (O.encode(ragged_lf, 3, 8, 4, 3).stream, 5, 3, 37, 29, 3)]:
        st = H.Stream(data)
        geo = S.lf_geometry(nu, nv, W, Hh)
        views = S.views_to_array(S.random_views(31, geo, 6, [(48, 40), (17, 64)]))
        for k in range(L + 1):
            outs = []
            for path in (0, 1, 2):
                H.set_render_path(path)
                outs.append(H.render_views([st], views, level=k))
            H.set_render_path(0)
            try:
                for cap in (3 * W * Hh * 4, 3 * st.info["block"] ** 2 * 4):   # three camera images; less than one
                    H.set_block_cache_bytes(cap)
                    outs.append(H.render_views([st], views, level=k))
            finally:
                H.set_block_cache_bytes(H.DEFAULT_CACHE_BYTES)
            for o in outs[1:]:
                assert torch.equal(outs[0], o), k


def test_progressive_touched_bytes_match_oracle(torch_cuda, tiny_streams, tiny_cfg):
    """The product's counter at level k (union over one view) equals the
    oracle's per-view count at level k, and falls with k."""
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    data = tiny_streams[c.qstep].stream
    st, ost = H.Stream(data), O.Stream(data)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(41, geo, 3, [(40, 40)]))
    prev = None
    for k in range(c.levels + 1):
        want = ost.touched_bytes(views, level=k)
        for v in range(len(views)):
            assert abs(H.touched_bytes_union([st], views[v:v + 1], level=k) - want[v]) < 1e-6
        tot = H.touched_bytes_union([st], views, level=k)
        assert prev is None or tot <= prev
        prev = tot
