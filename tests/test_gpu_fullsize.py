"""Parity at the paper-scale configuration, in the launch configuration the
benchmark times: 17x17 grid of 512x512 views, L=4, B=16, quarter-pel MC,
q=4, thresholds (400, 800), the 64-pose circular path of 512x512 views.

The stream is encoded by the oracle.  Checked: the product's host and device
encoders write the same bytes; 10^6 random samples decode bit-exactly; 30,000 sampled output
pixels of the 64 views (rendered by the benchmark's cached path, the batched
pass and the per-tile path) are within 1e-3 of the oracle's FP64
random-access render of the same pixels.
"""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def paper():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = S.CONFIGS["paper"]
    lf = S.make_lf(c.seed, c.nu, c.nv, c.width, c.height, c.n_planes, c.disp_max, c.texture)
    data = O.encode(lf, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800).stream
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.circle_path(geo, 64, 512, 512))
    return torch, c, lf, data, views


def test_product_encoder_bytes_at_full_size(paper):
    import paper_1902_09396_gb300 as H
    torch, c, lf, data, _ = paper
    assert H.encode(lf, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800) == data


def test_device_encoder_bytes_at_full_size(paper):
    import paper_1902_09396_gb300 as H
    torch, c, lf, data, _ = paper
    d = torch.from_numpy(lf).cuda()
    assert H.encode_device(d, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800) == data


def test_million_samples_bit_exact(paper):
    import paper_1902_09396_gb300 as H
    torch, c, _, data, _ = paper
    rng = np.random.default_rng(71)
    n = 1_000_000
    coords = np.stack([rng.integers(0, c.nu, n), rng.integers(0, c.nv, n), rng.integers(0, c.width, n),
                       rng.integers(0, c.height, n)], -1).astype(np.int32)
    st = H.Stream(data)
    got = st.decode_pixels(torch.from_numpy(coords).cuda())
    torch.cuda.synchronize()
    st.check_status()
    assert np.array_equal(got.cpu().numpy(), O.Stream(data).decode_samples(coords))


@pytest.mark.parametrize("how", ["cached", "batched", "tile"])
def test_path_views_sampled_pixels(paper, how):
    import paper_1902_09396_gb300 as H
    torch, c, _, data, views = paper
    st = H.Stream(data)
    if how == "cached":
        out = H.render_views([st], views)
    elif how == "batched":
        out = H.render_batch([st], views)
    else:
        H.set_render_path(2)
        try:
            out = H.render_views([st], views)
        finally:
            H.set_render_path(0)
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(72)
    n = 30_000
    pix = np.stack([rng.integers(0, 64, n), rng.integers(0, 512, n), rng.integers(0, 512, n)], -1).astype(np.int32)
    want = O.Stream(data).render_pixels(views, pix)
    idx = (views["out_offset"][pix[:, 0]] + (pix[:, 2] * 512 + pix[:, 1]) * 3)[:, None] + np.arange(3)[None, :]
    assert np.max(np.abs(out[idx] - want)) <= 1e-3


@pytest.mark.parametrize("level", [1, 2])
def test_progressive_decode_at_full_size(paper, level):
    """Progressive decode at the benchmark's configuration: 200,000 random
    samples bit-exact at the level, and 10,000 sampled pixels of the 64
    cached-path views within 1e-3 of the oracle's FP64 render at the level."""
    import paper_1902_09396_gb300 as H
    torch, c, _, data, views = paper
    st, ost = H.Stream(data), O.Stream(data)
    rng = np.random.default_rng(80 + level)
    n = 200_000
    coords = np.stack([rng.integers(0, c.nu, n), rng.integers(0, c.nv, n), rng.integers(0, c.width, n),
                       rng.integers(0, c.height, n)], -1).astype(np.int32)
    got = st.decode_pixels(torch.from_numpy(coords).cuda(), level=level)
    assert np.array_equal(got.cpu().numpy(), ost.decode_samples(coords, level=level))
    out = H.render_views([st], views, level=level)
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.float64)
    m = 10_000
    pix = np.stack([rng.integers(0, 64, m), rng.integers(0, 512, m), rng.integers(0, 512, m)], -1).astype(np.int32)
    want = ost.render_pixels(views, pix, level=level)
    idx = (views["out_offset"][pix[:, 0]] + (pix[:, 2] * 512 + pix[:, 1]) * 3)[:, None] + np.arange(3)[None, :]
    assert np.max(np.abs(out[idx] - want)) <= 1e-3
