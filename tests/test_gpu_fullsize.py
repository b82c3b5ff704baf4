"""Parity at the paper-scale configuration, in the launch configuration the
benchmark times: 17x17 grid of 512x512 views, L=4, B=16, quarter-pel MC,
q=4, thresholds (400, 800), the 64-pose circular path of 512x512 views.

The stream is encoded by the oracle.  Checked, without sampling: the
product's host and device encoders write the same bytes; every one of the
75.8M samples decodes bit-exactly against the oracle's full decode (and at
progressive levels 1 and 2 against the oracle's random-access decode of
every sample); every pixel of the 64 views, rendered by the benchmark's
cached path, the batched pass, the per-tile path and the per-ray path, is
within 1e-3 of the oracle's FP64 dense render of the oracle-decoded field.
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


@pytest.fixture(scope="module")
def paper_decoded(paper):
    """The oracle's full top-down decode of the paper-scale stream."""
    _, _, _, data, _ = paper
    return O.Stream(data).decode_all()


def _row_coords(c, i):
    """(i, j, x, y) of every sample of camera row i, camera-major then
    row-major pixels."""
    yy, xx = np.meshgrid(np.arange(c.height), np.arange(c.width), indexing="ij")
    jj = np.repeat(np.arange(c.nv), c.width * c.height)
    return np.stack([np.full(jj.size, i), jj, np.tile(xx.ravel(), c.nv), np.tile(yy.ravel(), c.nv)],
                    -1).astype(np.int32)


def _gpu_decode_all(torch, H, st, c, level=0):
    """Every sample of the light field through hmlfc_decode_pixels[_lod],
    a row of cameras per call: uint8 [nu][nv][H][W][3]."""
    out = np.zeros((c.nu, c.nv, c.height, c.width, 3), np.uint8)
    for i in range(c.nu):
        got = st.decode_pixels(torch.from_numpy(_row_coords(c, i)).cuda(), level=level)
        out[i] = got.cpu().numpy().reshape(c.nv, c.height, c.width, 3)
    torch.cuda.synchronize()
    st.check_status()
    return out


def test_product_encoder_bytes_at_full_size(paper):
    import paper_1902_09396_gb300 as H
    torch, c, lf, data, _ = paper
    assert H.encode(lf, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800) == data


def test_device_encoder_bytes_at_full_size(paper):
    import paper_1902_09396_gb300 as H
    torch, c, lf, data, _ = paper
    d = torch.from_numpy(lf).cuda()
    assert H.encode_device(d, c.levels, c.block, c.search, c.qstep, t_ref=400, t_pred=800) == data


def test_every_sample_bit_exact(paper, paper_decoded):
    """All 17 x 17 x 512 x 512 samples (75.8M) against the oracle's full
    decode (Sec. 4.8.1)."""
    import paper_1902_09396_gb300 as H
    torch, c, _, data, _ = paper
    got = _gpu_decode_all(torch, H, H.Stream(data), c)
    assert np.array_equal(got, paper_decoded)


@pytest.mark.parametrize("how", ["cached", "batched", "tile", "direct"])
def test_path_views_every_pixel(paper, paper_decoded, how):
    """Every output pixel of the 64 views against the FP64 dense render of
    the oracle-decoded field, for each render path."""
    import paper_1902_09396_gb300 as H
    torch, c, _, data, views = paper
    st = H.Stream(data)
    if how == "cached":
        out = H.render_views([st], views)
    elif how == "batched":
        out = H.render_batch([st], views)
    else:
        H.set_render_path(2 if how == "tile" else 1)
        try:
            out = H.render_views([st], views)
        finally:
            H.set_render_path(0)
    torch.cuda.synchronize()
    want = O.render_dense(paper_decoded, views)
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - want)) <= 1e-3


@pytest.mark.parametrize("level", [1, 2])
def test_progressive_decode_at_full_size(paper, level):
    """Progressive decode at the benchmark's configuration: every sample
    bit-exact at the level against the oracle's random-access decode, and
    every pixel of the 64 cached-path views within 1e-3 of the FP64 dense
    render of that level field."""
    import paper_1902_09396_gb300 as H
    torch, c, _, data, views = paper
    st, ost = H.Stream(data), O.Stream(data)
    got = _gpu_decode_all(torch, H, st, c, level=level)
    want = np.stack([ost.decode_samples(_row_coords(c, i), level=level).reshape(c.nv, c.height, c.width, 3)
                     for i in range(c.nu)])
    assert np.array_equal(got, want)
    out = H.render_views([st], views, level=level)
    torch.cuda.synchronize()
    ref = O.render_dense(want, views)
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref)) <= 1e-3
