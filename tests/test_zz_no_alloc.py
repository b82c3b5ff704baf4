"""The allocation-free render entry point, called through the C ABI.

hmlfc_render_views_noalloc serves callers that cannot allocate device memory
when they render: a frame loop with a hard deadline that must not wait on
the allocator or fail on fragmentation midway, code under a caching
allocator that has to account for every byte, and code capturing work into
a CUDA graph in a capture mode that forbids cudaMalloc.  Its index and
decoded camera images live in a fixed device array that every call shares
and finds as the previous call left it, so it is checked on two calls in a
row, with different streams and views, against hmlfc_render_views: the
results must be the same bits.  A larger field whose reached cameras
overflow the array exercises the direct decode of their rays, and a stream
whose index alone does not fit must be rejected.  This file is collected
last so that a run stopping at its first failure has already run every
other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_09396_gb300 as H
    lib = H.lib()
    fn = lib.hmlfc_render_views_noalloc
    fn.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return torch, H, lib, fn


def _noalloc(torch, H, fn, streams, arr, fill=-7.0):
    got = torch.full((H.out_size(arr),), fill, dtype=torch.float32, device="cuda")
    va = H._views_array(arr)
    cuda_stream = C.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    rc = fn(H._streams_array(streams), len(streams), va, len(va), C.c_void_p(int(got.data_ptr())), cuda_stream)
    return rc, got


def test_noalloc_render_matches_render_views(tiny_streams, tiny_cfg, ragged_lf):
    torch, H, lib, fn = _setup()
    c = tiny_cfg
    s_tiny = H.Stream(tiny_streams[c.qstep].stream)
    s_ragged = H.Stream(O.encode(ragged_lf, 3, 8, 4, 2, t_ref=20, t_pred=30).stream)
    geo_t = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    geo_r = S.lf_geometry(5, 3, 37, 29)
    calls = [
        ([s_tiny], S.random_views(41, geo_t, 5, [(64, 64), (37, 23), (1, 1)])),
        ([s_ragged, s_tiny], S.random_views(42, geo_r, 3, [(40, 31)], lf=0) +
         S.random_views(43, geo_t, 2, [(64, 48)], lf=1)),
    ]
    for streams, views in calls:
        arr = S.views_to_array(views)
        want = H.render_views(streams, arr)
        rc, got = _noalloc(torch, H, fn, streams, arr)
        assert rc == 0, lib.hmlfc_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(got, want)


def test_noalloc_overflow_into_per_ray_decode():
    """A 9x9 grid of 512x512 views with 16x16 blocks: the decoded camera
    images that 64 circling views reach do not all fit the 32 MiB array
    (1 MiB per camera), so the rays of the cameras beyond it decode their
    samples directly.  Two calls in a row (different views), each the same
    bits as hmlfc_render_views; sampled pixels within 1e-3 of the oracle."""
    torch, H, lib, fn = _setup()
    lf = S.make_lf(91, 9, 9, 512, 512, 6, 12.0, "pink")
    data = O.encode(lf, 3, 16, 4, 4, t_ref=400, t_pred=800).stream
    st = H.Stream(data)
    geo = S.lf_geometry(9, 9, 512, 512)
    reached = []
    for k, (n, radius) in enumerate(((64, 0.45), (48, 0.2))):
        arr = S.views_to_array(S.circle_path(geo, n, 512, 512, radius_frac=radius))
        _, cam_blocks = H.touched_bytes_union([st], arr, with_blocks=True)
        reached.append(cam_blocks)
        want = H.render_views([st], arr)
        rc, got = _noalloc(torch, H, fn, [st], arr, fill=float(k))
        assert rc == 0, lib.hmlfc_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        rng = np.random.default_rng(92 + k)
        m = 4000
        pix = np.stack([rng.integers(0, n, m), rng.integers(0, 512, m), rng.integers(0, 512, m)], -1).astype(np.int32)
        ref = O.Stream(data).render_pixels(arr, pix)
        idx = (arr["out_offset"][pix[:, 0]] + (pix[:, 2] * 512 + pix[:, 1]) * 3)[:, None] + np.arange(3)[None, :]
        assert np.max(np.abs(got.cpu().numpy().astype(np.float64)[idx] - ref)) <= 1e-3
    # even the blocks alone (16 * 16 * 4 B each) exceed the array: the first call overflowed it
    assert reached[0] * 16 * 16 * 4 > (32 << 20)          # HMLFC_FIXED_SCRATCH_BYTES


def test_noalloc_rejects_a_block_index_beyond_the_array():
    """8x8 cameras of 1024x512 with 2x2 blocks and one SRV level: 8.4M
    (camera, block) pairs and 2.1M (level-1 node, block) decode items, a
    block index of about 42 MB.  The call returns HMLFC_E_UNSUPPORTED with a
    message and writes nothing; hmlfc_render_views still renders."""
    torch, H, lib, fn = _setup()
    lf = S.make_lf(93, 8, 8, 1024, 512, 3, 4.0, "noise_gradient")
    data = O.encode(lf, 1, 2, 1, 8, mc=O.MC_OFF).stream
    st = H.Stream(data)
    geo = S.lf_geometry(8, 8, 1024, 512)
    arr = S.views_to_array(S.random_views(94, geo, 2, [(64, 64)]))
    rc, got = _noalloc(torch, H, fn, [st], arr, fill=-7.0)
    assert rc == H.E_UNSUPPORTED
    assert "fixed scratch" in lib.hmlfc_last_error().decode()
    torch.cuda.synchronize()
    assert bool((got == -7.0).all())
    out = H.render_views([st], arr)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
