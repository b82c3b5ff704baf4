"""Parity at the batched configuration, in the launch configuration the
batched benchmark form times: 8 light fields of uneven size (5x5x256^2 ..
17x17x1024^2, 3-5 levels, B=16, quarter-pel MC, q=4, T=(400, 800)) and 256
novel views of mixed resolution 256^2-1024^2 in one batched pass, replayed
from a CUDA graph.  The streams are encoded by the oracle; sampled pixels of
every one of the 256 views are checked against the oracle's FP64
random-access render (Sec. 4.8.1, Sec. 2.1) within 1e-3, and the graph
replay against the direct call bit for bit."""
import numpy as np
import pytest

import oracle as O
import synthlf as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_batched_configuration_against_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_09396_gb300 as H
    cfgs = S.batched_workload()
    datas = []
    for c in cfgs:
        lf = S.make_lf(c.seed, c.nu, c.nv, c.width, c.height, c.n_planes, c.disp_max, c.texture)
        datas.append(O.encode(lf, c.levels, c.block, c.search, 4, t_ref=400, t_pred=800).stream)
        del lf
    streams = [H.Stream(d) for d in datas]
    arr = S.views_to_array(S.batched_views(4, cfgs, 256))
    out = H.render_batch(streams, arr)
    torch.cuda.synchronize()
    g_out = torch.full_like(out, -1.0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        H.render_batch(streams, arr, g_out)          # first call outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g_out.fill_(-1.0)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        H.render_batch(streams, arr, g_out)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(g_out, out)
    got = out.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(96)
    per_view = 60
    for lf, d in enumerate(datas):
        vi = np.nonzero(arr["lf"] == lf)[0]
        if len(vi) == 0:
            continue
        sub = arr[vi].copy()
        pix = np.concatenate([np.stack([np.full(per_view, k), rng.integers(0, sub[k]["width"], per_view),
                                        rng.integers(0, sub[k]["height"], per_view)], -1) for k in range(len(sub))])
        pix = pix.astype(np.int32)
        want = O.Stream(d).render_pixels(sub, pix)
        w = sub["width"][pix[:, 0]].astype(np.int64)
        idx = (sub["out_offset"][pix[:, 0]] + (pix[:, 2] * w + pix[:, 1]) * 3)[:, None] + np.arange(3)[None, :]
        assert np.max(np.abs(got[idx] - want)) <= 1e-3, f"light field {lf}"
