"""GPU encoder: byte-identical streams to the oracle's encoder (Sec. 4.3-4.7)
for every motion-compensation mode, on the tiny field, on an odd grid with
partial edge blocks and thresholds, with wide search windows, and at block
sizes from 4 to 64; search windows the device does not hold are refused."""
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


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL, O.MC_ZERO, O.MC_INTEGER])
def test_device_encoder_matches_oracle(torch_cuda, tiny_lf, tiny_cfg, ragged_lf, mc):
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    for lf, L, B, q, tr, tp in [(tiny_lf, c.levels, c.block, 1, 0, 0), (tiny_lf, c.levels, c.block, 4, 0, 0),
                                (ragged_lf, 2, 8, 4, 40, 90), (ragged_lf, 3, 16, 2, 0, 0)]:
        a = O.encode(lf, L, B, c.search, q, t_ref=tr, t_pred=tp, mc=mc).stream
        b = H.encode_device(lf, L, B, c.search, q, t_ref=tr, t_pred=tp, mc=mc)
        assert a == b, (L, B, q, tr, tp)


@pytest.mark.parametrize("search", [0, 1, 7, 16])
def test_device_encoder_search_windows(torch_cuda, ragged_lf, search):
    import paper_1902_09396_gb300 as H
    for mc in (O.MC_QPEL, O.MC_INTEGER):
        a = O.encode(ragged_lf, 2, 8, search, 3, mc=mc).stream
        assert H.encode_device(ragged_lf, 2, 8, search, 3, mc=mc) == a


@pytest.mark.parametrize("block", [4, 5, 32, 64])
def test_device_encoder_block_sizes(torch_cuda, block):
    import paper_1902_09396_gb300 as H
    lf = S.make_lf(23, 3, 4, 70, 45, 3, 5.0, "pink")
    for q, tr, tp in [(1, 0, 0), (6, 100, 300)]:
        a = O.encode(lf, 2, block, 3, q, t_ref=tr, t_pred=tp).stream
        assert H.encode_device(lf, 2, block, 3, q, t_ref=tr, t_pred=tp) == a


def test_device_encoder_from_device_tensor_and_decode(torch_cuda, tiny_lf, tiny_cfg):
    """A CUDA tensor is encoded in place; the stream loads and decodes to
    the oracle's samples."""
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    d = torch.from_numpy(tiny_lf).cuda()
    data = H.encode_device(d, c.levels, c.block, c.search, c.qstep)
    assert torch.equal(d.cpu(), torch.from_numpy(tiny_lf))
    st = H.Stream(data)
    coords = np.stack(np.meshgrid(np.arange(c.nu), np.arange(c.nv), np.arange(c.width), np.arange(c.height),
                                  indexing="ij"), -1).reshape(-1, 4).astype(np.int32)
    got = st.decode_pixels(torch.from_numpy(coords).cuda()).cpu().numpy()
    assert np.array_equal(got, O.Stream(data).decode_samples(coords))


def test_device_encoder_refuses_wide_search(torch_cuda, tiny_lf):
    import paper_1902_09396_gb300 as H
    with pytest.raises(H.HmlfcError) as ei:
        H.encode_device(tiny_lf, 2, 8, 33, 4, mc=O.MC_QPEL)
    assert ei.value.code == H.E_UNSUPPORTED
    # no search: any window is fine
    assert H.encode_device(tiny_lf, 2, 8, 40, 4, mc=O.MC_ZERO) == O.encode(tiny_lf, 2, 8, 40, 4, mc=O.MC_ZERO).stream


def test_device_encoder_work_counts_and_events(torch_cuda, tiny_lf, tiny_cfg):
    """Work counts: the integer stage evaluates (2 Ws + 1)^2 candidates for
    both signs at every pixel of every predictive node-channel; the
    refinement at most 48 per sign; significant blocks = the stream's
    records.  The per-level search events bracket positive times."""
    torch = torch_cuda
    import paper_1902_09396_gb300 as H
    c = tiny_cfg
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * c.levels)]
    H.set_encode_events(ev)
    try:
        st = {}
        data = H.encode_device(tiny_lf, c.levels, c.block, c.search, c.qstep, stats=st)
    finally:
        H.set_encode_events(None)
    ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(c.levels)]
    assert all(m > 0 for m in ms)
    info = H.Stream(data).info
    px = c.width * c.height
    # reference members of level l: one per 2x2 cluster = the node count of level l + 1
    n_pred_nc = info["n_nc"] - 3 * sum(((c.nu + (2 << l) - 1) >> (l + 1)) * ((c.nv + (2 << l) - 1) >> (l + 1))
                                       for l in range(c.levels))
    assert st["int_terms"] == n_pred_nc * 2 * (2 * c.search + 1) ** 2 * px
    assert 0 < st["frac_terms"] <= n_pred_nc * 96 * px
    assert st["sig_blocks"] == info["n_sig"]
    assert st["blocks_searched"] == n_pred_nc * ((c.width + c.block - 1) // c.block) * ((c.height + c.block - 1) // c.block)
    st0 = {}
    H.encode_device(tiny_lf, c.levels, c.block, c.search, c.qstep, mc=O.MC_ZERO, stats=st0)
    assert st0["blocks_searched"] == 0 and st0["int_terms"] == 0 and st0["frac_terms"] == 0
