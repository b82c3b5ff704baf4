"""Host-side tests of the product library (no GPU needed): the shared object
builds and exports every entry point of include/hmlfc.h; its encoder writes
the same bytes as the oracle's; the loader rejects corrupt streams before
touching a device; the touched-bytes counter agrees with the oracle's."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

import oracle as O
import paper_1902_09396_gb300 as H
import synthlf as S

ROOT = Path(__file__).resolve().parent.parent


def test_library_exports_every_declared_symbol():
    header = (ROOT / "include" / "hmlfc.h").read_text()
    names = sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(hmlfc_\w+)\s*\(", header, re.M)))
    assert len(names) >= 15
    lib = C.CDLL(str(H.build()))
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL, O.MC_ZERO, O.MC_INTEGER])
def test_encoder_matches_oracle_bytes(tiny_lf, tiny_cfg, ragged_lf, mc):
    """The product encoder follows the same readings (tie-breaks, quantiser,
    thresholds, layout) and writes byte-identical streams."""
    c = tiny_cfg
    for lf, L, B, q, tr, tp in [(tiny_lf, c.levels, c.block, 1, 0, 0), (tiny_lf, c.levels, c.block, 4, 0, 0),
                                (ragged_lf, 2, 8, 4, 40, 90), (ragged_lf, 3, 16, 2, 0, 0)]:
        a = O.encode(lf, L, B, c.search, q, t_ref=tr, t_pred=tp, mc=mc).stream
        b = H.encode(lf, L, B, c.search, q, t_ref=tr, t_pred=tp, mc=mc, threads=3)
        assert a == b


@pytest.mark.parametrize("search", [0, 1, 7, 16])
def test_encoder_matches_oracle_search_windows(ragged_lf, search):
    for mc in (O.MC_QPEL, O.MC_INTEGER):
        assert H.encode(ragged_lf, 2, 8, search, 3, mc=mc, threads=4) == O.encode(ragged_lf, 2, 8, search, 3, mc=mc).stream


@pytest.mark.parametrize("block", [4, 5, 32, 64])
def test_encoder_matches_oracle_block_sizes(block):
    lf = S.make_lf(23, 3, 4, 70, 45, 3, 5.0, "pink")
    for q, tr, tp in [(1, 0, 0), (6, 100, 300)]:
        a = O.encode(lf, 2, block, 3, q, t_ref=tr, t_pred=tp).stream
        assert H.encode(lf, 2, block, 3, q, t_ref=tr, t_pred=tp, threads=4) == a


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL, O.MC_ZERO, O.MC_INTEGER])
def test_encoder_matches_oracle_bytes_chroma_420(tiny_lf, tiny_cfg, ragged_lf, mc):
    """Chroma sub-sampled 4:2:0 streams (Sec. 4.5): the product encoder
    writes the oracle's bytes, odd image sizes and block sizes 4-32 included;
    an odd block size is refused."""
    c = tiny_cfg
    for lf, L, B, q, tr, tp in [(tiny_lf, c.levels, c.block, 1, 0, 0), (tiny_lf, c.levels, c.block, 4, 0, 0),
                                (ragged_lf, 2, 8, 4, 40, 90), (ragged_lf, 3, 4, 2, 0, 0), (ragged_lf, 1, 32, 3, 0, 0)]:
        a = O.encode(lf, L, B, c.search, q, t_ref=tr, t_pred=tp, mc=mc, sub=1).stream
        b = H.encode(lf, L, B, c.search, q, t_ref=tr, t_pred=tp, mc=mc, threads=3, sub=1)
        assert a == b
    with pytest.raises(H.HmlfcError):
        H.encode(ragged_lf, 2, 5, c.search, 4, sub=1)


def test_encoder_thread_count_does_not_change_output(ragged_lf):
    a = H.encode(ragged_lf, 2, 8, 4, 4, threads=1)
    b = H.encode(ragged_lf, 2, 8, 4, 4, threads=7)
    assert a == b


def _load_error(data: bytes) -> int:
    h = C.c_void_p()
    return H.lib().hmlfc_load_stream(data, len(data), 0, None, C.byref(h))


def test_loader_rejects_corrupt_streams(tiny_streams, tiny_cfg):
    """Truncated or bit-flipped streams fail with HMLFC_E_CORRUPT (or
    UNSUPPORTED) during host validation, before any device work."""
    good = tiny_streams[tiny_cfg.qstep].stream
    bad_cases = {
        "truncated": good[:-16],
        "short": good[:64],
        "magic": b"XXXX" + good[4:],
        "total": good[:104] + (len(good) + 16).to_bytes(4, "little") + good[108:],
    }
    b = bytearray(good)
    # first group entry: a record base far past the end
    off_groups = int.from_bytes(good[88:92], "little")
    b[off_groups + 4:off_groups + 8] = (0x7FFFFFF0).to_bytes(4, "little")
    bad_cases["record_base"] = bytes(b)
    b = bytearray(good)
    b[off_groups + 8:off_groups + 12] = (5).to_bytes(4, "little")
    bad_cases["offset_base"] = bytes(b)
    b = bytearray(good)
    assert b[off_groups:off_groups + 4] != b"\x00\x00\x00\x00"
    b[off_groups:off_groups + 4] = b"\x00\x00\x00\x00"      # drops blocks: offsets no longer line up
    bad_cases["bitmap"] = bytes(b)
    b = bytearray(good)
    off_recs = int.from_bytes(good[96:100], "little")
    b[off_recs + 2:off_recs + 4] = (0x7F | 0x60).to_bytes(2, "little")   # mode 3 / b > 16
    bad_cases["record_header"] = bytes(b)
    for name, data in bad_cases.items():
        rc = _load_error(data)
        assert rc in (H.E_CORRUPT, H.E_UNSUPPORTED), (name, rc)
        assert H.lib().hmlfc_last_error()


def test_null_and_invalid_arguments():
    L = H.lib()
    h = C.c_void_p()
    assert L.hmlfc_load_stream(None, 0, 0, None, C.byref(h)) == H.E_CORRUPT
    assert L.hmlfc_decode_pixels(None, None, 0, None, None) == H.E_INVALID_ARG
    assert L.hmlfc_render_views(None, 0, None, 0, None, None) == H.E_INVALID_ARG
    L.hmlfc_free_stream(None)


@pytest.mark.gpu
def test_touched_bytes_matches_oracle(tiny_streams, tiny_cfg):
    """The product's counter (the roofline numerator of the benchmark)
    reproduces the oracle's definition exactly on the same views (a stream
    object lives on a device, hence the GPU mark)."""
    c = tiny_cfg
    data = tiny_streams[c.qstep].stream
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(21, geo, 4, [(64, 64), (40, 24)]) +
                             [S.grid_view(1.0, 2.0, 0.0, 0.0, 64, 64)])
    want = O.Stream(data).touched_bytes(views)
    got = H.touched_bytes([H.Stream(data)], views)
    assert np.allclose(got, want, rtol=0, atol=1e-6)


@pytest.mark.gpu
def test_touched_bytes_union(tiny_streams, tiny_cfg):
    """Union over a call: one view alone equals its per-view count (and the
    oracle's); a repeated view adds only its output; the union never exceeds
    the sum of the per-view counts."""
    c = tiny_cfg
    data = tiny_streams[c.qstep].stream
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    vs = S.random_views(22, geo, 3, [(48, 40)])
    st = H.Stream(data)
    one = S.views_to_array(vs[:1])
    want = O.Stream(data).touched_bytes(one)[0]
    assert abs(H.touched_bytes_union([st], one) - want) < 1e-6
    twice = S.views_to_array([vs[0], vs[0]])
    assert abs(H.touched_bytes_union([st], twice) - (want + 48 * 40 * 12)) < 1e-6
    three = S.views_to_array(vs)
    assert H.touched_bytes_union([st], three) <= float(np.sum(H.touched_bytes([st], three))) + 1e-6


@pytest.mark.gpu
def test_touched_bytes_significant_blocks_match_oracle():
    """On the hand-derived field with significant predictive records and
    reference tiles reached directly and through motion-compensation taps,
    the product's counter equals the oracle's (whose values are pinned by
    closed forms), per view and over the union."""
    from tests.test_oracle_pins import _sig_field
    data = O.encode(_sig_field(), 1, 8, 4, 1, mc=O.MC_ZERO).stream
    views = S.views_to_array([S.grid_view(1.0, 1.0, 4.5, 2.5, 2, 2), S.grid_view(1.0, 1.0, 5.5, 2.5, 2, 2),
                              S.grid_view(0.0, 0.0, 5.5, 2.5, 2, 2)])
    want = O.Stream(data).touched_bytes(views)
    st = H.Stream(data)
    assert np.allclose(H.touched_bytes([st], views), want, rtol=0, atol=1e-6)
    for v in range(len(views)):
        assert abs(H.touched_bytes_union([st], views[v:v + 1]) - want[v]) < 1e-6
