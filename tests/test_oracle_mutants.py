"""Each test plants one plausible mistake in a copy of the oracle's C source,
builds it on the CPU, and checks that the pins catch it.  Every planted
mistake keeps the oracle's reads in bounds, so a copy never crashes.  A mistake that is
consistent between the encoder and the decoder (a swapped motion-vector axis,
transposed bilinear taps) still round-trips losslessly, so these show which
pin stands guard over it."""
import numpy as np
import pytest

import oracle as O
import tests.test_oracle_pins as pins

MUTANTS = {
    # name: (original text, replacement, pins that must fail)
    "inverse_ycocg_sign": ("*r = bb + co;", "*r = bb - co;",
                           ["ycocg_lossless"]),
    "predictor_transposed_taps": ("fx * (4 - fy) * b + (4 - fx) * fy * c",
                                  "(4 - fx) * fy * b + fx * (4 - fy) * c",
                                  ["pred_plane"]),
    "predictor_mv_axes_swapped": ("int X = 4 * x + mvx;\n    int Y = 4 * y + mvy;\n    int x0 = (int)fdiv(X, 4), y0 = (int)fdiv(Y, 4);\n    int fx = X - 4 * x0, fy = Y - 4 * y0;\n    int xa = clampi(x0, 0, W - 1)",
                                  "int X = 4 * x + mvy;\n    int Y = 4 * y + mvx;\n    int x0 = (int)fdiv(X, 4), y0 = (int)fdiv(Y, 4);\n    int fx = X - 4 * x0, fy = Y - 4 * y0;\n    int xa = clampi(x0, 0, W - 1)",
                                  ["pred_shift"]),
    "search_cost_sign": ("acc += iabs(S[y * g->W + x] - sign * p);", "acc += iabs(S[y * g->W + x] + sign * p);",
                         ["search_sign"]),
    "quantiser_rounding": ("int lv = (int)fdiv(a + q / 2, q);", "int lv = (int)fdiv(a + q, q);",
                           ["quantiser"]),
    "bise_trit_radix": ("            packed += (val >> b) * mul;\n            mul *= radix;",
                        "            packed += (val >> b) * mul;\n            mul *= radix + 1;",
                        ["bise_golden"]),
    "decoder_node_axes": ("v[c] += srv_at(s, l, i >> l, j >> l, c, cx[c], cy[c]);",
                          "v[c] += srv_at(s, l, j >> l, i >> l, c, cx[c], cy[c]);",
                          ["random_access"]),
    "mv_symbol_axes": ("*mvx = (int)((sym / 2u) / side) - 4 * g->Ws;\n    *mvy = (int)((sym / 2u) % side) - 4 * g->Ws;",
                       "*mvy = (int)((sym / 2u) / side) - 4 * g->Ws;\n    *mvx = (int)((sym / 2u) % side) - 4 * g->Ws;",
                       ["lossless"]),
    "render_weights_swapped": ("r->ws[0] = 1.0 - fs; r->ws[1] = fs;", "r->ws[0] = fs; r->ws[1] = 1.0 - fs;",
                               ["render_grid"]),
    "adjoint_ycocg_transpose": ("gv[1] = 0.5 * gR - 0.5 * gB;", "gv[1] = 0.5 * gB - 0.5 * gR;",
                                ["adjoint_dot"]),
    "touched_root_bytes": ("if (!root_seen[rp]) { root_seen[rp] = 1; acc += 2.0; }",
                           "if (!root_seen[rp]) { root_seen[rp] = 1; acc += 1.0; }",
                           ["touched"]),
    "touched_record_header_dropped": ("acc += 2.0 + 4.0 * (1 + (orc_bise_bits(md, bb, (uint64_t)bw * bh) + 31) / 32);",
                                      "acc += 2.0 + 4.0 * ((orc_bise_bits(md, bb, (uint64_t)bw * bh) + 31) / 32);",
                                      ["touched_sig"]),
    "touched_tap_tile_double_counted": ("if (!blk_seen[rk]) {\n                                                    blk_seen[rk] = 1;",
                                        "if (1) {\n                                                    blk_seen[rk] = 1;",
                                        ["touched_sig", "touched_direct_and_taps"]),
    "touched_tap_tile_bytes": ("if (find_record(s, rnc, kk)) acc += g->B * g->B * 2.0 + 4.0;",
                               "if (find_record(s, rnc, kk)) acc += g->B * g->B * 2.0;",
                               ["touched_sig"]),
    "chroma_filter_rounding": ("d[(size_t)yc * g->cW[c] + xc] = (int16_t)fdiv(sum + k / 2, k);",
                               "d[(size_t)yc * g->cW[c] + xc] = (int16_t)fdiv(sum, k);",
                               ["chroma_closed_form"]),
    "chroma_sample_mapping": ("cx[c] = (g->sub && c > 0) ? x >> 1 : x;",
                              "cx[c] = (g->sub && c > 0) ? (x >> 2) << 1 : x;",
                              ["chroma_closed_form"]),
    "chroma_full_decode_mapping": ("int xc = (g->sub && c > 0) ? x >> 1 : x, yc = (g->sub && c > 0) ? y >> 1 : y;",
                                   "int xc = (g->sub && c > 0) ? x >> 1 : x, yc = (g->sub && c > 0) ? (y >> 2) << 1 : y;",
                                   ["chroma_closed_form"]),
    "chroma_root_bytes": ("size_t rp = ((size_t)(i >> g->L) * g->gv[g->L] + (j >> g->L)) * g->npx + g->coff[c] +",
                          "size_t rp = ((size_t)(i >> g->L) * g->gv[g->L] + (j >> g->L)) * g->npx + g->coff[0] +",
                          ["chroma_touched"]),
    "relax_bias_ycocg_sign": ("double t = v[0] - v[2] / 2.0 + (bias ? 0.25 : 0.0);",
                              "double t = v[0] - v[2] / 2.0 - (bias ? 0.25 : 0.0);", ["relax_bias_ycocg"]),
    "mc_rounding_bias_scale": ("return gcd4(fx) * gcd4(fy) / 32.0;", "return gcd4(fx) * gcd4(fy) / 16.0;",
                               ["mc_rounding_bias"]),
    "progressive_one_level_too_deep": ("for (int l = lod; l < L; l++)", "for (int l = lod > 0 ? lod - 1 : 0; l < L; l++)",
                                       ["progressive"]),
}


def _run(name, tiny_lf, tiny_cfg, ragged_lf):
    c = tiny_cfg
    if name == "ycocg_lossless":
        pins.test_ycocg_lossless_and_ranges()
    elif name == "pred_plane":
        pins.test_predictor_reproduces_planes_at_quarter_positions()
    elif name == "pred_shift":
        pins.test_predictor_integer_shift_is_a_copy()
    elif name == "search_sign":
        pins.test_search_sign_convention(False)
    elif name == "quantiser":
        pins.test_quantiser_error_bound_and_symmetry(4)
    elif name == "bise_golden":
        pins.test_bise_golden_layout()
    elif name == "random_access":
        streams = {q: O.encode(tiny_lf, c.levels, c.block, c.search, q, debug=True) for q in (1, 4)}
        pins.test_random_access_equals_full_decode(streams, ragged_lf)
    elif name == "lossless":
        pins.test_lossless_round_trip(tiny_lf, tiny_cfg, ragged_lf, O.MC_QPEL)
    elif name == "render_grid":
        pins.test_render_exact_at_grid_samples(tiny_lf)
    elif name == "adjoint_dot":
        st = O.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, 4).stream)
        import synthlf as S
        geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
        views = S.views_to_array(S.random_views(11, geo, 1, [(12, 10)]))
        pins.test_adjoint_dot_product((st, views))
    elif name == "touched":
        pins.test_touched_bytes_closed_form(tiny_cfg)
    elif name == "touched_sig":
        pins.test_touched_bytes_significant_blocks_closed_form()
    elif name == "touched_direct_and_taps":
        pins.test_touched_bytes_reference_reached_directly_and_by_taps()
    elif name == "chroma_closed_form":
        pins.test_chroma_420_lossless_luma_and_filter_closed_form(tiny_lf, tiny_cfg, ragged_lf, O.MC_QPEL)
    elif name == "chroma_touched":
        pins.test_chroma_420_touched_bytes_closed_form(tiny_cfg)
    elif name == "relax_bias_ycocg":
        pins.test_relax_bias_ycocg_closed_form(tiny_lf, tiny_cfg)
    elif name == "mc_rounding_bias":
        pins.test_mc_rounding_bias_equals_brute_force()
    elif name == "progressive":
        pins.test_progressive_lossless_equals_level_images(tiny_lf, tiny_cfg, ragged_lf, O.MC_QPEL)
    else:
        raise KeyError(name)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant, tmp_path, tiny_lf, tiny_cfg, ragged_lf):
    old, new, guards = MUTANTS[mutant]
    src = O.source_text()
    assert src.count(old) == 1, f"mutation site for {mutant} not found exactly once"
    so = O.build_variant(src.replace(old, new), tmp_path / f"{mutant}.so")
    with O.using(so):
        for g in guards:
            with pytest.raises(AssertionError):
                _run(g, tiny_lf, tiny_cfg, ragged_lf)


def test_unmutated_copy_passes_the_same_pins(tmp_path, tiny_lf, tiny_cfg, ragged_lf):
    so = O.build_variant(O.source_text(), tmp_path / "same.so")
    with O.using(so):
        for g in sorted({g for _, _, gs in MUTANTS.values() for g in gs}):
            _run(g, tiny_lf, tiny_cfg, ragged_lf)
