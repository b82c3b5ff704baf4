"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
invariant the paper states (lossless integer coding, Sec. 4.5-4.6), a
hand-derived layout example, a brute-force enumeration, or a special case that
reduces to a textbook definition.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle as O
import synthlf as S

GOLDEN = Path(__file__).parent / "golden"


# --------------------------------------------------------------------------
# Sec. 4.5: YCoCg-R
# --------------------------------------------------------------------------

def _rgb_grid(n=20000, seed=0):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, 256, size=(n, 3))
    edges = np.array([[r, g, b] for r in (0, 1, 254, 255) for g in (0, 1, 254, 255) for b in (0, 1, 254, 255)])
    return np.concatenate([edges, pts])


def test_ycocg_lossless_and_ranges():
    """Sec. 4.5: the colour transform is lossless on 8-bit RGB, and its
    outputs fit the widened range (Y in [0,255], Co/Cg in [-255,255])."""
    for r, g, b in _rgb_grid():
        y, co, cg = O.rgb_to_ycocg(int(r), int(g), int(b))
        assert 0 <= y <= 255 and -255 <= co <= 255 and -255 <= cg <= 255
        assert O.ycocg_to_rgb(y, co, cg) == (r, g, b)


def test_ycocg_closed_form():
    """YCoCg: Co = R - B, Cg = G - (R + B)/2, Y = (R + 2G + B)/4; the lifting
    form agrees up to its floor roundings (catches swapped channels/signs)."""
    for r, g, b in _rgb_grid(5000, 1):
        y, co, cg = O.rgb_to_ycocg(int(r), int(g), int(b))
        assert co == r - b
        assert abs(cg - (g - (r + b) / 2.0)) <= 0.5
        assert abs(y - (r + 2 * g + b) / 4.0) <= 1.0


# --------------------------------------------------------------------------
# quantiser (configs; not in the paper)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q", [1, 2, 3, 4, 8])
def test_quantiser_error_bound_and_symmetry(q):
    prev = None
    for r in range(-1100, 1101):
        lv = O.quantise(r, q)
        assert abs(r - q * lv) <= q // 2
        assert O.quantise(-r, q) == -lv
        if prev is not None:
            assert lv >= prev
        prev = lv
    if q == 1:
        assert all(O.quantise(r, 1) == r for r in range(-50, 51))


# --------------------------------------------------------------------------
# Sec. 4.4 + Sec. 6: quarter-pel predictor
# --------------------------------------------------------------------------

def test_predictor_integer_shift_is_a_copy():
    """mv = 4*(dx, dy) reads R(x+dx, y+dy), clamped to the image: the shift
    direction and axes of the motion vector (Sec. 4.4: B_R^{xy})."""
    rng = np.random.default_rng(2)
    R = rng.integers(-300, 300, size=(13, 17)).astype(np.int16)   # H=13, W=17
    for _ in range(400):
        x, y = int(rng.integers(0, 17)), int(rng.integers(0, 13))
        dx, dy = int(rng.integers(-5, 6)), int(rng.integers(-5, 6))
        want = R[min(max(y + dy, 0), 12), min(max(x + dx, 0), 16)]
        assert O.pred_qpel(R, x, y, 4 * dx, 4 * dy) == want


def test_predictor_reproduces_planes_at_quarter_positions():
    """Bilinear interpolation is exact on affine functions: for
    R = a*x + b*y the prediction at quarter position (X/4, Y/4) equals
    round_half_up((a*X + b*Y)/4).  a != b catches transposed taps/weights."""
    H, W = 24, 24
    for a, b in [(4, -8), (-12, 4), (7, 3), (0, 5)]:
        yy, xx = np.mgrid[0:H, 0:W]
        R = (a * xx + b * yy).astype(np.int16)
        for x in range(6, 18, 3):
            for y in range(6, 18, 3):
                for mvx in range(-7, 8):
                    for mvy in range(-7, 8, 3):
                        X, Y = 4 * x + mvx, 4 * y + mvy
                        want = math.floor((a * X + b * Y) / 4.0 + 0.5)
                        assert O.pred_qpel(R, x, y, mvx, mvy) == want


def test_predictor_constant_and_edges():
    R = np.full((8, 8), -37, np.int16)
    for mvx in range(-9, 10):
        for mvy in range(-9, 10):
            assert O.pred_qpel(R, 0, 7, mvx, mvy) == -37
    # clamp: a motion vector pointing far outside reads the edge
    R = np.arange(64, dtype=np.int16).reshape(8, 8)
    assert O.pred_qpel(R, 0, 0, -40, -40) == R[0, 0]
    assert O.pred_qpel(R, 7, 7, 40, 40) == R[7, 7]
    assert O.pred_qpel(R, 7, 0, 40, -40) == R[0, 7]


# --------------------------------------------------------------------------
# Sec. 4.4: phase-shifted search (Eq. 1-2, the argmin displays)
# --------------------------------------------------------------------------

def _shifted(R, dx, dy):
    H, W = R.shape
    yy, xx = np.mgrid[0:H, 0:W]
    return R[np.clip(yy + dy, 0, H - 1), np.clip(xx + dx, 0, W - 1)].astype(np.int32)


@pytest.mark.parametrize("refine", [False, True])
def test_search_sign_convention(refine):
    """Eq. 1 (subtractive) finds P = +R shifted; Eq. 2 (additive) finds
    P = -R shifted, with zero residual."""
    rng = np.random.default_rng(3)
    R = rng.integers(-200, 200, size=(32, 32)).astype(np.int16)
    for dx, dy in [(2, -1), (-3, 3), (0, 0), (4, -4)]:
        k = 1 * 4 + 1                        # block (1, 1) of 8x8 blocks
        P = _shifted(R, dx, dy)
        assert O.mc_search_block(P, R, 8, k, 4, refine) == (4 * dx, 4 * dy, 1, 0)
        assert O.mc_search_block(-P, R, 8, k, 4, refine) == (4 * dx, 4 * dy, -1, 0)


def test_search_finds_quarter_pel_motion():
    """A block predicted from a smooth random reference at a quarter-pel
    vector is matched exactly by the refinement stage and not by the integer
    stage.  (A plane would not do: many vectors predict it equally well.)"""
    H, W = 32, 32
    rng = np.random.default_rng(14)
    g = rng.integers(-400, 400, size=(20, 20)).astype(np.float64)
    yy, xx = np.mgrid[0:H, 0:W] / 3.0
    y0, x0 = np.floor(yy).astype(int), np.floor(xx).astype(int)
    fy, fx = yy - y0, xx - x0
    R = ((g[y0, x0] * (1 - fx) + g[y0, x0 + 1] * fx) * (1 - fy)
         + (g[y0 + 1, x0] * (1 - fx) + g[y0 + 1, x0 + 1] * fx) * fy).round().astype(np.int16)
    k = 5
    mvx, mvy = 6, -3        # 1.5 px, -0.75 px
    P = np.zeros((H, W), np.int32)
    for y in range(H):
        for x in range(W):
            P[y, x] = O.pred_qpel(R, x, y, mvx, mvy)
    assert O.mc_search_block(P, R, 8, k, 4, True) == (mvx, mvy, 1, 0)
    assert O.mc_search_block(P, R, 8, k, 4, False)[3] > 0


def _np_pred(R, x0, y0, bw, bh, mvx, mvy):
    """Vectorised quarter-pel predictor for one block (checked against the
    oracle's pinned scalar predictor before use)."""
    H, W = R.shape
    yy, xx = np.mgrid[y0:y0 + bh, x0:x0 + bw]
    X, Y = 4 * xx + mvx, 4 * yy + mvy
    xa, ya = X // 4, Y // 4
    fx, fy = X - 4 * xa, Y - 4 * ya
    cx = lambda v: np.clip(v, 0, W - 1)
    cy = lambda v: np.clip(v, 0, H - 1)
    R = R.astype(np.int64)
    s = ((4 - fx) * (4 - fy) * R[cy(ya), cx(xa)] + fx * (4 - fy) * R[cy(ya), cx(xa + 1)]
         + (4 - fx) * fy * R[cy(ya + 1), cx(xa)] + fx * fy * R[cy(ya + 1), cx(xa + 1)])
    return (s + 8) // 16


def test_vectorised_predictor_matches_oracle():
    rng = np.random.default_rng(4)
    R = rng.integers(-500, 500, size=(20, 28)).astype(np.int16)
    for _ in range(50):
        mvx, mvy = (int(v) for v in rng.integers(-20, 21, 2))
        got = _np_pred(R, 8, 4, 8, 8, mvx, mvy)
        for (yy, xx), v in np.ndenumerate(got):
            assert v == O.pred_qpel(R, 8 + xx, 4 + yy, mvx, mvy)


@pytest.mark.parametrize("mode", [O.MC_INTEGER, O.MC_QPEL])
def test_encoder_search_attains_brute_force_minimum(tiny_lf, tiny_cfg, mode):
    """Brute force over every candidate: with the per-pel search (the paper's
    own) the stored (mv, sign) attains min(Delta_-, Delta_+) over the whole
    window; with quarter-pel refinement it attains the minimum over the
    refinement neighbourhood of each sign's integer winner, and is never
    worse than the integer minimum.  Ties follow the documented keys."""
    c = tiny_cfg
    enc = O.encode(tiny_lf, c.levels, c.block, c.search, 1, mc=mode, debug=True)
    st = O.Stream(enc.stream)
    B, Ws = c.block, c.search
    nbx = c.width // B
    checked = 0
    for l in range(c.levels - 1, -1, -1):
        gu = (c.nu + (1 << l) - 1) >> l
        gv = (c.nv + (1 << l) - 1) >> l
        base = 3 * sum(((c.nu + (1 << m) - 1) >> m) * ((c.nv + (1 << m) - 1) >> m)
                       for m in range(c.levels - 1, l, -1))
        for a in range(gu):
            for b in range(gv):
                if a % 2 == 0 and b % 2 == 0:
                    continue
                for ch in range(3):
                    nc = base + (a * gv + b) * 3 + ch
                    rnc = base + ((a & ~1) * gv + (b & ~1)) * 3 + ch
                    P = enc.S[nc]
                    R = enc.Rhat[rnc].astype(np.int16)
                    for k in range(0, st.nblocks, 7):
                        x0, y0 = (k % nbx) * B, (k // nbx) * B
                        blk = P[y0:y0 + B, x0:x0 + B].astype(np.int64)
                        cost = {}
                        for sgn in (1, -1):
                            for dy in range(-Ws, Ws + 1):
                                for dx in range(-Ws, Ws + 1):
                                    pr = _np_pred(R, x0, y0, B, B, 4 * dx, 4 * dy)
                                    cost[(4 * dx, 4 * dy, sgn)] = int(np.abs(blk - sgn * pr).sum())
                        _, mvx, mvy, sgn = st.block_info(nc, k)
                        best_int = min(cost.values())
                        if mode == O.MC_INTEGER:
                            assert cost[(mvx, mvy, sgn)] == best_int
                            winners = [kk for kk, v in cost.items() if v == best_int]
                            key = lambda t: (0 if t[2] == 1 else 1, abs(t[0]) + abs(t[1]), t[1], t[0])
                            assert min(winners, key=key) == (mvx, mvy, sgn)
                        else:
                            got = int(np.abs(blk - sgn * _np_pred(R, x0, y0, B, B, mvx, mvy)).sum())
                            assert got <= best_int
                            # neighbourhood of the same sign's integer winner
                            ints = {kk: v for kk, v in cost.items() if kk[2] == sgn}
                            bi = min(ints.values())
                            wk = min((kk for kk, v in ints.items() if v == bi),
                                     key=lambda t: (abs(t[0]) + abs(t[1]), t[1], t[0]))
                            for oy in range(-3, 4):
                                for ox in range(-3, 4):
                                    mx, my = wk[0] + ox, wk[1] + oy
                                    if abs(mx) > 4 * Ws or abs(my) > 4 * Ws:
                                        continue
                                    v = int(np.abs(blk - sgn * _np_pred(R, x0, y0, B, B, mx, my)).sum())
                                    assert got <= v
                        checked += 1
    assert checked > 100


# --------------------------------------------------------------------------
# Sec. 4.6: BISE
# --------------------------------------------------------------------------

def test_bise_choose_smallest_alphabet():
    """N is the smallest of {2^b, 3*2^b, 5*2^b} covering the range."""
    table = {1: (0, 0), 2: (0, 1), 3: (1, 0), 4: (0, 2), 5: (2, 0), 6: (1, 1), 7: (0, 3), 8: (0, 3),
             9: (2, 1), 10: (2, 1), 11: (1, 2), 12: (1, 2), 13: (0, 4), 16: (0, 4), 17: (2, 2),
             20: (2, 2), 21: (1, 3), 24: (1, 3), 25: (0, 5), 2178: (2, 9), 2560: (2, 9), 2561: (1, 10)}
    for rng, want in table.items():
        assert O.bise_choose(rng) == want, rng
    for rng in range(1, 5000):
        mode, b = O.bise_choose(rng)
        N = (1, 3, 5)[mode] << b
        assert N >= rng
        for m2 in range(3):
            for b2 in range(0, 14):
                N2 = (1, 3, 5)[m2] << b2
                if N2 >= rng:
                    assert N2 >= N


def test_bise_near_information_bound():
    """Trits cost 8/5 bits and quints 7/3 bits: within 0.016 bit of log2 N
    per value (up to last-group padding)."""
    for rng in range(2, 3000, 7):
        mode, b = O.bise_choose(rng)
        N = (1, 3, 5)[mode] << b
        n = 15 * 64
        bits = O.bise_bits(mode, b, n)
        assert bits / n <= math.log2(N) + 0.016


def test_bise_golden_layout():
    cases = json.loads((GOLDEN / "bise_layout.json").read_text())["cases"]
    for c in cases:
        words = O.bise_pack(c["values"], c["mode"], c["b"])
        assert list(map(int, words)) == c["words"], c
        for i, v in enumerate(c["values"]):
            assert O.bise_get(np.array(c["words"], np.uint32), c["mode"], c["b"], i) == v


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_bise_roundtrip_random_access_and_sequential(mode):
    rng = np.random.default_rng(5 + mode)
    for b in range(0, 13):
        N = (1, 3, 5)[mode] << b
        n = int(rng.integers(1, 300))
        vals = rng.integers(0, N, size=n).astype(np.uint32)
        words = O.bise_pack(vals, mode, b)
        assert len(words) == (O.bise_bits(mode, b, n) + 31) // 32
        assert np.array_equal(O.bise_unpack(words, mode, b, n), vals)
        for i in rng.integers(0, n, size=min(n, 40)):
            assert O.bise_get(words, mode, b, int(i)) == vals[i]


# --------------------------------------------------------------------------
# whole codec: the paper's lossless claims and the closed-loop bound
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL, O.MC_ZERO, O.MC_INTEGER])
def test_lossless_round_trip(tiny_lf, tiny_cfg, ragged_lf, mc):
    """Sec. 4.5-4.6: lossless integer coding -- with q = 1 and zero
    thresholds every decoded sample equals the input, for every MC mode, on
    square and ragged fields (partial blocks, 1- and 2-member clusters)."""
    c = tiny_cfg
    for lf, L, B in [(tiny_lf, c.levels, c.block), (ragged_lf, 2, 8), (ragged_lf, 3, 16)]:
        st = O.Stream(O.encode(lf, L, B, c.search, 1, mc=mc).stream)
        assert np.array_equal(st.decode_all(), lf)


@pytest.mark.parametrize("q", [2, 4, 8])
def test_closed_loop_error_bound(tiny_lf, tiny_cfg, ragged_lf, q):
    """Closed loop: with zero thresholds the only error is the leaf-level
    quantiser error, |decoded - original| <= floor(q/2) in Y, Co and Cg."""
    c = tiny_cfg
    for lf, L, B in [(tiny_lf, c.levels, c.block), (ragged_lf, 2, 8)]:
        st = O.Stream(O.encode(lf, L, B, c.search, q).stream)
        _, ycc = st.decode_all(with_ycocg=True)
        nu, nv, H, W, _ = lf.shape
        orig = np.zeros((nu, nv, 3, H, W), np.int64)
        for i in range(nu):
            for j in range(nv):
                for yy in range(0, H, 3):
                    for xx in range(0, W, 2):
                        r, g, b = (int(v) for v in lf[i, j, yy, xx])
                        orig[i, j, :, yy, xx] = O.rgb_to_ycocg(r, g, b)
                        assert np.all(np.abs(ycc[i, j, :, yy, xx] - orig[i, j, :, yy, xx]) <= q // 2)


def test_thresholds_drop_blocks_and_stay_decodable(tiny_lf, tiny_cfg):
    """Sec. 4.5: raising the block thresholds removes significant blocks
    (fewer stored), and the stream still decodes consistently."""
    c = tiny_cfg
    base = O.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, 4).stream)
    thr = O.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, 4, t_ref=400, t_pred=800).stream)
    assert thr.n_sig < base.n_sig
    coords = np.array([[i, j, x, y] for i in range(4) for j in range(4) for x in (0, 31, 63) for y in (0, 40, 63)])
    full = thr.decode_all()
    assert np.array_equal(thr.decode_samples(coords), full[coords[:, 0], coords[:, 1], coords[:, 3], coords[:, 2]])


def test_random_access_equals_full_decode(tiny_streams, ragged_lf):
    """Sec. 4.8.4: random access to any sample gives the same value as the
    full reconstruction (two independent paths through the stream)."""
    for enc in tiny_streams.values():
        st = O.Stream(enc.stream)
        full = st.decode_all()
        ii, jj, xx, yy = np.meshgrid(np.arange(st.nu), np.arange(st.nv), np.arange(st.W), np.arange(st.H),
                                     indexing="ij")
        coords = np.stack([ii, jj, xx, yy], -1).reshape(-1, 4)
        got = st.decode_samples(coords).reshape(st.nu, st.nv, st.W, st.H, 3).transpose(0, 1, 3, 2, 4)
        assert np.array_equal(got, full)
    st = O.Stream(O.encode(ragged_lf, 2, 8, 4, 4).stream)
    full = st.decode_all()
    rng = np.random.default_rng(6)
    coords = np.stack([rng.integers(0, 5, 3000), rng.integers(0, 3, 3000), rng.integers(0, 37, 3000),
                       rng.integers(0, 29, 3000)], -1)
    assert np.array_equal(st.decode_samples(coords), full[coords[:, 0], coords[:, 1], coords[:, 3], coords[:, 2]])


def _nc_layout(nu, nv, L):
    """(level, a, b, ch) of every node-channel in breadth-first order."""
    out = []
    for l in range(L - 1, -1, -1):
        gu, gv = (nu + (1 << l) - 1) >> l, (nv + (1 << l) - 1) >> l
        for a in range(gu):
            for b in range(gv):
                for ch in range(3):
                    out.append((l, a, b, ch))
    return out


def test_without_mc_is_plain_residual_coding(tiny_lf, tiny_cfg):
    """MC off: a predictive SRV is coded directly, so its dequantised
    coefficients equal q * Q(SRV); no motion vectors are stored."""
    c = tiny_cfg
    for q in (1, 4):
        enc = O.encode(tiny_lf, c.levels, c.block, c.search, q, mc=O.MC_OFF, debug=True)
        st = O.Stream(enc.stream)
        assert st.n_mv == 0 and st.mc == 0
        coeff, _ = st.dequant()
        quant = np.vectorize(lambda r: O.quantise(int(r), q))
        for nc in range(0, st.n_nc, 5):
            assert np.array_equal(coeff[nc], q * quant(enc.S[nc]))


def test_zero_motion_predicts_from_reference(tiny_lf, tiny_cfg):
    """Zero motion, subtractive sign: a predictive SRV's residual is
    SRV - R^ (the sibling reference's dequantised SRV), quantised."""
    c = tiny_cfg
    q = 2
    enc = O.encode(tiny_lf, c.levels, c.block, c.search, q, mc=O.MC_ZERO, debug=True)
    st = O.Stream(enc.stream)
    coeff, _ = st.dequant()
    lay = _nc_layout(c.nu, c.nv, c.levels)
    index = {t: n for n, t in enumerate(lay)}
    quant = np.vectorize(lambda r: O.quantise(int(r), q))
    for nc, (l, a, b, ch) in enumerate(lay):
        if a % 2 == 0 and b % 2 == 0:
            assert np.array_equal(coeff[nc], enc.Rhat[nc])
            continue
        rnc = index[(l, a & ~1, b & ~1, ch)]
        assert np.array_equal(coeff[nc], q * quant(enc.S[nc] - enc.Rhat[rnc]))
        for k in range(0, st.nblocks, 9):
            assert st.block_info(nc, k)[1:] == (0, 0, 1)


def test_identical_views_give_empty_residuals(tiny_cfg):
    """All views equal: every RKV equals the view, every SRV is zero, so no
    block is significant and the stream is the roots plus the index."""
    c = tiny_cfg
    one = S.make_lf(7, 1, 1, 64, 64, 3, 0.0, "noise_gradient")[0, 0]
    lf = np.broadcast_to(one, (4, 4, 64, 64, 3)).copy()
    st = O.Stream(O.encode(lf, c.levels, c.block, c.search, 4).stream)
    assert st.n_sig == 0
    assert np.array_equal(st.decode_all(), lf)


def test_bpp_unit_from_table1():
    """Table 1's sizes are nu*nv*rows*cols*3 bytes, so bpp counts bits per
    24-bit sample of one view; the abstract's 30-800x range is 24/bpp."""
    d = json.loads((GOLDEN / "table1_sizes.json").read_text())
    ratios = []
    for name, nu, nv, rows, cols, mb, bpp in d["rows"]:
        assert nu * nv * rows * cols * 3 / 2 ** 20 == mb, name
        ratios.append(24.0 / bpp)
    lo, hi = d["abstract_ratio_range"]
    assert min(ratios) >= lo and max(ratios) >= hi


# --------------------------------------------------------------------------
# Sec. 2.1 / Sec. 5: rendering
# --------------------------------------------------------------------------

def _one(view):
    return S.views_to_array([view])


def test_render_exact_at_grid_samples(tiny_lf):
    """(u, v) on a camera and (s, t) on pixel centres: the render is that
    camera's image."""
    for i, j in [(0, 0), (2, 1), (3, 3)]:
        v = _one(S.grid_view(float(i), float(j), 0.0, 0.0, 64, 64))
        out = O.render_dense(tiny_lf, v).reshape(64, 64, 3)
        assert np.max(np.abs(out - tiny_lf[i, j] / 255.0)) <= 1e-12


def test_render_linear_precision():
    """Quadrilinear interpolation reproduces affine functions of (u,v,s,t)."""
    nu, nv, H, W = 4, 5, 16, 20
    i, j, y, x = np.meshgrid(np.arange(nu), np.arange(nv), np.arange(H), np.arange(W), indexing="ij")
    lf = np.stack([10 + 3 * x + 7 * i, 200 - 5 * y + 2 * j, 40 + 2 * x + 3 * y + 11 * i + 13 * j], -1)
    assert lf.min() >= 0 and lf.max() <= 255
    lf = lf.astype(np.uint8)
    rng = np.random.default_rng(8)
    for _ in range(20):
        u0, v0 = rng.random() * (nu - 1), rng.random() * (nv - 1)
        so, to = rng.random() * 2, rng.random() * 2
        view = S.grid_view(u0, v0, so, to, 12, 10)
        out = O.render_dense(lf, _one(view)).reshape(10, 12, 3)
        Huv = view.H_uv.astype(np.float64)
        u, vv = Huv[2], Huv[5]
        for py in range(10):
            for px in range(12):
                s = px + 0.5 + float(view.H_st[2])
                t = py + 0.5 + float(view.H_st[5])
                want = np.array([10 + 3 * s + 7 * u, 200 - 5 * t + 2 * vv, 40 + 2 * s + 3 * t + 11 * u + 13 * vv])
                assert np.max(np.abs(out[py, px] * 255.0 - want)) < 1e-9


def test_render_matches_tent_sum(tiny_lf, tiny_cfg):
    """Brute force: the render equals the sum over all samples of the
    product of 1-D tent kernels (inside the grid)."""
    c = tiny_cfg
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.random_views(9, geo, 3, [(9, 7)], radius_frac=0.15)
    arr = S.views_to_array(views)
    out = O.render_dense(tiny_lf, arr)
    lf = tiny_lf.astype(np.float64)
    tent = lambda d: np.maximum(0.0, 1.0 - np.abs(d))
    for vi, v in enumerate(views):
        Huv = v.H_uv.astype(np.float64).reshape(3, 3)
        Hst = v.H_st.astype(np.float64).reshape(3, 3)
        for py in range(v.height):
            for px in range(v.width):
                p = np.array([px + 0.5, py + 0.5, 1.0])
                a = Huv @ p
                b = Hst @ p
                u, vv, s, t = a[0] / a[2], a[1] / a[2], b[0] / b[2], b[1] / b[2]
                if not (0 <= u <= c.nu - 1 and 0 <= vv <= c.nv - 1 and 0 <= s <= c.width - 1 and 0 <= t <= c.height - 1):
                    continue
                w = (tent(u - np.arange(c.nu))[:, None, None, None] * tent(vv - np.arange(c.nv))[None, :, None, None]
                     * tent(t - np.arange(c.height))[None, None, :, None] * tent(s - np.arange(c.width))[None, None, None, :])
                want = np.einsum("ijyx,ijyxc->c", w, lf) / 255.0
                got = out[int(arr[vi]["out_offset"]) + (py * v.width + px) * 3:][:3]
                assert np.max(np.abs(got - want)) < 1e-9


def test_render_clamps_to_edges(tiny_lf):
    a = O.render_dense(tiny_lf, _one(S.grid_view(-2.5, 1.25, -9.0, 3.0, 16, 16)))
    b = O.render_dense(tiny_lf, _one(S.grid_view(0.0, 1.25, -9.0, 3.0, 16, 16)))
    assert np.array_equal(a, b)


def test_random_access_render_equals_dense_render(tiny_streams, tiny_cfg):
    c = tiny_cfg
    st = O.Stream(tiny_streams[c.qstep].stream)
    lf = st.decode_all()
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(10, geo, 2, [(32, 24)]))
    dense = O.render_dense(lf, views)
    pix = np.array([[v, x, y] for v in range(2) for y in range(24) for x in range(32)], np.int32)
    ra = st.render_pixels(views, pix)
    assert np.array_equal(ra.reshape(-1), dense)


# --------------------------------------------------------------------------
# differentiable relaxation and its adjoint
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def relax_setup(tiny_streams, tiny_cfg):
    c = tiny_cfg
    st = O.Stream(tiny_streams[c.qstep].stream)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(11, geo, 2, [(20, 16)]))
    return st, views


def test_relaxation_close_to_integer_render(relax_setup):
    """With the dequantised coefficients the relaxed render differs from the
    integer decode only by the dropped roundings: the bilinear >>4 (<= 1/2
    per level) and the YCoCg >>1 (<= 1 per channel); no clamp is active
    here."""
    st, views = relax_setup
    co, ro = st.dequant()
    rel = st.relax_render(co, ro, views)
    integer = O.render_dense(st.decode_all(), views)
    assert np.max(np.abs(rel - integer)) * 255.0 <= 0.5 * st.L + 2.0 + 1e-9


def test_adjoint_dot_product(relax_setup):
    """<J a, b> = <a, J^T b> for random a, b (the relaxation is linear)."""
    st, views = relax_setup
    rng = np.random.default_rng(12)
    a_c = rng.standard_normal((st.n_nc, st.H, st.W))
    a_r = rng.standard_normal((st.n_roots, 3, st.H, st.W))
    Ja = st.relax_render(a_c, a_r, views)
    b = rng.standard_normal(Ja.shape)
    gc, gr = st.relax_adjoint(views, b)
    lhs = float(np.dot(Ja, b))
    rhs = float(np.sum(a_c * gc) + np.sum(a_r * gr))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    assert np.count_nonzero(gc) > 0


def test_adjoint_finite_differences(relax_setup):
    """Central differences of L = <render(c), b> along single coefficients
    equal the adjoint's entries (exact up to rounding: L is linear)."""
    st, views = relax_setup
    rng = np.random.default_rng(13)
    co, ro = st.dequant()
    b = rng.standard_normal(st.relax_render(co, ro, views).shape)
    gc, gr = st.relax_adjoint(views, b)
    hot = np.argwhere(gc != 0)
    pick = hot[rng.choice(len(hot), size=12, replace=False)]
    h = 0.5
    for nc, y, x in pick:
        cp = co.copy(); cp[nc, y, x] += h
        cm = co.copy(); cm[nc, y, x] -= h
        fd = (np.dot(st.relax_render(cp, ro, views), b) - np.dot(st.relax_render(cm, ro, views), b)) / (2 * h)
        assert abs(fd - gc[nc, y, x]) <= 1e-9 * max(1.0, abs(fd))
    r = tuple(np.argwhere(gr != 0)[0])
    rp = ro.copy(); rp[r] += h
    rm = ro.copy(); rm[r] -= h
    fd = (np.dot(st.relax_render(co, rp, views), b) - np.dot(st.relax_render(co, rm, views), b)) / (2 * h)
    assert abs(fd - gr[r]) <= 1e-9 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# touched-set counter (algorithmic bytes of a view)
# --------------------------------------------------------------------------

def test_touched_bytes_closed_form(tiny_cfg):
    """Identical views (no significant block) seen from camera (0, 0) with
    (s, t) on pixel centres: every pixel of cameras {0,1}x{0,1} is touched.
    Bytes = output 12/px + root 6/px + 3 predictive level-0 nodes x 3
    channels x 2 group entries x 16 + 3 x 3 x 64 blocks x MV bits / 8."""
    c = tiny_cfg
    one = S.make_lf(7, 1, 1, 64, 64, 3, 0.0, "noise_gradient")[0, 0]
    lf = np.broadcast_to(one, (4, 4, 64, 64, 3)).copy()
    st = O.Stream(O.encode(lf, c.levels, c.block, c.search, 4).stream)
    v = _one(S.grid_view(0.0, 0.0, 0.0, 0.0, 64, 64))
    mode, b = O.bise_choose(2 * (8 * c.search + 1) ** 2)
    mv_bits = O.bise_bits(mode, b, 15) / 15.0
    want = 64 * 64 * 12 + 64 * 64 * 6 + 3 * 3 * 2 * 16 + 3 * 3 * 64 * mv_bits / 8.0
    assert abs(st.touched_bytes(v)[0] - want) < 1e-6



def _sig_field(seed=5):
    """A 2x2 grid of 16x16 views (L = 1, B = 8) whose significant blocks are
    known by hand.  Cameras (0,0), (0,1), (1,0) show one texture; camera (1,1)
    adds d(x, y) = (x mod 8) + 8y to all three of R, G, B in the top block row
    (y < 8).  Adding d to R, G and B moves only Y of YCoCg-R (Co = R - B and
    Cg = G - t cancel it), so in the YCoCg-R domain, with q = 1, T = 0 and
    zero motion (mv = 0, sign +):
    - the root (rounded mean of 4) is Y + floor((d + 2) / 4), Co, Cg;
    - reference (0,0)'s SRV is -floor((d + 2) / 4) in Y: Y blocks 0 and 1
      significant (resident tiles), every other block zero;
    - predictive (0,1), (1,0) equal the reference's SRV: zero residual;
    - predictive (1,1)'s residual is d: Y blocks 0 and 1 significant with
      levels 0..63, i.e. BISE alphabet 2^6, 6 bits a value, 64 * 6 / 32 = 12
      payload words behind the one header word."""
    rng = np.random.default_rng(seed)
    base = rng.integers(0, 150, size=(16, 16, 3))
    lf = np.broadcast_to(base, (2, 2, 16, 16, 3)).copy()
    yy, xx = np.mgrid[0:8, 0:16]
    lf[1, 1, 0:8, :, :] += ((xx % 8) + 8 * yy)[..., None]
    return lf.astype(np.uint8)


def test_touched_bytes_significant_blocks_closed_form():
    """Algorithmic bytes with significant predictive records and reference
    tiles (Sec. 4.6 records, Sec. 4.8.2 resident references): a view at
    camera (1,1) only, reaching pixels x in {x0..x0+2}, y in {2, 3, 4} of its
    block 0.  Bytes = 12 per output pixel + 6 per root pixel + per touched
    predictive block (16 B group entry + MV bits / 8) + the significant Y
    record of block 0 (2 B offset + 4 B header + 12 x 4 B payload = 54 B)
    + every significant reference tile its zero-motion taps reach, once
    (8 * 8 * 2 + 4 = 132 B).  Taps of (x, y) read (x + 1, y + 1) too, so
    x0 = 5 reaches reference block 1 through its taps alone; x0 = 4 does not."""
    lf = _sig_field()
    st = O.Stream(O.encode(lf, 1, 8, 4, 1, mc=O.MC_ZERO).stream)
    # the hand derivation of which blocks are significant
    nc = {(a, b, c): (a * 2 + b) * 3 + c for a in range(2) for b in range(2) for c in range(3)}
    for (a, b, c), n in nc.items():
        for k in range(4):
            sig = st.block_info(n, k)[0]
            want = c == 0 and k < 2 and (a, b) in ((0, 0), (1, 1))
            assert bool(sig) == want, (a, b, c, k)
    mode, b = O.bise_choose(2 * (8 * 4 + 1) ** 2)
    mv_bits = O.bise_bits(mode, b, 15) / 15.0
    record, tile = 2 + 4 * (1 + 64 * 6 // 32), 8 * 8 * 2 + 4
    fixed = 2 * 2 * 12 + 9 * 6 + 3 * (16 + mv_bits / 8.0) + record
    got = st.touched_bytes(S.views_to_array([S.grid_view(1.0, 1.0, 4.5, 2.5, 2, 2),
                                             S.grid_view(1.0, 1.0, 5.5, 2.5, 2, 2)]))
    assert abs(got[0] - (fixed + tile)) < 1e-6
    assert abs(got[1] - (fixed + 2 * tile)) < 1e-6


def test_touched_bytes_reference_reached_directly_and_by_taps():
    """The field of the test above seen from (u, v) = (0, 0): the ray's
    neighbours are all four cameras (u = 0 gives cameras 0 and 1 with
    weights 1 and 0).  Reference (0,0)'s Y tiles 0 and 1 are reached directly
    and through the taps of three predictive nodes, and count once each; the
    three predictive nodes add 3 channels x (group entry + MV bits) each, and
    only (1,1)'s Y block 0 has a record."""
    lf = _sig_field()
    st = O.Stream(O.encode(lf, 1, 8, 4, 1, mc=O.MC_ZERO).stream)
    mode, b = O.bise_choose(2 * (8 * 4 + 1) ** 2)
    mv_bits = O.bise_bits(mode, b, 15) / 15.0
    record, tile = 2 + 4 * (1 + 64 * 6 // 32), 8 * 8 * 2 + 4
    want = 2 * 2 * 12 + 9 * 6 + 3 * 3 * (16 + mv_bits / 8.0) + record + 2 * tile
    got = st.touched_bytes(S.views_to_array([S.grid_view(0.0, 0.0, 5.5, 2.5, 2, 2)]))
    assert abs(got[0] - want) < 1e-6

# --------------------------------------------------------------------------
# progressive decoding (Sec. 1, Sec. 4: the upper levels of the tree carry
# what the views share, the lower levels their detail)
# --------------------------------------------------------------------------

def _level_images(lf, L):
    """Level images I_0..I_L of the input in YCoCg-R, straight from their
    definition: I_0 = the views, I_{l+1} = the rounded mean of each 2x2
    cluster of I_l (1, 2 or 4 members at the edges; Sec. 4.3).  Shape of
    I_l: [gu_l][gv_l][3][H][W]."""
    r, g, b = (lf[..., k].astype(np.int64) for k in range(3))
    co = r - b
    t = b + (co >> 1)
    cg = g - t
    y = t + (cg >> 1)
    levels = [np.stack([y, co, cg], axis=2)]
    for _ in range(L):
        P = levels[-1]
        pu, pv = (P.shape[0] + 1) // 2, (P.shape[1] + 1) // 2
        N = np.zeros((pu, pv) + P.shape[2:], np.int64)
        for A in range(pu):
            for Bn in range(pv):
                m = P[2 * A:2 * A + 2, 2 * Bn:2 * Bn + 2]
                k = m.shape[0] * m.shape[1]
                N[A, Bn] = np.floor_divide(m.sum(axis=(0, 1)) + k // 2, k)
        levels.append(N)
    return levels


def _all_coords(nu, nv, W, H):
    return np.stack(np.meshgrid(np.arange(nu), np.arange(nv), np.arange(W), np.arange(H), indexing="ij"),
                    -1).reshape(-1, 4).astype(np.int32)


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL])
def test_progressive_lossless_equals_level_images(tiny_lf, tiny_cfg, ragged_lf, mc):
    """With q = 1 and zero thresholds the closed loop reconstructs every
    level exactly, so decoding sample (i, j, x, y) down to level k gives
    I_k at node (i >> k, j >> k); level L gives the stored roots."""
    c = tiny_cfg
    for lf, L, B in [(tiny_lf, c.levels, c.block), (ragged_lf, 3, 16)]:
        nu, nv, H, W, _ = lf.shape
        st = O.Stream(O.encode(lf, L, B, c.search, 1, mc=mc).stream)
        I = _level_images(lf, L)
        co = _all_coords(nu, nv, W, H)
        for k in range(L + 1):
            _, ycc = st.decode_samples(co, with_ycocg=True, level=k)
            want = I[k][co[:, 0] >> k, co[:, 1] >> k, :, co[:, 3], co[:, 2]]
            assert np.array_equal(ycc, want), (L, k)


@pytest.mark.parametrize("q", [4, 8])
def test_progressive_closed_loop_bound(tiny_lf, tiny_cfg, ragged_lf, q):
    """Closed loop at every level: with zero thresholds the level-k
    reconstruction differs from I_k by at most floor(q/2) per channel."""
    c = tiny_cfg
    for lf, L, B in [(tiny_lf, c.levels, c.block), (ragged_lf, 3, 8)]:
        nu, nv, H, W, _ = lf.shape
        st = O.Stream(O.encode(lf, L, B, c.search, q).stream)
        I = _level_images(lf, L)
        co = _all_coords(nu, nv, W, H)
        for k in range(L):
            _, ycc = st.decode_samples(co, with_ycocg=True, level=k)
            want = I[k][co[:, 0] >> k, co[:, 1] >> k, :, co[:, 3], co[:, 2]]
            assert np.max(np.abs(ycc - want)) <= q // 2, (L, k)


def test_progressive_render_equals_dense_render_of_level_field(tiny_streams, tiny_cfg):
    """Rendering at level k by random access equals the dense FP64 render of
    the light field whose view (i, j) is its level-k node's reconstruction."""
    c = tiny_cfg
    st = O.Stream(tiny_streams[c.qstep].stream)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(12, geo, 2, [(24, 20)]))
    pix = np.array([[v, x, y] for v in range(2) for y in range(20) for x in range(24)], np.int32)
    co = _all_coords(c.nu, c.nv, c.width, c.height)
    for k in range(1, c.levels + 1):
        rgb = st.decode_samples(co, level=k)
        lf_k = np.zeros((c.nu, c.nv, c.height, c.width, 3), np.uint8)
        lf_k[co[:, 0], co[:, 1], co[:, 3], co[:, 2]] = rgb
        assert np.array_equal(st.render_pixels(views, pix, level=k).reshape(-1), O.render_dense(lf_k, views))


def test_progressive_touched_bytes_closed_form(tiny_cfg):
    """The identical-views case of test_touched_bytes_closed_form decoded to
    level 1 or 2: cameras {0,1}x{0,1} share the level-1 node (0, 0), a
    reference node without significant blocks, so only the output and the
    root pixels remain: 12 + 6 bytes per pixel."""
    c = tiny_cfg
    one = S.make_lf(7, 1, 1, 64, 64, 3, 0.0, "noise_gradient")[0, 0]
    lf = np.broadcast_to(one, (4, 4, 64, 64, 3)).copy()
    st = O.Stream(O.encode(lf, c.levels, c.block, c.search, 4).stream)
    v = _one(S.grid_view(0.0, 0.0, 0.0, 0.0, 64, 64))
    for k in (1, 2):
        assert abs(st.touched_bytes(v, level=k)[0] - 64 * 64 * 18) < 1e-6
    with pytest.raises(Exception):
        st.touched_bytes(v, level=3)


# --------------------------------------------------------------------------
# Sec. 4.5: chroma sub-sampling (4:2:0 stream mode)
# --------------------------------------------------------------------------

def _ycocg_planes(lf):
    """YCoCg-R of every sample, written out from its lifting definition
    (Co = R - B, t = B + floor(Co/2), Cg = G - t, Y = t + floor(Cg/2)):
    int64 [..., 3]."""
    r, g, b = (lf[..., k].astype(np.int64) for k in range(3))
    co = r - b
    t = b + np.floor_divide(co, 2)
    cg = g - t
    y = t + np.floor_divide(cg, 2)
    return np.stack([y, co, cg], -1)


def _subsampled(plane):
    """The 4:2:0 reading of a chroma plane [..., H, W]: each 2x2 pixel group
    (1-4 members at odd edges) reduced to floor((sum + floor(k/2)) / k), then
    replicated back to every pixel of the group (nearest-pixel
    reconstruction)."""
    H, W = plane.shape[-2:]
    Hc, Wc = (H + 1) // 2, (W + 1) // 2
    pad = np.zeros(plane.shape[:-2] + (2 * Hc, 2 * Wc), np.int64)
    cnt = np.zeros((2 * Hc, 2 * Wc), np.int64)
    pad[..., :H, :W] = plane
    cnt[:H, :W] = 1
    s = pad.reshape(plane.shape[:-2] + (Hc, 2, Wc, 2)).sum(axis=(-3, -1))
    k = cnt.reshape(Hc, 2, Wc, 2).sum(axis=(-3, -1))
    m = np.floor_divide(s + k // 2, k)
    return np.repeat(np.repeat(m, 2, axis=-2), 2, axis=-1)[..., :H, :W]


def _want_ycocg_420(lf):
    """[nu][nv][H][W][3]: Y of the input, Co and Cg of its 2x2 groups."""
    ycc = _ycocg_planes(lf)
    out = ycc.copy()
    for c in (1, 2):
        out[..., c] = _subsampled(ycc[..., c])
    return out


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL, O.MC_ZERO, O.MC_INTEGER])
def test_chroma_420_lossless_luma_and_filter_closed_form(tiny_lf, tiny_cfg, ragged_lf, mc):
    """At q = 1 with no thresholds the 4:2:0 stream decodes (full decode and
    random access) to exactly the input's Y and the rounded 2x2 means of its
    Co and Cg, replicated over each group -- odd sizes included."""
    c = tiny_cfg
    for lf, L, B in ((tiny_lf, c.levels, c.block), (ragged_lf, 3, 8)):
        st = O.Stream(O.encode(lf, L, B, c.search, 1, mc=mc, sub=1).stream)
        assert st.sub == 1
        want = _want_ycocg_420(lf)                               # [nu][nv][H][W][3]
        _, ycc = st.decode_all(with_ycocg=True)                  # [nu][nv][3][H][W]
        assert np.array_equal(np.moveaxis(ycc, 2, -1), want)
        nu, nv, H, W = lf.shape[:4]
        co = _all_coords(nu, nv, W, H)
        _, ra = st.decode_samples(co, with_ycocg=True)
        assert np.array_equal(ra, want[co[:, 0], co[:, 1], co[:, 3], co[:, 2]])


@pytest.mark.parametrize("q", [2, 4, 8])
def test_chroma_420_closed_loop_bound(tiny_lf, tiny_cfg, ragged_lf, q):
    """With q > 1 every decoded Y, Co, Cg stays within floor(q/2) of the
    4:2:0 reading of the input (the closed loop leaves only the leaf
    quantiser's error), and random access equals the full decode."""
    c = tiny_cfg
    for lf, L, B in ((tiny_lf, c.levels, c.block), (ragged_lf, 3, 8)):
        st = O.Stream(O.encode(lf, L, B, c.search, q, sub=1).stream)
        rgb, ycc = st.decode_all(with_ycocg=True)
        err = np.abs(np.moveaxis(ycc, 2, -1) - _want_ycocg_420(lf))
        assert err.max() <= q // 2
        nu, nv, H, W = lf.shape[:4]
        co = _all_coords(nu, nv, W, H)
        assert np.array_equal(st.decode_samples(co), rgb[co[:, 0], co[:, 1], co[:, 3], co[:, 2]])


def test_chroma_420_stream_layout(tiny_lf, tiny_cfg, ragged_lf):
    """Header flag bit 1 marks the mode; the root section holds, per root,
    H x W luma and two ceil(H/2) x ceil(W/2) chroma planes of int16; the MV
    sequence has one symbol per block of each predictive node-channel at its
    channel's block grid; and the 4:2:0 stream is the smaller one."""
    c = tiny_cfg
    for lf, L, B in ((tiny_lf, c.levels, c.block), (ragged_lf, 3, 8)):
        nu, nv, H, W = lf.shape[:4]
        d420 = O.encode(lf, L, B, c.search, 4, sub=1).stream
        d444 = O.encode(lf, L, B, c.search, 4).stream
        h = np.frombuffer(d420[:128], np.uint32)
        assert h[12] == 3                                        # MC on, chroma sub-sampled
        roots = ((nu + (1 << L) - 1) >> L) * ((nv + (1 << L) - 1) >> L)
        Hc, Wc = (H + 1) // 2, (W + 1) // 2
        root_bytes = roots * (H * W + 2 * Hc * Wc) * 2
        assert h[21] + root_bytes <= h[22] < h[21] + root_bytes + 16
        nb = lambda w, hh: ((w + B - 1) // B) * ((hh + B - 1) // B)
        n_pred = sum(((nu + (1 << l) - 1) >> l) * ((nv + (1 << l) - 1) >> l) -
                     (((nu + (1 << l) - 1) >> l) + 1) // 2 * ((((nv + (1 << l) - 1) >> l) + 1) // 2)
                     for l in range(L))
        assert h[19] == n_pred * (nb(W, H) + 2 * nb(Wc, Hc))
        assert len(d420) < len(d444)


def test_chroma_420_touched_bytes_closed_form(tiny_cfg):
    """The identical-views field of the 4:4:4 closed form, coded 4:2:0 and
    seen from camera (0, 0) with (s, t) on pixel centres: 12 B per output
    pixel + 2 B per luma root pixel (64 x 64) + 2 B per chroma root pixel
    (2 x 32 x 32) + for each of the 3 predictive level-0 nodes its luma
    (2 groups, 64 blocks) and two chroma node-channels (1 group, 16 blocks
    each): 16 B per group entry and the MV bits of every block."""
    c = tiny_cfg
    one = S.make_lf(7, 1, 1, 64, 64, 3, 0.0, "noise_gradient")[0, 0]
    lf = np.broadcast_to(one, (4, 4, 64, 64, 3)).copy()
    st = O.Stream(O.encode(lf, c.levels, c.block, c.search, 4, sub=1).stream)
    v = _one(S.grid_view(0.0, 0.0, 0.0, 0.0, 64, 64))
    mode, b = O.bise_choose(2 * (8 * c.search + 1) ** 2)
    mv_bits = O.bise_bits(mode, b, 15) / 15.0
    want = (64 * 64 * 12 + 64 * 64 * 2 + 2 * 32 * 32 * 2 + 3 * (2 + 1 + 1) * 16 +
            3 * (64 + 16 + 16) * mv_bits / 8.0)
    assert abs(st.touched_bytes(v)[0] - want) < 1e-6


def test_chroma_420_render_equals_dense_render(tiny_lf, tiny_cfg):
    """The random-access render of a 4:2:0 stream equals the FP64 dense
    render of its full decode (the render sees decoded RGB8 samples only)."""
    c = tiny_cfg
    st = O.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, 4, sub=1).stream)
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(17, geo, 3, [(40, 36)]))
    dense = O.render_dense(st.decode_all(), views)
    rng = np.random.default_rng(18)
    pix = np.stack([rng.integers(0, 3, 600), rng.integers(0, 40, 600), rng.integers(0, 36, 600)], -1).astype(np.int32)
    got = st.render_pixels(views, pix)
    idx = (views["out_offset"][pix[:, 0]] + (pix[:, 2] * 40 + pix[:, 1]) * 3)[:, None] + np.arange(3)[None, :]
    assert np.max(np.abs(got - dense[idx])) < 1e-12


# --------------------------------------------------------------------------
# the relaxation carrying the expected rounding of the integer decode
# --------------------------------------------------------------------------

def test_mc_rounding_bias_equals_brute_force():
    """floor((S + 8) / 16) - S / 16 averaged over every residue of four
    reference values (0..15 each) equals the oracle's predictor bias at every
    quarter-pel phase, for negative vectors too (Sec. 4.4 filter)."""
    a = np.stack(np.meshgrid(*[np.arange(16)] * 4, indexing="ij"), -1).reshape(-1, 4)
    for mvx in range(-5, 5):
        for mvy in range(-5, 5):
            fx, fy = mvx & 3, mvy & 3
            w = np.array([(4 - fx) * (4 - fy), fx * (4 - fy), (4 - fx) * fy, fx * fy])
            s = a @ w
            want = float(np.mean(np.floor((s + 8) / 16.0) - s / 16.0))
            assert O.mc_rounding_bias(mvx, mvy) == pytest.approx(want, abs=1e-12), (mvx, mvy)


def test_relax_bias_ycocg_closed_form(tiny_lf, tiny_cfg):
    """Without motion compensation the biased relaxation is the relaxation
    plus (1/2, 1/4, 1/2) levels in (R, G, B): each >> 1 of the YCoCg-R
    inverse averages v/2 - 1/4, t carries +1/4, B = t - Co/2 twice that."""
    c = tiny_cfg
    st = O.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, 4, mc=O.MC_OFF).stream)
    co, ro = st.dequant()
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(21, geo, 2, [(19, 13)]))
    d = (st.relax_render(co, ro, views, bias=True) - st.relax_render(co, ro, views)).reshape(-1, 3) * 255.0
    assert np.max(np.abs(d - np.array([0.5, 0.25, 0.5]))) < 1e-9


@pytest.mark.parametrize("mc", [O.MC_OFF, O.MC_QPEL])
def test_relax_bias_removes_the_mean_offset(tiny_lf, tiny_cfg, mc):
    """At the dequantised coefficients the integer render exceeds the plain
    relaxation by about (1/2, 1/4, 1/2) levels on average; the biased
    relaxation leaves no mean offset (within 0.05 level per channel)."""
    c = tiny_cfg
    st = O.Stream(O.encode(tiny_lf, c.levels, c.block, c.search, 4, mc=mc).stream)
    co, ro = st.dequant()
    geo = S.lf_geometry(c.nu, c.nv, c.width, c.height)
    views = S.views_to_array(S.random_views(3, geo, 6, [(64, 64)]))
    ri = O.render_dense(st.decode_all(), views)
    plain = ((ri - st.relax_render(co, ro, views)).reshape(-1, 3) * 255.0).mean(0)
    biased = ((ri - st.relax_render(co, ro, views, bias=True)).reshape(-1, 3) * 255.0).mean(0)
    assert np.all(np.abs(plain - np.array([0.5, 0.25, 0.5])) < 0.05), plain
    assert np.all(np.abs(biased) < 0.05), biased

