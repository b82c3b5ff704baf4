/*
 * hmlfc_oracle.c -- plain CPU oracle of HMLFC (Pratapa & Manocha, "HMLFC:
 * Hierarchical Motion-Compensated Light Field Compression for Interactive
 * Rendering", arXiv 1902.09396).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
 * object that the tests, the smoke check and the CPU baseline of the
 * benchmark load.  The product library never includes, links or calls it and
 * shares no code, header or table with it.
 *
 * It is written to be read against the paper, not to be fast: integer
 * arithmetic is done with explicit floor division, bit fields are read and
 * written one bit at a time, and every step follows the paper's order.
 *
 *   colour       Sec. 4.5   YCoCg-R lifting ("InvertibleYCoCg"), lossless
 *   hierarchy    Sec. 4.3   2x2 clusters in (u,v), RKV = rounded mean, SRV =
 *                           child - parent, recursively up to the tree height
 *   MC           Sec. 4.4   Eq. 1-2 and the two argmin displays: phase-shifted
 *                           block search (subtractive and additive residual),
 *                           then the replacement step; sub-pel (Sec. 6 future
 *                           work) as a quarter-pel integer bilinear refinement
 *   thresholds   Sec. 4.5   per-block energy (sum of |pixel|), two thresholds
 *   BISE         Sec. 4.6   values in [0, N-1], N in {2^b, 3*2^b, 5*2^b}
 *   stream       Sec. 4.7   breadth-first from the top of the tree
 *   decode       Sec. 4.8.1 roots + per-level SRV blocks + motion
 *                           re-compensation, random access per sample;
 *                           progressive decoding (Sec. 1, Sec. 4) stops the
 *                           sum at a level k: the level-k node's image
 *   render       Sec. 2.1, Sec. 5  two-plane (u,v,s,t) rays, quadrilinear
 *                           interpolation of the 16 neighbouring samples
 *
 * Readings where the paper is silent (cluster shape, reference choice,
 * closed-loop coding, tie-breaks, quantiser, block index, bit layout,
 * render geometry) are fixed identically in the stream format description
 * of the product header and in the design notes; each is repeated below
 * where it is used.
 *
 * Functions whose results are not pinned by an independent test say so.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAGIC 0x464C4D48u /* "HMLF" little-endian */
#define ORC_VERSION 1u
#define ORC_HEADER_WORDS 32

/* error codes */
#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_CORRUPT -2
#define ORC_E_OOM -3
#define ORC_E_RANGE -4

/* ------------------------------------------------------------------ */
/* integer helpers                                                     */
/* ------------------------------------------------------------------ */

/* floor(a / b) for b > 0, for any sign of a. */
static int64_t fdiv(int64_t a, int64_t b) {
    int64_t qt = a / b;
    if ((a % b) != 0 && (a < 0)) qt -= 1;
    return qt;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int iabs(int v) { return v < 0 ? -v : v; }

/* ------------------------------------------------------------------ */
/* Sec. 4.5: YCoCg-R (lifting form; the paper cites it as InvertibleYCoCg)   */
/* ------------------------------------------------------------------ */

void orc_rgb_to_ycocg(int r, int g, int b, int *y, int *co, int *cg) {
    int o = r - b;
    int t = b + (int)fdiv(o, 2);
    int gg = g - t;
    *co = o;
    *cg = gg;
    *y = t + (int)fdiv(gg, 2);
}

void orc_ycocg_to_rgb(int y, int co, int cg, int *r, int *g, int *b) {
    int t = y - (int)fdiv(cg, 2);
    int gg = cg + t;
    int bb = t - (int)fdiv(co, 2);
    *g = gg;
    *b = bb;
    *r = bb + co;
}

/* ------------------------------------------------------------------ */
/* quantiser (not in the paper; uniform step q, dead-zone free rounding) */
/* ------------------------------------------------------------------ */

int orc_quantise(int r, int q) {
    int a = iabs(r);
    int lv = (int)fdiv(a + q / 2, q);
    return r < 0 ? -lv : lv;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.4 + Sec. 6: quarter-pel motion-compensated predictor          */
/* mv in quarter pixels; taps clamped to the image; integer bilinear    */
/* weights that sum to 16, rounded half up.                            */
/* ------------------------------------------------------------------ */

int orc_pred_qpel(const int16_t *plane, int W, int H, int x, int y, int mvx, int mvy) {
    int X = 4 * x + mvx;
    int Y = 4 * y + mvy;
    int x0 = (int)fdiv(X, 4), y0 = (int)fdiv(Y, 4);
    int fx = X - 4 * x0, fy = Y - 4 * y0;
    int xa = clampi(x0, 0, W - 1), xb = clampi(x0 + 1, 0, W - 1);
    int ya = clampi(y0, 0, H - 1), yb = clampi(y0 + 1, 0, H - 1);
    int a = plane[ya * W + xa], b = plane[ya * W + xb];
    int c = plane[yb * W + xa], d = plane[yb * W + xb];
    int s = (4 - fx) * (4 - fy) * a + fx * (4 - fy) * b + (4 - fx) * fy * c + fx * fy * d;
    return (int)fdiv(s + 8, 16);
}

/* ------------------------------------------------------------------ */
/* Sec. 4.6: BISE.  A sequence of n values in [0, N-1].                 */
/*   mode 0: N = 2^b      b bits per value                              */
/*   mode 1: N = 3 * 2^b  groups of 5: an 8-bit trit byte               */
/*                        t0 + 3 t1 + 9 t2 + 27 t3 + 81 t4, then 5 x b  */
/*                        low bits; value = t * 2^b + low               */
/*   mode 2: N = 5 * 2^b  groups of 3: a 7-bit quint field              */
/*                        q0 + 5 q1 + 25 q2, then 3 x b low bits        */
/* The last group is padded with zero values.  Bits are numbered LSB    */
/* first within little-endian 32-bit words.                             */
/* ------------------------------------------------------------------ */

static void put_bits(uint32_t *buf, uint64_t pos, uint32_t val, int w) {
    for (int k = 0; k < w; k++) {
        if ((val >> k) & 1u) buf[(pos + k) >> 5] |= 1u << ((pos + k) & 31);
    }
}

static uint32_t get_bits(const uint32_t *buf, uint64_t pos, int w) {
    uint32_t v = 0;
    for (int k = 0; k < w; k++) {
        v |= ((buf[(pos + k) >> 5] >> ((pos + k) & 31)) & 1u) << k;
    }
    return v;
}

/* Smallest N in {2^b, 3*2^b, 5*2^b} that holds `range` distinct values. */
void orc_bise_choose(uint32_t range, int *mode, int *b) {
    int bp = 0, bt = 0, bq = 0;
    while ((1ull << bp) < range) bp++;
    while ((3ull << bt) < range) bt++;
    while ((5ull << bq) < range) bq++;
    uint64_t np = 1ull << bp, nt = 3ull << bt, nq = 5ull << bq;
    if (np <= nt && np <= nq) { *mode = 0; *b = bp; }
    else if (nt <= nq) { *mode = 1; *b = bt; }
    else { *mode = 2; *b = bq; }
}

uint64_t orc_bise_bits(int mode, int b, uint64_t n) {
    if (mode == 0) return n * (uint64_t)b;
    if (mode == 1) return ((n + 4) / 5) * (uint64_t)(8 + 5 * b);
    return ((n + 2) / 3) * (uint64_t)(7 + 3 * b);
}

/* Pack n values (each < N of the mode) into buf (zeroed by the caller). */
void orc_bise_pack(uint32_t *buf, int mode, int b, const uint32_t *v, uint64_t n) {
    if (mode == 0) {
        for (uint64_t i = 0; i < n; i++) put_bits(buf, i * (uint64_t)b, v[i], b);
        return;
    }
    int per = mode == 1 ? 5 : 3;
    int radix = mode == 1 ? 3 : 5;
    int hw = mode == 1 ? 8 : 7;
    uint64_t gbits = (uint64_t)hw + (uint64_t)per * b;
    uint64_t ng = (n + per - 1) / per;
    for (uint64_t g = 0; g < ng; g++) {
        uint32_t packed = 0, mul = 1;
        for (int r = 0; r < per; r++) {
            uint64_t i = g * per + r;
            uint32_t val = i < n ? v[i] : 0;
            packed += (val >> b) * mul;
            mul *= radix;
            put_bits(buf, g * gbits + hw + (uint64_t)r * b, val & ((1u << b) - 1u), b);
        }
        put_bits(buf, g * gbits, packed, hw);
    }
}

/* Random access to value i.  Returns -1 when the packed trit/quint field is
 * outside its alphabet (a corrupt stream). */
int64_t orc_bise_get(const uint32_t *buf, int mode, int b, uint64_t i) {
    if (mode == 0) return get_bits(buf, i * (uint64_t)b, b);
    int per = mode == 1 ? 5 : 3;
    int radix = mode == 1 ? 3 : 5;
    int hw = mode == 1 ? 8 : 7;
    uint32_t maxpacked = mode == 1 ? 242u : 124u;
    uint64_t gbits = (uint64_t)hw + (uint64_t)per * b;
    uint64_t g = i / per;
    int r = (int)(i % per);
    uint32_t packed = get_bits(buf, g * gbits, hw);
    if (packed > maxpacked) return -1;
    for (int k = 0; k < r; k++) packed /= radix;
    uint32_t hi = packed % radix;
    uint32_t lo = get_bits(buf, g * gbits + hw + (uint64_t)r * b, b);
    return ((int64_t)hi << b) + lo;
}

/* Sequential unpack of all n values (a second, independent reading path). */
int orc_bise_unpack(const uint32_t *buf, int mode, int b, uint32_t *v, uint64_t n) {
    if (mode == 0) {
        uint64_t pos = 0;
        for (uint64_t i = 0; i < n; i++) { v[i] = get_bits(buf, pos, b); pos += b; }
        return ORC_OK;
    }
    int per = mode == 1 ? 5 : 3;
    int radix = mode == 1 ? 3 : 5;
    int hw = mode == 1 ? 8 : 7;
    uint32_t maxpacked = mode == 1 ? 242u : 124u;
    uint64_t pos = 0;
    for (uint64_t first = 0; first < n; first += per) {
        uint32_t packed = get_bits(buf, pos, hw);
        pos += hw;
        if (packed > maxpacked) return ORC_E_CORRUPT;
        for (int r = 0; r < per; r++) {
            uint32_t lo = get_bits(buf, pos, b);
            pos += b;
            uint32_t hi = packed % radix;
            packed /= radix;
            if (first + r < n) v[first + r] = (hi << b) + lo;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tree geometry (Sec. 4.3 reading: 2x2 clusters of the node grid,     */
/* ceil(n / 2^l) nodes per axis at level l, level 0 = leaf SRVs, the   */
/* roots are the RKVs of level L)                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    int nu, nv, W, H, L, B, Ws, q, t_ref, t_pred, mc;
    int nbx, nby, nblocks, ngroups;
    int gu[33], gv[33];
    int64_t nc_base[33]; /* BFS index of the first node-channel of level l */
    int64_t n_nc;
    /* chroma sub-sampling (Sec. 4.5): sub = 1 codes Co and Cg at
     * ceil(W/2) x ceil(H/2); per channel c its plane size, block grid and
     * the offset of its plane within one node's planes (npx values) */
    int sub;
    int cW[3], cH[3], cnbx[3], cnby[3], cnb[3];
    size_t coff[3], npx;
} geom;

static int grid_n(int n, int l) { return (n + (1 << l) - 1) >> l; }

static int make_geom(geom *g, int nu, int nv, int W, int H, int L, int B, int sub) {
    if (nu < 1 || nv < 1 || W < 1 || H < 1 || L < 1 || L > 30 || B < 1 || B > 64) return ORC_E_ARG;
    if (sub != 0 && (sub != 1 || B % 2 != 0)) return ORC_E_ARG;
    memset(g, 0, sizeof(*g));
    g->nu = nu; g->nv = nv; g->W = W; g->H = H; g->L = L; g->B = B; g->sub = sub;
    g->nbx = (W + B - 1) / B;
    g->nby = (H + B - 1) / B;
    g->nblocks = g->nbx * g->nby;
    g->ngroups = (g->nblocks + 31) / 32;
    size_t off = 0;
    for (int c = 0; c < 3; c++) {
        g->cW[c] = (sub && c > 0) ? (W + 1) / 2 : W;
        g->cH[c] = (sub && c > 0) ? (H + 1) / 2 : H;
        g->cnbx[c] = (g->cW[c] + B - 1) / B;
        g->cnby[c] = (g->cH[c] + B - 1) / B;
        g->cnb[c] = g->cnbx[c] * g->cnby[c];
        g->coff[c] = off;
        off += (size_t)g->cW[c] * g->cH[c];
    }
    g->npx = off;
    for (int l = 0; l <= L; l++) { g->gu[l] = grid_n(nu, l); g->gv[l] = grid_n(nv, l); }
    /* breadth-first from the top: level L-1 first, nodes row-major (u major),
     * channels Y, Co, Cg innermost (Sec. 4.7) */
    int64_t acc = 0;
    for (int l = L - 1; l >= 0; l--) {
        g->nc_base[l] = acc;
        acc += 3ll * g->gu[l] * g->gv[l];
    }
    g->n_nc = acc;
    return ORC_OK;
}

static int64_t nc_of(const geom *g, int l, int a, int b, int c) {
    return g->nc_base[l] + ((int64_t)a * g->gv[l] + b) * 3 + c;
}

/* The geometry of channel c's planes: a copy of g with the plane size and
 * block grid of that channel (the other fields unchanged). */
static geom chan_geom(const geom *g, int c) {
    geom gc = *g;
    gc.W = g->cW[c]; gc.H = g->cH[c];
    gc.nbx = g->cnbx[c]; gc.nby = g->cnby[c]; gc.nblocks = g->cnb[c];
    return gc;
}

/* Channel of a node-channel (the channels are innermost in BFS order, and
 * every level's first node-channel index is a multiple of 3). */
static int chan_of(int64_t nc) { return (int)(nc % 3); }

/* Reference member of a sibling cluster: the node with both grid
 * coordinates even (the top-left member of its 2x2 cluster). */
static int is_ref(int a, int b) { return (a % 2 == 0) && (b % 2 == 0); }

static void block_rect(const geom *g, int k, int *x0, int *y0, int *bw, int *bh) {
    int bx = k % g->nbx, by = k / g->nbx;
    *x0 = bx * g->B;
    *y0 = by * g->B;
    *bw = (g->W - *x0) < g->B ? (g->W - *x0) : g->B;
    *bh = (g->H - *y0) < g->B ? (g->H - *y0) : g->B;
}

/* MV symbol: ((mvx + 4Ws) * (8Ws + 1) + (mvy + 4Ws)) * 2 + signbit, where
 * signbit = 1 for the additive (phase-inverted) prediction. */
static uint32_t mv_range(int Ws) { return 2u * (uint32_t)(8 * Ws + 1) * (uint32_t)(8 * Ws + 1); }

/* ------------------------------------------------------------------ */
/* encoder                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t nu, nv, W, H, L, B, Ws, q, t_ref, t_pred, mc, sub;
} orc_params;
/* sub: 1 = chroma sub-sampled 4:2:0 (Co, Cg at half resolution; B even). */
/* mc: 0 = no motion compensation (plain hierarchical residual coding),
 *     1 = phase-shifted search, integer then quarter-pel refinement,
 *     2 = zero motion (mv = 0, subtractive sign) for every block,
 *     3 = phase-shifted integer-pel search only (the paper's per-pel MC). */

typedef struct {
    uint8_t *sig;      /* [nblocks] */
    uint32_t *roff;    /* [nblocks] word offset of the record in `rec` */
    uint32_t *rec;     /* records */
    uint64_t nrec, caprec;
    uint32_t *mvsym;   /* [nblocks] or NULL */
} nc_out;

static int rec_append(nc_out *o, const uint32_t *w, uint64_t n) {
    if (o->nrec + n > o->caprec) {
        uint64_t cap = o->caprec ? o->caprec * 2 : 1024;
        while (cap < o->nrec + n) cap *= 2;
        uint32_t *p = (uint32_t *)realloc(o->rec, cap * sizeof(uint32_t));
        if (!p) return ORC_E_OOM;
        o->rec = p;
        o->caprec = cap;
    }
    memcpy(o->rec + o->nrec, w, n * sizeof(uint32_t));
    o->nrec += n;
    return ORC_OK;
}

/* Code one block of quantiser levels as a BISE record (Sec. 4.6):
 * header word = (uint16) min | b << 16 | mode << 21, then the payload. */
static int code_block(nc_out *o, int k, const int *lv, int n) {
    int m = lv[0], M = lv[0];
    for (int i = 1; i < n; i++) { if (lv[i] < m) m = lv[i]; if (lv[i] > M) M = lv[i]; }
    if (m < -32768 || M > 32767 || (int64_t)M - m + 1 > 65536) return ORC_E_RANGE;
    int mode, b;
    orc_bise_choose((uint32_t)(M - m + 1), &mode, &b);
    uint64_t bits = orc_bise_bits(mode, b, (uint64_t)n);
    uint64_t words = 1 + (bits + 31) / 32;
    uint32_t *w = (uint32_t *)calloc(words, sizeof(uint32_t));
    uint32_t *v = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!w || !v) { free(w); free(v); return ORC_E_OOM; }
    for (int i = 0; i < n; i++) v[i] = (uint32_t)(lv[i] - m);
    w[0] = ((uint32_t)(uint16_t)(int16_t)m) | ((uint32_t)b << 16) | ((uint32_t)mode << 21);
    orc_bise_pack(w + 1, mode, b, v, (uint64_t)n);
    o->sig[k] = 1;
    o->roff[k] = (uint32_t)o->nrec;
    int rc = rec_append(o, w, words);
    free(w);
    free(v);
    return rc;
}

/* Sum over the block of |S - sign * pred(mv)| (Eq. 1 for sign = +1, Eq. 2
 * for sign = -1). */
static int64_t block_cost(const int32_t *S, const int16_t *R, const geom *g, int k,
                          int mvx, int mvy, int sign) {
    int x0, y0, bw, bh;
    block_rect(g, k, &x0, &y0, &bw, &bh);
    int64_t acc = 0;
    for (int y = y0; y < y0 + bh; y++)
        for (int x = x0; x < x0 + bw; x++) {
            int p = orc_pred_qpel(R, g->W, g->H, x, y, mvx, mvy);
            acc += iabs(S[y * g->W + x] - sign * p);
        }
    return acc;
}

/* Phase-shifted search (Sec. 4.4).  For each sign, the integer stage
 * minimises over (x, y) in [-Ws, Ws]^2 with key (cost, |x|+|y|, raster
 * order of (y, x)); with mode 1 a quarter-pel refinement then looks at the
 * 7x7 quarter offsets around the integer winner (inside the symbol range)
 * with key (cost, fractional, |mvx|+|mvy|, raster order).  The smaller of
 * the two signs wins, the subtractive one on a tie. */
static void mc_search(const int32_t *S, const int16_t *R, const geom *g, int k, int Ws,
                      int refine, int *out_mvx, int *out_mvy, int *out_sign, int64_t *out_cost) {
    int64_t bestc[2];
    int bmx[2], bmy[2];
    for (int si = 0; si < 2; si++) {
        int sign = si == 0 ? 1 : -1;
        int64_t bc = -1;
        int bl1 = 0, bx = 0, by = 0;
        for (int dy = -Ws; dy <= Ws; dy++)
            for (int dx = -Ws; dx <= Ws; dx++) {
                int64_t c = block_cost(S, R, g, k, 4 * dx, 4 * dy, sign);
                int l1 = iabs(dx) + iabs(dy);
                if (bc < 0 || c < bc || (c == bc && l1 < bl1)) { bc = c; bl1 = l1; bx = 4 * dx; by = 4 * dy; }
            }
        if (refine) {
            int64_t rc = bc;
            int rfrac = 0, rl1 = iabs(bx) + iabs(by), rx = bx, ry = by;
            for (int oy = -3; oy <= 3; oy++)
                for (int ox = -3; ox <= 3; ox++) {
                    if (ox == 0 && oy == 0) continue;
                    int mx = bx + ox, my = by + oy;
                    if (iabs(mx) > 4 * Ws || iabs(my) > 4 * Ws) continue;
                    int64_t c = block_cost(S, R, g, k, mx, my, sign);
                    int l1 = iabs(mx) + iabs(my);
                    int better = 0;
                    if (c < rc) better = 1;
                    else if (c == rc) {
                        if (rfrac == 1 && l1 < rl1) better = 1; /* never displaces the integer winner */
                    }
                    if (better) { rc = c; rfrac = 1; rl1 = l1; rx = mx; ry = my; }
                }
            bc = rc; bx = rx; by = ry;
        }
        bestc[si] = bc; bmx[si] = bx; bmy[si] = by;
    }
    int pick = bestc[0] <= bestc[1] ? 0 : 1;
    *out_mvx = bmx[pick];
    *out_mvy = bmy[pick];
    *out_sign = pick == 0 ? 1 : -1;
    *out_cost = bestc[pick];
}

/* The search of one block k of an S plane against an R plane, exposed on its
 * own: out4 = (mvx, mvy, sign, cost). */
int orc_mc_search_block(const int32_t *S, const int16_t *R, int W, int H, int B, int k, int Ws, int refine,
                        int64_t *out4) {
    geom g;
    if (make_geom(&g, 1, 1, W, H, 1, B, 0) != ORC_OK || k < 0 || k >= g.nblocks || Ws < 0) return ORC_E_ARG;
    int mvx, mvy, sign;
    int64_t cost;
    mc_search(S, R, &g, k, Ws, refine, &mvx, &mvy, &sign, &cost);
    out4[0] = mvx; out4[1] = mvy; out4[2] = sign; out4[3] = cost;
    return ORC_OK;
}

/* Level images I_l (int16, [node][npx]: channel c's plane at coff[c]).
 * I_0 = YCoCg-R of the views (Sec. 4.5); with chroma sub-sampling, Co and Cg
 * are then reduced to ceil(W/2) x ceil(H/2) by the rounded mean of each 2x2
 * pixel group (1-4 members at odd edges) -- the reading fixed for "the
 * chroma channels are sub-sampled".  I_{l+1}(node) = floor((sum of the
 * cluster's members + floor(k/2)) / k), per pixel and channel (Sec. 4.3
 * reading: uniform pixel-wise filter). */
static int16_t *build_levels(const geom *g, const uint8_t *lf, int l_top, int16_t **lev) {
    size_t plane = (size_t)g->W * g->H, npx = g->npx;
    lev[0] = (int16_t *)malloc((size_t)g->nu * g->nv * npx * sizeof(int16_t));
    int16_t *full = (int16_t *)malloc(3 * plane * sizeof(int16_t));
    if (!lev[0] || !full) { free(full); return NULL; }
    for (int i = 0; i < g->nu; i++)
        for (int j = 0; j < g->nv; j++) {
            for (size_t p = 0; p < plane; p++) {
                const uint8_t *px = lf + (((size_t)i * g->nv + j) * plane + p) * 3;
                int y, co, cg;
                orc_rgb_to_ycocg(px[0], px[1], px[2], &y, &co, &cg);
                full[p] = (int16_t)y;
                full[plane + p] = (int16_t)co;
                full[2 * plane + p] = (int16_t)cg;
            }
            int16_t *dst = lev[0] + ((size_t)i * g->nv + j) * npx;
            for (int c = 0; c < 3; c++) {
                const int16_t *src = full + c * plane;
                int16_t *d = dst + g->coff[c];
                if (!(g->sub && c > 0)) { memcpy(d, src, plane * sizeof(int16_t)); continue; }
                for (int yc = 0; yc < g->cH[c]; yc++)
                    for (int xc = 0; xc < g->cW[c]; xc++) {
                        int64_t sum = 0;
                        int k = 0;
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++) {
                                int x = 2 * xc + dx, y = 2 * yc + dy;
                                if (x >= g->W || y >= g->H) continue;
                                sum += src[(size_t)y * g->W + x];
                                k++;
                            }
                        d[(size_t)yc * g->cW[c] + xc] = (int16_t)fdiv(sum + k / 2, k);
                    }
            }
        }
    free(full);
    for (int l = 0; l < l_top; l++) {
        int gu = g->gu[l], gv = g->gv[l], pu = g->gu[l + 1], pv = g->gv[l + 1];
        lev[l + 1] = (int16_t *)malloc((size_t)pu * pv * npx * sizeof(int16_t));
        if (!lev[l + 1]) return NULL;
        for (int A = 0; A < pu; A++)
            for (int Bn = 0; Bn < pv; Bn++)
                for (size_t p = 0; p < npx; p++) {
                    int64_t sum = 0;
                    int k = 0;
                    for (int da = 0; da < 2; da++)
                        for (int db = 0; db < 2; db++) {
                            int a = 2 * A + da, b = 2 * Bn + db;
                            if (a >= gu || b >= gv) continue;
                            sum += lev[l][((size_t)a * gv + b) * npx + p];
                            k++;
                        }
                    lev[l + 1][((size_t)A * pv + Bn) * npx + p] = (int16_t)fdiv(sum + k / 2, k);
                }
    }
    return lev[0];
}

/* Quantise-and-code one SRV node-channel whose per-pixel values to be coded
 * are `res` (the SRV itself for a reference, the MC residual for a
 * predictive node); writes the dequantised values to `deq`. */
static int code_plane_block(const geom *g, nc_out *o, int k, const int32_t *res, int thr,
                            int32_t *deq, int *lvbuf) {
    int x0, y0, bw, bh;
    block_rect(g, k, &x0, &y0, &bw, &bh);
    int64_t energy = 0;
    int any = 0, n = 0;
    for (int y = y0; y < y0 + bh; y++)
        for (int x = x0; x < x0 + bw; x++) {
            int r = res[y * g->W + x];
            energy += iabs(r);
            int lv = orc_quantise(r, g->q);
            lvbuf[n++] = lv;
            if (lv != 0) any = 1;
        }
    /* Sec. 4.5: a block whose energy is below the threshold is insignificant
     * and not stored; a block whose levels are all zero is not stored either. */
    int sig = any && energy >= thr;
    n = 0;
    for (int y = y0; y < y0 + bh; y++)
        for (int x = x0; x < x0 + bw; x++) {
            deq[y * g->W + x] = sig ? g->q * lvbuf[n] : 0;
            n++;
        }
    if (!sig) { o->sig[k] = 0; return ORC_OK; }
    return code_block(o, k, lvbuf, bw * bh);
}

/* Code one node-channel.  S is its SRV (child - reconstructed parent), R16
 * the dequantised SRV of its cluster's reference (predictive nodes only).
 * Writes the reconstructed SRV (prediction + dequantised residual) to shat. */
static int code_nc(const geom *g, nc_out *o, int ref, const int32_t *S, const int16_t *R16,
                   int32_t *res, int32_t *deq, int32_t *shat) {
    const int W = g->W, H = g->H;
    int use_mc = !ref && g->mc != 0;
    int *mvx = (int *)calloc((size_t)g->nblocks, sizeof(int));
    int *mvy = (int *)calloc((size_t)g->nblocks, sizeof(int));
    int *sgn = (int *)malloc((size_t)g->nblocks * sizeof(int));
    int *lvbuf = (int *)malloc((size_t)g->B * g->B * sizeof(int));
    int rc = ORC_OK;
    if (!mvx || !mvy || !sgn || !lvbuf) rc = ORC_E_OOM;
    if (rc == ORC_OK) {
        /* motion search, block by block (Sec. 4.4) */
        #pragma omp parallel for schedule(dynamic, 4)
        for (int k = 0; k < g->nblocks; k++) {
            sgn[k] = 1;
            if (use_mc && (g->mc == 1 || g->mc == 3)) {
                int64_t cost;
                mc_search(S, R16, g, k, g->Ws, g->mc == 1, &mvx[k], &mvy[k], &sgn[k], &cost);
            }
        }
        for (int k = 0; k < g->nblocks && rc == ORC_OK; k++) {
            int x0, y0, bw, bh;
            block_rect(g, k, &x0, &y0, &bw, &bh);
            /* replacement step: the block is replaced by its prediction residual */
            for (int y = y0; y < y0 + bh; y++)
                for (int x = x0; x < x0 + bw; x++) {
                    int pr = use_mc ? sgn[k] * orc_pred_qpel(R16, W, H, x, y, mvx[k], mvy[k]) : 0;
                    res[y * W + x] = S[y * W + x] - pr;
                }
            if (o->mvsym) {
                uint32_t sb = sgn[k] < 0 ? 1u : 0u;
                o->mvsym[k] = ((uint32_t)(mvx[k] + 4 * g->Ws) * (uint32_t)(8 * g->Ws + 1) +
                               (uint32_t)(mvy[k] + 4 * g->Ws)) * 2u + sb;
            }
            rc = code_plane_block(g, o, k, res, ref ? g->t_ref : g->t_pred, deq, lvbuf);
            for (int y = y0; y < y0 + bh; y++)
                for (int x = x0; x < x0 + bw; x++) {
                    int pr = use_mc ? sgn[k] * orc_pred_qpel(R16, W, H, x, y, mvx[k], mvy[k]) : 0;
                    shat[y * W + x] = pr + deq[y * W + x];
                }
        }
    }
    (void)H;
    free(mvx); free(mvy); free(sgn); free(lvbuf);
    return rc;
}

static void free_ncs(nc_out *o, int64_t n) {
    if (!o) return;
    for (int64_t i = 0; i < n; i++) { free(o[i].sig); free(o[i].roff); free(o[i].rec); free(o[i].mvsym); }
    free(o);
}

static void put_u32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }
static uint32_t rd_u32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }
static size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

/*
 * Encode a light field lf[nu][nv][H][W][3] (uint8).  On success *out holds a
 * malloc'd stream of *out_len bytes (free with orc_free).
 *
 * dbg_S / dbg_R (optional, [n_nc][H][W] int32 each): the SRV of every
 * node-channel before motion compensation, and the dequantised reference
 * SRV R^ of every reference node-channel (zero elsewhere).
 */
int orc_encode(const orc_params *P, const uint8_t *lf, uint8_t **out, size_t *out_len,
               int32_t *dbg_S, int32_t *dbg_R) {
    geom g;
    if (!P || !lf || !out || !out_len) return ORC_E_ARG;
    if (make_geom(&g, P->nu, P->nv, P->W, P->H, P->L, P->B, P->sub) != ORC_OK) return ORC_E_ARG;
    if (P->q < 1 || P->Ws < 0 || P->Ws > 64 || P->mc < 0 || P->mc > 3 || P->t_ref < 0 || P->t_pred < 0)
        return ORC_E_ARG;
    g.Ws = P->Ws; g.q = P->q; g.t_ref = P->t_ref; g.t_pred = P->t_pred; g.mc = P->mc;
    const int L = g.L, W = g.W, H = g.H;
    const size_t plane = (size_t)W * H, npx = g.npx;
    int rc = ORC_OK;

    int16_t *lev[33] = {0};
    int32_t *rec[33] = {0};
    nc_out *ncs = (nc_out *)calloc((size_t)g.n_nc, sizeof(nc_out));
    if (!ncs) return ORC_E_OOM;
    if (!build_levels(&g, lf, L, lev)) { rc = ORC_E_OOM; goto done; }

    /* roots: the level-L RKVs, stored losslessly (reconstruction = exact) */
    {
        size_t n = (size_t)g.gu[L] * g.gv[L] * npx;
        rec[L] = (int32_t *)malloc(n * sizeof(int32_t));
        if (!rec[L]) { rc = ORC_E_OOM; goto done; }
        for (size_t i = 0; i < n; i++) rec[L][i] = lev[L][i];
    }

    for (int l = L - 1; l >= 0 && rc == ORC_OK; l--) {
        const int gu = g.gu[l], gv = g.gv[l], pv = g.gv[l + 1];
        rec[l] = (int32_t *)malloc((size_t)gu * gv * npx * sizeof(int32_t));
        int32_t *Rhat = (int32_t *)calloc((size_t)gu * gv * npx, sizeof(int32_t));
        if (!rec[l] || !Rhat) { free(Rhat); rc = ORC_E_OOM; break; }
        /* references first: their dequantised SRVs predict the siblings */
        for (int pass = 0; pass < 2 && rc == ORC_OK; pass++) {
            for (int a = 0; a < gu && rc == ORC_OK; a++)
                for (int b = 0; b < gv && rc == ORC_OK; b++) {
                    int ref = is_ref(a, b);
                    if ((pass == 0) != ref) continue;
                    for (int c = 0; c < 3 && rc == ORC_OK; c++) {
                        /* every plane of channel c has that channel's size and block grid */
                        const geom gc = chan_geom(&g, c);
                        const size_t cpl = (size_t)gc.W * gc.H;
                        int64_t nc = nc_of(&g, l, a, b, c);
                        nc_out *o = &ncs[nc];
                        o->sig = (uint8_t *)calloc((size_t)gc.nblocks, 1);
                        o->roff = (uint32_t *)calloc((size_t)gc.nblocks, sizeof(uint32_t));
                        if (!ref && g.mc != 0) o->mvsym = (uint32_t *)calloc((size_t)gc.nblocks, sizeof(uint32_t));
                        int32_t *S = (int32_t *)malloc(cpl * sizeof(int32_t));
                        int32_t *res = (int32_t *)malloc(cpl * sizeof(int32_t));
                        int32_t *deq = (int32_t *)malloc(cpl * sizeof(int32_t));
                        int16_t *R16 = (int16_t *)malloc(cpl * sizeof(int16_t));
                        if (!o->sig || !o->roff || (!ref && g.mc != 0 && !o->mvsym) || !S || !res || !deq || !R16) {
                            free(S); free(res); free(deq); free(R16); rc = ORC_E_OOM; break;
                        }
                        /* SRV = child - reconstructed parent (closed loop) */
                        const int16_t *child = lev[l] + ((size_t)a * gv + b) * npx + g.coff[c];
                        const int32_t *par = rec[l + 1] + ((size_t)(a / 2) * pv + b / 2) * npx + g.coff[c];
                        for (size_t p = 0; p < cpl; p++) S[p] = (int32_t)child[p] - par[p];
                        if (dbg_S) {
                            int32_t *d = dbg_S + (size_t)nc * plane;       /* [n_nc][H][W], channel plane top-left */
                            memset(d, 0, plane * sizeof(int32_t));
                            for (int y = 0; y < gc.H; y++) memcpy(d + (size_t)y * W, S + (size_t)y * gc.W, gc.W * sizeof(int32_t));
                        }
                        const int32_t *Rref = NULL;
                        if (!ref) {
                            Rref = Rhat + ((size_t)(a & ~1) * gv + (b & ~1)) * npx + g.coff[c];
                            for (size_t p = 0; p < cpl; p++) R16[p] = (int16_t)Rref[p];
                        }
                        int32_t *shat = rec[l] + ((size_t)a * gv + b) * npx + g.coff[c];
                        int brc = code_nc(&gc, o, ref, S, R16, res, deq, shat);
                        if (dbg_R) {
                            int32_t *d = dbg_R + (size_t)nc * plane;
                            memset(d, 0, plane * sizeof(int32_t));
                            if (ref)
                                for (int y = 0; y < gc.H; y++)
                                    memcpy(d + (size_t)y * W, shat + (size_t)y * gc.W, gc.W * sizeof(int32_t));
                        }
                        if (ref) memcpy(Rhat + ((size_t)a * gv + b) * npx + g.coff[c], shat, cpl * sizeof(int32_t));
                        /* reconstruction of this node: parent + reconstructed SRV */
                        for (size_t p = 0; p < cpl; p++) {
                            int64_t v = (int64_t)par[p] + shat[p];
                            if (v < -32768 || v > 32767) brc = ORC_E_RANGE;
                            shat[p] = (int32_t)v;
                        }
                        free(S); free(res); free(deq); free(R16);
                        rc = brc;
                    }
                }
        }
        free(Rhat);
        free(rec[l + 1]);
        rec[l + 1] = NULL;
    }
    if (rc != ORC_OK) goto done;

    /* ---- Sec. 4.7: serialise breadth-first ---- */
    {
        uint64_t nsig = 0, nrecw = 0, nmv = 0;
        for (int64_t nc = 0; nc < g.n_nc; nc++) {
            const int nb = g.cnb[chan_of(nc)];
            for (int k = 0; k < nb; k++) nsig += ncs[nc].sig[k];
            nrecw += ncs[nc].nrec;
            if (ncs[nc].mvsym) nmv += (uint64_t)nb;          /* one symbol per block of a predictive node-channel */
        }
        int mv_mode = 0, mv_b = 0;
        if (g.mc != 0) orc_bise_choose(mv_range(g.Ws), &mv_mode, &mv_b);
        uint64_t nmvw = g.mc != 0 ? (orc_bise_bits(mv_mode, mv_b, nmv) + 31) / 32 : 0;
        size_t nroot = (size_t)g.gu[L] * g.gv[L];
        size_t off_roots = ORC_HEADER_WORDS * 4;
        size_t off_groups = align16(off_roots + nroot * npx * 2);
        size_t off_offs = align16(off_groups + (size_t)g.n_nc * g.ngroups * 16);
        size_t off_recs = align16(off_offs + nsig * 2);
        size_t off_mvs = align16(off_recs + nrecw * 4);
        size_t total = align16(off_mvs + nmvw * 4);
        if (total > 0xFFFFFFF0ull || nrecw > 0xFFFFFFF0ull) { rc = ORC_E_RANGE; goto done; }
        uint8_t *s = (uint8_t *)calloc(total, 1);
        if (!s) { rc = ORC_E_OOM; goto done; }
        uint32_t hdr[ORC_HEADER_WORDS] = {0};
        hdr[0] = ORC_MAGIC; hdr[1] = ORC_VERSION;
        hdr[2] = (uint32_t)g.nu; hdr[3] = (uint32_t)g.nv; hdr[4] = (uint32_t)W; hdr[5] = (uint32_t)H;
        hdr[6] = (uint32_t)L; hdr[7] = (uint32_t)g.B; hdr[8] = (uint32_t)g.Ws; hdr[9] = (uint32_t)g.q;
        hdr[10] = (uint32_t)g.t_ref; hdr[11] = (uint32_t)g.t_pred;
        hdr[12] = (g.mc != 0 ? 1u : 0u) | (g.sub ? 2u : 0u);
        hdr[13] = (uint32_t)mv_mode; hdr[14] = (uint32_t)mv_b;
        hdr[15] = (uint32_t)g.n_nc; hdr[16] = (uint32_t)g.ngroups; hdr[17] = (uint32_t)nsig;
        hdr[18] = (uint32_t)nrecw; hdr[19] = (uint32_t)nmv; hdr[20] = (uint32_t)nmvw;
        hdr[21] = (uint32_t)off_roots; hdr[22] = (uint32_t)off_groups; hdr[23] = (uint32_t)off_offs;
        hdr[24] = (uint32_t)off_recs; hdr[25] = (uint32_t)off_mvs; hdr[26] = (uint32_t)total;
        for (int i = 0; i < ORC_HEADER_WORDS; i++) put_u32(s + 4 * i, hdr[i]);
        /* roots: int16, per root its Y, Co, Cg planes at their channel sizes */
        for (size_t i = 0; i < nroot * npx; i++) {
            int16_t v = lev[L][i];
            memcpy(s + off_roots + 2 * i, &v, 2);
        }
        /* groups of 32 blocks: {bitmap, record word base, offset base, 0};
         * per significant block a u16 word offset from the group's base */
        uint64_t sig_cursor = 0, rec_cursor = 0;
        uint32_t *mvbuf = nmvw ? (uint32_t *)calloc(nmvw, sizeof(uint32_t)) : NULL;
        uint32_t *mvvals = nmv ? (uint32_t *)malloc(nmv * sizeof(uint32_t)) : NULL;
        if ((nmvw && !mvbuf) || (nmv && !mvvals)) { free(s); free(mvbuf); free(mvvals); rc = ORC_E_OOM; goto done; }
        uint64_t mv_cursor = 0;
        for (int64_t nc = 0; nc < g.n_nc; nc++) {
            nc_out *o = &ncs[nc];
            const geom gc = chan_geom(&g, chan_of(nc));
            /* ngroups groups per node-channel (the luma block count); a chroma
             * node-channel with fewer blocks leaves its last groups empty */
            for (int gi = 0; gi < g.ngroups; gi++) {
                uint32_t bitmap = 0;
                uint64_t gbase = rec_cursor, obase = sig_cursor;
                for (int r = 0; r < 32; r++) {
                    int k = gi * 32 + r;
                    if (k >= gc.nblocks || !o->sig[k]) continue;
                    bitmap |= 1u << r;
                    /* record length from its header */
                    uint32_t h0 = o->rec[o->roff[k]];
                    int md = (int)((h0 >> 21) & 3u), bb = (int)((h0 >> 16) & 31u);
                    int x0, y0, bw, bh;
                    block_rect(&gc, k, &x0, &y0, &bw, &bh);
                    uint64_t len = 1 + (orc_bise_bits(md, bb, (uint64_t)bw * bh) + 31) / 32;
                    uint64_t rel = rec_cursor - gbase;
                    if (rel > 0xFFFFu) { free(s); free(mvbuf); free(mvvals); rc = ORC_E_RANGE; goto done; }
                    uint16_t r16 = (uint16_t)rel;
                    memcpy(s + off_offs + 2 * sig_cursor, &r16, 2);
                    memcpy(s + off_recs + 4 * rec_cursor, o->rec + o->roff[k], len * 4);
                    rec_cursor += len;
                    sig_cursor++;
                }
                uint8_t *ge = s + off_groups + ((size_t)nc * g.ngroups + gi) * 16;
                put_u32(ge, bitmap);
                put_u32(ge + 4, (uint32_t)gbase);
                put_u32(ge + 8, (uint32_t)obase);
                put_u32(ge + 12, 0);
            }
            if (o->mvsym)
                for (int k = 0; k < gc.nblocks; k++) mvvals[mv_cursor++] = o->mvsym[k];
        }
        if (nmv) {
            orc_bise_pack(mvbuf, mv_mode, mv_b, mvvals, nmv);
            memcpy(s + off_mvs, mvbuf, nmvw * 4);
        }
        free(mvbuf);
        free(mvvals);
        *out = s;
        *out_len = total;
    }

done:
    for (int l = 0; l <= L; l++) { free(lev[l]); free(rec[l]); }
    free_ncs(ncs, g.n_nc);
    return rc;
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* stream parsing                                                       */
/* ------------------------------------------------------------------ */

typedef struct {
    geom g;
    int mcflag, mv_mode, mv_b;
    uint32_t n_sig, n_recw, n_mv, n_mvw;
    uint8_t *bytes;
    size_t nbytes;
    const int16_t *roots;
    const uint32_t *groups;
    const uint16_t *offs;
    const uint32_t *recs;
    const uint32_t *mvs;
    int64_t *mv_base; /* [n_nc]: index of the node-channel's first MV symbol, -1 for a reference */
} orc_stream;

void orc_close(orc_stream *s) {
    if (!s) return;
    free(s->bytes);
    free(s->mv_base);
    free(s);
}

int orc_open(const uint8_t *bytes, size_t n, orc_stream **out) {
    if (!bytes || !out || n < ORC_HEADER_WORDS * 4) return ORC_E_CORRUPT;
    uint32_t h[ORC_HEADER_WORDS];
    for (int i = 0; i < ORC_HEADER_WORDS; i++) h[i] = rd_u32(bytes + 4 * i);
    if (h[0] != ORC_MAGIC || h[1] != ORC_VERSION) return ORC_E_CORRUPT;
    orc_stream *s = (orc_stream *)calloc(1, sizeof(orc_stream));
    if (!s) return ORC_E_OOM;
    if (h[2] > 65536 || h[3] > 65536 || h[4] > 65536 || h[5] > 65536 || h[6] > 30 || h[7] > 64 || (h[12] & ~3u) ||
        make_geom(&s->g, (int)h[2], (int)h[3], (int)h[4], (int)h[5], (int)h[6], (int)h[7], (int)((h[12] >> 1) & 1u)) !=
            ORC_OK) {
        free(s); return ORC_E_CORRUPT;
    }
    s->g.Ws = (int)h[8]; s->g.q = (int)h[9]; s->g.t_ref = (int)h[10]; s->g.t_pred = (int)h[11];
    s->mcflag = (int)(h[12] & 1u);
    s->mv_mode = (int)h[13]; s->mv_b = (int)h[14];
    s->n_sig = h[17]; s->n_recw = h[18]; s->n_mv = h[19]; s->n_mvw = h[20];
    const geom *g = &s->g;
    size_t nroot = (size_t)g->gu[g->L] * g->gv[g->L];
    int bad = 0;
    if (s->g.q < 1 || h[8] > 64 || h[15] != (uint32_t)g->n_nc || h[16] != (uint32_t)g->ngroups) bad = 1;
    if (h[26] != n) bad = 1;
    if (h[21] + nroot * g->npx * 2 > n) bad = 1;
    if (h[22] + (uint64_t)g->n_nc * g->ngroups * 16 > n) bad = 1;
    if (h[23] + (uint64_t)s->n_sig * 2 > n || h[24] + (uint64_t)s->n_recw * 4 > n ||
        h[25] + (uint64_t)s->n_mvw * 4 > n) bad = 1;
    if ((h[21] | h[22] | h[23] | h[24] | h[25]) & 3u) bad = 1;
    if (bad) { free(s); return ORC_E_CORRUPT; }
    s->bytes = (uint8_t *)malloc(n);
    s->mv_base = (int64_t *)malloc((size_t)g->n_nc * sizeof(int64_t));
    if (!s->bytes || !s->mv_base) { orc_close(s); return ORC_E_OOM; }
    memcpy(s->bytes, bytes, n);
    s->nbytes = n;
    s->roots = (const int16_t *)(s->bytes + h[21]);
    s->groups = (const uint32_t *)(s->bytes + h[22]);
    s->offs = (const uint16_t *)(s->bytes + h[23]);
    s->recs = (const uint32_t *)(s->bytes + h[24]);
    s->mvs = (const uint32_t *)(s->bytes + h[25]);
    int64_t nsym = 0;          /* MV symbols before this node-channel: one per block of each predictive one */
    for (int l = g->L - 1; l >= 0; l--)
        for (int a = 0; a < g->gu[l]; a++)
            for (int b = 0; b < g->gv[l]; b++)
                for (int c = 0; c < 3; c++) {
                    int64_t nc = nc_of(g, l, a, b, c);
                    s->mv_base[nc] = is_ref(a, b) ? -1 : nsym;
                    if (!is_ref(a, b)) nsym += g->cnb[c];
                }
    if (s->mcflag) {
        int md, bb;
        orc_bise_choose(mv_range(g->Ws), &md, &bb);
        if (md != s->mv_mode || bb != s->mv_b || (uint64_t)s->n_mv != (uint64_t)nsym ||
            (orc_bise_bits(md, bb, s->n_mv) + 31) / 32 != s->n_mvw) { orc_close(s); return ORC_E_CORRUPT; }
    } else if (s->n_mv != 0) { orc_close(s); return ORC_E_CORRUPT; }
    *out = s;
    return ORC_OK;
}

int orc_stream_info(const orc_stream *s, int32_t *info /* [17] */) {
    const geom *g = &s->g;
    info[0] = g->nu; info[1] = g->nv; info[2] = g->W; info[3] = g->H; info[4] = g->L;
    info[5] = g->B; info[6] = g->Ws; info[7] = g->q; info[8] = s->mcflag;
    info[9] = (int32_t)g->n_nc; info[10] = g->nblocks; info[11] = (int32_t)s->n_sig;
    info[12] = (int32_t)s->n_recw; info[13] = (int32_t)s->n_mv; info[14] = g->gu[g->L] * g->gv[g->L];
    info[15] = (int32_t)s->nbytes; info[16] = g->sub;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.8.1: random-access decoding of one sample                    */
/* ------------------------------------------------------------------ */

/* Locate block k of node-channel nc: returns the record pointer or NULL for
 * an insignificant block. */
static const uint32_t *find_record(const orc_stream *s, int64_t nc, int k) {
    const uint32_t *ge = s->groups + ((size_t)nc * s->g.ngroups + k / 32) * 4;
    uint32_t bitmap = ge[0];
    int r = k % 32;
    if (!((bitmap >> r) & 1u)) return NULL;
    int rank = 0;
    for (int t = 0; t < r; t++) rank += (bitmap >> t) & 1u;
    uint16_t off = s->offs[ge[2] + rank];
    return s->recs + ge[1] + off;
}

/* Dequantised coefficient q * level of pixel (x, y) of node-channel nc, in
 * the coordinates and block grid of its channel's plane. */
static int coef_at(const orc_stream *s, int64_t nc, int x, int y) {
    const geom gc = chan_geom(&s->g, chan_of(nc));
    const geom *g = &gc;
    int bx = x / g->B, by = y / g->B;
    int k = by * g->nbx + bx;
    const uint32_t *rec = find_record(s, nc, k);
    if (!rec) return 0;
    int x0, y0, bw, bh;
    block_rect(g, k, &x0, &y0, &bw, &bh);
    uint32_t hdr = rec[0];
    int m = (int16_t)(hdr & 0xFFFFu);
    int b = (int)((hdr >> 16) & 31u);
    int mode = (int)((hdr >> 21) & 3u);
    int64_t v = orc_bise_get(rec + 1, mode, b, (uint64_t)(y - y0) * bw + (uint64_t)(x - x0));
    return g->q * (m + (int)v);
}

static void mv_of(const orc_stream *s, int64_t nc, int k, int *mvx, int *mvy, int *sign) {
    const geom *g = &s->g;
    uint64_t idx = (uint64_t)s->mv_base[nc] + k;
    uint32_t sym = (uint32_t)orc_bise_get(s->mvs, s->mv_mode, s->mv_b, idx);
    uint32_t side = (uint32_t)(8 * g->Ws + 1);
    *sign = (sym & 1u) ? -1 : 1;
    *mvx = (int)((sym / 2u) / side) - 4 * g->Ws;
    *mvy = (int)((sym / 2u) % side) - 4 * g->Ws;
}

/* Reconstructed SRV value of node (a, b) at level l, channel c, at (x, y) of
 * that channel's plane. */
static int srv_at(const orc_stream *s, int l, int a, int b, int c, int x, int y) {
    const geom gc = chan_geom(&s->g, c);
    const geom *g = &gc;
    int64_t nc = nc_of(g, l, a, b, c);
    int r = coef_at(s, nc, x, y);
    if (is_ref(a, b) || !s->mcflag) return r;
    int k = (y / g->B) * g->nbx + x / g->B;
    int mvx, mvy, sign;
    mv_of(s, nc, k, &mvx, &mvy, &sign);
    int64_t rnc = nc_of(g, l, a & ~1, b & ~1, c);
    /* motion re-compensation from the resident reference SRV */
    int X = 4 * x + mvx, Y = 4 * y + mvy;
    int x0 = (int)fdiv(X, 4), y0 = (int)fdiv(Y, 4);
    int fx = X - 4 * x0, fy = Y - 4 * y0;
    int xa = clampi(x0, 0, g->W - 1), xb = clampi(x0 + 1, 0, g->W - 1);
    int ya = clampi(y0, 0, g->H - 1), yb = clampi(y0 + 1, 0, g->H - 1);
    int ta = coef_at(s, rnc, xa, ya), tb = coef_at(s, rnc, xb, ya);
    int tc = coef_at(s, rnc, xa, yb), td = coef_at(s, rnc, xb, yb);
    int sum = (4 - fx) * (4 - fy) * ta + fx * (4 - fy) * tb + (4 - fx) * fy * tc + fx * fy * td;
    int pred = (int)fdiv(sum + 8, 16);
    return sign * pred + r;
}

/* YCoCg value of LF sample (i, j, x, y): root + sum over levels (Sec. 4.8.1).
 * Progressive decoding (Sec. 1, Sec. 4: the upper levels carry what the views
 * share, the lower ones their detail) stops the sum at level lod: the value is
 * then the reconstruction of the level-lod node (i >> lod, j >> lod). */
/* With chroma sub-sampling, Co and Cg of sample (x, y) are those of chroma
 * pixel (x >> 1, y >> 1): nearest-pixel reconstruction (the reading fixed
 * for Sec. 4.5's sub-sampled chroma). */
static void sample_ycocg(const orc_stream *s, int i, int j, int x, int y, int lod, int v[3]) {
    const geom *g = &s->g;
    int L = g->L;
    int ra = i >> L, rb = j >> L;
    int cx[3], cy[3];
    for (int c = 0; c < 3; c++) {
        cx[c] = (g->sub && c > 0) ? x >> 1 : x;
        cy[c] = (g->sub && c > 0) ? y >> 1 : y;
        v[c] = s->roots[((size_t)ra * g->gv[L] + rb) * g->npx + g->coff[c] + (size_t)cy[c] * g->cW[c] + cx[c]];
    }
    for (int l = lod; l < L; l++)
        for (int c = 0; c < 3; c++) v[c] += srv_at(s, l, i >> l, j >> l, c, cx[c], cy[c]);
}

static void sample_rgb(const orc_stream *s, int i, int j, int x, int y, int lod, int rgb[3]) {
    int v[3], r, g, b;
    sample_ycocg(s, i, j, x, y, lod, v);
    orc_ycocg_to_rgb(v[0], v[1], v[2], &r, &g, &b);
    rgb[0] = clampi(r, 0, 255);
    rgb[1] = clampi(g, 0, 255);
    rgb[2] = clampi(b, 0, 255);
}

/* coords [n][4] = (i, j, x, y); rgb [n][3]; ycocg [n][3] (optional); decoded
 * down to level lod (0 = full decode, L = roots only). */
int orc_decode_samples_lod(const orc_stream *s, const int32_t *coords, int64_t n, int lod, uint8_t *rgb,
                           int32_t *ycocg) {
    const geom *g = &s->g;
    if (lod < 0 || lod > g->L) return ORC_E_ARG;
    for (int64_t k = 0; k < n; k++) {
        const int32_t *c = coords + 4 * k;
        if (c[0] < 0 || c[0] >= g->nu || c[1] < 0 || c[1] >= g->nv || c[2] < 0 || c[2] >= g->W || c[3] < 0 ||
            c[3] >= g->H) return ORC_E_ARG;
    }
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < n; k++) {
        const int32_t *c = coords + 4 * k;
        int v[3], o[3];
        sample_ycocg(s, c[0], c[1], c[2], c[3], lod, v);
        if (ycocg) { ycocg[3 * k] = v[0]; ycocg[3 * k + 1] = v[1]; ycocg[3 * k + 2] = v[2]; }
        int r, gg, b;
        orc_ycocg_to_rgb(v[0], v[1], v[2], &r, &gg, &b);
        o[0] = clampi(r, 0, 255); o[1] = clampi(gg, 0, 255); o[2] = clampi(b, 0, 255);
        for (int t = 0; t < 3; t++) rgb[3 * k + t] = (uint8_t)o[t];
    }
    return ORC_OK;
}

int orc_decode_samples(const orc_stream *s, const int32_t *coords, int64_t n, uint8_t *rgb, int32_t *ycocg) {
    return orc_decode_samples_lod(s, coords, n, 0, rgb, ycocg);
}

/* ------------------------------------------------------------------ */
/* full decoding: top-down reconstruction of every level image, cluster */
/* by cluster, with a sequential BISE reader (an independent path)     */
/* ------------------------------------------------------------------ */

/* Decode all dequantised coefficients of node-channel nc into plane[H][W]
 * (its channel's plane size). */
static int decode_plane_seq(const orc_stream *s, int64_t nc, int32_t *plane) {
    const geom gc = chan_geom(&s->g, chan_of(nc));
    const geom *g = &gc;
    uint32_t vals[64 * 64];
    for (int k = 0; k < g->nblocks; k++) {
        int x0, y0, bw, bh;
        block_rect(g, k, &x0, &y0, &bw, &bh);
        const uint32_t *ge = s->groups + ((size_t)nc * g->ngroups + k / 32) * 4;
        int sig = (ge[0] >> (k % 32)) & 1u;
        if (!sig) {
            for (int y = y0; y < y0 + bh; y++)
                for (int x = x0; x < x0 + bw; x++) plane[y * g->W + x] = 0;
            continue;
        }
        const uint32_t *rec = find_record(s, nc, k);
        uint32_t hdr = rec[0];
        int m = (int16_t)(hdr & 0xFFFFu);
        int b = (int)((hdr >> 16) & 31u);
        int mode = (int)((hdr >> 21) & 3u);
        if (mode == 3 || b > 16) return ORC_E_CORRUPT;
        if (orc_bise_unpack(rec + 1, mode, b, vals, (uint64_t)bw * bh) != ORC_OK) return ORC_E_CORRUPT;
        int n = 0;
        for (int y = y0; y < y0 + bh; y++)
            for (int x = x0; x < x0 + bw; x++) plane[y * g->W + x] = g->q * (m + (int)vals[n++]);
    }
    return ORC_OK;
}

/* out: uint8 [nu][nv][H][W][3]; if ycocg != NULL also int32 [nu][nv][3][H][W]
 * (with chroma sub-sampling, Co and Cg at (x, y) are those of chroma pixel
 * (x >> 1, y >> 1)). */
int orc_decode_all(const orc_stream *s, uint8_t *out, int32_t *ycocg) {
    const geom *g = &s->g;
    const int L = g->L, W = g->W;
    const size_t plane = (size_t)W * g->H, npx = g->npx;
    int rc = ORC_OK;
    /* level reconstructions, [node][npx] (channel c's plane at coff[c]) */
    int32_t *cur = (int32_t *)malloc((size_t)g->gu[L] * g->gv[L] * npx * sizeof(int32_t));
    if (!cur) return ORC_E_OOM;
    for (size_t i = 0; i < (size_t)g->gu[L] * g->gv[L] * npx; i++) cur[i] = s->roots[i];
    for (int l = L - 1; l >= 0 && rc == ORC_OK; l--) {
        int gu = g->gu[l], gv = g->gv[l], pu = g->gu[l + 1], pv = g->gv[l + 1];
        int32_t *nxt = (int32_t *)malloc((size_t)gu * gv * npx * sizeof(int32_t));
        if (!nxt) { rc = ORC_E_OOM; break; }
        #pragma omp parallel for collapse(2) schedule(dynamic, 1)
        for (int A = 0; A < pu; A++)
            for (int Bn = 0; Bn < pv; Bn++) {
                int32_t *refp = (int32_t *)malloc(plane * sizeof(int32_t));
                int32_t *srv = (int32_t *)malloc(plane * sizeof(int32_t));
                int16_t *ref16 = (int16_t *)malloc(plane * sizeof(int16_t));
                if (!refp || !srv || !ref16) { free(refp); free(srv); free(ref16); rc = ORC_E_OOM; continue; }
                for (int c = 0; c < 3; c++) {
                    const geom gc = chan_geom(g, c);
                    const size_t cpl = (size_t)gc.W * gc.H;
                    const int32_t *par = cur + ((size_t)A * pv + Bn) * npx + g->coff[c];
                    /* the cluster's reference member first */
                    int ra = 2 * A, rb = 2 * Bn;
                    if (decode_plane_seq(s, nc_of(g, l, ra, rb, c), refp) != ORC_OK) rc = ORC_E_CORRUPT;
                    for (size_t p = 0; p < cpl; p++) ref16[p] = (int16_t)refp[p];
                    for (int da = 0; da < 2; da++)
                        for (int db = 0; db < 2; db++) {
                            int a = 2 * A + da, b = 2 * Bn + db;
                            if (a >= gu || b >= gv) continue;
                            int64_t nc = nc_of(g, l, a, b, c);
                            if (da == 0 && db == 0) {
                                memcpy(srv, refp, cpl * sizeof(int32_t));
                            } else {
                                if (decode_plane_seq(s, nc, srv) != ORC_OK) rc = ORC_E_CORRUPT;
                                if (s->mcflag) {
                                    for (int k = 0; k < gc.nblocks; k++) {
                                        int mvx, mvy, sign, x0, y0, bw, bh;
                                        mv_of(s, nc, k, &mvx, &mvy, &sign);
                                        block_rect(&gc, k, &x0, &y0, &bw, &bh);
                                        for (int y = y0; y < y0 + bh; y++)
                                            for (int x = x0; x < x0 + bw; x++)
                                                srv[y * gc.W + x] += sign * orc_pred_qpel(ref16, gc.W, gc.H, x, y, mvx, mvy);
                                    }
                                }
                            }
                            int32_t *dst = nxt + ((size_t)a * gv + b) * npx + g->coff[c];
                            for (size_t p = 0; p < cpl; p++) dst[p] = par[p] + srv[p];
                        }
                }
                free(refp); free(srv); free(ref16);
            }
        free(cur);
        cur = nxt;
    }
    if (rc == ORC_OK) {
        for (int i = 0; i < g->nu; i++)
            for (int j = 0; j < g->nv; j++) {
                const int32_t *src = cur + ((size_t)i * g->nv + j) * npx;
                for (int y = 0; y < g->H; y++)
                    for (int x = 0; x < W; x++) {
                        int v[3];
                        for (int c = 0; c < 3; c++) {
                            int xc = (g->sub && c > 0) ? x >> 1 : x, yc = (g->sub && c > 0) ? y >> 1 : y;
                            v[c] = src[g->coff[c] + (size_t)yc * g->cW[c] + xc];
                        }
                        size_t p = (size_t)y * W + x;
                        if (ycocg)
                            for (int c = 0; c < 3; c++) ycocg[(((size_t)i * g->nv + j) * 3 + c) * plane + p] = v[c];
                        int r, gg, b;
                        orc_ycocg_to_rgb(v[0], v[1], v[2], &r, &gg, &b);
                        uint8_t *o = out + (((size_t)i * g->nv + j) * plane + p) * 3;
                        o[0] = (uint8_t)clampi(r, 0, 255);
                        o[1] = (uint8_t)clampi(gg, 0, 255);
                        o[2] = (uint8_t)clampi(b, 0, 255);
                    }
            }
    }
    free(cur);
    return rc;
}

/* Per block of node-channel nc: significance, mv and sign (mv/sign are 0/+1
 * for references or streams without motion compensation). */
int orc_block_info(const orc_stream *s, int64_t nc, int k, int32_t *out4) {
    const geom *g = &s->g;
    if (nc < 0 || nc >= g->n_nc || k < 0 || k >= g->cnb[chan_of(nc)]) return ORC_E_ARG;
    const uint32_t *ge = s->groups + ((size_t)nc * g->ngroups + k / 32) * 4;
    out4[0] = (ge[0] >> (k % 32)) & 1u;
    out4[1] = 0; out4[2] = 0; out4[3] = 1;
    if (s->mcflag && s->mv_base[nc] >= 0) mv_of(s, nc, k, &out4[1], &out4[2], &out4[3]);
    return ORC_OK;
}

/* All dequantised coefficients (BFS node-channel order) and roots, as
 * float64 -- the starting point of the differentiable relaxation. */
int orc_dequant(const orc_stream *s, double *coeff /* [n_nc][H][W] */, double *roots /* [nroot][3][H][W] */) {
    const geom *g = &s->g;
    if (g->sub) return ORC_E_ARG;          /* the relaxation is defined on full-resolution chroma only */
    size_t plane = (size_t)g->W * g->H;
    int32_t *tmp = (int32_t *)malloc(plane * sizeof(int32_t));
    if (!tmp) return ORC_E_OOM;
    for (int64_t nc = 0; nc < g->n_nc; nc++) {
        if (decode_plane_seq(s, nc, tmp) != ORC_OK) { free(tmp); return ORC_E_CORRUPT; }
        for (size_t p = 0; p < plane; p++) coeff[(size_t)nc * plane + p] = tmp[p];
    }
    size_t nr = (size_t)g->gu[g->L] * g->gv[g->L] * 3 * plane;
    for (size_t i = 0; i < nr; i++) roots[i] = s->roots[i];
    free(tmp);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* rendering (Sec. 2.1 two-plane rays; Sec. 5 ray-traced novel views)  */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t lf, width, height;
    float H_uv[9], H_st[9];
    int32_t pad;
    int64_t out_offset;
} orc_view;

static void apply_h(const float *Hm, double X, double Y, double *a, double *b) {
    double w = (double)Hm[6] * X + (double)Hm[7] * Y + (double)Hm[8];
    *a = ((double)Hm[0] * X + (double)Hm[1] * Y + (double)Hm[2]) / w;
    *b = ((double)Hm[3] * X + (double)Hm[4] * Y + (double)Hm[5]) / w;
}

/* Neighbour indices and fraction along one axis with clamp-to-edge.  The
 * coordinate is first limited to [-1, n] (which does not change the
 * interpolated value and keeps the integer conversion defined). */
static double axis_nb(double c, int n, int *i0, int *i1) {
    double cc = fmin(fmax(c, -1.0), (double)n);
    double fl = floor(cc);
    int k = (int)fl;
    *i0 = clampi(k, 0, n - 1);
    *i1 = clampi(k + 1, 0, n - 1);
    return cc - fl;
}

typedef struct { int i[2], j[2], x[2], y[2]; double wu[2], wv[2], ws[2], wt[2]; } ray_nb;

static void ray_setup(const orc_view *v, int nu, int nv, int W, int H, int px, int py, ray_nb *r) {
    double X = px + 0.5, Y = py + 0.5, u, vv, s, t;
    apply_h(v->H_uv, X, Y, &u, &vv);
    apply_h(v->H_st, X, Y, &s, &t);
    double fu = axis_nb(u, nu, &r->i[0], &r->i[1]);
    double fv = axis_nb(vv, nv, &r->j[0], &r->j[1]);
    double fs = axis_nb(s, W, &r->x[0], &r->x[1]);
    double ft = axis_nb(t, H, &r->y[0], &r->y[1]);
    r->wu[0] = 1.0 - fu; r->wu[1] = fu;
    r->wv[0] = 1.0 - fv; r->wv[1] = fv;
    r->ws[0] = 1.0 - fs; r->ws[1] = fs;
    r->wt[0] = 1.0 - ft; r->wt[1] = ft;
}

/* Render views from a dense RGB8 light field lf[nu][nv][H][W][3]; output is
 * float64 [H][W][3] per view at its out_offset (in elements). */
int orc_render_dense(const uint8_t *lf, int nu, int nv, int W, int H, const orc_view *views, int nviews,
                     double *out) {
    for (int vi = 0; vi < nviews; vi++) {
        const orc_view *v = &views[vi];
        double *o = out + v->out_offset;
        #pragma omp parallel for schedule(static)
        for (int py = 0; py < v->height; py++)
            for (int px = 0; px < v->width; px++) {
                ray_nb r;
                ray_setup(v, nu, nv, W, H, px, py, &r);
                double acc[3] = {0, 0, 0};
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int xs = 0; xs < 2; xs++)
                            for (int ys = 0; ys < 2; ys++) {
                                double w = r.wu[a] * r.wv[b] * r.ws[xs] * r.wt[ys];
                                const uint8_t *p = lf + ((((size_t)r.i[a] * nv + r.j[b]) * H + r.y[ys]) * W + r.x[xs]) * 3;
                                for (int c = 0; c < 3; c++) acc[c] += w * p[c];
                            }
                for (int c = 0; c < 3; c++) o[((size_t)py * v->width + px) * 3 + c] = acc[c] / 255.0;
            }
    }
    return ORC_OK;
}

/* Render selected pixels straight from the stream by random-access decoding
 * of their 16 samples.  pix [n][3] = (view index, px, py); out [n][3]. */
int orc_render_pixels_lod(const orc_stream *s, const orc_view *views, int nviews, const int32_t *pix, int64_t n,
                          int lod, double *out) {
    const geom *g = &s->g;
    if (lod < 0 || lod > g->L) return ORC_E_ARG;
    for (int64_t k = 0; k < n; k++) {
        const int32_t *p = pix + 3 * k;
        if (p[0] < 0 || p[0] >= nviews || p[1] < 0 || p[1] >= views[p[0]].width || p[2] < 0 ||
            p[2] >= views[p[0]].height) return ORC_E_ARG;
    }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; k++) {
        const int32_t *p = pix + 3 * k;
        ray_nb r;
        ray_setup(&views[p[0]], g->nu, g->nv, g->W, g->H, p[1], p[2], &r);
        double acc[3] = {0, 0, 0};
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int xs = 0; xs < 2; xs++)
                    for (int ys = 0; ys < 2; ys++) {
                        double w = r.wu[a] * r.wv[b] * r.ws[xs] * r.wt[ys];
                        int rgb[3];
                        sample_rgb(s, r.i[a], r.j[b], r.x[xs], r.y[ys], lod, rgb);
                        for (int c = 0; c < 3; c++) acc[c] += w * rgb[c];
                    }
        for (int c = 0; c < 3; c++) out[3 * k + c] = acc[c] / 255.0;
    }
    return ORC_OK;
}

int orc_render_pixels(const orc_stream *s, const orc_view *views, int nviews, const int32_t *pix, int64_t n,
                      double *out) {
    return orc_render_pixels_lod(s, views, nviews, pix, n, 0, out);
}

/* ------------------------------------------------------------------ */
/* differentiable relaxation: the decode with real-valued coefficients, */
/* exact bilinear weights (no >>4 rounding), YCoCg inverse with /2 (no  */
/* floor) and no clamp.  It is linear in (coefficients, roots) for      */
/* fixed motion vectors and signs.                                      */
/* ------------------------------------------------------------------ */

static void relax_taps(const geom *g, int x, int y, int mvx, int mvy, int tx[4], int ty[4], double tw[4]) {
    int X = 4 * x + mvx, Y = 4 * y + mvy;
    int x0 = (int)fdiv(X, 4), y0 = (int)fdiv(Y, 4);
    int fx = X - 4 * x0, fy = Y - 4 * y0;
    int xa = clampi(x0, 0, g->W - 1), xb = clampi(x0 + 1, 0, g->W - 1);
    int ya = clampi(y0, 0, g->H - 1), yb = clampi(y0 + 1, 0, g->H - 1);
    tx[0] = xa; ty[0] = ya; tw[0] = (4 - fx) * (4 - fy) / 16.0;
    tx[1] = xb; ty[1] = ya; tw[1] = fx * (4 - fy) / 16.0;
    tx[2] = xa; ty[2] = yb; tw[2] = (4 - fx) * fy / 16.0;
    tx[3] = xb; ty[3] = yb; tw[3] = fx * fy / 16.0;
}

/* Expected rounding of the integer predictor (Sec. 4.4 filter, +8 >> 4)
 * against the exact weighted sum S / 16, over reference values whose sum
 * is equally likely in every residue class its weights allow: the four
 * weights (4 - fx)(4 - fy), fx(4 - fy), (4 - fx)fy, fx fy share the factor
 * g = gcd(4 - fx, fx) * gcd(4 - fy, fy), S + 8 takes the residues 0, g, ..,
 * 16 - g mod 16 (mean 8 - g/2), so floor((S + 8) / 16) - S / 16 averages
 * g / 32.  Integer motion (g = 16) rounds nothing. */
static int gcd4(int f) { return f == 0 ? 4 : (f == 2 ? 2 : 1); }

double orc_mc_rounding_bias(int mvx, int mvy) {
    int fx = mvx & 3, fy = mvy & 3;
    if (fx == 0 && fy == 0) return 0.0;
    return gcd4(fx) * gcd4(fy) / 32.0;
}

/* with `bias`, each operation the relaxation drops carries its expected
 * value: every predictor its rounding bias above, each >> 1 of the YCoCg-R
 * inverse -1/4 (floor(v/2) - v/2 over both parities). */
static void relax_sample(const orc_stream *s, const double *coeff, const double *roots, int i, int j, int x, int y,
                         int bias, double rgb[3]) {
    const geom *g = &s->g;
    size_t plane = (size_t)g->W * g->H;
    int L = g->L;
    double v[3];
    for (int c = 0; c < 3; c++)
        v[c] = roots[(((size_t)(i >> L) * g->gv[L] + (j >> L)) * 3 + c) * plane + (size_t)y * g->W + x];
    int k = (y / g->B) * g->nbx + x / g->B;
    for (int l = 0; l < L; l++) {
        int a = i >> l, b = j >> l;
        for (int c = 0; c < 3; c++) {
            int64_t nc = nc_of(g, l, a, b, c);
            v[c] += coeff[(size_t)nc * plane + (size_t)y * g->W + x];
            if (!is_ref(a, b) && s->mcflag) {
                int mvx, mvy, sign, tx[4], ty[4];
                double tw[4];
                mv_of(s, nc, k, &mvx, &mvy, &sign);
                relax_taps(g, x, y, mvx, mvy, tx, ty, tw);
                int64_t rnc = nc_of(g, l, a & ~1, b & ~1, c);
                double p = bias ? orc_mc_rounding_bias(mvx, mvy) : 0.0;
                for (int t = 0; t < 4; t++) p += tw[t] * coeff[(size_t)rnc * plane + (size_t)ty[t] * g->W + tx[t]];
                v[c] += sign * p;
            }
        }
    }
    double t = v[0] - v[2] / 2.0 + (bias ? 0.25 : 0.0);
    double G = v[2] + t;
    double Bb = t - v[1] / 2.0 + (bias ? 0.25 : 0.0);
    rgb[0] = Bb + v[1];
    rgb[1] = G;
    rgb[2] = Bb;
}

int orc_relax_render_ex(const orc_stream *s, const double *coeff, const double *roots, const orc_view *views,
                        int nviews, int bias, double *out) {
    const geom *g = &s->g;
    if (g->sub) return ORC_E_ARG;          /* the relaxation is defined on full-resolution chroma only */
    for (int vi = 0; vi < nviews; vi++) {
        const orc_view *v = &views[vi];
        double *o = out + v->out_offset;
        #pragma omp parallel for schedule(static)
        for (int py = 0; py < v->height; py++)
            for (int px = 0; px < v->width; px++) {
                ray_nb r;
                ray_setup(v, g->nu, g->nv, g->W, g->H, px, py, &r);
                double acc[3] = {0, 0, 0};
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int xs = 0; xs < 2; xs++)
                            for (int ys = 0; ys < 2; ys++) {
                                double w = r.wu[a] * r.wv[b] * r.ws[xs] * r.wt[ys];
                                double rgb[3];
                                relax_sample(s, coeff, roots, r.i[a], r.j[b], r.x[xs], r.y[ys], bias, rgb);
                                for (int c = 0; c < 3; c++) acc[c] += w * rgb[c];
                            }
                for (int c = 0; c < 3; c++) o[((size_t)py * v->width + px) * 3 + c] = acc[c] / 255.0;
            }
    }
    return ORC_OK;
}

int orc_relax_render(const orc_stream *s, const double *coeff, const double *roots, const orc_view *views,
                     int nviews, double *out) {
    return orc_relax_render_ex(s, coeff, roots, views, nviews, 0, out);
}

/* Transpose of orc_relax_render: accumulates into grad_coeff [n_nc][H][W]
 * and grad_roots [nroot][3][H][W] (both zeroed by the caller). Single
 * threaded: the scatter is written plainly, in ray order. */
int orc_relax_adjoint(const orc_stream *s, const orc_view *views, int nviews, const double *grad_out,
                      double *grad_coeff, double *grad_roots) {
    const geom *g = &s->g;
    if (g->sub) return ORC_E_ARG;          /* the relaxation is defined on full-resolution chroma only */
    size_t plane = (size_t)g->W * g->H;
    int L = g->L;
    for (int vi = 0; vi < nviews; vi++) {
        const orc_view *v = &views[vi];
        const double *go = grad_out + v->out_offset;
        for (int py = 0; py < v->height; py++)
            for (int px = 0; px < v->width; px++) {
                ray_nb r;
                ray_setup(v, g->nu, g->nv, g->W, g->H, px, py, &r);
                const double *gp = go + ((size_t)py * v->width + px) * 3;
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int xs = 0; xs < 2; xs++)
                            for (int ys = 0; ys < 2; ys++) {
                                double w = r.wu[a] * r.wv[b] * r.ws[xs] * r.wt[ys] / 255.0;
                                double gR = w * gp[0], gG = w * gp[1], gB = w * gp[2];
                                /* transpose of the linear YCoCg inverse */
                                double gv[3];
                                gv[0] = gR + gG + gB;
                                gv[1] = 0.5 * gR - 0.5 * gB;
                                gv[2] = -0.5 * gR + 0.5 * gG - 0.5 * gB;
                                int i = r.i[a], j = r.j[b], x = r.x[xs], y = r.y[ys];
                                for (int c = 0; c < 3; c++)
                                    grad_roots[(((size_t)(i >> L) * g->gv[L] + (j >> L)) * 3 + c) * plane + (size_t)y * g->W + x] += gv[c];
                                int k = (y / g->B) * g->nbx + x / g->B;
                                for (int l = 0; l < L; l++) {
                                    int na = i >> l, nb = j >> l;
                                    for (int c = 0; c < 3; c++) {
                                        int64_t nc = nc_of(g, l, na, nb, c);
                                        grad_coeff[(size_t)nc * plane + (size_t)y * g->W + x] += gv[c];
                                        if (!is_ref(na, nb) && s->mcflag) {
                                            int mvx, mvy, sign, tx[4], ty[4];
                                            double tw[4];
                                            mv_of(s, nc, k, &mvx, &mvy, &sign);
                                            relax_taps(g, x, y, mvx, mvy, tx, ty, tw);
                                            int64_t rnc = nc_of(g, l, na & ~1, nb & ~1, c);
                                            for (int t = 0; t < 4; t++)
                                                grad_coeff[(size_t)rnc * plane + (size_t)ty[t] * g->W + tx[t]] += sign * tw[t] * gv[c];
                                        }
                                    }
                                }
                            }
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* touched-set counter: the bytes a view must read at least once        */
/* (compulsory traffic) plus its FP32 output, per view                  */
/* ------------------------------------------------------------------ */

/* bytes[v] = W*H*12 (output) + 2 per unique root pixel of each channel plane + per unique touched
 * predictive block (16 per unique group entry, 2 + 4*record words if
 * significant, MV bits/8) + per unique touched significant reference block
 * (B*B*2 resident tile + 4 table entry). */
/* Compulsory bytes of each view decoded down to level lod: a sample of camera
 * (i, j) stands for its level-lod node (keyed by the node's first camera). */
int orc_touched_bytes_lod(const orc_stream *s, const orc_view *views, int nviews, int lod, double *bytes) {
    const geom *g = &s->g;
    if (lod < 0 || lod > g->L) return ORC_E_ARG;
    size_t nroot = (size_t)g->gu[g->L] * g->gv[g->L];
    size_t nb_all = (size_t)g->n_nc * g->nblocks;
    double mv_bits = 0;
    if (s->mcflag) mv_bits = (double)orc_bise_bits(s->mv_mode, s->mv_b, 15) / 15.0;
    for (int vi = 0; vi < nviews; vi++) {
        const orc_view *v = &views[vi];
        uint8_t *root_seen = (uint8_t *)calloc(nroot * g->npx, 1);
        uint8_t *blk_seen = (uint8_t *)calloc(nb_all, 1);
        uint8_t *grp_seen = (uint8_t *)calloc((size_t)g->n_nc * g->ngroups, 1);
        if (!root_seen || !blk_seen || !grp_seen) { free(root_seen); free(blk_seen); free(grp_seen); return ORC_E_OOM; }
        double acc = (double)v->width * v->height * 12.0;
        for (int py = 0; py < v->height; py++)
            for (int px = 0; px < v->width; px++) {
                ray_nb r;
                ray_setup(v, g->nu, g->nv, g->W, g->H, px, py, &r);
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int xs = 0; xs < 2; xs++)
                            for (int ys = 0; ys < 2; ys++) {
                                int i = (r.i[a] >> lod) << lod, j = (r.j[b] >> lod) << lod;
                                for (int c = 0; c < 3; c++) {
                                    /* the sample's pixel in channel c's plane (half resolution for sub-sampled chroma) */
                                    const geom gc = chan_geom(g, c);
                                    int x = (g->sub && c > 0) ? r.x[xs] >> 1 : r.x[xs];
                                    int y = (g->sub && c > 0) ? r.y[ys] >> 1 : r.y[ys];
                                    size_t rp = ((size_t)(i >> g->L) * g->gv[g->L] + (j >> g->L)) * g->npx + g->coff[c] +
                                                (size_t)y * gc.W + x;
                                    if (!root_seen[rp]) { root_seen[rp] = 1; acc += 2.0; }
                                    int k = (y / g->B) * gc.nbx + x / g->B;
                                    for (int l = lod; l < g->L; l++) {
                                        int na = i >> l, nb = j >> l;
                                        int64_t nc = nc_of(g, l, na, nb, c);
                                        if (is_ref(na, nb)) {
                                            size_t key = (size_t)nc * g->nblocks + k;
                                            if (!blk_seen[key]) {
                                                blk_seen[key] = 1;
                                                if (find_record(s, nc, k)) acc += g->B * g->B * 2.0 + 4.0;
                                            }
                                            continue;
                                        }
                                        size_t key = (size_t)nc * g->nblocks + k;
                                        if (!blk_seen[key]) {
                                            blk_seen[key] = 1;
                                            size_t gk = (size_t)nc * g->ngroups + k / 32;
                                            if (!grp_seen[gk]) { grp_seen[gk] = 1; acc += 16.0; }
                                            const uint32_t *rec = find_record(s, nc, k);
                                            if (rec) {
                                                int x0, y0, bw, bh;
                                                block_rect(&gc, k, &x0, &y0, &bw, &bh);
                                                int md = (int)((rec[0] >> 21) & 3u), bb = (int)((rec[0] >> 16) & 31u);
                                                acc += 2.0 + 4.0 * (1 + (orc_bise_bits(md, bb, (uint64_t)bw * bh) + 31) / 32);
                                            }
                                            acc += mv_bits / 8.0;
                                        }
                                        if (s->mcflag) {
                                            int mvx, mvy, sign, tx[4], ty[4];
                                            double tw[4];
                                            mv_of(s, nc, k, &mvx, &mvy, &sign);
                                            relax_taps(&gc, x, y, mvx, mvy, tx, ty, tw);
                                            int64_t rnc = nc_of(g, l, na & ~1, nb & ~1, c);
                                            for (int t = 0; t < 4; t++) {
                                                int kk = (ty[t] / g->B) * gc.nbx + tx[t] / g->B;
                                                size_t rk = (size_t)rnc * g->nblocks + kk;
                                                if (!blk_seen[rk]) {
                                                    blk_seen[rk] = 1;
                                                    if (find_record(s, rnc, kk)) acc += g->B * g->B * 2.0 + 4.0;
                                                }
                                            }
                                        }
                                    }
                                }
                            }
            }
        bytes[vi] = acc;
        free(root_seen); free(blk_seen); free(grp_seen);
    }
    return ORC_OK;
}

int orc_touched_bytes(const orc_stream *s, const orc_view *views, int nviews, double *bytes) {
    return orc_touched_bytes_lod(s, views, nviews, 0, bytes);
}

int orc_version(void) { return (int)ORC_VERSION; }

/* Thread count of the OpenMP loops (results do not depend on it). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
