// HMLFC encoder of the product library (host threads): hierarchy (Sec. 4.3),
// closed-loop phase-shifted motion compensation (Sec. 4.4), quantiser and
// block thresholds (Sec. 4.5), BISE (Sec. 4.6), breadth-first stream
// (Sec. 4.7).  Also the re-quantiser that writes a stream from refined
// coefficients with the motion vectors of an existing stream.
//
// Deterministic: every choice follows fixed keys, so the output does not
// depend on the thread count.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hmlfc_host.h"

using namespace hmlfc;

namespace {

int fdiv(int a, int b) {  // floor(a / b), b > 0
    int q = a / b;
    if ((a % b) != 0 && a < 0) q--;
    return q;
}

int quant(int r, int q) {
    const int m = (std::abs(r) + q / 2) / q;
    return r < 0 ? -m : m;
}

struct Plane {
    int W, H;
    const int16_t *p;
    int at(int x, int y) const { return p[y * W + x]; }
};

// Quarter-pel bilinear prediction (weights sum to 16, rounded half up, taps
// clamped to the image).
inline int qpel(const Plane &R, int x, int y, int mvx, int mvy) {
    const int X = 4 * x + mvx, Y = 4 * y + mvy;
    const int x0 = X >> 2, y0 = Y >> 2, fx = X & 3, fy = Y & 3;
    const int xa = std::min(std::max(x0, 0), R.W - 1), xb = std::min(std::max(x0 + 1, 0), R.W - 1);
    const int ya = std::min(std::max(y0, 0), R.H - 1), yb = std::min(std::max(y0 + 1, 0), R.H - 1);
    const int s = (4 - fx) * (4 - fy) * R.at(xa, ya) + fx * (4 - fy) * R.at(xb, ya) + (4 - fx) * fy * R.at(xa, yb) +
                  fx * fy * R.at(xb, yb);
    return (s + 8) >> 4;
}

struct Enc {
    Geometry g;
    int mc = 1;
};

struct BlockOut {
    bool sig = false;
    std::vector<uint32_t> rec;  // header + payload
};

struct NcOut {
    std::vector<BlockOut> blocks;
    std::vector<uint32_t> mv;   // symbols (predictive nodes with MC)
};

void bits_put(uint32_t *buf, uint64_t pos, uint32_t v, int w) {
    if (w == 0) return;
    const uint64_t k = pos >> 5;
    const int sh = (int)(pos & 31u);
    const uint64_t wide = (uint64_t)(v & ((w >= 32) ? 0xFFFFFFFFu : ((1u << w) - 1u))) << sh;
    buf[k] |= (uint32_t)wide;
    if (sh + w > 32) buf[k + 1] |= (uint32_t)(wide >> 32);
}

// BISE packing of n values of alphabet (mode, b) at bit 0 of buf (zeroed,
// one spare word).
void bise_pack(uint32_t *buf, int mode, int b, const uint32_t *v, uint64_t n) {
    if (mode == 0) {
        for (uint64_t i = 0; i < n; i++) bits_put(buf, i * (uint64_t)b, v[i], b);
        return;
    }
    const int per = mode == 1 ? 5 : 3, radix = mode == 1 ? 3 : 5, hw = mode == 1 ? 8 : 7;
    const uint64_t gbits = (uint64_t)hw + (uint64_t)per * b;
    const uint32_t mask = (1u << b) - 1u;
    for (uint64_t g0 = 0, gi = 0; g0 < n; g0 += per, gi++) {
        uint32_t packed = 0, mul = 1;
        const uint64_t base = gi * gbits;
        for (int r = 0; r < per; r++) {
            const uint32_t val = g0 + r < n ? v[g0 + r] : 0u;
            packed += (val >> b) * mul;
            mul *= (uint32_t)radix;
            bits_put(buf, base + hw + (uint64_t)r * b, val & mask, b);
        }
        bits_put(buf, base, packed, hw);
    }
}

// Record of one block's levels (header word + BISE payload).
void make_record(const int *lv, int n, std::vector<uint32_t> &rec) {
    int m = lv[0], M = lv[0];
    for (int i = 1; i < n; i++) {
        m = std::min(m, lv[i]);
        M = std::max(M, lv[i]);
    }
    int mode, b;
    bise_choose((uint64_t)(M - m + 1), mode, b);
    const uint64_t bits = bise_bits(mode, b, (uint64_t)n);
    const size_t words = 1 + (size_t)((bits + 31) / 32);
    rec.assign(words + 1, 0u);
    std::vector<uint32_t> v(n);
    for (int i = 0; i < n; i++) v[i] = (uint32_t)(lv[i] - m);
    rec[0] = (uint32_t)(uint16_t)(int16_t)m | ((uint32_t)b << 16) | ((uint32_t)mode << 21);
    bise_pack(rec.data() + 1, mode, b, v.data(), (uint64_t)n);
    rec.resize(words);
}

// Phase-shifted block search (Sec. 4.4, Eq. 1-2 and the argmin displays):
// per sign an integer stage over [-Ws, Ws]^2 keyed (cost, |x|+|y|, raster),
// then (refine) the 7x7 quarter offsets around it keyed (cost, fractional,
// |mv|_1, raster); the subtractive sign wins ties.
void search(const int32_t *S, const Plane &R, int W, int H, int x0, int y0, int bw, int bh, int Ws, bool refine,
            int &omx, int &omy, int &osign) {
    int64_t best[2] = {-1, -1};
    int bmx[2] = {0, 0}, bmy[2] = {0, 0}, bl1[2] = {0, 0};
    const bool interior = x0 - Ws >= 0 && y0 - Ws >= 0 && x0 + bw + Ws <= W && y0 + bh + Ws <= H;
    for (int dy = -Ws; dy <= Ws; dy++)
        for (int dx = -Ws; dx <= Ws; dx++) {
            int64_t cp = 0, cm = 0;
            for (int y = y0; y < y0 + bh; y++) {
                const int32_t *srow = S + (size_t)y * W;
                int yy = y + dy;
                if (!interior) yy = std::min(std::max(yy, 0), H - 1);
                const int16_t *rrow = R.p + (size_t)yy * W;
                if (interior) {
                    for (int x = x0; x < x0 + bw; x++) {
                        const int s = srow[x], r = rrow[x + dx];
                        cp += std::abs(s - r);
                        cm += std::abs(s + r);
                    }
                } else {
                    for (int x = x0; x < x0 + bw; x++) {
                        const int s = srow[x], r = rrow[std::min(std::max(x + dx, 0), W - 1)];
                        cp += std::abs(s - r);
                        cm += std::abs(s + r);
                    }
                }
            }
            const int l1 = std::abs(dx) + std::abs(dy);
            const int64_t c[2] = {cp, cm};
            for (int s = 0; s < 2; s++)
                if (best[s] < 0 || c[s] < best[s] || (c[s] == best[s] && l1 < bl1[s])) {
                    best[s] = c[s];
                    bmx[s] = 4 * dx;
                    bmy[s] = 4 * dy;
                    bl1[s] = l1;
                }
        }
    if (refine) {
        for (int s = 0; s < 2; s++) {
            const int sg = s == 0 ? 1 : -1;
            const int cx = bmx[s], cy = bmy[s];
            int64_t bc = best[s];
            bool frac = false;
            int l1b = std::abs(cx) + std::abs(cy), rx = cx, ry = cy;
            for (int oy = -3; oy <= 3; oy++)
                for (int ox = -3; ox <= 3; ox++) {
                    if (ox == 0 && oy == 0) continue;
                    const int mx = cx + ox, my = cy + oy;
                    if (std::abs(mx) > 4 * Ws || std::abs(my) > 4 * Ws) continue;
                    int64_t c = 0;
                    for (int y = y0; y < y0 + bh && c <= bc; y++)
                        for (int x = x0; x < x0 + bw; x++) c += std::abs(S[(size_t)y * W + x] - sg * qpel(R, x, y, mx, my));
                    const int l1 = std::abs(mx) + std::abs(my);
                    if (c < bc || (c == bc && frac && l1 < l1b)) {
                        bc = c;
                        frac = true;
                        l1b = l1;
                        rx = mx;
                        ry = my;
                    }
                }
            best[s] = bc;
            bmx[s] = rx;
            bmy[s] = ry;
        }
    }
    const int pick = best[0] <= best[1] ? 0 : 1;
    omx = bmx[pick];
    omy = bmy[pick];
    osign = pick == 0 ? 1 : -1;
}

// Serialise the coded tree in the breadth-first stream layout.
int serialise(const Geometry &g, const std::vector<int16_t> &roots, const std::vector<NcOut> &ncs, void **h_out,
              size_t *nbytes) {
    uint64_t nsig = 0, nrecw = 0, nmv = 0;
    for (const auto &o : ncs) {
        for (const auto &b : o.blocks)
            if (b.sig) {
                nsig++;
                nrecw += b.rec.size();
            }
        nmv += o.mv.size();
    }
    int mv_mode = 0, mv_b = 0;
    if (g.mc) bise_choose(2ull * g.side * g.side, mv_mode, mv_b);
    const uint64_t nmvw = g.mc ? (bise_bits(mv_mode, mv_b, nmv) + 31) / 32 : 0;
    auto a16 = [](uint64_t v) { return (v + 15) & ~(uint64_t)15; };
    const uint64_t plane = (uint64_t)g.W * g.H;
    const uint64_t o_roots = (uint64_t)kHeaderWords * 4;
    const uint64_t o_groups = a16(o_roots + roots.size() * 2);
    const uint64_t o_offs = a16(o_groups + (uint64_t)g.n_nc * g.ngroups * 16);
    const uint64_t o_recs = a16(o_offs + nsig * 2);
    const uint64_t o_mvs = a16(o_recs + nrecw * 4);
    const uint64_t total = a16(o_mvs + nmvw * 4);
    (void)plane;
    if (total > 0xFFFFFFF0ull) return fail(HMLFC_E_UNSUPPORTED, "stream larger than 4 GB");
    uint8_t *s = static_cast<uint8_t *>(std::calloc((size_t)total, 1));
    if (!s) return fail(HMLFC_E_OOM, "stream allocation");
    uint32_t h[kHeaderWords] = {0};
    h[0] = kMagic; h[1] = kVersion; h[2] = (uint32_t)g.nu; h[3] = (uint32_t)g.nv; h[4] = (uint32_t)g.W;
    h[5] = (uint32_t)g.H; h[6] = (uint32_t)g.L; h[7] = (uint32_t)g.B; h[8] = (uint32_t)g.Ws; h[9] = (uint32_t)g.q;
    h[10] = (uint32_t)g.t_ref; h[11] = (uint32_t)g.t_pred; h[12] = (g.mc ? 1u : 0u) | (g.sub ? 2u : 0u);
    h[13] = (uint32_t)mv_mode;
    h[14] = (uint32_t)mv_b; h[15] = (uint32_t)g.n_nc; h[16] = (uint32_t)g.ngroups; h[17] = (uint32_t)nsig;
    h[18] = (uint32_t)nrecw; h[19] = (uint32_t)nmv; h[20] = (uint32_t)nmvw; h[21] = (uint32_t)o_roots;
    h[22] = (uint32_t)o_groups; h[23] = (uint32_t)o_offs; h[24] = (uint32_t)o_recs; h[25] = (uint32_t)o_mvs;
    h[26] = (uint32_t)total;
    std::memcpy(s, h, sizeof h);
    std::memcpy(s + o_roots, roots.data(), roots.size() * 2);
    uint64_t sc = 0, rc = 0;
    std::vector<uint32_t> mvall;
    mvall.reserve(nmv);
    for (int64_t nc = 0; nc < g.n_nc; nc++) {
        const NcOut &o = ncs[nc];
        for (int gi = 0; gi < g.ngroups; gi++) {
            uint32_t bitmap = 0;
            const uint64_t gbase = rc, obase = sc;
            for (int r = 0; r < 32; r++) {
                const int k = gi * 32 + r;
                if (k >= (int)o.blocks.size() || !o.blocks[k].sig) continue;   // the node-channel's own block grid
                bitmap |= 1u << r;
                const uint64_t rel = rc - gbase;
                if (rel > 0xFFFFu) {
                    std::free(s);
                    return fail(HMLFC_E_UNSUPPORTED, "block group larger than 64 K words");
                }
                const uint16_t r16 = (uint16_t)rel;
                std::memcpy(s + o_offs + 2 * sc, &r16, 2);
                std::memcpy(s + o_recs + 4 * rc, o.blocks[k].rec.data(), o.blocks[k].rec.size() * 4);
                rc += o.blocks[k].rec.size();
                sc++;
            }
            const uint32_t ge[4] = {bitmap, (uint32_t)gbase, (uint32_t)obase, 0u};
            std::memcpy(s + o_groups + ((uint64_t)nc * g.ngroups + gi) * 16, ge, 16);
        }
        mvall.insert(mvall.end(), o.mv.begin(), o.mv.end());
    }
    if (nmv) {
        std::vector<uint32_t> buf((size_t)nmvw + 1, 0u);
        bise_pack(buf.data(), mv_mode, mv_b, mvall.data(), nmv);
        std::memcpy(s + o_mvs, buf.data(), (size_t)nmvw * 4);
    }
    *h_out = s;
    *nbytes = (size_t)total;
    return HMLFC_OK;
}

}  // namespace

void hmlfc::fill_channels(Geometry &g) {
    int64_t off = 0, mv = 0;
    for (int c = 0; c < 3; c++) {
        g.cW[c] = (g.sub && c > 0) ? (g.W + 1) / 2 : g.W;
        g.cH[c] = (g.sub && c > 0) ? (g.H + 1) / 2 : g.H;
        g.cnbx[c] = (g.cW[c] + g.B - 1) / g.B;
        g.cnby[c] = (g.cH[c] + g.B - 1) / g.B;
        g.cnb[c] = g.cnbx[c] * g.cnby[c];
        g.coff[c] = off;
        g.mv_coff[c] = mv;
        off += (int64_t)g.cW[c] * g.cH[c];
        mv += g.cnb[c];
    }
    g.npx = off;
    g.mv_node = mv;
}

void hmlfc::fill_geometry(Geometry &g, int nu, int nv, int W, int H, int L, int B, int Ws, int q, int tr, int tp, int mc,
                          int sub) {
    std::memset(&g, 0, sizeof g);
    g.nu = nu; g.nv = nv; g.W = W; g.H = H; g.L = L; g.B = B; g.Ws = Ws; g.q = q; g.t_ref = tr; g.t_pred = tp;
    g.mc = mc ? 1 : 0;
    g.sub = sub ? 1 : 0;
    g.nbx = (W + B - 1) / B;
    g.nby = (H + B - 1) / B;
    g.nblocks = g.nbx * g.nby;
    g.ngroups = (g.nblocks + 31) / 32;
    g.side = 8 * Ws + 1;
    for (int l = 0; l <= L; l++) {
        g.gu[l] = (nu + (1 << l) - 1) >> l;
        g.gv[l] = (nv + (1 << l) - 1) >> l;
    }
    int64_t nc = 0;
    for (int l = L - 1; l >= 0; l--) {
        g.nc_base[l] = nc;
        nc += 3ll * g.gu[l] * g.gv[l];
    }
    g.n_nc = nc;
    g.n_roots = (int64_t)g.gu[L] * g.gv[L];
    fill_channels(g);
}

extern "C" int hmlfc_encode(const uint8_t *h_lf, int nu, int nv, int W, int H, const hmlfc_encode_params *p,
                            void **h_out, size_t *nbytes) {
    if (!h_lf || !p || !h_out || !nbytes) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    if (nu < 1 || nv < 1 || W < 1 || H < 1 || nu > 65536 || nv > 65536 || W > 65536 || H > 65536)
        return fail(HMLFC_E_INVALID_ARG, "light-field size");
    if (p->levels < 1 || p->levels > kMaxLevels || p->block < 1 || p->block > kMaxBlock || p->search < 0 ||
        p->search > 64 || p->qstep < 1 || p->qstep > kCoefLimit || p->t_ref < 0 || p->t_pred < 0 || p->mc < 0 ||
        p->mc > 3 || p->chroma < 0 || p->chroma > 1 || (p->chroma && p->block % 2 != 0))
        return fail(HMLFC_E_INVALID_ARG, "encoder parameters");
    Geometry g;
    fill_geometry(g, nu, nv, W, H, p->levels, p->block, p->search, p->qstep, p->t_ref, p->t_pred, p->mc != 0,
                  p->chroma);
    const int L = g.L, B = g.B, q = g.q, threads = p->threads;
    const size_t plane = (size_t)W * H, npx = (size_t)g.npx;

    // I_0: YCoCg-R of every view (Sec. 4.5), int16 [node][npx] with channel c's plane at coff[c]; with
    // sub-sampled chroma, Co and Cg at ceil(W/2) x ceil(H/2), each the rounded mean of a 2x2 pixel group
    std::vector<std::vector<int16_t>> lev(L + 1);
    lev[0].resize((size_t)nu * nv * npx);
    parallel_for((int64_t)nu * nv, threads, [&](int64_t v) {
        const uint8_t *src = h_lf + (size_t)v * plane * 3;
        int16_t *dst = lev[0].data() + (size_t)v * npx;
        std::vector<int16_t> full(g.sub ? 2 * plane : 0);
        int16_t *co_out = g.sub ? full.data() : dst + g.coff[1];
        int16_t *cg_out = g.sub ? full.data() + plane : dst + g.coff[2];
        for (size_t px = 0; px < plane; px++) {
            const int R = src[3 * px], G = src[3 * px + 1], Bc = src[3 * px + 2];
            const int co = R - Bc;
            const int t = Bc + (co >> 1);
            const int cg = G - t;
            dst[px] = (int16_t)(t + (cg >> 1));
            co_out[px] = (int16_t)co;
            cg_out[px] = (int16_t)cg;
        }
        if (g.sub)
            for (int c = 1; c < 3; c++) {
                const int16_t *f = full.data() + (size_t)(c - 1) * plane;
                int16_t *d = dst + g.coff[c];
                for (int yc = 0; yc < g.cH[c]; yc++)
                    for (int xc = 0; xc < g.cW[c]; xc++) {
                        int sum = 0, k = 0;
                        for (int y = 2 * yc; y < std::min(2 * yc + 2, H); y++)
                            for (int x = 2 * xc; x < std::min(2 * xc + 2, W); x++, k++) sum += f[(size_t)y * W + x];
                        d[(size_t)yc * g.cW[c] + xc] = (int16_t)fdiv(sum + k / 2, k);
                    }
            }
    });
    // RKVs: rounded mean of each 2x2 cluster (Sec. 4.3), per pixel of every channel plane
    for (int l = 0; l < L; l++) {
        const int gv = g.gv[l], pu = g.gu[l + 1], pv = g.gv[l + 1], gu = g.gu[l];
        lev[l + 1].resize((size_t)pu * pv * npx);
        parallel_for((int64_t)pu * pv * 3, threads, [&](int64_t e) {
            const int c = (int)(e % 3), node = (int)(e / 3), A = node / pv, Bn = node % pv;
            const size_t cpl = (size_t)g.cW[c] * g.cH[c];
            const int16_t *mem[4];
            int k = 0;
            for (int da = 0; da < 2; da++)
                for (int db = 0; db < 2; db++) {
                    const int a = 2 * A + da, b = 2 * Bn + db;
                    if (a < gu && b < gv) mem[k++] = lev[l].data() + ((size_t)a * gv + b) * npx + g.coff[c];
                }
            int16_t *dst = lev[l + 1].data() + ((size_t)A * pv + Bn) * npx + g.coff[c];
            for (size_t px = 0; px < cpl; px++) {
                int s = 0;
                for (int t = 0; t < k; t++) s += mem[t][px];
                dst[px] = (int16_t)fdiv(s + k / 2, k);
            }
        });
    }

    std::vector<NcOut> ncs((size_t)g.n_nc);
    std::vector<int16_t> roots(lev[L]);
    // closed loop, top-down (reconstructions recon[l] as int16)
    std::vector<int16_t> recon_parent(lev[L]);
    int err = HMLFC_OK;
    for (int l = L - 1; l >= 0 && err == HMLFC_OK; l--) {
        const int gu = g.gu[l], gv = g.gv[l], pv = g.gv[l + 1];
        std::vector<int16_t> recon((size_t)gu * gv * npx);
        std::vector<int16_t> rhat((size_t)gu * gv * npx, 0);
        for (int pass = 0; pass < 2; pass++) {
            std::vector<int64_t> items;
            for (int a = 0; a < gu; a++)
                for (int b = 0; b < gv; b++) {
                    const bool ref = (a % 2 == 0) && (b % 2 == 0);
                    if ((pass == 0) == ref)
                        for (int c = 0; c < 3; c++) items.push_back(((int64_t)a * gv + b) * 3 + c);
                }
            std::vector<int> errs(items.size(), HMLFC_OK);
            parallel_for((int64_t)items.size(), threads, [&](int64_t it) {
                const int64_t e = items[it];
                const int c = (int)(e % 3), node = (int)(e / 3), a = node / gv, b = node % gv;
                const bool ref = pass == 0;
                const int64_t nc = g.nc_base[l] + e;
                // every plane of channel c has that channel's size and block grid
                const int Wc = g.cW[c], Hc = g.cH[c], nbc = g.cnb[c], nbxc = g.cnbx[c];
                const size_t cpl = (size_t)Wc * Hc;
                NcOut &o = ncs[nc];
                o.blocks.assign(nbc, BlockOut());
                const bool use_mc = !ref && p->mc != 0;
                if (use_mc) o.mv.assign(nbc, 0u);
                const int16_t *child = lev[l].data() + (size_t)node * npx + g.coff[c];
                const int16_t *par = recon_parent.data() + ((size_t)(a / 2) * pv + b / 2) * npx + g.coff[c];
                std::vector<int32_t> S(cpl);
                for (size_t px = 0; px < cpl; px++) S[px] = (int32_t)child[px] - par[px];
                const Plane R{Wc, Hc, rhat.data() + ((size_t)(a & ~1) * gv + (b & ~1)) * npx + g.coff[c]};
                int16_t *rec_out = recon.data() + (size_t)node * npx + g.coff[c];
                int16_t *rhat_out = rhat.data() + (size_t)node * npx + g.coff[c];
                std::vector<int> lv((size_t)B * B), res((size_t)B * B), pr((size_t)B * B);
                for (int k = 0; k < nbc; k++) {
                    const int x0 = (k % nbxc) * B, y0 = (k / nbxc) * B;
                    const int bw = std::min(B, Wc - x0), bh = std::min(B, Hc - y0);
                    int mvx = 0, mvy = 0, sign = 1;
                    if (use_mc && (p->mc == 1 || p->mc == 3))
                        search(S.data(), R, Wc, Hc, x0, y0, bw, bh, g.Ws, p->mc == 1, mvx, mvy, sign);
                    int64_t energy = 0;
                    bool any = false;
                    int n = 0;
                    for (int y = y0; y < y0 + bh; y++)
                        for (int x = x0; x < x0 + bw; x++, n++) {
                            pr[n] = use_mc ? sign * qpel(R, x, y, mvx, mvy) : 0;
                            res[n] = S[(size_t)y * Wc + x] - pr[n];
                            energy += std::abs(res[n]);
                            lv[n] = quant(res[n], q);
                            any |= lv[n] != 0;
                        }
                    const bool sig = any && energy >= (ref ? g.t_ref : g.t_pred);
                    if (use_mc)
                        o.mv[k] = ((uint32_t)(mvx + 4 * g.Ws) * (uint32_t)g.side + (uint32_t)(mvy + 4 * g.Ws)) * 2u +
                                  (sign < 0 ? 1u : 0u);
                    if (sig) {
                        for (int t = 0; t < n; t++)
                            if (lv[t] < -32768 || lv[t] > 32767) errs[it] = HMLFC_E_UNSUPPORTED;
                        o.blocks[k].sig = true;
                        make_record(lv.data(), n, o.blocks[k].rec);
                    }
                    n = 0;
                    for (int y = y0; y < y0 + bh; y++)
                        for (int x = x0; x < x0 + bw; x++, n++) {
                            const int shat = pr[n] + (sig ? q * lv[n] : 0);
                            const int v = par[(size_t)y * Wc + x] + shat;
                            if (v < -32768 || v > 32767 || shat < -32768 || shat > 32767) errs[it] = HMLFC_E_UNSUPPORTED;
                            rec_out[(size_t)y * Wc + x] = (int16_t)v;
                            if (ref) rhat_out[(size_t)y * Wc + x] = (int16_t)shat;
                        }
                }
            });
            for (int e2 : errs)
                if (e2 != HMLFC_OK) err = e2;
        }
        recon_parent.swap(recon);
        lev[l + 1].clear();
        lev[l + 1].shrink_to_fit();
    }
    if (err != HMLFC_OK) return fail(err, "values outside the int16 range while encoding");
    return serialise(g, roots, ncs, h_out, nbytes);
}

extern "C" int hmlfc_requantize(const hmlfc_stream *s, const float *h_coeff, const float *h_root, void **h_out,
                                size_t *nbytes) {
    if (!s || !h_coeff || !h_root || !h_out || !nbytes) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    if (s->g.sub) return fail(HMLFC_E_UNSUPPORTED, "re-quantising a stream with sub-sampled chroma");
    const Geometry &g0 = s->g;
    Geometry g;
    fill_geometry(g, g0.nu, g0.nv, g0.W, g0.H, g0.L, g0.B, g0.Ws, g0.q, g0.t_ref, g0.t_pred, g0.mc);
    const size_t plane = (size_t)g.W * g.H;
    std::vector<int16_t> roots((size_t)g.n_roots * 3 * plane);
    for (size_t i = 0; i < roots.size(); i++) {
        const double v = std::floor((double)h_root[i] + 0.5);
        if (!(v >= -32768.0 && v <= 32767.0)) return fail(HMLFC_E_UNSUPPORTED, "root value outside int16");
        roots[i] = (int16_t)v;
    }
    // motion-vector symbols of the source stream, in order
    const uint8_t *bytes = s->bytes.data();
    std::vector<uint32_t> mvsyms;
    if (g.mc) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(bytes + g0.off_mvs);
        std::vector<uint32_t> buf(w, w + g0.n_mvw);
        buf.push_back(0);
        buf.push_back(0);
        const int mode = g0.mv_mode, b = g0.mv_b;
        mvsyms.resize(g0.n_mv);
        for (uint64_t i = 0; i < g0.n_mv; i++) {
            auto get = [&](uint64_t pos, int wd) -> uint32_t {
                if (wd == 0) return 0u;
                const uint64_t k = pos >> 5;
                const uint64_t v = ((uint64_t)buf[k + 1] << 32 | buf[k]) >> (pos & 31u);
                return (uint32_t)(v & ((1ull << wd) - 1));
            };
            if (mode == 0) {
                mvsyms[i] = get(i * (uint64_t)b, b);
            } else {
                const int per = mode == 1 ? 5 : 3, radix = mode == 1 ? 3 : 5, hw = mode == 1 ? 8 : 7;
                const uint64_t gi = i / per;
                const int r = (int)(i % per);
                const uint64_t base = gi * (uint64_t)(hw + per * b);
                uint32_t packed = get(base, hw);
                for (int t = 0; t < r; t++) packed /= (uint32_t)radix;
                mvsyms[i] = ((packed % (uint32_t)radix) << b) | get(base + hw + (uint64_t)r * b, b);
            }
        }
    }
    std::vector<NcOut> ncs((size_t)g.n_nc);
    int64_t nc = 0, mvpos = 0;
    std::vector<int> lv((size_t)g.B * g.B);
    int err = HMLFC_OK;
    for (int l = g.L - 1; l >= 0; l--)
        for (int a = 0; a < g.gu[l]; a++)
            for (int b = 0; b < g.gv[l]; b++)
                for (int c = 0; c < 3; c++, nc++) {
                    NcOut &o = ncs[nc];
                    o.blocks.assign(g.nblocks, BlockOut());
                    const bool ref = (a % 2 == 0) && (b % 2 == 0);
                    if (!ref && g.mc) {
                        o.mv.assign(mvsyms.begin() + mvpos, mvsyms.begin() + mvpos + g.nblocks);
                        mvpos += g.nblocks;
                    }
                    const float *cp = h_coeff + (size_t)nc * plane;
                    for (int k = 0; k < g.nblocks; k++) {
                        const int x0 = (k % g.nbx) * g.B, y0 = (k / g.nbx) * g.B;
                        const int bw = std::min(g.B, g.W - x0), bh = std::min(g.B, g.H - y0);
                        bool any = false;
                        int n = 0;
                        for (int y = y0; y < y0 + bh; y++)
                            for (int x = x0; x < x0 + bw; x++, n++) {
                                const double v = std::floor((double)cp[(size_t)y * g.W + x] / g.q + 0.5);
                                if (!(std::fabs(v) * g.q <= (double)kCoefLimit)) err = HMLFC_E_UNSUPPORTED;
                                lv[n] = std::fabs(v) * g.q <= (double)kCoefLimit ? (int)v : 0;
                                any |= lv[n] != 0;
                            }
                        if (any) {
                            o.blocks[k].sig = true;
                            make_record(lv.data(), n, o.blocks[k].rec);
                        }
                    }
                }
    if (err != HMLFC_OK) return fail(err, "coefficient beyond the supported range");
    return serialise(g, roots, ncs, h_out, nbytes);
}
