// Compulsory traffic of a render: the bytes a view's rays must move at least
// once (a measurement aid for the roofline, host threads only).
//
// Per view: FP32 output (12 B per pixel) + 2 B per distinct root pixel of each
// channel plane (6 B per sample without chroma sub-sampling) + per
// distinct predictive block (16 B group entry once per group, 2 B offset and
// the record if significant, the motion-vector symbol's bits) + per distinct
// significant reference block reached directly or by a motion-compensation
// tap (B * B * 2 B resident tile + 4 B table entry).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <cstring>
#include <vector>

#include "hmlfc_host.h"

using namespace hmlfc;

namespace {

struct Counter {
    const Geometry &g;
    const uint8_t *bytes;
    std::vector<uint32_t> mvw;   // padded copy of the motion-vector words
    double mv_bits = 0.0;

    Counter(const Geometry &geo, const uint8_t *b) : g(geo), bytes(b) {
        if (g.mc) {
            const uint32_t *w = reinterpret_cast<const uint32_t *>(b + g.off_mvs);
            mvw.assign(w, w + g.n_mvw);
            mvw.push_back(0);
            mvw.push_back(0);
            mv_bits = (double)bise_bits(g.mv_mode, g.mv_b, 15) / 15.0;
        }
    }

    uint32_t field(uint64_t pos, int w) const {
        if (w == 0) return 0u;
        const uint64_t k = pos >> 5;
        const uint64_t v = (((uint64_t)mvw[k + 1] << 32) | mvw[k]) >> (pos & 31u);
        return (uint32_t)(v & ((1ull << w) - 1));
    }

    uint32_t mv_symbol(uint64_t i) const {
        const int mode = g.mv_mode, b = g.mv_b;
        if (mode == 0) return field(i * (uint64_t)b, b);
        const int per = mode == 1 ? 5 : 3, radix = mode == 1 ? 3 : 5, hw = mode == 1 ? 8 : 7;
        const uint64_t base = (i / per) * (uint64_t)(hw + per * b);
        const int r = (int)(i % per);
        uint32_t packed = field(base, hw);
        for (int t = 0; t < r; t++) packed /= (uint32_t)radix;
        return ((packed % (uint32_t)radix) << b) | field(base + hw + (uint64_t)r * b, b);
    }

    // Record size in bytes of block k of node-channel nc, or -1 if insignificant.
    int64_t record_bytes(int64_t nc, int k) const {
        const uint8_t *ge = bytes + g.off_groups + ((size_t)nc * g.ngroups + k / 32) * 16;
        const uint32_t bitmap = rd32(ge);
        const int r = k % 32;
        if (!((bitmap >> r) & 1u)) return -1;
        const int rank = __builtin_popcount(bitmap & ((1u << r) - 1u));
        uint16_t off;
        std::memcpy(&off, bytes + g.off_offs + 2 * ((size_t)rd32(ge + 8) + rank), 2);
        const uint32_t hdr = rd32(bytes + g.off_recs + 4 * ((size_t)rd32(ge + 4) + off));
        const int c = (int)(nc % 3);                            // the node-channel's channel: its block grid
        const int x0 = (k % g.cnbx[c]) * g.B, y0 = (k / g.cnbx[c]) * g.B;
        const int bw = std::min(g.B, g.cW[c] - x0), bh = std::min(g.B, g.cH[c] - y0);
        return 4 * (1 + (int64_t)((bise_bits((hdr >> 21) & 3, (hdr >> 16) & 31, (uint64_t)bw * bh) + 31) / 32));
    }
};

void nb(double c, int n, int &i0, int &i1, double &f) {
    const double cc = std::fmin(std::fmax(c, -1.0), (double)n);
    const double fl = std::floor(cc);
    const int k = (int)fl;
    i0 = std::min(std::max(k, 0), n - 1);
    i1 = std::min(std::max(k + 1, 0), n - 1);
    f = cc - fl;
}

// Seen-sets as atomic bitsets, so that several views can share them (the
// union over a call) while host threads count in parallel.
struct Bits {
    std::unique_ptr<std::atomic<uint64_t>[]> w;
    explicit Bits(size_t n) : w(new std::atomic<uint64_t>[(n + 63) / 64]) {
        for (size_t i = 0; i < (n + 63) / 64; i++) w[i].store(0, std::memory_order_relaxed);
    }
    // true if the bit was clear (first visit)
    bool set(size_t k) {
        const uint64_t m = 1ull << (k & 63);
        return !(w[k >> 6].fetch_or(m, std::memory_order_relaxed) & m);
    }
};

struct Seen {
    Bits sample, root, blk, grp;
    explicit Seen(const Geometry &g)
        : sample((size_t)g.nu * g.nv * g.W * g.H), root((size_t)g.n_roots * g.npx),
          blk((size_t)g.n_nc * g.nblocks), grp((size_t)g.n_nc * g.ngroups) {}
};

// Bytes first reached by view V (all of its bytes when `seen` is fresh).  At
// a progressive-decode level lod a sample of camera (i, j) is its level-lod
// node's reconstruction: the representative camera stands for it and only
// levels L-1 .. lod are reached.
double count_view(const Counter &C, const hmlfc_view &V, Seen &seen, int lod = 0, bool with_output = true) {
    const Geometry &g = C.g;
    const size_t plane = (size_t)g.W * g.H;
    double acc = with_output ? (double)V.width * V.height * 12.0 : 0.0;
    const double tile_bytes = (double)g.B * g.B * 2.0 + 4.0;
    auto nc_of = [&](int l, int a, int b, int c) { return g.nc_base[l] + ((int64_t)a * g.gv[l] + b) * 3 + c; };
    auto touch_ref = [&](int64_t nc, int k) {
        if (seen.blk.set((size_t)nc * g.nblocks + k) && C.record_bytes(nc, k) >= 0) acc += tile_bytes;
    };
    for (int py = 0; py < V.height; py++)
        for (int px = 0; px < V.width; px++) {
            const double X = px + 0.5, Y = py + 0.5;
            const float *h = V.H_uv, *hs = V.H_st;
            const double wu = (double)h[6] * X + (double)h[7] * Y + (double)h[8];
            const double u = ((double)h[0] * X + (double)h[1] * Y + (double)h[2]) / wu;
            const double v = ((double)h[3] * X + (double)h[4] * Y + (double)h[5]) / wu;
            const double ws = (double)hs[6] * X + (double)hs[7] * Y + (double)hs[8];
            const double s = ((double)hs[0] * X + (double)hs[1] * Y + (double)hs[2]) / ws;
            const double t = ((double)hs[3] * X + (double)hs[4] * Y + (double)hs[5]) / ws;
            int ii[2], jj[2], xx[2], yy[2];
            double f;
            nb(u, g.nu, ii[0], ii[1], f);
            nb(v, g.nv, jj[0], jj[1], f);
            nb(s, g.W, xx[0], xx[1], f);
            nb(t, g.H, yy[0], yy[1], f);
            for (int q = 0; q < 16; q++) {
                const int i = (ii[q >> 3] >> lod) << lod, j = (jj[(q >> 2) & 1] >> lod) << lod;
                const int x = xx[(q >> 1) & 1], y = yy[q & 1];
                const size_t sk = ((size_t)i * g.nv + j) * plane + (size_t)y * g.W + x;
                if (!seen.sample.set(sk)) continue;
                const size_t root_node = (size_t)(i >> g.L) * g.gv[g.L] + (j >> g.L);
                for (int c = 0; c < 3; c++) {
                    // the sample's pixel in channel c's plane (half resolution for sub-sampled chroma)
                    const bool half = g.sub && c > 0;
                    const int xc = half ? x >> 1 : x, yc = half ? y >> 1 : y;
                    if (seen.root.set(root_node * g.npx + g.coff[c] + (size_t)yc * g.cW[c] + xc)) acc += 2.0;
                    const int k = (yc / g.B) * g.cnbx[c] + xc / g.B;
                    for (int l = lod; l < g.L; l++) {
                        const int a = i >> l, b = j >> l;
                        const bool ref = (a % 2 == 0) && (b % 2 == 0);
                        const int64_t nc = nc_of(l, a, b, c);
                        if (ref) {
                            touch_ref(nc, k);
                            continue;
                        }
                        const size_t key = (size_t)nc * g.nblocks + k;
                        if (seen.blk.set(key)) {
                            if (seen.grp.set((size_t)nc * g.ngroups + k / 32)) acc += 16.0;
                            const int64_t rb = C.record_bytes(nc, k);
                            if (rb >= 0) acc += 2.0 + (double)rb;
                            acc += C.mv_bits / 8.0;
                        }
                        if (!g.mc) continue;
                        // predictive node rank of (l, a, b) in breadth-first order; its symbols start at
                        // rank * mv_node, channel c's at mv_coff[c]
                        const int gv = g.gv[l];
                        const int64_t before = (int64_t)((a + 1) / 2) * ((gv + 1) / 2) + ((a % 2 == 0) ? (b + 1) / 2 : 0);
                        const int64_t pnode = g.pred_base[l] / 3 + ((int64_t)a * gv + b - before);
                        const uint32_t sym = C.mv_symbol((uint64_t)pnode * g.mv_node + g.mv_coff[c] + k);
                        const int mvx = (int)((sym >> 1) / (uint32_t)g.side) - 4 * g.Ws;
                        const int mvy = (int)((sym >> 1) % (uint32_t)g.side) - 4 * g.Ws;
                        const int Xq = 4 * xc + mvx, Yq = 4 * yc + mvy;
                        const int x0 = Xq >> 2, y0 = Yq >> 2;
                        const int xa = std::min(std::max(x0, 0), g.cW[c] - 1), xb = std::min(std::max(x0 + 1, 0), g.cW[c] - 1);
                        const int ya = std::min(std::max(y0, 0), g.cH[c] - 1), yb = std::min(std::max(y0 + 1, 0), g.cH[c] - 1);
                        const int64_t rnc = nc_of(l, a & ~1, b & ~1, c);
                        const int tx[4] = {xa, xb, xa, xb}, ty[4] = {ya, ya, yb, yb};
                        for (int tp = 0; tp < 4; tp++) touch_ref(rnc, (ty[tp] / g.B) * g.cnbx[c] + tx[tp] / g.B);
                    }
                }
            }
        }
    return acc;
}

}  // namespace

extern "C" int hmlfc_touched_bytes(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views,
                                   int n_views, double *h_bytes) {
    if (!streams || n_streams < 1 || n_streams > HMLFC_MAX_STREAMS || n_views < 0 || (n_views && (!h_views || !h_bytes)))
        return fail(HMLFC_E_INVALID_ARG, "bad arguments");
    std::vector<Counter> counters;
    counters.reserve(n_streams);
    for (int k = 0; k < n_streams; k++) {
        if (!streams[k]) return fail(HMLFC_E_INVALID_ARG, "stream %d is NULL", k);
        counters.emplace_back(streams[k]->g, streams[k]->bytes.data());
    }
    for (int v = 0; v < n_views; v++)
        if (h_views[v].lf < 0 || h_views[v].lf >= n_streams || h_views[v].width < 0 || h_views[v].height < 0)
            return fail(HMLFC_E_INVALID_ARG, "view %d", v);
    parallel_for(n_views, 0, [&](int64_t v) {
        Seen seen(streams[h_views[v].lf]->g);
        h_bytes[v] = count_view(counters[h_views[v].lf], h_views[v], seen);
    });
    return HMLFC_OK;
}

extern "C" int hmlfc_touched_bytes_union(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views,
                                         int n_views, double *h_total, double *h_cam_blocks) {
    return hmlfc_touched_bytes_union_lod(streams, n_streams, h_views, n_views, 0, h_total, h_cam_blocks);
}

extern "C" int hmlfc_touched_bytes_union_lod(const hmlfc_stream *const *streams, int n_streams,
                                             const hmlfc_view *h_views, int n_views, int level, double *h_total,
                                             double *h_cam_blocks) {
    if (!streams || n_streams < 1 || n_streams > HMLFC_MAX_STREAMS || n_views < 0 || !h_total ||
        (n_views && !h_views))
        return fail(HMLFC_E_INVALID_ARG, "bad arguments");
    for (int k = 0; k < n_streams; k++)
        if (streams[k] && (level < 0 || level > streams[k]->g.L))
            return fail(HMLFC_E_INVALID_ARG, "level %d outside 0..%d", level, streams[k]->g.L);
    std::vector<Counter> counters;
    std::vector<std::unique_ptr<Seen>> seen;
    for (int k = 0; k < n_streams; k++) {
        if (!streams[k]) return fail(HMLFC_E_INVALID_ARG, "stream %d is NULL", k);
        counters.emplace_back(streams[k]->g, streams[k]->bytes.data());
        seen.emplace_back(new Seen(streams[k]->g));
    }
    for (int v = 0; v < n_views; v++)
        if (h_views[v].lf < 0 || h_views[v].lf >= n_streams || h_views[v].width < 0 || h_views[v].height < 0)
            return fail(HMLFC_E_INVALID_ARG, "view %d", v);
    std::vector<double> part(n_views, 0.0);
    parallel_for(n_views, 0, [&](int64_t v) {
        part[v] = count_view(counters[h_views[v].lf], h_views[v], *seen[h_views[v].lf], level);
    });
    double t = 0.0;
    for (double p : part) t += p;
    *h_total = t;
    if (h_cam_blocks) {
        // distinct (camera, block) pairs holding a reached sample
        double nb = 0.0;
        for (int k = 0; k < n_streams; k++) {
            const Geometry &g = streams[k]->g;
            const size_t plane = (size_t)g.W * g.H;
            for (int64_t cam = 0; cam < (int64_t)g.nu * g.nv; cam++)
                for (int blk = 0; blk < g.nblocks; blk++) {
                    const int x0 = (blk % g.nbx) * g.B, y0 = (blk / g.nbx) * g.B;
                    const int bw = std::min(g.B, g.W - x0), bh = std::min(g.B, g.H - y0);
                    bool any = false;
                    for (int y = y0; y < y0 + bh && !any; y++)
                        for (int x = x0; x < x0 + bw && !any; x++) {
                            const size_t sk = (size_t)cam * plane + (size_t)y * g.W + x;
                            any = (seen[k]->sample.w[sk >> 6].load(std::memory_order_relaxed) >> (sk & 63)) & 1u;
                        }
                    nb += any ? 1.0 : 0.0;
                }
        }
        *h_cam_blocks = nb;
    }
    return HMLFC_OK;
}
