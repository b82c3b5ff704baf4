// Host-only internal definitions of the product library (stream geometry
// and the stream object); never used by the CPU oracle.
#pragma once

#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>

#include "hmlfc_internal.h"

namespace hmlfc {

// Geometry derived from a stream header.
struct Geometry {
    int nu, nv, W, H, L, B, Ws, q, t_ref, t_pred, mc, mv_mode, mv_b;
    int nbx, nby, nblocks, ngroups, side;
    int gu[kMaxLevels + 1], gv[kMaxLevels + 1];
    int64_t nc_base[kMaxLevels], ref_base[kMaxLevels], pred_base[kMaxLevels];
    int64_t n_nc, n_ref_nc, n_pred_nc, n_roots;
    // chroma sub-sampling (Sec. 4.5): sub = 1 codes Co and Cg at ceil(W/2) x
    // ceil(H/2); per channel its plane size and block grid, the offset of its
    // plane within one root's planes (npx values per root), and the offset of
    // its blocks' motion-vector symbols within one predictive node's
    // (mv_node symbols per node)
    int sub;
    int cW[3], cH[3], cnbx[3], cnby[3], cnb[3];
    int64_t coff[3], npx, mv_coff[3], mv_node;
    uint32_t n_sig, n_recw, n_mv, n_mvw;
    uint32_t off_roots, off_groups, off_offs, off_recs, off_mvs, total;
};

// Set the thread-local error message and return `code`.
int fail(int code, const char *fmt, ...);

// Parse and check a header (sizes, counts, section layout) into g.
int parse_header(const uint8_t *p, size_t n, Geometry &g);

inline uint32_t rd32(const uint8_t *p) {
    uint32_t v;
    std::memcpy(&v, p, 4);
    return v;
}

// BISE sizes (Sec. 4.6): bits of n values of alphabet mode/b.
inline uint64_t bise_bits(int mode, int b, uint64_t n) {
    if (mode == 0) return n * (uint64_t)b;
    if (mode == 1) return ((n + 4) / 5) * (uint64_t)(8 + 5 * b);
    return ((n + 2) / 3) * (uint64_t)(7 + 3 * b);
}

inline uint64_t bise_alphabet(int mode, int b) { return (uint64_t)(mode == 0 ? 1 : mode == 1 ? 3 : 5) << b; }

// Smallest alphabet N in {2^b, 3*2^b, 5*2^b} with N >= range.
inline void bise_choose(uint64_t range, int &mode, int &b) {
    int bp = 0, bt = 0, bq = 0;
    while ((1ull << bp) < range) bp++;
    while ((3ull << bt) < range) bt++;
    while ((5ull << bq) < range) bq++;
    const uint64_t np = 1ull << bp, nt = 3ull << bt, nq = 5ull << bq;
    if (np <= nt && np <= nq) { mode = 0; b = bp; }
    else if (nt <= nq) { mode = 1; b = bt; }
    else { mode = 2; b = bq; }
}

// Geometry of a stream about to be encoded (header fields, level grids and
// breadth-first node-channel bases; no section offsets or counts).
void fill_geometry(Geometry &g, int nu, int nv, int W, int H, int L, int B, int Ws, int q, int tr, int tp, int mc,
                   int sub = 0);

// The per-channel fields of g from W, H, B and sub.
void fill_channels(Geometry &g);

// Run fn(item) for item in [0, n) on up to `threads` host threads.
void parallel_for(int64_t n, int threads, const std::function<void(int64_t)> &fn);

}  // namespace hmlfc

struct hmlfc_stream {
    int device = 0;
    hmlfc::Geometry g{};
    hmlfc::DevStream ds{};
    void *d_mem = nullptr;
    size_t d_bytes = 0;
    std::vector<uint8_t> bytes;      // host copy of the stream (re-encoding, counting)
    int64_t n_tiles = 0;
    int64_t n_ptiles = 0;           // predictive residual tiles (significant predictive blocks)
    std::vector<uint32_t> ref_tab;   // host copy of the tile table
};

struct hmlfc_server {
    const hmlfc_stream *s = nullptr;
    uint32_t capacity = 0;
    uint32_t call = 0;                 // epoch of the last render call
    int64_t n_keys = 0, n_ck = 0;
    void *d_mem = nullptr;
    size_t bytes = 0;
    uint8_t *flags = nullptr;
    uint32_t *slotmap = nullptr, *owner = nullptr, *epoch = nullptr, *clock = nullptr;
    unsigned long long *counters = nullptr, *totals = nullptr;
    uint4 *items = nullptr;
    uint32_t *cache = nullptr;
};
