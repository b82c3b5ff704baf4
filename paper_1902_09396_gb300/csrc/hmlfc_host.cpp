// Host side of the HMLFC library: stream parsing and validation, device
// residency (Sec. 4.8.2), and the C ABI entry points that launch the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hmlfc_host.h"

#include <nvtx3/nvToolsExt.h>

using namespace hmlfc;

namespace {

// A named range on the host timeline (NVTX; free when no profiler listens):
// the load, render, decode and serve calls of the library.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

thread_local std::string g_err;
int g_render_path = 0;                      // 0 cached blocks, 1 direct per ray, 2 per-tile staging
size_t g_cache_bytes = (size_t)8 << 30;     // cap on the scratch of one cached render call: index and camera images
cudaEvent_t g_phase_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // optional phase markers of the cached render

struct BatchTuning {
    int tile_shape = 0;                   // 0: 16x16, 1: 32x8, 2: 8x8 rays per tile
    int group = 4;                        // decode items per pass
    int ctas_per_sm = 8;                  // persistent CTAs per SM
    size_t cache_bytes = (size_t)2 << 30; // decoded-block cache of one batched call
} g_batch;

// Stream-ordered scratch of the render calls comes from one library pool per
// device that keeps the memory it has mapped (release threshold: never), so
// that back-to-back calls reuse it instead of mapping it again after each
// synchronisation.  Falls back to the device's default pool.
cudaError_t lib_malloc_async(void **p, size_t n, int device, cudaStream_t st) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if ((int)pools.size() <= device) pools.resize(device + 1, nullptr);
        if (!pools[device]) {
            cudaMemPoolProps props;
            std::memset(&props, 0, sizeof props);
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            if (cudaMemPoolCreate(&pools[device], &props) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
            } else {
                cudaGetLastError();
                pools[device] = nullptr;
            }
        }
        pool = pools[device];
    }
    return pool ? cudaMallocFromPoolAsync(p, n, pool, st) : cudaMallocAsync(p, n, st);
}

void phase_mark(int k, cudaStream_t st) {
    if (g_phase_ev[k]) cudaEventRecord(g_phase_ev[k], st);
}

}  // namespace

int hmlfc::fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace {

int cuda_fail(cudaError_t e, const char *what) {
    return fail(HMLFC_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

void hmlfc::parallel_for(int64_t n, int threads, const std::function<void(int64_t)> &fn) {
    if (n <= 0) return;
    int hw = (int)std::thread::hardware_concurrency();
    if (threads <= 0) threads = hw > 0 ? hw : 1;
    threads = (int)std::min<int64_t>(threads, n);
    if (threads <= 1) {
        for (int64_t i = 0; i < n; i++) fn(i);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; t++)
        pool.emplace_back([&] {
            for (int64_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) fn(i);
        });
    for (auto &th : pool) th.join();
}

int hmlfc::parse_header(const uint8_t *p, size_t n, Geometry &g) {
    if (!p || n < (size_t)kHeaderWords * 4) return fail(HMLFC_E_CORRUPT, "stream shorter than its header");
    uint32_t h[kHeaderWords];
    for (int i = 0; i < kHeaderWords; i++) h[i] = rd32(p + 4 * i);
    if (h[0] != kMagic) return fail(HMLFC_E_CORRUPT, "bad magic");
    if (h[1] != kVersion) return fail(HMLFC_E_UNSUPPORTED, "stream version %u", h[1]);
    if (h[2] < 1 || h[2] > 65536 || h[3] < 1 || h[3] > 65536 || h[4] < 1 || h[4] > 65536 || h[5] < 1 ||
        h[5] > 65536)
        return fail(HMLFC_E_CORRUPT, "grid or image size out of range");
    if (h[6] < 1 || h[6] > (uint32_t)kMaxLevels) return fail(HMLFC_E_UNSUPPORTED, "tree height %u", h[6]);
    if (h[7] < 1 || h[7] > (uint32_t)kMaxBlock) return fail(HMLFC_E_UNSUPPORTED, "block size %u", h[7]);
    if (h[8] > 64) return fail(HMLFC_E_UNSUPPORTED, "search window %u", h[8]);
    if (h[9] < 1 || h[9] > (uint32_t)kCoefLimit) return fail(HMLFC_E_UNSUPPORTED, "quantiser step %u", h[9]);
    if (h[12] > 3) return fail(HMLFC_E_CORRUPT, "flags");
    if ((h[12] & 2u) && (h[7] % 2) != 0) return fail(HMLFC_E_CORRUPT, "sub-sampled chroma needs an even block size");
    g.nu = (int)h[2]; g.nv = (int)h[3]; g.W = (int)h[4]; g.H = (int)h[5]; g.L = (int)h[6]; g.B = (int)h[7];
    g.Ws = (int)h[8]; g.q = (int)h[9]; g.t_ref = (int)h[10]; g.t_pred = (int)h[11];
    g.mc = (int)(h[12] & 1u);
    g.sub = (int)((h[12] >> 1) & 1u);
    g.mv_mode = (int)h[13]; g.mv_b = (int)h[14];
    g.nbx = (g.W + g.B - 1) / g.B;
    g.nby = (g.H + g.B - 1) / g.B;
    g.nblocks = g.nbx * g.nby;
    g.ngroups = (g.nblocks + 31) / 32;
    g.side = 8 * g.Ws + 1;
    for (int l = 0; l <= g.L; l++) {
        g.gu[l] = (g.nu + (1 << l) - 1) >> l;
        g.gv[l] = (g.nv + (1 << l) - 1) >> l;
    }
    int64_t nc = 0, rr = 0, pr = 0;
    for (int l = g.L - 1; l >= 0; l--) {
        g.nc_base[l] = nc;
        g.ref_base[l] = rr;
        g.pred_base[l] = pr;
        const int64_t nodes = (int64_t)g.gu[l] * g.gv[l];
        const int64_t refs = (int64_t)((g.gu[l] + 1) / 2) * ((g.gv[l] + 1) / 2);
        nc += 3 * nodes;
        rr += 3 * refs;
        pr += 3 * (nodes - refs);
    }
    g.n_nc = nc;
    g.n_ref_nc = rr;
    g.n_pred_nc = pr;
    g.n_roots = (int64_t)g.gu[g.L] * g.gv[g.L];
    fill_channels(g);
    if (nc * g.nblocks >= (int64_t)INT32_MAX || (int64_t)g.W * g.H * 3 * std::max<int64_t>(nc, g.n_roots) >= (1ll << 40))
        return fail(HMLFC_E_UNSUPPORTED, "light field too large for one stream object");
    if (h[15] != (uint32_t)nc || h[16] != (uint32_t)g.ngroups) return fail(HMLFC_E_CORRUPT, "node-channel count");
    g.n_sig = h[17]; g.n_recw = h[18]; g.n_mv = h[19]; g.n_mvw = h[20];
    g.off_roots = h[21]; g.off_groups = h[22]; g.off_offs = h[23]; g.off_recs = h[24]; g.off_mvs = h[25];
    g.total = h[26];
    if ((uint64_t)g.total != (uint64_t)n) return fail(HMLFC_E_CORRUPT, "stream length %zu, header says %u", n, g.total);
    if (g.mc) {
        int md, bb;
        bise_choose(2ull * g.side * g.side, md, bb);
        if (md != g.mv_mode || bb != g.mv_b) return fail(HMLFC_E_CORRUPT, "motion-vector alphabet");
        if ((uint64_t)g.n_mv != (uint64_t)(g.n_pred_nc / 3) * g.mv_node) return fail(HMLFC_E_CORRUPT, "motion-vector count");
        if ((uint64_t)g.n_mvw != (bise_bits(md, bb, g.n_mv) + 31) / 32) return fail(HMLFC_E_CORRUPT, "motion-vector words");
    } else if (g.n_mv != 0 || g.n_mvw != 0) {
        return fail(HMLFC_E_CORRUPT, "motion vectors without motion compensation");
    }
    struct Sec { uint64_t off, len; } secs[5] = {
        {g.off_roots, (uint64_t)g.n_roots * g.npx * 2},
        {g.off_groups, (uint64_t)nc * g.ngroups * 16},
        {g.off_offs, (uint64_t)g.n_sig * 2},
        {g.off_recs, (uint64_t)g.n_recw * 4},
        {g.off_mvs, (uint64_t)g.n_mvw * 4}};
    uint64_t prev_end = (uint64_t)kHeaderWords * 4;
    for (auto &s : secs) {
        if (s.off % 4 != 0 || s.off < prev_end || s.off + s.len > n) return fail(HMLFC_E_CORRUPT, "section layout");
        prev_end = s.off + s.len;
    }
    return HMLFC_OK;
}

namespace {

// Walk the block index; check every significant block's record against the
// stream bounds and the coefficient limit; build the reference tile table
// and the record list of the reference tiles (tile_src) and of the
// predictive residual tiles (ptile_src, {record, width, height, 0} each),
// with the first residual tile of every group (gtile, 0 for the groups of
// reference node-channels).
int validate_index(const uint8_t *p, const Geometry &g, std::vector<uint32_t> &ref_tab, std::vector<uint32_t> &tile_src,
                   std::vector<uint32_t> &ptile_src, std::vector<uint32_t> &gtile) {
    const uint8_t *groups = p + g.off_groups;
    const uint8_t *offs = p + g.off_offs;
    const uint8_t *recs = p + g.off_recs;
    ref_tab.assign((size_t)g.n_ref_nc * g.nblocks, 0u);
    tile_src.clear();
    ptile_src.clear();
    gtile.assign((size_t)g.n_nc * g.ngroups, 0u);
    uint64_t sig = 0;
    int64_t nc = 0, rr = 0;
    for (int l = g.L - 1; l >= 0; l--)
        for (int a = 0; a < g.gu[l]; a++)
            for (int b = 0; b < g.gv[l]; b++) {
                const bool ref = (a % 2 == 0) && (b % 2 == 0);
                for (int c = 0; c < 3; c++, nc++) {
                    for (int gi = 0; gi < g.ngroups; gi++) {
                        const uint8_t *ge = groups + ((size_t)nc * g.ngroups + gi) * 16;
                        const uint32_t bitmap = rd32(ge), rbase = rd32(ge + 4), obase = rd32(ge + 8);
                        // the channel's blocks (fewer for sub-sampled chroma, whose last groups stay empty)
                        const int valid = std::max(0, std::min(32, g.cnb[c] - gi * 32));
                        if (valid < 32 && (valid == 0 ? bitmap : bitmap >> valid) != 0)
                            return fail(HMLFC_E_CORRUPT, "bitmap past the last block");
                        if ((uint64_t)obase != sig) return fail(HMLFC_E_CORRUPT, "block-offset base");
                        if (!ref) gtile[(size_t)nc * g.ngroups + gi] = (uint32_t)(ptile_src.size() / 4);
                        for (int r = 0; r < valid; r++) {
                            if (!((bitmap >> r) & 1u)) continue;
                            if (sig >= g.n_sig) return fail(HMLFC_E_CORRUPT, "more significant blocks than offsets");
                            uint16_t off;
                            std::memcpy(&off, offs + 2 * sig, 2);
                            sig++;
                            const uint64_t rec = (uint64_t)rbase + off;
                            if (rec >= g.n_recw) return fail(HMLFC_E_CORRUPT, "record outside the stream");
                            const uint32_t hdr = rd32(recs + 4 * rec);
                            const int mode = (int)((hdr >> 21) & 3u), bb = (int)((hdr >> 16) & 31u);
                            if (mode == 3 || bb > 16 || (hdr >> 23) != 0) return fail(HMLFC_E_CORRUPT, "record header");
                            const int k = gi * 32 + r;
                            const int x0 = (k % g.cnbx[c]) * g.B, y0 = (k / g.cnbx[c]) * g.B;
                            const int bw = std::min(g.B, g.cW[c] - x0), bh = std::min(g.B, g.cH[c] - y0);
                            const uint64_t words = 1 + (bise_bits(mode, bb, (uint64_t)bw * bh) + 31) / 32;
                            if (rec + words > g.n_recw) return fail(HMLFC_E_CORRUPT, "record overruns the stream");
                            const int64_t m = (int16_t)(hdr & 0xFFFFu);
                            const int64_t lo = (int64_t)g.q * m, hi = (int64_t)g.q * (m + (int64_t)bise_alphabet(mode, bb) - 1);
                            if (lo < -kCoefLimit || hi > kCoefLimit)
                                return fail(HMLFC_E_UNSUPPORTED, "coefficients beyond +-%d", kCoefLimit);
                            if (ref) {
                                tile_src.push_back((uint32_t)rec);
                                tile_src.push_back((uint32_t)bw);
                                tile_src.push_back((uint32_t)bh);
                                tile_src.push_back(0u);
                                ref_tab[(size_t)(rr + c) * g.nblocks + k] = (uint32_t)(tile_src.size() / 4);
                            } else {
                                ptile_src.push_back((uint32_t)rec);
                                ptile_src.push_back((uint32_t)bw);
                                ptile_src.push_back((uint32_t)bh);
                                ptile_src.push_back(0u);
                            }
                        }
                    }
                }
                if (ref) rr += 3;
            }
    if (sig != g.n_sig) return fail(HMLFC_E_CORRUPT, "offset count");
    return HMLFC_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int check_views(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *views, int n_views) {
    if (n_streams < 1 || n_streams > HMLFC_MAX_STREAMS || !streams)
        return fail(HMLFC_E_INVALID_ARG, "need 1..%d streams", HMLFC_MAX_STREAMS);
    for (int k = 0; k < n_streams; k++) {
        if (!streams[k]) return fail(HMLFC_E_INVALID_ARG, "stream %d is NULL", k);
        if (streams[k]->device != streams[0]->device) return fail(HMLFC_E_INVALID_ARG, "streams on different devices");
    }
    if (n_views < 0 || n_views > HMLFC_MAX_VIEWS || (n_views > 0 && !views))
        return fail(HMLFC_E_INVALID_ARG, "bad view count or view array");
    for (int v = 0; v < n_views; v++) {
        const hmlfc_view &V = views[v];
        if (V.lf < 0 || V.lf >= n_streams) return fail(HMLFC_E_INVALID_ARG, "view %d: lf %d out of range", v, V.lf);
        if (V.width < 0 || V.height < 0 || V.width > 65536 || V.height > 65536 || V.out_offset < 0)
            return fail(HMLFC_E_INVALID_ARG, "view %d: bad size or offset", v);
    }
    return HMLFC_OK;
}

// Quotient multiplier for a view's tile index: floor((2^32 - 1) / d) + 1 (0
// for d = 1), exact with __umulhi for n, d < 2^16; 1 (an impossible
// multiplier) asks the kernel for a plain division when the view has 2^16
// tiles or more.
uint32_t tile_div_magic(const hmlfc_view &V) {
    const int64_t d = (V.width + 15) / 16, n = d * ((V.height + 15) / 16);
    if (n >= 65536) return 1u;
    return d <= 1 ? 0u : (uint32_t)(0xFFFFFFFFull / (uint32_t)d) + 1u;
}

// The views of stream `lf`, in launch chunks that fit the by-value view table.
int view_chunks(const hmlfc_view *views, int n_views, int lf, std::vector<LaunchViews> &chunks,
                std::vector<int> &tiles, int per_chunk = kMaxViewsPerLaunch) {
    chunks.clear();
    tiles.clear();
    std::vector<int> idx;
    for (int v = 0; v < n_views; v++)
        if (views[v].lf == lf && views[v].width > 0 && views[v].height > 0) idx.push_back(v);
    for (size_t s = 0; s < idx.size(); s += (size_t)per_chunk) {
        chunks.emplace_back();
        LaunchViews &lv = chunks.back();
        std::memset(&lv, 0, sizeof lv);
        lv.tile_w = 16;
        lv.tile_h = 16;
        const size_t e = std::min(idx.size(), s + (size_t)per_chunk);
        int64_t t = 0;
        for (size_t k = s; k < e; k++) {
            const hmlfc_view &V = views[idx[k]];
            lv.tile_start[k - s] = (int)t;
            lv.tiles_x_magic[k - s] = tile_div_magic(V);
            lv.views[k - s] = V;
            t += (int64_t)((V.width + 15) / 16) * ((V.height + 15) / 16);
        }
        lv.n_views = (int)(e - s);
        lv.tile_start[lv.n_views] = (int)t;
        if (t >= INT32_MAX) return fail(HMLFC_E_INVALID_ARG, "too many tiles in one launch");
        tiles.push_back((int)t);
    }
    return HMLFC_OK;
}

// The next launch chunk of stream lf's views, scanning from *pos, without
// any allocation; returns the number of views in the chunk (0 at the end).
int next_chunk(const hmlfc_view *views, int n_views, int lf, int *pos, LaunchViews &lv, int &tiles) {
    std::memset(&lv, 0, sizeof lv);
    lv.tile_w = 16;
    lv.tile_h = 16;
    int64_t t = 0;
    int k = 0;
    while (*pos < n_views && k < kMaxViewsPerLaunch) {
        const hmlfc_view &V = views[*pos];
        (*pos)++;
        if (V.lf != lf || V.width <= 0 || V.height <= 0) continue;
        lv.tile_start[k] = (int)t;
        lv.tiles_x_magic[k] = tile_div_magic(V);
        lv.views[k] = V;
        k++;
        t += (int64_t)((V.width + 15) / 16) * ((V.height + 15) / 16);
        if (t >= INT32_MAX) return -1;
    }
    lv.n_views = k;
    lv.tile_start[k] = (int)t;
    tiles = (int)t;
    return k;
}

// Launch one kernel family over the views of each stream, chunk by chunk.
template <class F>
int for_view_chunks(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *views, int n_views, F launch) {
    std::vector<LaunchViews> chunks;
    std::vector<int> tiles;
    for (int lf = 0; lf < n_streams; lf++) {
        int rc = view_chunks(views, n_views, lf, chunks, tiles);
        if (rc != HMLFC_OK) return rc;
        for (size_t c = 0; c < chunks.size(); c++) {
            rc = launch(streams[lf], chunks[c], tiles[c]);
            if (rc != HMLFC_OK) return rc;
        }
    }
    return HMLFC_OK;
}

int sm_count(int device) {
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device]) return cached[device];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) n = 1;
    if (device >= 0 && device < 64) cached[device] = n;
    return n;
}

// Cached render of the views of one stream: mark the (camera, block) pairs
// the tiles reach, give each a slot of a stream-ordered scratch cache, decode
// those blocks once, then blend every ray from the cache.  Returns 1 (and
// launches nothing) when the scratch cannot be had, so the caller falls back.
// Device-to-host copies that follow each blend chunk of a render into host
// memory: after chunk c's blend, `copy` waits for it and copies that chunk's
// views from d_out to h_out, so the copies overlap the later chunks.
struct HostSink {
    float *h_out = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev = nullptr;
};

cudaError_t sink_chunk(const HostSink *sink, const LaunchViews &lv, const float *d_out, cudaStream_t st) {
    if (!sink) return cudaSuccess;
    cudaError_t e = cudaEventRecord(sink->ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sink->copy, sink->ev, 0);
    // one copy per run of views whose output ranges follow each other
    for (int v = 0; v < lv.n_views && e == cudaSuccess;) {
        const size_t first = (size_t)lv.views[v].out_offset;
        size_t end = first + (size_t)lv.views[v].width * lv.views[v].height * 3;
        int w = v + 1;
        while (w < lv.n_views && (size_t)lv.views[w].out_offset == end) {
            end += (size_t)lv.views[w].width * lv.views[w].height * 3;
            w++;
        }
        e = cudaMemcpyAsync(sink->h_out + first, d_out + first, (end - first) * sizeof(float), cudaMemcpyDeviceToHost,
                            sink->copy);
        v = w;
    }
    return e;
}

// Scratch of one cached render call: flags (one per (camera, block) pair,
// grouped by super key), the camera slots, the decode items, two counters,
// then the camera images (W x H RGB8 u32 each).
struct CachedLayout {
    size_t o_flags = 0, o_slot = 0, o_items = 0, o_count = 0, index_bytes = 0;
    int64_t n_keys = 0, n_cam = 0;
    size_t image_bytes = 0;
};

CachedLayout cached_layout(const hmlfc_stream *s) {
    const Geometry &g = s->g;
    CachedLayout c;
    c.n_cam = (int64_t)g.nu * g.nv;
    const int K = g.L < 2 ? g.L : 2;
    const int64_t n_sk = (int64_t)g.gu[K] * g.gv[K] * g.nblocks;
    c.n_keys = n_sk << (2 * K);            // flags grouped by super key, (2^K)^2 cameras each (zero-padded at edges)
    c.o_flags = 0;
    c.o_slot = up256((size_t)c.n_keys);
    c.o_items = up256(c.o_slot + (size_t)c.n_cam * 4);
    c.o_count = up256(c.o_items + (size_t)n_sk * 16);
    c.index_bytes = up256(c.o_count + 16);
    c.image_bytes = (size_t)g.W * g.H * 4;
    return c;
}

// The cached render's launches on scratch `b` laid out by `c`, with room for
// `capacity` camera images after the index.  each_chunk(f) calls f(launch
// views, tiles) for every launch chunk of the stream's views, in order, and
// returns the first error (or cudaSuccess); after each blend chunk, `sink`
// (if any) copies it.
template <class EachChunk>
int cached_launches(const hmlfc_stream *s, const DevStream &ds, const CachedLayout &c, uint8_t *b, uint32_t capacity,
                    EachChunk each_chunk, float *d_out, cudaStream_t st, const HostSink *sink, bool phases) {
    uint8_t *flags = b + c.o_flags;
    uint32_t *camslot = reinterpret_cast<uint32_t *>(b + c.o_slot);
    uint4 *items = reinterpret_cast<uint4 *>(b + c.o_items);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(b + c.o_count);
    uint32_t *cache = reinterpret_cast<uint32_t *>(b + c.index_bytes);
    if (phases) phase_mark(0, st);
    NvtxRange range("hmlfc cached render: mark, assign, decode, blend launches");
    // the scratch keeps an earlier call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)c.n_keys, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 16, st);
    if (e == cudaSuccess)
        e = each_chunk([&](const LaunchViews &lv, int t) { return launch_mark(ds, lv, t, flags, true, st); });
    if (e == cudaSuccess) e = launch_assign(ds, flags, camslot, items, counters, capacity, st);
    if (phases) phase_mark(1, st);
    if (e == cudaSuccess)
        e = launch_decode_blocks(ds, items, counters, camslot, cache, sm_count(s->device) * kDecodeCtasPerSm, st);
    if (phases) phase_mark(2, st);
    if (e == cudaSuccess)
        e = each_chunk([&](const LaunchViews &lv, int t) {
            cudaError_t r = launch_render_cached(ds, lv, t, camslot, cache, capacity >= c.n_cam, d_out, st);
            if (r == cudaSuccess) r = sink_chunk(sink, lv, d_out, st);
            return r;
        });
    if (phases) phase_mark(3, st);
    return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "cached render");
}

// Camera images that fit `budget` bytes of scratch after the index (0 when
// not even one fits).
uint32_t cached_capacity(const CachedLayout &c, size_t budget) {
    if (budget <= c.index_bytes) return 0;
    return (uint32_t)std::min<int64_t>({c.n_cam, (int64_t)((budget - c.index_bytes) / c.image_bytes), kMaxSlots});
}

int render_cached(const hmlfc_stream *s, const std::vector<LaunchViews> &chunks, const std::vector<int> &tiles,
                  float *d_out, cudaStream_t st, int lod = 0, const HostSink *sink = nullptr) {
    DevStream ds = s->ds;
    ds.lod = lod;
    const CachedLayout c = cached_layout(s);
    const uint32_t capacity = cached_capacity(c, g_cache_bytes);
    if (capacity == 0) return 1;
    const size_t total = up256(c.index_bytes + (size_t)capacity * c.image_bytes);
    void *base = nullptr;
    if (lib_malloc_async(&base, total, s->device, st) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    auto each_chunk = [&](auto f) {
        cudaError_t e = cudaSuccess;
        for (size_t k = 0; k < chunks.size() && e == cudaSuccess; k++) e = f(chunks[k], tiles[k]);
        return e;
    };
    int rc = cached_launches(s, ds, c, static_cast<uint8_t *>(base), capacity, each_chunk, d_out, st, sink, true);
    const cudaError_t ef = cudaFreeAsync(base, st);
    if (rc == HMLFC_OK && ef != cudaSuccess) rc = cuda_fail(ef, "cached render scratch");
    return rc;
}

}  // namespace

extern "C" {

const char *hmlfc_last_error(void) { return g_err.c_str(); }

int hmlfc_set_render_path(int path) {
    if (path < 0 || path > 2) return fail(HMLFC_E_INVALID_ARG, "render path %d", path);
    g_render_path = path;
    return HMLFC_OK;
}

int hmlfc_set_phase_events(void *const *events) {
    for (int k = 0; k < 4; k++) g_phase_ev[k] = events ? static_cast<cudaEvent_t>(events[k]) : nullptr;
    return HMLFC_OK;
}

int hmlfc_set_block_cache_bytes(size_t bytes) {
    g_cache_bytes = bytes;
    return HMLFC_OK;
}

int hmlfc_load_stream(const void *h_bytes, size_t nbytes, int device, void *cuda_stream, hmlfc_stream **out) {
    NvtxRange nvtx_range("hmlfc load_stream");
    if (!out) return fail(HMLFC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const uint8_t *p = static_cast<const uint8_t *>(h_bytes);
    Geometry g{};
    int rc = parse_header(p, nbytes, g);
    if (rc != HMLFC_OK) return rc;
    std::vector<uint32_t> ref_tab, tile_src, ptile_src, gtile;
    rc = validate_index(p, g, ref_tab, tile_src, ptile_src, gtile);
    if (rc != HMLFC_OK) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(HMLFC_E_INVALID_ARG, "device %d not available", device);
    DeviceGuard guard(device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    auto *s = new (std::nothrow) hmlfc_stream();
    if (!s) return fail(HMLFC_E_OOM, "host allocation");
    s->device = device;
    s->g = g;
    s->bytes.assign(p, p + nbytes);
    s->n_tiles = (int64_t)tile_src.size() / 4;
    s->n_ptiles = (int64_t)ptile_src.size() / 4;
    s->ref_tab = ref_tab;
    const int B2 = g.B * g.B;
    const int pstride = g.B + (g.B & 1);
    const uint64_t plane = (uint64_t)g.W * g.H;
    // one device allocation, carved into 256-byte aligned sections
    const size_t sz_roots = (size_t)g.n_roots * g.npx * 2;
    const size_t sz_groups = (size_t)g.n_nc * g.ngroups * 16;
    const size_t sz_offs = (size_t)g.n_sig * 2 + 4;
    const size_t sz_recs = ((size_t)g.n_recw + 2) * 4;
    const size_t sz_mvs = ((size_t)g.n_mvw + 2) * 4;
    const size_t sz_tab = ref_tab.size() * 4 + 4;
    const size_t sz_tiles = (size_t)(s->n_tiles + 1) * B2 * 2;
    const size_t sz_src = tile_src.size() * 4 + 16;
    const size_t sz_planes = (size_t)g.n_ref_nc * plane * 2 + 256;   // padded: a pixel pair may read one past
    const size_t sz_ptiles = (size_t)(s->n_ptiles + 1) * g.B * pstride * 2;   // tile 0: zeros
    const size_t sz_psrc = ptile_src.size() * 4 + 16;
    size_t o_roots = 0, o_groups = up256(o_roots + sz_roots), o_offs = up256(o_groups + sz_groups),
           o_recs = up256(o_offs + sz_offs), o_mvs = up256(o_recs + sz_recs), o_tab = up256(o_mvs + sz_mvs),
           o_tiles = up256(o_tab + sz_tab), o_src = up256(o_tiles + sz_tiles), o_status = up256(o_src + sz_src),
           o_planes = up256(o_status + 256), o_ptiles = up256(o_planes + sz_planes),
           o_psrc = up256(o_ptiles + sz_ptiles), total = up256(o_psrc + sz_psrc);
    cudaError_t e = cudaMalloc(&s->d_mem, total);
    if (e != cudaSuccess) {
        delete s;
        cudaGetLastError();
        return fail(HMLFC_E_OOM, "device allocation of %zu bytes: %s", total, cudaGetErrorString(e));
    }
    s->d_bytes = total;
    // staging image of the device layout, one copy
    std::vector<uint8_t> img(o_tiles, 0);
    std::memcpy(img.data() + o_roots, p + g.off_roots, sz_roots);
    std::memcpy(img.data() + o_groups, p + g.off_groups, sz_groups);
    for (size_t e = 0; e < gtile.size(); e++)      // word 3 of each group entry: its residual tiles' first rank
        std::memcpy(img.data() + o_groups + e * 16 + 12, &gtile[e], 4);
    std::memcpy(img.data() + o_offs, p + g.off_offs, (size_t)g.n_sig * 2);
    std::memcpy(img.data() + o_recs, p + g.off_recs, (size_t)g.n_recw * 4);
    std::memcpy(img.data() + o_mvs, p + g.off_mvs, (size_t)g.n_mvw * 4);
    if (!ref_tab.empty()) std::memcpy(img.data() + o_tab, ref_tab.data(), ref_tab.size() * 4);
    uint8_t *base = static_cast<uint8_t *>(s->d_mem);
    DevStream &ds = s->ds;
    ds.nu = g.nu; ds.nv = g.nv; ds.W = g.W; ds.H = g.H; ds.L = g.L; ds.B = g.B; ds.Ws = g.Ws; ds.q = g.q;
    ds.mc = g.mc; ds.mv_mode = g.mv_mode; ds.mv_b = g.mv_b; ds.nbx = g.nbx; ds.nby = g.nby;
    ds.nblocks = g.nblocks; ds.ngroups = g.ngroups; ds.side = g.side;
    ds.sub = g.sub;
    for (int c = 0; c < 3; c++) {
        ds.cW[c] = g.cW[c]; ds.cH[c] = g.cH[c]; ds.cnbx[c] = g.cnbx[c]; ds.cnb[c] = g.cnb[c];
        ds.roff[c] = (int)g.coff[c];
        ds.mv_coff[c] = (int)g.mv_coff[c];
    }
    ds.rnpx = g.npx;
    ds.mv_node = (int)g.mv_node;
    ds.lim_roots = (int64_t)g.n_roots * g.npx;
    ds.lim_groups = g.n_nc * g.ngroups;
    ds.lim_offs = g.n_sig;
    ds.lim_recs = (int64_t)g.n_recw + 2;          // with the padding words a funnel-shift read may touch
    ds.lim_mvs = (int64_t)g.n_mvw + 2;
    ds.lim_ref_tab = g.n_ref_nc * g.nblocks;
    ds.lim_tiles = (s->n_tiles + 1) * B2;
    ds.lim_planes = (int64_t)g.n_ref_nc * (int64_t)plane + 128;   // + the padding (256 B)
    ds.lim_mv = g.n_mv;
    ds.lim_ptiles = (s->n_ptiles + 1) * g.B * pstride;
    ds.pstride = pstride;
    for (int l = 0; l <= kMaxLevels; l++) {
        ds.gu[l] = l <= g.L ? g.gu[l] : 1;
        ds.gv[l] = l <= g.L ? g.gv[l] : 1;
    }
    for (int l = 0; l < kMaxLevels; l++) {
        ds.nc_base[l] = l < g.L ? (int)g.nc_base[l] : 0;
        ds.ref_base[l] = l < g.L ? (int)g.ref_base[l] : 0;
        ds.pred_base[l] = l < g.L ? (int)g.pred_base[l] : 0;
    }
    ds.roots = reinterpret_cast<const int16_t *>(base + o_roots);
    ds.groups = reinterpret_cast<const uint4 *>(base + o_groups);
    ds.offs = reinterpret_cast<const uint16_t *>(base + o_offs);
    ds.recs = reinterpret_cast<const uint32_t *>(base + o_recs);
    ds.mvs = reinterpret_cast<const uint32_t *>(base + o_mvs);
    ds.ref_tab = reinterpret_cast<const uint32_t *>(base + o_tab);
    ds.tiles = reinterpret_cast<const int16_t *>(base + o_tiles);
    ds.status = reinterpret_cast<uint32_t *>(base + o_status);
    ds.planes = reinterpret_cast<const int16_t *>(base + o_planes);
    ds.ptiles = reinterpret_cast<const int16_t *>(base + o_ptiles);
    e = cudaMemcpyAsync(base, img.data(), img.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !tile_src.empty())
        e = cudaMemcpyAsync(base + o_src, tile_src.data(), tile_src.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !ptile_src.empty())
        e = cudaMemcpyAsync(base + o_psrc, ptile_src.data(), ptile_src.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_tiles, 0, (size_t)B2 * 2, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_status, 0, 256, st);
    if (e == cudaSuccess)
        e = launch_decode_tiles(ds, reinterpret_cast<const uint32_t *>(base + o_src), (int)s->n_tiles,
                                reinterpret_cast<int16_t *>(base + o_tiles), g.B, 1, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(base + o_ptiles, 0, (size_t)g.B * pstride * 2, st);
    if (e == cudaSuccess)
        e = launch_decode_tiles(ds, reinterpret_cast<const uint32_t *>(base + o_psrc), (int)s->n_ptiles,
                                reinterpret_cast<int16_t *>(base + o_ptiles), pstride, 1, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_planes + sz_planes - 256, 0, 256, st);
    if (e == cudaSuccess) e = launch_build_planes(ds, g.n_ref_nc, reinterpret_cast<int16_t *>(base + o_planes), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        hmlfc_free_stream(s);
        return cuda_fail(e, "loading the stream");
    }
    *out = s;
    return HMLFC_OK;
}

void hmlfc_free_stream(hmlfc_stream *s) {
    if (!s) return;
    if (s->d_mem) {
        DeviceGuard guard(s->device);
        cudaFree(s->d_mem);
    }
    delete s;
}

int hmlfc_stream_info(const hmlfc_stream *s, hmlfc_stream_info_t *out) {
    if (!s || !out) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    const Geometry &g = s->g;
    out->nu = g.nu; out->nv = g.nv; out->width = g.W; out->height = g.H; out->levels = g.L; out->block = g.B;
    out->search = g.Ws; out->qstep = g.q; out->mc = g.mc; out->n_roots = (int32_t)g.n_roots;
    out->chroma = g.sub;
    out->n_nc = g.n_nc; out->n_blocks = g.nblocks; out->n_sig = g.n_sig; out->n_ref_tiles = s->n_tiles;
    out->stream_bytes = (int64_t)s->bytes.size();
    out->device_bytes = (int64_t)s->d_bytes;
    return HMLFC_OK;
}

int hmlfc_decode_pixels_lod(const hmlfc_stream *s, const int32_t *d_coords, int64_t n, int level, uint8_t *d_rgb,
                            void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc decode_pixels");
    if (!s) return fail(HMLFC_E_INVALID_ARG, "stream is NULL");
    if (n < 0) return fail(HMLFC_E_INVALID_ARG, "negative count");
    if (level < 0 || level > s->g.L) return fail(HMLFC_E_INVALID_ARG, "level %d outside 0..%d", level, s->g.L);
    if (n == 0) return HMLFC_OK;
    if (!d_coords || !d_rgb) return fail(HMLFC_E_INVALID_ARG, "NULL buffer");
    DeviceGuard guard(s->device);
    DevStream ds = s->ds;
    ds.lod = level;
    const cudaError_t e = launch_decode_pixels(ds, d_coords, n, d_rgb, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "decode_pixels launch");
}

int hmlfc_decode_pixels(const hmlfc_stream *s, const int32_t *d_coords, int64_t n, uint8_t *d_rgb, void *cuda_stream) {
    return hmlfc_decode_pixels_lod(s, d_coords, n, 0, d_rgb, cuda_stream);
}

int hmlfc_check_status(const hmlfc_stream *s, void *cuda_stream) {
    if (!s) return fail(HMLFC_E_INVALID_ARG, "stream is NULL");
    DeviceGuard guard(s->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    uint32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, s->ds.status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v) e = cudaMemsetAsync(s->ds.status, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (v & kStatusBounds)
        return fail(HMLFC_E_CORRUPT, "a kernel index fell outside its stream array (bounds-checked build)");
    if (v & kStatusCoord) return fail(HMLFC_E_INVALID_ARG, "a decoded coordinate was outside the light field");
    return HMLFC_OK;
}

int hmlfc_render_views(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                       float *d_out, void *cuda_stream) {
    return hmlfc_render_views_lod(streams, n_streams, h_views, n_views, 0, d_out, cuda_stream);
}

int hmlfc_render_views_lod(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                           int level, float *d_out, void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc render_views");
    int rc = check_views(streams, n_streams, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    for (int k = 0; k < n_streams; k++)
        if (level < 0 || level > streams[k]->g.L)
            return fail(HMLFC_E_INVALID_ARG, "level %d outside 0..%d of stream %d", level, streams[k]->g.L, k);
    if (n_views > 0 && !d_out) return fail(HMLFC_E_INVALID_ARG, "d_out is NULL");
    if (n_views == 0) return HMLFC_OK;
    DeviceGuard guard(streams[0]->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<LaunchViews> chunks;
    std::vector<int> tiles;
    for (int lf = 0; lf < n_streams; lf++) {
        rc = view_chunks(h_views, n_views, lf, chunks, tiles);
        if (rc != HMLFC_OK) return rc;
        if (chunks.empty()) continue;
        int path = g_render_path;
        if (path == 0) {
            rc = render_cached(streams[lf], chunks, tiles, d_out, st, level);
            if (rc == HMLFC_OK) continue;
            if (rc != 1) return rc;
            path = 2;   // no scratch: per-tile staging needs none
        }
        // the per-tile staging decodes every level and full-resolution chroma only; the direct walk stops at
        // `level` and reads sub-sampled chroma
        if (level > 0 || streams[lf]->g.sub) path = 1;
        DevStream ds = streams[lf]->ds;
        ds.lod = level;
        for (size_t c = 0; c < chunks.size(); c++) {
            const cudaError_t e = launch_render(ds, chunks[c], tiles[c], d_out, path == 1 ? 1 : 0, st);
            if (e != cudaSuccess) return cuda_fail(e, "render launch");
        }
    }
    return HMLFC_OK;
}

// Render into host memory: the output is staged in device memory from the
// call's stream-ordered pool; the decode runs once for all views, then the
// blend runs in groups of kHostChunkViews views and each group is copied to
// the host on a per-device copy stream while the next group blends.
constexpr int kHostChunkViews = 8;

cudaStream_t copy_stream(int device) {
    static std::mutex mu;
    static std::vector<cudaStream_t> per_dev;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)per_dev.size() <= device) per_dev.resize(device + 1, nullptr);
    if (!per_dev[device] && cudaStreamCreateWithFlags(&per_dev[device], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        per_dev[device] = nullptr;
    }
    return per_dev[device];
}

int hmlfc_render_views_host(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                            float *h_out, void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc render_views_host");
    int rc = check_views(streams, n_streams, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    if (n_views > 0 && !h_out) return fail(HMLFC_E_INVALID_ARG, "h_out is NULL");
    if (n_views == 0) return HMLFC_OK;
    DeviceGuard guard(streams[0]->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    size_t n_out = 0;
    for (int v = 0; v < n_views; v++)
        n_out = std::max(n_out, (size_t)h_views[v].out_offset + (size_t)h_views[v].width * h_views[v].height * 3);
    HostSink sink;
    sink.h_out = h_out;
    sink.copy = copy_stream(streams[0]->device);
    if (!sink.copy) return fail(HMLFC_E_CUDA, "copy stream");
    void *dbuf = nullptr;
    cudaError_t e = lib_malloc_async(&dbuf, std::max<size_t>(n_out, 1) * sizeof(float), streams[0]->device, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HMLFC_E_OOM, "device staging of %zu output floats", n_out);
    }
    float *d_out = static_cast<float *>(dbuf);
    cudaEvent_t done = nullptr;
    e = cudaEventCreateWithFlags(&sink.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    std::vector<LaunchViews> chunks;
    std::vector<int> tiles;
    for (int lf = 0; lf < n_streams && e == cudaSuccess && rc == HMLFC_OK; lf++) {
        rc = view_chunks(h_views, n_views, lf, chunks, tiles, kHostChunkViews);
        if (rc != HMLFC_OK || chunks.empty()) continue;
        if (g_render_path == 0) {
            rc = render_cached(streams[lf], chunks, tiles, d_out, st, 0, &sink);
            if (rc == HMLFC_OK) continue;
            if (rc != 1) break;
            rc = HMLFC_OK;   // no scratch: per-tile staging needs none
        }
        for (size_t c = 0; c < chunks.size() && e == cudaSuccess; c++) {
            const int mode = (g_render_path == 1 || streams[lf]->g.sub) ? 1 : 0;   // staging: full chroma only
            e = launch_render(streams[lf]->ds, chunks[c], tiles[c], d_out, mode, st);
            if (e == cudaSuccess) e = sink_chunk(&sink, chunks[c], d_out, st);
        }
    }
    // the caller's stream waits for the last copy; the staging is freed behind it
    if (e == cudaSuccess) e = cudaEventRecord(done, sink.copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, done, 0);
    const cudaError_t ef = cudaFreeAsync(dbuf, st);
    if (sink.ev) cudaEventDestroy(sink.ev);
    if (done) cudaEventDestroy(done);
    if (rc != HMLFC_OK) return rc;
    if (e == cudaSuccess) e = ef;
    return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "render to host");
}

// Allocation-free variant of the cached render: the flags, camera slots,
// decode items and camera images live in the fixed device array set up by
// fixed_scratch() (hmlfc_kernels.cu).  Nothing is allocated, on the device
// or on the host.
int hmlfc_render_views_noalloc(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views,
                               int n_views, float *d_out, void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc render_views_noalloc");
    int rc = check_views(streams, n_streams, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    if (n_views > 0 && !d_out) return fail(HMLFC_E_INVALID_ARG, "d_out is NULL");
    if (n_views == 0) return HMLFC_OK;
    const int dev = streams[0]->device;
    DeviceGuard guard(dev);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    for (int lf = 0; lf < n_streams; lf++) {
        const CachedLayout c = cached_layout(streams[lf]);
        if (c.index_bytes > kFixedScratchBytes)
            return fail(HMLFC_E_UNSUPPORTED,
                        "stream %d needs %zu bytes of block index in the fixed scratch, which holds %zu; "
                        "use hmlfc_render_views",
                        lf, c.index_bytes, kFixedScratchBytes);
    }
    void *scratch = nullptr;
    cudaError_t e = fixed_scratch(dev, &scratch);
    if (e != cudaSuccess) return cuda_fail(e, "fixed scratch set-up");
    for (int lf = 0; lf < n_streams; lf++) {
        const hmlfc_stream *s = streams[lf];
        const CachedLayout c = cached_layout(s);
        const uint32_t capacity = cached_capacity(c, kFixedScratchBytes);
        // launch chunks built one at a time on the stack: no host allocation either
        bool too_many = false;
        auto each_chunk = [&](auto f) {
            LaunchViews lv;
            int pos = 0, k = 0, t = 0;
            cudaError_t r = cudaSuccess;
            while (r == cudaSuccess && (k = next_chunk(h_views, n_views, lf, &pos, lv, t)) != 0) {
                if (k < 0) {
                    too_many = true;
                    return cudaErrorInvalidValue;
                }
                r = f(lv, t);
            }
            return r;
        };
        rc = cached_launches(s, s->ds, c, static_cast<uint8_t *>(scratch), capacity, each_chunk, d_out, st, nullptr,
                             false);
        if (too_many) return fail(HMLFC_E_INVALID_ARG, "too many tiles in one launch");
        if (rc != HMLFC_OK) return rc;
    }
    return HMLFC_OK;
}

int hmlfc_set_batch_tuning(int tile_shape, int group, int ctas_per_sm, size_t cache_bytes) {
    if (tile_shape < 0 || tile_shape > 2 || group < 1 || group > 8 || ctas_per_sm < 1 || ctas_per_sm > 32)
        return fail(HMLFC_E_INVALID_ARG, "batch tuning (%d, %d, %d)", tile_shape, group, ctas_per_sm);
    g_batch.tile_shape = tile_shape;
    g_batch.group = group;
    g_batch.ctas_per_sm = ctas_per_sm;
    if (cache_bytes) g_batch.cache_bytes = cache_bytes;
    return HMLFC_OK;
}

int hmlfc_render_batch(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                       float *d_out, void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc render_batch");
    int rc = check_views(streams, n_streams, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    if (n_views > 0 && !d_out) return fail(HMLFC_E_INVALID_ARG, "d_out is NULL");
    if (n_views == 0) return HMLFC_OK;
    // one kernel instantiation per call: the streams' common block size, or the generic one when they differ
    int B = streams[0]->g.B;
    for (int k = 1; k < n_streams; k++)
        if (streams[k]->g.B != B) B = 0;
    const int dev = streams[0]->device;
    DeviceGuard guard(dev);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int TW = g_batch.tile_shape == 1 ? 32 : (g_batch.tile_shape == 2 ? 8 : 16);
    const int TH = g_batch.tile_shape == 1 ? 8 : (g_batch.tile_shape == 2 ? 8 : 16);
    // the host image: header | light fields | views | tile prefix
    std::vector<hmlfc_view> views;
    std::vector<int> tile_start;
    int64_t tiles = 0;
    for (int v = 0; v < n_views; v++) {
        const hmlfc_view &V = h_views[v];
        if (V.width <= 0 || V.height <= 0) continue;
        views.push_back(V);
        tile_start.push_back((int)tiles);
        tiles += (int64_t)((V.width + TW - 1) / TW) * ((V.height + TH - 1) / TH);
        if (tiles >= INT32_MAX) return fail(HMLFC_E_INVALID_ARG, "too many tiles in one call");
    }
    tile_start.push_back((int)tiles);
    if (views.empty()) return HMLFC_OK;
    int64_t n_keys = 0, n_sk = 0, n_cam = 0;
    const size_t lf_bytes = batch_lf_bytes(), hdr_bytes = batch_hdr_bytes();
    auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    int offs[4];
    offs[0] = 0;
    offs[1] = (int)a16(hdr_bytes);
    offs[2] = (int)a16(offs[1] + lf_bytes * n_streams);
    offs[3] = (int)a16(offs[2] + sizeof(hmlfc_view) * views.size());
    const size_t img_bytes = a16(offs[3] + sizeof(int) * tile_start.size());
    std::vector<unsigned char> img(img_bytes, 0);
    for (int k = 0; k < n_streams; k++) {
        const Geometry &g = streams[k]->g;
        const int K = g.L < 2 ? g.L : 2;
        const int64_t sk = (int64_t)g.gu[K] * g.gv[K] * g.nblocks;
        batch_fill_lf(img.data() + offs[1] + lf_bytes * k, streams[k]->ds, n_keys, n_sk, n_cam);
        n_keys += (((sk << (2 * K)) + 15) / 16) * 16;     // each light field's flags start on 16 bytes
        n_sk += sk;
        n_cam += (int64_t)g.nu * g.nv;
    }
    batch_fill_hdr(img.data(), n_streams, (int)views.size(), (int)tiles, TW, TH, n_keys, n_sk, n_cam);
    std::memcpy(img.data() + offs[2], views.data(), sizeof(hmlfc_view) * views.size());
    std::memcpy(img.data() + offs[3], tile_start.data(), sizeof(int) * tile_start.size());
    // the image pool: camera images of W x H RGB8 pixels (u32), offsets below 2^31 so that kNone stays apart
    const unsigned long long capacity = std::min<unsigned long long>(g_batch.cache_bytes / 4, (unsigned long long)kMaxSlots);
    const size_t o_flags = up256(img_bytes), o_slot = up256(o_flags + (size_t)n_keys),
                 o_items = up256(o_slot + (size_t)n_cam * 4), o_count = up256(o_items + (size_t)n_sk * 16),
                 o_cache = up256(o_count + 24), total = up256(o_cache + (size_t)capacity * 4);
    void *base = nullptr;
    cudaError_t e = cudaMallocAsync(&base, total, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return hmlfc_render_views(streams, n_streams, h_views, n_views, d_out, cuda_stream);
    }
    uint8_t *b = static_cast<uint8_t *>(base);
    BatchLaunch L;
    L.total_tiles = (int)tiles;
    L.flags = b + o_flags;
    L.camslot = reinterpret_cast<uint32_t *>(b + o_slot);
    L.items = reinterpret_cast<uint4 *>(b + o_items);
    L.counters = reinterpret_cast<unsigned long long *>(b + o_count);
    L.work = reinterpret_cast<unsigned int *>(b + o_count + 16);
    L.cache = reinterpret_cast<uint32_t *>(b + o_cache);
    L.capacity = capacity;
    L.n_sk = n_sk;
    L.n_cam = n_cam;
    L.group = g_batch.group;
    L.sm_count = sm_count(dev);
    L.decode_ctas = L.sm_count * g_batch.ctas_per_sm;
    L.d_out = d_out;
    e = launch_copy_blob(img.data(), (int)img_bytes, b, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_flags, 0, (size_t)n_keys, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_count, 0, 24, st);
    if (e == cudaSuccess)
        e = launch_batch(B, g_batch.tile_shape, b, offs, L, g_phase_ev[0] ? g_phase_ev : nullptr, st);
    const cudaError_t ef = cudaFreeAsync(base, st);
    if (e == cudaSuccess) e = ef;
    return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "batched render");
}

int hmlfc_server_create(const hmlfc_stream *s, size_t cache_bytes, void *cuda_stream, hmlfc_server **out) {
    if (!s || !out) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const Geometry &g = s->g;
    DeviceGuard guard(s->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t n_keys = (int64_t)g.nu * g.nv * g.nblocks;
    const int64_t n_ck = (int64_t)g.gu[1] * g.gv[1] * g.nblocks;
    const size_t blk = (size_t)g.B * g.B * 4;
    const uint32_t capacity = (uint32_t)std::min<int64_t>({n_keys, (int64_t)(cache_bytes / blk), kMaxSlots});
    if (capacity == 0) return fail(HMLFC_E_INVALID_ARG, "cache of %zu bytes holds no block", cache_bytes);
    auto *sv = new (std::nothrow) hmlfc_server();
    if (!sv) return fail(HMLFC_E_OOM, "host allocation");
    sv->s = s;
    sv->capacity = capacity;
    sv->n_keys = n_keys;
    sv->n_ck = n_ck;
    const size_t o_flags = 0, o_slot = up256((size_t)n_keys), o_owner = up256(o_slot + (size_t)n_keys * 4),
                 o_epoch = up256(o_owner + (size_t)capacity * 4), o_clock = up256(o_epoch + (size_t)capacity * 4),
                 o_items = up256(o_clock + 64), o_cache = up256(o_items + (size_t)n_ck * 32),
                 total = up256(o_cache + (size_t)capacity * blk);
    cudaError_t e = cudaMalloc(&sv->d_mem, total);
    if (e != cudaSuccess) {
        delete sv;
        cudaGetLastError();
        return fail(HMLFC_E_OOM, "server allocation of %zu bytes", total);
    }
    uint8_t *b = static_cast<uint8_t *>(sv->d_mem);
    sv->bytes = total;
    sv->flags = b + o_flags;
    sv->slotmap = reinterpret_cast<uint32_t *>(b + o_slot);
    sv->owner = reinterpret_cast<uint32_t *>(b + o_owner);
    sv->epoch = reinterpret_cast<uint32_t *>(b + o_epoch);
    sv->clock = reinterpret_cast<uint32_t *>(b + o_clock);
    sv->counters = reinterpret_cast<unsigned long long *>(b + o_clock + 8);
    sv->totals = reinterpret_cast<unsigned long long *>(b + o_clock + 16);
    sv->items = reinterpret_cast<uint4 *>(b + o_items);
    sv->cache = reinterpret_cast<uint32_t *>(b + o_cache);
    e = cudaMemsetAsync(sv->slotmap, 0xFF, (size_t)n_keys * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->owner, 0xFF, (size_t)capacity * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->epoch, 0, (size_t)capacity * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->clock, 0, 64, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        hmlfc_server_free(sv);
        return cuda_fail(e, "server set-up");
    }
    *out = sv;
    return HMLFC_OK;
}

void hmlfc_server_free(hmlfc_server *sv) {
    if (!sv) return;
    if (sv->d_mem) {
        DeviceGuard guard(sv->s->device);
        cudaFree(sv->d_mem);
    }
    delete sv;
}

int hmlfc_server_render(hmlfc_server *sv, const hmlfc_view *h_views, int n_views, float *d_out, void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc server_render");
    if (!sv) return fail(HMLFC_E_INVALID_ARG, "server is NULL");
    const hmlfc_stream *s = sv->s;
    int rc = check_views(&s, 1, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    if (n_views == 0) return HMLFC_OK;
    if (!d_out) return fail(HMLFC_E_INVALID_ARG, "d_out is NULL");
    DeviceGuard guard(s->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<LaunchViews> chunks;
    std::vector<int> tiles;
    rc = view_chunks(h_views, n_views, 0, chunks, tiles);
    if (rc != HMLFC_OK) return rc;
    const uint32_t cur = ++sv->call;
    phase_mark(0, st);
    cudaError_t e = cudaMemsetAsync(sv->flags, 0, (size_t)sv->n_keys, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->counters, 0, 8, st);
    for (size_t c = 0; c < chunks.size() && e == cudaSuccess; c++)
        e = launch_mark(s->ds, chunks[c], tiles[c], sv->flags, false, st);
    phase_mark(1, st);
    if (e == cudaSuccess)
        e = launch_resident(s->ds, sv->flags, sv->n_keys, sv->slotmap, sv->owner, sv->epoch, sv->clock, sv->capacity, cur,
                            sv->items, sv->counters, sv->cache, sm_count(s->device) * 8, st);
    phase_mark(2, st);
    for (size_t c = 0; c < chunks.size() && e == cudaSuccess; c++)
        e = launch_render_slots(s->ds, chunks[c], tiles[c], sv->slotmap, sv->cache, d_out, st);
    phase_mark(3, st);
    if (e == cudaSuccess) e = launch_accumulate(sv->counters, sv->totals, st);
    return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "server render");
}

int hmlfc_server_stats(const hmlfc_server *sv, void *cuda_stream, int64_t *out3) {
    if (!sv || !out3) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    DeviceGuard guard(sv->s->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long t[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(t, sv->totals, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "server stats");
    out3[0] = (int64_t)t[0];           // blocks decoded (cache misses) since creation
    out3[1] = (int64_t)t[1];           // decode items
    out3[2] = (int64_t)sv->capacity;   // slots of the resident cache
    return HMLFC_OK;
}

int hmlfc_render_views_relaxed(const hmlfc_stream *const *streams, int n_streams, const float *const *d_coeff,
                               const float *const *d_root, const hmlfc_view *h_views, int n_views, float *d_out,
                               void *cuda_stream) {
    return hmlfc_render_views_relaxed_ex(streams, n_streams, d_coeff, d_root, h_views, n_views, 0u, d_out,
                                         cuda_stream);
}

int hmlfc_render_views_relaxed_ex(const hmlfc_stream *const *streams, int n_streams, const float *const *d_coeff,
                                  const float *const *d_root, const hmlfc_view *h_views, int n_views, uint32_t flags,
                                  float *d_out, void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc render_views_relaxed");
    if (flags & ~HMLFC_RELAX_BIAS) return fail(HMLFC_E_INVALID_ARG, "unknown relaxation flags 0x%x", flags);
    const bool bias = (flags & HMLFC_RELAX_BIAS) != 0;
    int rc = check_views(streams, n_streams, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    for (int k = 0; k < n_streams; k++)
        if (streams[k]->g.sub) return fail(HMLFC_E_UNSUPPORTED, "the relaxation is defined on full-resolution chroma");
    if (n_views == 0) return HMLFC_OK;
    if (!d_out || !d_coeff || !d_root) return fail(HMLFC_E_INVALID_ARG, "NULL buffer");
    DeviceGuard guard(streams[0]->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const hmlfc_stream *s0 = streams[0];
    (void)s0;
    return for_view_chunks(streams, n_streams, h_views, n_views,
                           [&](const hmlfc_stream *s, const LaunchViews &lv, int tiles) {
                               const int k = lv.views[0].lf;
                               if (!d_coeff[k] || !d_root[k]) return fail(HMLFC_E_INVALID_ARG, "NULL coefficients");
                               const cudaError_t e =
                                   launch_render_relaxed(s->ds, lv, tiles, d_coeff[k], d_root[k], d_out, bias, st);
                               return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "relaxed render launch");
                           });
}

int hmlfc_render_backward(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                          const float *d_grad_out, float *const *d_grad_coeff, float *const *d_grad_root,
                          void *cuda_stream) {
    NvtxRange nvtx_range("hmlfc render_backward");
    int rc = check_views(streams, n_streams, h_views, n_views);
    if (rc != HMLFC_OK) return rc;
    for (int k = 0; k < n_streams; k++)
        if (streams[k]->g.sub) return fail(HMLFC_E_UNSUPPORTED, "the relaxation is defined on full-resolution chroma");
    if (n_views == 0) return HMLFC_OK;
    if (!d_grad_out || !d_grad_coeff || !d_grad_root) return fail(HMLFC_E_INVALID_ARG, "NULL buffer");
    DeviceGuard guard(streams[0]->device);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return for_view_chunks(streams, n_streams, h_views, n_views,
                           [&](const hmlfc_stream *s, const LaunchViews &lv, int tiles) {
                               const int k = lv.views[0].lf;
                               if (!d_grad_coeff[k] || !d_grad_root[k]) return fail(HMLFC_E_INVALID_ARG, "NULL gradient");
                               const cudaError_t e = launch_render_backward(s->ds, lv, tiles, d_grad_out,
                                                                            d_grad_coeff[k], d_grad_root[k], st);
                               return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "backward launch");
                           });
}

int hmlfc_dequant(const hmlfc_stream *s, float *d_coeff, float *d_root, void *cuda_stream) {
    if (!s || !d_coeff || !d_root) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    if (s->g.sub) return fail(HMLFC_E_UNSUPPORTED, "the relaxation is defined on full-resolution chroma");
    DeviceGuard guard(s->device);
    const cudaError_t e = launch_dequant(s->ds, s->g.n_nc, d_coeff, d_root, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? HMLFC_OK : cuda_fail(e, "dequant launch");
}

void hmlfc_free_host(void *p) { std::free(p); }

}  // extern "C"

