// CUDA kernels of the HMLFC library for sm_103a (GB300).
//
// The decode is a gather over a small, L2-resident working set, not a dense
// contraction, so no tensor cores are used.  The render kernel stages the
// samples a CTA's rays share: it reduces the tile's footprint (cameras and
// pixels its 16-sample neighbourhoods reach), decodes every block record and
// motion vector of that footprint once into shared memory (per level, node,
// channel and block), reconstructs the level-1 images of the footprint once
// (root + levels L-1..1, shared by up to four cameras), then the level-0
// samples, and finally blends each ray's 16 samples from shared memory.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "hmlfc_internal.h"

namespace hmlfc {

namespace {

// ---------------------------------------------------------------------------
// checked reads (HMLFC_CHECK builds)
// ---------------------------------------------------------------------------
//
// A build with HMLFC_CHECK defined bounds-checks every index into the stream
// object's arrays before the read: an index outside [0, n) sets
// kStatusBounds in the stream's status word (hmlfc_check_status reports it)
// and reads element 0 instead.  Other builds compile the checks away.

__device__ __forceinline__ int64_t chk(const DevStream &S, int64_t i, int64_t n) {
#ifdef HMLFC_CHECK
    if (i < 0 || i >= n) {
        atomicOr(S.status, kStatusBounds);
        return 0;
    }
#else
    (void)S;
    (void)n;
#endif
    return i;
}

// true when [p, p + span) lies inside array [base, base + n) (always in other builds)
template <class T>
__device__ __forceinline__ bool chk_span(const DevStream &S, const T *base, int64_t n, const T *p, int64_t span) {
#ifdef HMLFC_CHECK
    const int64_t o = p - base;
    if (o < 0 || o + span > n) {
        atomicOr(S.status, kStatusBounds);
        return false;
    }
#else
    (void)S; (void)base; (void)n; (void)p; (void)span;
#endif
    return true;
}

// __ldg of element `idx` of stream array `arr`, bounds-checked in HMLFC_CHECK builds
#define SLD(S, arr, idx) __ldg((S).arr + chk((S), (int64_t)(idx), (S).lim_##arr))

// ---------------------------------------------------------------------------
// bit fields and BISE (Sec. 4.6)
// ---------------------------------------------------------------------------

// `width` (<= 16) bits at bit `pos` of the word array; reads w[pos/32 + 1]
// too, which the device copies pad.
__device__ __forceinline__ uint32_t bits_at(const uint32_t *__restrict__ w, uint32_t pos, uint32_t width) {
    const uint32_t k = pos >> 5;
    const uint32_t v = __funnelshift_r(__ldg(w + k), __ldg(w + k + 1), pos & 31u);
    return v & ((1u << width) - 1u);
}

// Digit r (0-based, least significant first) of a packed trit byte or quint
// field, without a runtime divide: floor(p / 3^r) = (p * M3[r]) >> 16 for
// p < 256 and floor(p / 5^r) = (p * M5[r]) >> 16 for p < 128 (checked
// exhaustively), then the last digit by the same trick.
__device__ __forceinline__ uint32_t trit_digit(uint32_t packed, uint32_t r) {
    const uint32_t m = r == 0 ? 65536u : (uint32_t)((0x032A097C1C725556ull >> (16u * (r - 1u))) & 0xFFFFu);
    const uint32_t d = (packed * m) >> 16;
    return d - 3u * ((d * 171u) >> 9);
}

__device__ __forceinline__ uint32_t quint_digit(uint32_t packed, uint32_t r) {
    const uint32_t m = r == 0 ? 65536u : (r == 1 ? 13108u : 2622u);
    const uint32_t d = (packed * m) >> 16;
    return d - 5u * ((d * 205u) >> 10);
}

// Value i of a BISE sequence starting at word w (i < 2^16: block payloads).
// Branch-free over the three alphabets so that the lanes of a warp whose
// pixels fall in blocks of different modes do not diverge: mode 0 is the
// case "one value per group, no packed field".
__device__ __forceinline__ uint32_t bise_get_small(const uint32_t *__restrict__ w, uint32_t mode, uint32_t b,
                                                   uint32_t i) {
    // groups: mode 0 -> 1 value, mode 1 -> 5, mode 2 -> 3; packed field 0 / 8 / 7 bits
    const uint32_t g = mode == 1 ? (i * 52429u) >> 18 : (mode == 2 ? (i * 43691u) >> 17 : i);   // i / per
    const uint32_t per = mode == 1 ? 5u : (mode == 2 ? 3u : 1u);
    const uint32_t hw = mode == 1 ? 8u : (mode == 2 ? 7u : 0u);
    const uint32_t r = i - g * per;
    const uint32_t pos = g * (hw + per * b);
    const uint32_t packed = bits_at(w, pos, hw);
    const uint32_t hi = mode == 1 ? trit_digit(packed, r) : quint_digit(packed, r);   // 0 when hw == 0
    return (hi << b) | bits_at(w, pos + hw + r * b, b);
}

// Value i of a long BISE sequence (the motion-vector symbols).
__device__ __forceinline__ uint32_t bise_get_long(const uint32_t *__restrict__ w, uint32_t mode, uint32_t b,
                                                  uint64_t i) {
    uint64_t pos;
    uint32_t r = 0, hw = 0;
    if (mode == 0) {
        pos = i * b;
        return bits_at(w + (pos >> 5), (uint32_t)(pos & 31u), b);
    }
    if (mode == 1) {
        const uint64_t g = i / 5u;
        r = (uint32_t)(i - 5u * g);
        pos = g * (8u + 5u * b);
        hw = 8;
    } else {
        const uint64_t g = i / 3u;
        r = (uint32_t)(i - 3u * g);
        pos = g * (7u + 3u * b);
        hw = 7;
    }
    const uint32_t *base = w + (pos >> 5);
    const uint32_t p0 = (uint32_t)(pos & 31u);
    const uint32_t packed = bits_at(base, p0, hw);
    const uint32_t hi = mode == 1 ? trit_digit(packed, r) : quint_digit(packed, r);
    return (hi << b) | bits_at(base, p0 + hw + r * b, b);
}

// ---------------------------------------------------------------------------
// per-level tables, copied to shared memory by every CTA
// ---------------------------------------------------------------------------

struct LevelTabs {
    int gu[kMaxLevels + 1], gv[kMaxLevels + 1];
    int nc_base[kMaxLevels], ref_base[kMaxLevels], pred_base[kMaxLevels];
};

__device__ __forceinline__ void load_tabs(const DevStream &S, LevelTabs &T) {
    for (int t = threadIdx.x; t <= kMaxLevels; t += blockDim.x) {
        T.gu[t] = S.gu[t];
        T.gv[t] = S.gv[t];
        if (t < kMaxLevels) {
            T.nc_base[t] = S.nc_base[t];
            T.ref_base[t] = S.ref_base[t];
            T.pred_base[t] = S.pred_base[t];
        }
    }
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ bool is_ref(int a, int b) { return ((a | b) & 1) == 0; }

__device__ __forceinline__ int ref_rank(const LevelTabs &T, int l, int a, int b, int c) {
    return T.ref_base[l] + ((a >> 1) * ((T.gv[l] + 1) >> 1) + (b >> 1)) * 3 + c;
}

__device__ __forceinline__ int pred_rank(const LevelTabs &T, int l, int a, int b, int c) {
    const int gv = T.gv[l];
    const int refs_before = ((a + 1) >> 1) * ((gv + 1) >> 1) + ((a & 1) == 0 ? (b + 1) >> 1 : 0);
    return T.pred_base[l] + (a * gv + b - refs_before) * 3 + c;
}

__device__ __forceinline__ int nc_index(const LevelTabs &T, int l, int a, int b, int c) {
    return T.nc_base[l] + (a * T.gv[l] + b) * 3 + c;
}

// Block geometry, specialised on the block size (BS > 0: compile-time power
// of two; BS == 0: the runtime value S.B).
template <int BS>
struct Blk {
    int B;
    __device__ __forceinline__ explicit Blk(int b) : B(BS > 0 ? BS : b) {}
    __device__ __forceinline__ int div(int v) const { return BS > 0 ? (v / BS) : (v / B); }
    __device__ __forceinline__ int size() const { return BS > 0 ? BS : B; }
};

// Resident reference coefficient R^ at (x, y) of channel c's plane of
// reference node-channel row `row` (= ref rank * nblocks).
template <int BS>
__device__ __forceinline__ int ref_coef(const DevStream &S, const Blk<BS> &bk, int c, uint32_t row, int x, int y) {
    const int bx = bk.div(x), by = bk.div(y);
    const int B = bk.size();
    const uint32_t tile = SLD(S, ref_tab, row + (uint32_t)(by * S.cnbx[c] + bx));
    return SLD(S, tiles, (size_t)tile * (B * B) + (y - by * B) * B + (x - bx * B));
}

// Sec. 4.4 motion re-compensation with the quarter-pel bilinear predictor,
// taps clamped to channel c's plane.
template <int BS>
__device__ __forceinline__ int mc_pred(const DevStream &S, const Blk<BS> &bk, int c, uint32_t row, int x, int y,
                                       int mvx, int mvy) {
    const int X = 4 * x + mvx, Y = 4 * y + mvy;
    const int x0 = X >> 2, y0 = Y >> 2, fx = X & 3, fy = Y & 3;
    const int xa = clampi(x0, 0, S.cW[c] - 1), xb = clampi(x0 + 1, 0, S.cW[c] - 1);
    const int ya = clampi(y0, 0, S.cH[c] - 1), yb = clampi(y0 + 1, 0, S.cH[c] - 1);
    const int a = ref_coef(S, bk, c, row, xa, ya), b = ref_coef(S, bk, c, row, xb, ya);
    const int cc = ref_coef(S, bk, c, row, xa, yb), d = ref_coef(S, bk, c, row, xb, yb);
    const int s = (4 - fx) * (4 - fy) * a + fx * (4 - fy) * b + (4 - fx) * fy * cc + fx * fy * d;
    return (s + 8) >> 4;
}

// Index of the MV symbol of block k of predictive node (a, b), level l,
// channel c: per predictive node (breadth-first) mv_node symbols, channel
// c's blocks from mv_coff[c] (pred_rank * nblocks + k without sub-sampling).
__device__ __forceinline__ uint64_t mv_index(const DevStream &S, const LevelTabs &T, int l, int a, int b, int c,
                                            int k) {
    const int pr = pred_rank(T, l, a, b, c);       // pred_base (a multiple of 3) + node * 3 + c
    return (uint64_t)chk(S, (int64_t)((pr - c) / 3) * S.mv_node + S.mv_coff[c] + k, S.lim_mv);
}

// HMLFC_CHECK builds: true when the record at word `rec` (header hdr) with n
// values ends inside the record words (otherwise kStatusBounds is set and the
// caller treats the block as insignificant); always true in other builds.
__device__ __forceinline__ bool rec_ok(const DevStream &S, uint32_t rec, uint32_t hdr, int n) {
#ifdef HMLFC_CHECK
    const uint32_t mode = (hdr >> 21) & 3u, b = (hdr >> 16) & 31u;
    const uint64_t bits = mode == 0 ? (uint64_t)n * b
                                    : (mode == 1 ? (uint64_t)((n + 4) / 5) * (8 + 5 * b) : (uint64_t)((n + 2) / 3) * (7 + 3 * b));
    if (mode == 3 || (uint64_t)rec + 1 + (bits + 31) / 32 > (uint64_t)S.lim_recs - 2) {
        atomicOr(S.status, kStatusBounds);
        return false;
    }
#else
    (void)S; (void)rec; (void)hdr; (void)n;
#endif
    return true;
}

__device__ __forceinline__ void decode_mv(const DevStream &S, uint32_t sym, int &mvx, int &mvy, int &sign) {
    sign = (sym & 1u) ? -1 : 1;
    const uint32_t s2 = sym >> 1;
    const uint32_t qx = s2 / (uint32_t)S.side;
    mvx = (int)qx - 4 * S.Ws;
    mvy = (int)(s2 - qx * (uint32_t)S.side) - 4 * S.Ws;
}

// Residual r^ of block k, n values, at value index idx (record lookup through
// the group index).
__device__ __forceinline__ int residual(const DevStream &S, int nc, int k, uint32_t idx, int n) {
    const uint4 g = SLD(S, groups, (size_t)nc * S.ngroups + (k >> 5));
    const uint32_t bit = (uint32_t)k & 31u;
    if (!((g.x >> bit) & 1u)) return 0;
    const uint32_t rank = __popc(g.x & ((1u << bit) - 1u));
    const uint32_t rec = g.y + SLD(S, offs, g.z + rank);
    const uint32_t hdr = SLD(S, recs, rec);
    if (!rec_ok(S, rec, hdr, n)) return 0;
    const int m = (int)(int16_t)(hdr & 0xFFFFu);
    return S.q * (m + (int)bise_get_small(S.recs + rec + 1, (hdr >> 21) & 3u, (hdr >> 16) & 31u, idx));
}

// SRV value of node (a, b) at level l, channel c, at pixel (x, y) of that
// channel's plane, straight from the index (no staging).
template <int BS>
__device__ int srv_direct(const DevStream &S, const LevelTabs &T, const Blk<BS> &bk, int l, int a, int b, int c, int x,
                          int y) {
    const int B = bk.size();
    const int bx = bk.div(x), by = bk.div(y);
    const int k = by * S.cnbx[c] + bx;
    if (is_ref(a, b)) return ref_coef(S, bk, c, (uint32_t)ref_rank(T, l, a, b, c) * S.nblocks, x, y);
    const int x0 = bx * B, y0 = by * B;
    const int bw = min(B, S.cW[c] - x0), bh = min(B, S.cH[c] - y0);
    const int r = residual(S, nc_index(T, l, a, b, c), k, (uint32_t)((y - y0) * bw + (x - x0)), bw * bh);
    if (!S.mc) return r;
    const uint32_t sym = bise_get_long(S.mvs, S.mv_mode, S.mv_b, mv_index(S, T, l, a, b, c, k));
    int mvx, mvy, sign;
    decode_mv(S, sym, mvx, mvy, sign);
    const uint32_t row = (uint32_t)ref_rank(T, l, a & ~1, b & ~1, c) * S.nblocks;
    return sign * mc_pred(S, bk, c, row, x, y, mvx, mvy) + r;
}

__device__ __forceinline__ uint32_t ycocg_to_rgb8(int Y, int Co, int Cg) {
    const int t = Y - (Cg >> 1);
    const int G = Cg + t;
    const int Bc = t - (Co >> 1);
    const int R = Bc + Co;
    // __vimin_s32_relu(x, 255) = max(min(x, 255), 0)
    return (uint32_t)__vimin_s32_relu(R, 255) | ((uint32_t)__vimin_s32_relu(G, 255) << 8) |
           ((uint32_t)__vimin_s32_relu(Bc, 255) << 16);
}

// Random-access decoding of one sample (Sec. 4.8.1): root + SRV levels
// L-1 .. lod.  lod > 0 is the progressive decode: the sample of camera (i, j)
// is then its level-lod node's reconstruction.
template <int BS>
__device__ uint32_t sample_direct(const DevStream &S, const LevelTabs &T, const Blk<BS> &bk, int i, int j, int x,
                                  int y) {
    const int L = S.L;
    // with sub-sampled chroma, Co and Cg of (x, y) are those of chroma pixel (x >> 1, y >> 1)
    const int xc = S.sub ? x >> 1 : x, yc = S.sub ? y >> 1 : y;
    const size_t rbase = ((size_t)(i >> L) * T.gv[L] + (j >> L)) * (size_t)S.rnpx;
    int v0 = SLD(S, roots, rbase + S.roff[0] + (size_t)y * S.cW[0] + x);
    int v1 = SLD(S, roots, rbase + S.roff[1] + (size_t)yc * S.cW[1] + xc);
    int v2 = SLD(S, roots, rbase + S.roff[2] + (size_t)yc * S.cW[2] + xc);
    for (int l = S.lod; l < L; l++) {
        const int a = i >> l, b = j >> l;
        v0 += srv_direct(S, T, bk, l, a, b, 0, x, y);
        v1 += srv_direct(S, T, bk, l, a, b, 1, xc, yc);
        v2 += srv_direct(S, T, bk, l, a, b, 2, xc, yc);
    }
    return ycocg_to_rgb8(v0, v1, v2);
}

// ---------------------------------------------------------------------------
// K3: load-time decode of the reference SRV blocks into resident tiles
// ---------------------------------------------------------------------------

// src[t] = {record word, block valid width, block valid height, unused} for
// tile t + first, B rows of `stride` values (the reference tiles: stride B,
// first 1, tile 0 being the shared zero tile; the predictive residual tiles:
// stride B rounded up to even, first 0).  Values outside the block's valid
// pixels are zero.
__global__ void k_decode_tiles(const DevStream S, const uint4 *__restrict__ src, int n_tiles,
                               int16_t *__restrict__ tiles, int stride, int first) {
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    const uint4 s = src[t];
    const uint32_t hdr = SLD(S, recs, s.x);
    if (!rec_ok(S, s.x, hdr, (int)(s.y * s.z))) return;
    const int m = (int)(int16_t)(hdr & 0xFFFFu);
    const uint32_t mode = (hdr >> 21) & 3u, b = (hdr >> 16) & 31u;
    const int B = S.B;
    int16_t *dst = tiles + (size_t)(t + first) * B * stride;
    for (int p = threadIdx.x; p < B * stride; p += blockDim.x) {
        const int yy = p / stride, xx = p - yy * stride;
        int v = 0;
        if (xx < (int)s.y && yy < (int)s.z)
            v = S.q * (m + (int)bise_get_small(S.recs + s.x + 1, mode, b, (uint32_t)(yy * (int)s.y + xx)));
        dst[p] = (int16_t)v;
    }
}

// Dense copy of the resident reference SRVs for the block decode: plane r
// (reference node-channel rank r, [H][W] int16, channel r % 3) holds every
// block's tile, the zero tile where the block is insignificant; a sub-sampled
// chroma plane fills its top-left ceil(H/2) x ceil(W/2).  One CTA per
// (block, plane).
__global__ void __launch_bounds__(256) k_build_planes(const DevStream S, int n_ref, int16_t *__restrict__ planes) {
    const int k = blockIdx.x;
    const int B = S.B;
    for (int r = blockIdx.y; r < n_ref; r += gridDim.y) {
        const int c = r % 3;                                     // ranks: a multiple of 3 per level + node * 3 + c
        if (k >= S.cnb[c]) continue;
        const int bx = k % S.cnbx[c], by = k / S.cnbx[c];
        const int bw = min(B, S.cW[c] - bx * B), bh = min(B, S.cH[c] - by * B);
        const uint32_t tile = SLD(S, ref_tab, (size_t)r * S.nblocks + k);
        const int16_t *src = S.tiles + (size_t)tile * B * B;
        int16_t *dst = planes + (size_t)r * S.W * S.H + (size_t)by * B * S.W + (size_t)bx * B;
        for (int e = threadIdx.x; e < bw * bh; e += blockDim.x) {
            const int yy = e / bw, xx = e - yy * bw;
            dst[(size_t)yy * S.W + xx] = src[yy * B + xx];
        }
    }
}

// ---------------------------------------------------------------------------
// K2: random-access decoding of a list of samples
// ---------------------------------------------------------------------------

template <int BS>
__global__ void __launch_bounds__(256) k_decode_pixels(const DevStream S, const int4 *__restrict__ coords, int64_t n,
                                                       uint8_t *__restrict__ rgb) {
    __shared__ LevelTabs T;
    load_tabs(S, T);
    __syncthreads();
    const Blk<BS> bk(S.B);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int4 c = __ldg(coords + k);
        uint32_t v = 0;
        if (c.x < 0 || c.x >= S.nu || c.y < 0 || c.y >= S.nv || c.z < 0 || c.z >= S.W || c.w < 0 || c.w >= S.H) {
            atomicOr(S.status, kStatusCoord);
        } else {
            v = sample_direct(S, T, bk, c.x, c.y, c.z, c.w);
        }
        rgb[3 * k] = (uint8_t)(v & 0xFFu);
        rgb[3 * k + 1] = (uint8_t)((v >> 8) & 0xFFu);
        rgb[3 * k + 2] = (uint8_t)((v >> 16) & 0xFFu);
    }
}

// ---------------------------------------------------------------------------
// ray setup (Sec. 2.1 two-plane parameterisation)
// ---------------------------------------------------------------------------

struct Ray {
    int i0, i1, j0, j1, x0, x1, y0, y1;
    float fu, fv, fs, ft;
};

__device__ __forceinline__ float axis_nb(float c, int n, int &i0, int &i1) {
    const float cc = fminf(fmaxf(c, -1.0f), (float)n);
    const float fl = floorf(cc);
    const int k = (int)fl;
    i0 = clampi(k, 0, n - 1);
    i1 = clampi(k + 1, 0, n - 1);
    return cc - fl;
}

__device__ __forceinline__ void ray_setup(const hmlfc_view &V, int nu, int nv, int W, int H, int px, int py, Ray &r) {
    const float X = (float)px + 0.5f, Y = (float)py + 0.5f;
    const float *h = V.H_uv;
    const float wu = h[6] * X + h[7] * Y + h[8];
    const float u = __fdividef(h[0] * X + h[1] * Y + h[2], wu);
    const float v = __fdividef(h[3] * X + h[4] * Y + h[5], wu);
    const float *g = V.H_st;
    const float ws = g[6] * X + g[7] * Y + g[8];
    const float s = __fdividef(g[0] * X + g[1] * Y + g[2], ws);
    const float t = __fdividef(g[3] * X + g[4] * Y + g[5], ws);
    r.fu = axis_nb(u, nu, r.i0, r.i1);
    r.fv = axis_nb(v, nv, r.j0, r.j1);
    r.fs = axis_nb(s, W, r.x0, r.x1);
    r.ft = axis_nb(t, H, r.y0, r.y1);
}

// Quadrilinear blend of the 16 samples, separably: the 2 x 2 pixels of each
// camera first (weights in s, t), then the 2 x 2 cameras (weights in u, v).
// The per-camera bilinear runs in 16-bit fixed point on the packed bytes:
// one byte permute gathers a channel of two samples, one dp2a adds both
// weighted samples (weights round(w * 65535): error <= 4 * 255 * 0.5 / 65535
// of a level per channel).  fetch(a, b, xs, ys, i, j, x, y) returns the
// packed RGB8 sample (R | G << 8 | B << 16).
template <class F>
__device__ __forceinline__ void blend16(const Ray &r, F fetch, float out[3]) {
    const float ws0 = 1.0f - r.fs, ws1 = r.fs, wt0 = 1.0f - r.ft, wt1 = r.ft;
    const float wu[2] = {1.0f - r.fu, r.fu}, wv[2] = {1.0f - r.fv, r.fv};
    const int ii[2] = {r.i0, r.i1}, jj[2] = {r.j0, r.j1}, xx[2] = {r.x0, r.x1}, yy[2] = {r.y0, r.y1};
    // sample q = xs * 2 + ys; pair (q0, q1) has xs = 0, pair (q2, q3) xs = 1
    const uint32_t wA = __float2uint_rn(ws0 * wt0 * 65535.0f) | (__float2uint_rn(ws0 * wt1 * 65535.0f) << 16);
    const uint32_t wB = __float2uint_rn(ws1 * wt0 * 65535.0f) | (__float2uint_rn(ws1 * wt1 * 65535.0f) << 16);
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const uint32_t p0 = fetch(a, b, 0, 0, ii[a], jj[b], xx[0], yy[0]);
            const uint32_t p1 = fetch(a, b, 0, 1, ii[a], jj[b], xx[0], yy[1]);
            const uint32_t p2 = fetch(a, b, 1, 0, ii[a], jj[b], xx[1], yy[0]);
            const uint32_t p3 = fetch(a, b, 1, 1, ii[a], jj[b], xx[1], yy[1]);
            const uint32_t rg01 = __byte_perm(p0, p1, 0x5140u), rg23 = __byte_perm(p2, p3, 0x5140u);   // R R G G
            const uint32_t b01 = __byte_perm(p0, p1, 0x0062u), b23 = __byte_perm(p2, p3, 0x0062u);     // B B
            const uint32_t cr = __dp2a_lo(wB, rg23, __dp2a_lo(wA, rg01, 0u));
            const uint32_t cg = __dp2a_hi(wB, rg23, __dp2a_hi(wA, rg01, 0u));
            const uint32_t cb = __dp2a_lo(wB, b23, __dp2a_lo(wA, b01, 0u));
            const float wc = wu[a] * wv[b];
            acc0 = fmaf(wc, (float)cr, acc0);
            acc1 = fmaf(wc, (float)cg, acc1);
            acc2 = fmaf(wc, (float)cb, acc2);
        }
    const float inv = 1.0f / (255.0f * 65535.0f);
    out[0] = acc0 * inv;
    out[1] = acc1 * inv;
    out[2] = acc2 * inv;
}

__device__ __forceinline__ int find_view(const LaunchViews &LV, int tile) {
    int lo = 0, hi = LV.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (LV.tile_start[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// K1: fused decode + render
// ---------------------------------------------------------------------------

constexpr int kMaxCam = 9;          // cameras of a staged footprint (3 x 3)
constexpr int kMaxPx = 400;         // pixels of a staged footprint
constexpr int kMaxDesc = 384;       // block descriptors of a staged footprint
constexpr int kMaxNodes = 4;        // nodes of one level >= 1 in a staged footprint

struct Footprint {
    int imin, imax, jmin, jmax, xmin, xmax, ymin, ymax;
    int ncv, nx, npx, nbxb, nblk, bx0, by0;
    uint32_t mag_nx, mag_npx;           // floor((2^32 - 1) / d) + 1, or 0 for d == 1
    int staged;
    int a0[kMaxLevels], b0[kMaxLevels], nnu[kMaxLevels], nnv[kMaxLevels], dbase[kMaxLevels + 1];
};

// Shared memory of a staged tile: block descriptors, then two level
// accumulators (int32 [kMaxNodes][3][kMaxPx]); the RGB8 samples of the
// level-0 cameras reuse whichever accumulator is free at the end.
constexpr size_t kDescBytes = (size_t)kMaxDesc * 32;
constexpr size_t kAccBytes = (size_t)kMaxNodes * 3 * kMaxPx * 4;
constexpr size_t kStageSmem = kDescBytes + 2 * kAccBytes;
static_assert((size_t)kMaxCam * kMaxPx * 4 <= kAccBytes, "RGB8 staging must fit an accumulator");

// A block descriptor (32 B): d0 = {record word or kNone, record header,
// packed motion vector, tap tile origin cx | cy << 16}; d1 = the tiles of the
// reference node covering the block's motion-compensated taps, {T(cx, cy),
// T(cx+1, cy), T(cx, cy+1), T(cx+1, cy+1)} -- the taps of one block always
// fall in a 2 x 2 tile neighbourhood.  A reference node's descriptor holds
// its own tile in d1.x.
struct Desc {
    uint4 d0, d1;
};

// Pixel geometry shared by every level and channel of one staged item.
struct PixGeom {
    int x, y;
    int blk;        // block index inside the footprint's block box
    int idx;        // index of the pixel in its (possibly partial) block
    int toff;       // offset of the pixel in a B x B tile
};

// q = floor(n / d) for n, d < 2^16 with m = floor((2^32 - 1) / d) + 1; that
// m would be 2^32 for d == 1, which is stored as 0 and means "q = n".
__device__ __forceinline__ int qdiv(int n, uint32_t m) { return m ? (int)__umulhi((uint32_t)n, m) : n; }

__host__ __device__ __forceinline__ uint32_t qdiv_magic(uint32_t d) {
    return d <= 1 ? 0u : (uint32_t)(0xFFFFFFFFull / d) + 1u;
}

template <int BS>
__device__ __forceinline__ PixGeom pix_geom(const DevStream &S, const Footprint &F, const Blk<BS> &bk, int p) {
    PixGeom g;
    const int row = qdiv(p, F.mag_nx);
    g.x = F.xmin + p - row * F.nx;
    g.y = F.ymin + row;
    const int B = bk.size();
    const int bx = bk.div(g.x), by = bk.div(g.y);
    const int x0 = bx * B, y0 = by * B;
    g.blk = (by - F.by0) * F.nbxb + (bx - F.bx0);
    g.idx = (g.y - y0) * min(B, S.W - x0) + (g.x - x0);
    g.toff = (g.y - y0) * B + (g.x - x0);
    return g;
}

// One tap of the resident reference SRV through a descriptor's 2x2 tiles.
template <int BS>
__device__ __forceinline__ int tap(const DevStream &S, const Blk<BS> &bk, const uint4 &t, int cx, int cy, int x, int y) {
    const int B = bk.size();
    const int tx = bk.div(x), ty = bk.div(y);
    const uint32_t tile = (ty == cy) ? (tx == cx ? t.x : t.y) : (tx == cx ? t.z : t.w);
    return SLD(S, tiles, (size_t)tile * (B * B) + (y - ty * B) * B + (x - tx * B));
}

// SRV of one node-channel at a pixel, from its staged descriptor.
template <int BS>
__device__ __forceinline__ int srv_desc(const DevStream &S, const Blk<BS> &bk, const Desc &D, bool ref,
                                        const PixGeom &g) {
    const int B = bk.size();
    if (ref) return SLD(S, tiles, (size_t)D.d1.x * (B * B) + g.toff);
    int r = 0;
    if (D.d0.x != kNone) {
        const int m = (int)(int16_t)(D.d0.y & 0xFFFFu);
        r = S.q * (m + (int)bise_get_small(S.recs + D.d0.x + 1, (D.d0.y >> 21) & 3u, (D.d0.y >> 16) & 31u,
                                           (uint32_t)g.idx));
    }
    if (!S.mc) return r;
    const int mvx = (int)(D.d0.z & 1023u) - 512, mvy = (int)((D.d0.z >> 10) & 1023u) - 512;
    const int X = 4 * g.x + mvx, Y = 4 * g.y + mvy;
    const int x0 = X >> 2, y0 = Y >> 2, fx = X & 3, fy = Y & 3;
    const int xa = clampi(x0, 0, S.W - 1), xb = clampi(x0 + 1, 0, S.W - 1);
    const int ya = clampi(y0, 0, S.H - 1), yb = clampi(y0 + 1, 0, S.H - 1);
    const int cx = (int)(D.d0.w & 0xFFFFu), cy = (int)(D.d0.w >> 16);
    const int a = tap(S, bk, D.d1, cx, cy, xa, ya), b = tap(S, bk, D.d1, cx, cy, xb, ya);
    const int c = tap(S, bk, D.d1, cx, cy, xa, yb), d = tap(S, bk, D.d1, cx, cy, xb, yb);
    const int pred = ((4 - fx) * (4 - fy) * a + fx * (4 - fy) * b + (4 - fx) * fy * c + fx * fy * d + 8) >> 4;
    return ((D.d0.z >> 20) & 1u) ? r - pred : r + pred;
}


template <int BS>
__device__ __forceinline__ const Desc &desc_at(const Desc *desc, const Footprint &F, int l, int a, int b, int c,
                                              int blk) {
    return desc[F.dbase[l] + (((a - F.a0[l]) * F.nnv[l] + (b - F.b0[l])) * 3 + c) * F.nblk + blk];
}

template <int BS, int TW, int TH>
__global__ void __launch_bounds__(TW *TH, 4) k_render(const __grid_constant__ DevStream S,
                                                  const __grid_constant__ LaunchViews LV, float *__restrict__ out,
                                                  int force_direct) {
    constexpr int NT = TW * TH;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ LevelTabs T;
    __shared__ Footprint F;
    __shared__ int s_view;
    __shared__ int s_red[NT / 32][8];

    load_tabs(S, T);
    if (threadIdx.x == 0) s_view = find_view(LV, blockIdx.x);
    __syncthreads();
    const hmlfc_view &V = LV.views[s_view];
    const int tiles_x = (V.width + TW - 1) / TW;
    const int local = blockIdx.x - LV.tile_start[s_view];
    const int px = (local % tiles_x) * TW + (int)threadIdx.x % TW;
    const int py = (local / tiles_x) * TH + (int)threadIdx.x / TW;
    const bool act = px < V.width && py < V.height;
    const Blk<BS> bk(S.B);

    Ray r;
    ray_setup(V, S.nu, S.nv, S.W, S.H, act ? px : 0, act ? py : 0, r);

    // ---- footprint of the tile (min/max over active rays) ----
    int red[8] = {act ? r.i0 : INT_MAX, act ? -r.i1 : INT_MAX, act ? r.j0 : INT_MAX, act ? -r.j1 : INT_MAX,
                  act ? r.x0 : INT_MAX, act ? -r.x1 : INT_MAX, act ? r.y0 : INT_MAX, act ? -r.y1 : INT_MAX};
#pragma unroll
    for (int q = 0; q < 8; q++) red[q] = __reduce_min_sync(0xFFFFFFFFu, red[q]);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < 8; q++) s_red[threadIdx.x >> 5][q] = red[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int m[8];
        for (int q = 0; q < 8; q++) m[q] = INT_MAX;
        for (int w = 0; w < NT / 32; w++)
            for (int q = 0; q < 8; q++) m[q] = min(m[q], s_red[w][q]);
        F.imin = m[0]; F.imax = -m[1]; F.jmin = m[2]; F.jmax = -m[3];
        F.xmin = m[4]; F.xmax = -m[5]; F.ymin = m[6]; F.ymax = -m[7];
        const int ncu = F.imax - F.imin + 1, ncv = F.jmax - F.jmin + 1;
        F.ncv = ncv;
        F.nx = F.xmax - F.xmin + 1;
        F.npx = F.nx * (F.ymax - F.ymin + 1);
        F.mag_nx = qdiv_magic((uint32_t)F.nx);
        F.mag_npx = qdiv_magic((uint32_t)F.npx);
        F.bx0 = F.xmin / S.B;
        F.by0 = F.ymin / S.B;
        F.nbxb = F.xmax / S.B - F.bx0 + 1;
        F.nblk = F.nbxb * (F.ymax / S.B - F.by0 + 1);
        int nd = 0, maxn = 0;
        for (int l = 0; l < S.L; l++) {
            F.a0[l] = F.imin >> l;
            F.b0[l] = F.jmin >> l;
            F.nnu[l] = (F.imax >> l) - F.a0[l] + 1;
            F.nnv[l] = (F.jmax >> l) - F.b0[l] + 1;
            F.dbase[l] = nd;
            nd += F.nnu[l] * F.nnv[l] * 3 * F.nblk;
            if (l >= 1) maxn = max(maxn, F.nnu[l] * F.nnv[l]);
        }
        F.dbase[S.L] = nd;
        F.staged = !force_direct && ncu * ncv <= kMaxCam && F.npx <= kMaxPx && nd <= kMaxDesc && maxn <= kMaxNodes;
    }
    __syncthreads();

    float o[3];
    if (!F.staged) {
        // ---- direct path: every ray decodes its own 16 samples ----
        if (act) {
            blend16(r, [&](int, int, int, int, int i, int j, int x, int y) { return sample_direct(S, T, bk, i, j, x, y); },
                    o);
        }
    } else {
        Desc *desc = reinterpret_cast<Desc *>(smem);
        int *acc_base = reinterpret_cast<int *>(smem + kDescBytes);
        constexpr int kAccInts = (int)(kAccBytes / 4);
        const int L = S.L;
        const int B = bk.size();
        const size_t plane = (size_t)S.W * S.H;
        // ---- 1: block descriptors (index, header, motion vector, tap tiles) ----
        for (int d = threadIdx.x; d < F.dbase[L]; d += NT) {
            int l = 0;
            while (d >= F.dbase[l + 1]) l++;
            int e = d - F.dbase[l];
            const int blk = e % F.nblk;
            e /= F.nblk;
            const int c = e % 3;
            e /= 3;
            const int b = F.b0[l] + e % F.nnv[l];
            const int a = F.a0[l] + e / F.nnv[l];
            const int bx = F.bx0 + blk % F.nbxb, by = F.by0 + blk / F.nbxb;
            const int k = by * S.nbx + bx;
            Desc D;
            D.d0 = make_uint4(kNone, 0u, 0u, 0u);
            D.d1 = make_uint4(0u, 0u, 0u, 0u);
            if (a < T.gu[l] && b < T.gv[l] && bx < S.nbx && by < S.nby) {
                if (is_ref(a, b)) {
                    D.d1.x = SLD(S, ref_tab, (size_t)ref_rank(T, l, a, b, c) * S.nblocks + k);
                } else {
                    const int nc = nc_index(T, l, a, b, c);
                    const uint4 g = SLD(S, groups, (size_t)nc * S.ngroups + (k >> 5));
                    const uint32_t bit = (uint32_t)k & 31u;
                    if ((g.x >> bit) & 1u) {
                        const uint32_t rec = g.y + SLD(S, offs, g.z + __popc(g.x & ((1u << bit) - 1u)));
                        D.d0.x = rec;
                        D.d0.y = SLD(S, recs, rec);
                        if (!rec_ok(S, rec, D.d0.y, min(B, S.W - bx * B) * min(B, S.H - by * B))) D.d0.x = kNone;
                    }
                    if (S.mc) {
                        const uint32_t sym = bise_get_long(S.mvs, S.mv_mode, S.mv_b,
                                                           mv_index(S, T, l, a, b, c, k));
                        int mvx, mvy, sign;
                        decode_mv(S, sym, mvx, mvy, sign);
                        D.d0.z = (uint32_t)(mvx + 512) | ((uint32_t)(mvy + 512) << 10) | ((sign < 0 ? 1u : 0u) << 20);
                        // the taps of this block start at the clamped (x0 + floor(mvx/4), y0 + floor(mvy/4))
                        const int cx = bk.div(clampi(bx * B + (mvx >> 2), 0, S.W - 1));
                        const int cy = bk.div(clampi(by * B + (mvy >> 2), 0, S.H - 1));
                        const size_t row = (size_t)ref_rank(T, l, a & ~1, b & ~1, c) * S.nblocks;
                        const int cx1 = min(cx + 1, S.nbx - 1), cy1 = min(cy + 1, S.nby - 1);
                        D.d0.w = (uint32_t)cx | ((uint32_t)cy << 16);
                        D.d1.x = SLD(S, ref_tab, row + cy * S.nbx + cx);
                        D.d1.y = SLD(S, ref_tab, row + cy * S.nbx + cx1);
                        D.d1.z = SLD(S, ref_tab, row + cy1 * S.nbx + cx);
                        D.d1.w = SLD(S, ref_tab, row + cy1 * S.nbx + cx1);
                    }
                }
            }
            desc[d] = D;
        }
        __syncthreads();
        // ---- 2: levels L-1 .. 1: acc_l(node) = acc_{l+1}(parent) + SRV_l(node) ----
        int cur = 0;
        for (int l = L - 1; l >= 1; l--) {
            const int nn = F.nnu[l] * F.nnv[l];
            const int *par = acc_base + (cur ^ 1) * kAccInts;
            int *acc = acc_base + cur * kAccInts;
            for (int e = threadIdx.x; e < nn * F.npx; e += NT) {
                const int nd = qdiv(e, F.mag_npx);
                const int p = e - nd * F.npx;
                const int nv = F.nnv[l];   // nd < 4 nodes: the quotient by a few compares
                const int qa = nd >= nv ? (nd >= 2 * nv ? (nd >= 3 * nv ? 3 : 2) : 1) : 0;
                const int a = F.a0[l] + qa, b = F.b0[l] + nd - qa * nv;
                const PixGeom g = pix_geom(S, F, bk, p);
                const bool ref = is_ref(a, b);
                int v[3];
                if (l == L - 1) {
                    const size_t rb = ((size_t)(a >> 1) * T.gv[L] + (b >> 1)) * 3 * plane + (size_t)g.y * S.W + g.x;
                    v[0] = SLD(S, roots, rb);
                    v[1] = SLD(S, roots, rb + plane);
                    v[2] = SLD(S, roots, rb + 2 * plane);
                } else {
                    const int pn = ((a >> 1) - F.a0[l + 1]) * F.nnv[l + 1] + ((b >> 1) - F.b0[l + 1]);
                    const int *pp = par + pn * 3 * kMaxPx + p;
                    v[0] = pp[0];
                    v[1] = pp[kMaxPx];
                    v[2] = pp[2 * kMaxPx];
                }
                int *dst = acc + nd * 3 * kMaxPx + p;
#pragma unroll
                for (int c = 0; c < 3; c++)
                    dst[c * kMaxPx] = v[c] + srv_desc(S, bk, desc_at<BS>(desc, F, l, a, b, c, g.blk), ref, g);
            }
            __syncthreads();
            cur ^= 1;
        }
        // ---- 3: level-0 samples of the footprint's cameras -> RGB8 ----
        const int *acc1 = acc_base + (cur ^ 1) * kAccInts;          // level 1 (unused when L == 1)
        uint32_t *rgb = reinterpret_cast<uint32_t *>(acc_base + cur * kAccInts);
        const int ncam = (F.imax - F.imin + 1) * F.ncv;
        for (int e = threadIdx.x; e < ncam * F.npx; e += NT) {
            const int cam = qdiv(e, F.mag_npx);
            const int p = e - cam * F.npx;
            const int i = F.imin + cam / F.ncv, j = F.jmin + cam % F.ncv;
            const PixGeom g = pix_geom(S, F, bk, p);
            int v[3];
            if (L == 1) {
                const size_t rb = ((size_t)(i >> 1) * T.gv[1] + (j >> 1)) * 3 * plane + (size_t)g.y * S.W + g.x;
                v[0] = SLD(S, roots, rb);
                v[1] = SLD(S, roots, rb + plane);
                v[2] = SLD(S, roots, rb + 2 * plane);
            } else {
                const int pn = ((i >> 1) - F.a0[1]) * F.nnv[1] + ((j >> 1) - F.b0[1]);
                const int *pp = acc1 + pn * 3 * kMaxPx + p;
                v[0] = pp[0];
                v[1] = pp[kMaxPx];
                v[2] = pp[2 * kMaxPx];
            }
            const bool ref = is_ref(i, j);
#pragma unroll
            for (int c = 0; c < 3; c++) v[c] += srv_desc(S, bk, desc_at<BS>(desc, F, 0, i, j, c, g.blk), ref, g);
            rgb[e] = ycocg_to_rgb8(v[0], v[1], v[2]);
        }
        (void)B;
        __syncthreads();
        // ---- 4: blend ----
        if (act) {
            const int npx = F.npx;
            const int ci[2] = {(r.i0 - F.imin) * F.ncv * npx, (r.i1 - F.imin) * F.ncv * npx};
            const int cj[2] = {(r.j0 - F.jmin) * npx, (r.j1 - F.jmin) * npx};
            const int cy[2] = {(r.y0 - F.ymin) * F.nx, (r.y1 - F.ymin) * F.nx};
            const int cx[2] = {r.x0 - F.xmin, r.x1 - F.xmin};
            blend16(r, [&](int a, int b, int xs, int ys, int, int, int, int) { return rgb[ci[a] + cj[b] + cy[ys] + cx[xs]]; },
                    o);
        }
    }
    if (act) {
        // write-streaming stores: the output must not evict the decode's working set from L2
        float *dst = out + V.out_offset + ((size_t)py * V.width + px) * 3;
        __stcs(dst, o[0]);
        __stcs(dst + 1, o[1]);
        __stcs(dst + 2, o[2]);
    }
}

// ---------------------------------------------------------------------------
// differentiable relaxation: forward and adjoint (one thread per ray)
// ---------------------------------------------------------------------------

struct RelaxTap {
    int x[4], y[4];
    float w[4];
};

__device__ __forceinline__ void relax_taps(const DevStream &S, int x, int y, int mvx, int mvy, RelaxTap &t) {
    const int X = 4 * x + mvx, Y = 4 * y + mvy;
    const int x0 = X >> 2, y0 = Y >> 2, fx = X & 3, fy = Y & 3;
    const int xa = clampi(x0, 0, S.W - 1), xb = clampi(x0 + 1, 0, S.W - 1);
    const int ya = clampi(y0, 0, S.H - 1), yb = clampi(y0 + 1, 0, S.H - 1);
    t.x[0] = xa; t.y[0] = ya; t.w[0] = (float)((4 - fx) * (4 - fy)) * 0.0625f;
    t.x[1] = xb; t.y[1] = ya; t.w[1] = (float)(fx * (4 - fy)) * 0.0625f;
    t.x[2] = xa; t.y[2] = yb; t.w[2] = (float)((4 - fx) * fy) * 0.0625f;
    t.x[3] = xb; t.y[3] = yb; t.w[3] = (float)(fx * fy) * 0.0625f;
}

// Expected rounding of the integer predictor (+8 >> 4) against its exact
// weighted sum S / 16 when S is equally likely in every residue class its
// weights allow: the weights share g = gcd(4 - fx, fx) * gcd(4 - fy, fy),
// so floor((S + 8) / 16) - S / 16 averages g / 32 (0 for integer motion).
__device__ __forceinline__ float mc_rounding_bias(int mvx, int mvy) {
    const int fx = mvx & 3, fy = mvy & 3;
    if ((fx | fy) == 0) return 0.f;
    const int gx = fx == 0 ? 4 : (fx == 2 ? 2 : 1), gy = fy == 0 ? 4 : (fy == 2 ? 2 : 1);
    return (float)(gx * gy) * (1.0f / 32.0f);
}

// bias (forward only): every rounding the relaxation drops carries its
// expected value -- each predictor mc_rounding_bias, each >> 1 of the YCoCg-R
// inverse -1/4.  The adjoint does not depend on it (the terms are constant).
template <int BS, bool kBackward>
__global__ void __launch_bounds__(256) k_relax(const __grid_constant__ DevStream S,
                                              const __grid_constant__ LaunchViews LV, const float *__restrict__ coeff,
                                              const float *__restrict__ root, float *__restrict__ out,
                                              const float *__restrict__ gout, float *__restrict__ gcoeff,
                                              float *__restrict__ groot, int bias) {
    constexpr int TW = 16, TH = 16;
    __shared__ LevelTabs T;
    __shared__ int s_view;
    load_tabs(S, T);
    if (threadIdx.x == 0) s_view = find_view(LV, blockIdx.x);
    __syncthreads();
    const hmlfc_view &V = LV.views[s_view];
    const int tiles_x = (V.width + TW - 1) / TW;
    const int local = blockIdx.x - LV.tile_start[s_view];
    const int px = (local % tiles_x) * TW + (int)threadIdx.x % TW;
    const int py = (local / tiles_x) * TH + (int)threadIdx.x / TW;
    if (px >= V.width || py >= V.height) return;
    const Blk<BS> bk(S.B);
    Ray r;
    ray_setup(V, S.nu, S.nv, S.W, S.H, px, py, r);
    const size_t plane = (size_t)S.W * S.H;
    const int L = S.L;
    const size_t opix = V.out_offset + ((size_t)py * V.width + px) * 3;
    float g[3] = {0.f, 0.f, 0.f};
    if (kBackward) {
        g[0] = gout[opix] * (1.0f / 255.0f);
        g[1] = gout[opix + 1] * (1.0f / 255.0f);
        g[2] = gout[opix + 2] * (1.0f / 255.0f);
    }
    const float wu[2] = {1.0f - r.fu, r.fu}, wv[2] = {1.0f - r.fv, r.fv};
    const float ws[2] = {1.0f - r.fs, r.fs}, wt[2] = {1.0f - r.ft, r.ft};
    const int ii[2] = {r.i0, r.i1}, jj[2] = {r.j0, r.j1}, xx[2] = {r.x0, r.x1}, yy[2] = {r.y0, r.y1};
    float acc[3] = {0.f, 0.f, 0.f};
    for (int s = 0; s < 16; s++) {
        const int a = s >> 3, b = (s >> 2) & 1, xs = (s >> 1) & 1, ys = s & 1;
        const float w = wu[a] * wv[b] * ws[xs] * wt[ys];
        const int i = ii[a], j = jj[b], x = xx[xs], y = yy[ys];
        const int B = bk.size();
        const int k = bk.div(y) * S.nbx + bk.div(x);
        const size_t pix = (size_t)y * S.W + x;
        const size_t rb = ((size_t)(i >> L) * T.gv[L] + (j >> L)) * 3 * plane + pix;
        (void)B;
        if (!kBackward) {
            float v[3];
            for (int c = 0; c < 3; c++) v[c] = root[rb + c * plane];
            for (int l = 0; l < L; l++) {
                const int na = i >> l, nb = j >> l;
                for (int c = 0; c < 3; c++) {
                    const int nc = nc_index(T, l, na, nb, c);
                    v[c] += coeff[(size_t)nc * plane + pix];
                    if (!is_ref(na, nb) && S.mc) {
                        const uint32_t sym = bise_get_long(S.mvs, S.mv_mode, S.mv_b,
                                                           mv_index(S, T, l, na, nb, c, k));
                        int mvx, mvy, sign;
                        decode_mv(S, sym, mvx, mvy, sign);
                        RelaxTap t;
                        relax_taps(S, x, y, mvx, mvy, t);
                        const int rnc = nc_index(T, l, na & ~1, nb & ~1, c);
                        float p = bias ? mc_rounding_bias(mvx, mvy) : 0.f;
                        for (int q = 0; q < 4; q++) p += t.w[q] * coeff[(size_t)rnc * plane + (size_t)t.y[q] * S.W + t.x[q]];
                        v[c] += (float)sign * p;
                    }
                }
            }
            const float rb2 = bias ? 0.25f : 0.f;
            const float tt = v[0] - 0.5f * v[2] + rb2;
            const float G = v[2] + tt;
            const float Bc = tt - 0.5f * v[1] + rb2;
            acc[0] += w * (Bc + v[1]);
            acc[1] += w * G;
            acc[2] += w * Bc;
        } else {
            const float gR = w * g[0], gG = w * g[1], gB = w * g[2];
            const float gv3[3] = {gR + gG + gB, 0.5f * gR - 0.5f * gB, -0.5f * gR + 0.5f * gG - 0.5f * gB};
            for (int c = 0; c < 3; c++) atomicAdd(groot + rb + c * plane, gv3[c]);
            for (int l = 0; l < L; l++) {
                const int na = i >> l, nb = j >> l;
                for (int c = 0; c < 3; c++) {
                    const int nc = nc_index(T, l, na, nb, c);
                    atomicAdd(gcoeff + (size_t)nc * plane + pix, gv3[c]);
                    if (!is_ref(na, nb) && S.mc) {
                        const uint32_t sym = bise_get_long(S.mvs, S.mv_mode, S.mv_b,
                                                           mv_index(S, T, l, na, nb, c, k));
                        int mvx, mvy, sign;
                        decode_mv(S, sym, mvx, mvy, sign);
                        RelaxTap t;
                        relax_taps(S, x, y, mvx, mvy, t);
                        const int rnc = nc_index(T, l, na & ~1, nb & ~1, c);
                        for (int q = 0; q < 4; q++)
                            if (t.w[q] != 0.f)
                                atomicAdd(gcoeff + (size_t)rnc * plane + (size_t)t.y[q] * S.W + t.x[q],
                                          (float)sign * t.w[q] * gv3[c]);
                    }
                }
            }
        }
    }
    if (!kBackward) {
        out[opix] = acc[0] * (1.0f / 255.0f);
        out[opix + 1] = acc[1] * (1.0f / 255.0f);
        out[opix + 2] = acc[2] * (1.0f / 255.0f);
    }
}

// Dequantised coefficients of every node-channel (float [n_nc][H][W]); the
// rows after the last node-channel copy the root planes (float
// [roots][3][H][W]).
template <int BS>
__global__ void __launch_bounds__(256) k_dequant(const __grid_constant__ DevStream S, int64_t n_nc,
                                                float *__restrict__ coeff, float *__restrict__ root) {
    __shared__ LevelTabs T;
    __shared__ int s_l, s_a, s_b, s_c;
    load_tabs(S, T);
    const int64_t plane = (int64_t)S.W * S.H;
    const int64_t row = blockIdx.y;
    if (threadIdx.x == 0 && row < n_nc) {
        int l = S.L - 1;
        while (l > 0 && row >= S.nc_base[l - 1]) l--;
        const int e = (int)(row - S.nc_base[l]);
        s_l = l;
        s_c = e % 3;
        s_a = (e / 3) / S.gv[l];
        s_b = (e / 3) % S.gv[l];
    }
    __syncthreads();
    const Blk<BS> bk(S.B);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < plane; p += (int64_t)gridDim.x * blockDim.x) {
        if (row >= n_nc) {
            const int64_t q = (row - n_nc) * plane + p;
            root[q] = (float)S.roots[q];
            continue;
        }
        const int x = (int)(p % S.W), y = (int)(p / S.W);
        const int B = bk.size();
        const int bx = bk.div(x), by = bk.div(y);
        int v;
        if (is_ref(s_a, s_b)) {
            v = ref_coef(S, bk, s_c, (uint32_t)ref_rank(T, s_l, s_a, s_b, s_c) * S.nblocks, x, y);
        } else {
            const int bw = min(B, S.W - bx * B), bh = min(B, S.H - by * B);
            v = residual(S, (int)row, by * S.nbx + bx, (uint32_t)((y - by * B) * bw + (x - bx * B)), bw * bh);
        }
        coeff[row * plane + p] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// K1 (cached form): decode every block a call's views reach once, then blend
// ---------------------------------------------------------------------------
//
// mark:   each 16 x 16 ray tile flags the (camera, block) pairs of its
//         footprint's bounding box (idempotent byte stores);
// assign: every camera with a flagged block gets a slot of the call's cache
//         (a whole W x H RGB8 image; cameras past the capacity keep kNone and
//         their rays decode directly), and every (level-2 node, block) with
//         a flagged camera becomes a decode item;
// decode: a persistent kernel decodes each item's flagged blocks -- root +
//         every level of the tree path with motion re-compensation, the
//         levels the item's cameras share evaluated once -- to RGB8 in the
//         camera images;
// render: each ray gathers its 16 RGB8 samples from the images and blends.

// Descriptor of block (bx, by) of node (a, b) at level l, channel c.
template <int BS>
__device__ Desc make_desc(const DevStream &S, const LevelTabs &T, const Blk<BS> &bk, int l, int a, int b, int c, int bx,
                          int by) {
    const int B = bk.size();
    const int k = by * S.nbx + bx;
    Desc D;
    D.d0 = make_uint4(kNone, 0u, 0u, 0u);
    D.d1 = make_uint4(0u, 0u, 0u, 0u);
    if (is_ref(a, b)) {
        D.d1.x = SLD(S, ref_tab, (size_t)ref_rank(T, l, a, b, c) * S.nblocks + k);
        return D;
    }
    const int nc = nc_index(T, l, a, b, c);
    const uint4 g = SLD(S, groups, (size_t)nc * S.ngroups + (k >> 5));
    const uint32_t bit = (uint32_t)k & 31u;
    if ((g.x >> bit) & 1u) {
        const uint32_t rec = g.y + SLD(S, offs, g.z + __popc(g.x & ((1u << bit) - 1u)));
        D.d0.x = rec;
        D.d0.y = SLD(S, recs, rec);
        if (!rec_ok(S, rec, D.d0.y, min(B, S.W - bx * B) * min(B, S.H - by * B))) D.d0.x = kNone;
    }
    if (S.mc) {
        const uint32_t sym =
            bise_get_long(S.mvs, S.mv_mode, S.mv_b, mv_index(S, T, l, a, b, c, k));
        int mvx, mvy, sign;
        decode_mv(S, sym, mvx, mvy, sign);
        D.d0.z = (uint32_t)(mvx + 512) | ((uint32_t)(mvy + 512) << 10) | ((sign < 0 ? 1u : 0u) << 20);
        const int cx = bk.div(clampi(bx * B + (mvx >> 2), 0, S.W - 1));
        const int cy = bk.div(clampi(by * B + (mvy >> 2), 0, S.H - 1));
        const size_t row = (size_t)ref_rank(T, l, a & ~1, b & ~1, c) * S.nblocks;
        const int cx1 = min(cx + 1, S.nbx - 1), cy1 = min(cy + 1, S.nby - 1);
        D.d0.w = (uint32_t)cx | ((uint32_t)cy << 16);
        D.d1.x = SLD(S, ref_tab, row + cy * S.nbx + cx);
        D.d1.y = SLD(S, ref_tab, row + cy * S.nbx + cx1);
        D.d1.z = SLD(S, ref_tab, row + cy1 * S.nbx + cx);
        D.d1.w = SLD(S, ref_tab, row + cy1 * S.nbx + cx1);
    }
    return D;
}

// Index of the flag of (camera (i, j), block k).  kSuper: grouped by super
// key -- the (2^K)^2 cameras of a (level-K node, block) pair, K = min(2, L),
// are consecutive bytes (a zero-padded group at the grid's edge); otherwise
// camera-major, i * nv * nblocks + j * nblocks + k.
template <bool kSuper>
__device__ __forceinline__ size_t flag_index(const DevStream &S, int i, int j, int k) {
    if (!kSuper) return ((size_t)i * S.nv + j) * S.nblocks + k;
    const int K = S.L < 2 ? S.L : 2, cpa = 1 << K;
    const size_t node = (size_t)(i >> K) * S.gv[K] + (j >> K);
    return ((node * S.nblocks + k) << (2 * K)) + (size_t)(((i & (cpa - 1)) << K) | (j & (cpa - 1)));
}

// Mark the (camera, block) pairs of the tiles' footprints; eight tiles per
// warp, one per group of 4 lanes.  Under a projective map with w > 0 over the
// tile, each coordinate's extremes over the tile's pixel centres are at its
// corner pixels, so the 4 corner rays bound the footprint; the box is widened
// by a margin (1e-3 in u and v, 1e-2 in s and t) orders of magnitude above
// the fp32 rounding of interior rays.  A tile whose w is not positive at all
// corners is marked ray by ray, with the blend's own ray arithmetic, by the
// whole warp.  A group's lanes share its box's (camera, block) pairs.
template <int BS, int TW, int TH, bool kSuper>
__global__ void __launch_bounds__(256) k_mark(const __grid_constant__ DevStream S,
                                             const __grid_constant__ LaunchViews LV, int total_tiles,
                                             uint8_t *__restrict__ flags) {
    const int lane = threadIdx.x & 31, q = lane & 3;
    // eight tiles per warp, one per group of 4 lanes; each lane evaluates one corner ray of its group's tile
    const int tile = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 8) + (lane >> 2);
    const bool valid = tile < total_tiles;
    const int vi = find_view(LV, valid ? tile : total_tiles - 1);
    const hmlfc_view &V = LV.views[vi];
    const int tiles_x = (V.width + TW - 1) / TW;
    const int local = (valid ? tile : total_tiles - 1) - LV.tile_start[vi];
    const int x0 = (local % tiles_x) * TW, y0 = (local / tiles_x) * TH;
    const int x1 = min(x0 + TW, V.width) - 1, y1 = min(y0 + TH, V.height) - 1;
    const Blk<BS> bk(S.B);
    const float eps_uv = 1e-3f, eps_st = 1e-2f;
    const float X = (float)((q & 1) ? x1 : x0) + 0.5f, Y = (float)((q & 2) ? y1 : y0) + 0.5f;
    const float *h = V.H_uv, *g = V.H_st;
    const float wu = h[6] * X + h[7] * Y + h[8], ws = g[6] * X + g[7] * Y + g[8];
    float lo[4] = {__fdividef(h[0] * X + h[1] * Y + h[2], wu), __fdividef(h[3] * X + h[4] * Y + h[5], wu),
                   __fdividef(g[0] * X + g[1] * Y + g[2], ws), __fdividef(g[3] * X + g[4] * Y + g[5], ws)};
    float hi[4] = {lo[0], lo[1], lo[2], lo[3]};
    bool ok = wu > 0.f && ws > 0.f;
#pragma unroll
    for (int k = 0; k < 4; k++) ok = ok && lo[k] == lo[k];   // NaN
    // a butterfly over the group's 4 lanes gives each the extremes of its tile's corners
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
        }
        const int ok_other = __shfl_xor_sync(0xFFFFFFFFu, (int)ok, o);   // every lane takes part
        ok = ok && ok_other != 0;
    }
    // tiles whose w is not positive at every corner: the whole warp marks them ray by ray, one at a time
    for (unsigned bad = __ballot_sync(0xFFFFFFFFu, valid && !ok) & 0x11111111u; bad; bad &= bad - 1u) {
        const int src = __ffs(bad) - 1;                    // the tile's group leader
        const int bvi = __shfl_sync(0xFFFFFFFFu, vi, src);
        const int bx0 = __shfl_sync(0xFFFFFFFFu, x0, src), by0 = __shfl_sync(0xFFFFFFFFu, y0, src);
        const int bx1 = __shfl_sync(0xFFFFFFFFu, x1, src), by1 = __shfl_sync(0xFFFFFFFFu, y1, src);
        const hmlfc_view &BV = LV.views[bvi];
        const int tw = bx1 - bx0 + 1, n = tw * (by1 - by0 + 1);
        for (int e = lane; e < n; e += 32) {
            const int py = by0 + e / tw, px = bx0 + e % tw;
            Ray r;
            ray_setup(BV, S.nu, S.nv, S.W, S.H, px, py, r);
            const int ci[2] = {(r.i0 >> S.lod) << S.lod, (r.i1 >> S.lod) << S.lod};
            const int cj[2] = {(r.j0 >> S.lod) << S.lod, (r.j1 >> S.lod) << S.lod};
            const int kb[4] = {bk.div(r.y0) * S.nbx + bk.div(r.x0), bk.div(r.y0) * S.nbx + bk.div(r.x1),
                               bk.div(r.y1) * S.nbx + bk.div(r.x0), bk.div(r.y1) * S.nbx + bk.div(r.x1)};
            for (int k = 0; k < 16; k++) flags[flag_index<kSuper>(S, ci[k >> 3], cj[(k >> 2) & 1], kb[k & 3])] = 1;
        }
    }
    if (!valid || !ok) return;                             // no warp-wide operation follows
    const int n[4] = {S.nu, S.nv, S.W, S.H};
    int bl[4], bh[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float e = k < 2 ? eps_uv : eps_st;
        int a0, a1, b0, b1;
        axis_nb(lo[k] - e, n[k], a0, a1);
        axis_nb(hi[k] + e, n[k], b0, b1);
        bl[k] = a0;
        bh[k] = b1;
    }
    const int bx0 = bk.div(bl[2]), by0 = bk.div(bl[3]);
    const int nbx = bk.div(bh[2]) - bx0 + 1, by1 = bk.div(bh[3]);
    const int sh = S.lod;                                  // progressive decode: one representative camera per node
    const int i0 = (bl[0] >> sh) << sh, j0 = (bl[1] >> sh) << sh;
    // the group's lanes take the box's (camera, block row) pairs in turn; each stores its row's blocks, whose
    // flags lie a fixed stride apart (one block further in either layout)
    const size_t stride = kSuper ? (size_t)1 << (2 * (S.L < 2 ? S.L : 2)) : 1;
    int e = 0;
    for (int i = i0; i <= bh[0]; i += 1 << sh)
        for (int j = j0; j <= bh[1]; j += 1 << sh)
            for (int by = by0; by <= by1; by++, e++) {
                if ((e & 3) != q) continue;
                uint8_t *f = flags + flag_index<kSuper>(S, i, j, by * S.nbx + bx0);
                for (int bx = 0; bx < nbx; bx++) f[bx * stride] = 1;
            }
}

// Per-camera decoded images: a call gives every camera its views reach (a
// camera with a flagged block) one slot of W x H RGB8 pixels (u32 each) in its
// scratch, in the order the cameras are found; cameras beyond the capacity
// keep kNone and their rays decode directly.  Only the flagged blocks of a
// slot are written.
//
// Decode items: a super key is a (level-K node, block) pair, K = min(2, L);
// every super key with a flagged camera among its (2^K)^2 cameras becomes one
// item {super key, camera mask, 0, 0}.  One launch does both: the first
// blocks of the grid the items, the rest the camera slots.
__global__ void __launch_bounds__(256) k_assign(const __grid_constant__ DevStream S, const uint8_t *__restrict__ flags,
                                                uint32_t *__restrict__ camslot, uint4 *__restrict__ items,
                                                unsigned long long *__restrict__ counters, uint32_t capacity,
                                                int item_blocks) {
    const int K = S.L < 2 ? S.L : 2, cpa = 1 << K, ncg = cpa * cpa;
    if ((int)blockIdx.x >= item_blocks) {           // camera slots: one warp per camera
        const int cam = ((int)blockIdx.x - item_blocks) * 8 + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
        if (cam >= S.nu * S.nv) return;
        const int i = cam / S.nv, j = cam - (cam / S.nv) * S.nv;
        const uint8_t *f = flags + flag_index<true>(S, i, j, 0);   // block k of this camera at f[k * ncg]
        uint32_t any = 0;
        for (int k = lane; k < S.nblocks; k += 32) any |= __ldg(f + (size_t)k * ncg);
        any = __any_sync(0xFFFFFFFFu, any != 0);
        if (lane == 0) {
            uint32_t slot = kNone;
            if (any) {
                const uint32_t s = (uint32_t)atomicAdd(counters + 1, 1ull);
                if (s < capacity) slot = s;
            }
            camslot[cam] = slot;
        }
        return;
    }
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_base;
    const int64_t n_sk = (int64_t)S.gu[K] * S.gv[K] * S.nblocks;
    const int64_t sk = (int64_t)blockIdx.x * 256 + threadIdx.x;
    uint32_t mask = 0;
    if (sk < n_sk) {
        const uint8_t *f = flags + ((size_t)sk << (2 * K));       // the super key's camera flags, consecutive
        if (K == 2) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(f));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 16; q++) mask |= ((w[q >> 2] >> (8 * (q & 3))) & 0xFFu) ? 1u << q : 0u;
        } else {
            for (int q = 0; q < ncg; q++) mask |= f[q] ? 1u << q : 0u;
        }
    }
    const uint32_t nitem = mask ? 1u : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ii = nitem;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, ii, o);
        if (lane >= o) ii += v;
    }
    if (lane == 31) s_warp[warp] = ii;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0;
        for (int w = 0; w < 8; w++) {
            const uint32_t v = s_warp[w];
            s_warp[w] = a;
            a += v;
        }
        s_base = (uint32_t)(atomicAdd(counters, (unsigned long long)a << 32) >> 32);
    }
    __syncthreads();
    if (mask) items[s_base + s_warp[warp] + ii - nitem] = make_uint4((uint32_t)sk, mask, 0u, 0u);
}

// Descriptor of one (level, node, channel) of a decode item, for the block
// decode (32 B, shared memory).  The resident reference SRVs are read as
// dense planes: `base` points at the value under the block's first pixel --
// the node's own plane for a reference node, the reference's plane shifted
// by the integer part of the motion vector for a predictive one -- so every
// tap of every pixel is base + (pixel offset in the block) + a constant.
// Blocks whose taps would leave the image take the clamped path instead,
// with base at the plane origin and the tap origin in (ox, oy).  A
// significant predictive block's residual r^ is read from its resident tile
// (decoded at load), `res` pointing at the tile's first value; every other
// descriptor points at the shared zero tile, so the read needs no branch.
constexpr uint32_t kDRef = 1u, kDNeg = 2u, kDClamp = 4u, kDInt = 8u, kDNoMC = 16u;

struct NDesc {
    const int16_t *base;
    const int16_t *res;    // residual tile; the zero tile when insignificant (r^ = 0)
    uint32_t w;            // bilinear weights w00 | w10 << 8 | w01 << 16 | w11 << 24 (sum 16)
    uint32_t flags;        // kD*
    int32_t ox, oy;        // clamped path: block origin + integer part of the motion vector
};
static_assert(sizeof(NDesc) == 32, "descriptor size");

// Descriptor of luma block (bx, by)'s region in channel c of node (a, b),
// level l.  Without sub-sampling, or for luma, the region is the block
// itself; for sub-sampled chroma it is the (B/2) x (B/2) chroma pixels under
// the luma block, at (bx * B/2, by * B/2) of the half-resolution plane, inside
// chroma block (bx >> 1, by >> 1) (B is even).
template <int BS>
__device__ NDesc make_ndesc(const DevStream &S, const LevelTabs &T, const Blk<BS> &bk, int l, int a, int b, int c,
                            int bx, int by) {
    const int B = bk.size();
    const bool half = S.sub && c > 0;
    const int span = half ? B / 2 : B;                         // extent of the region
    const int k = half ? (by >> 1) * S.cnbx[c] + (bx >> 1) : by * S.nbx + bx;
    const int x0 = bx * span, y0 = by * span;                  // region origin in the channel's plane
    const size_t plane = (size_t)S.W * S.H;                    // dense planes keep row stride W
    NDesc D;
    D.res = S.ptiles;                                          // tile 0: zeros
    D.w = 16u;
    D.ox = x0;
    D.oy = y0;
    if (is_ref(a, b)) {
        D.base = S.planes + (size_t)ref_rank(T, l, a, b, c) * plane + (size_t)y0 * S.W + x0;
        D.flags = kDRef;
        return D;
    }
    const int nc = nc_index(T, l, a, b, c);
    const uint4 g = SLD(S, groups, (size_t)nc * S.ngroups + (k >> 5));
    const uint32_t bit = (uint32_t)k & 31u;
    if ((g.x >> bit) & 1u) D.res = S.ptiles + (size_t)(1u + g.w + __popc(g.x & ((1u << bit) - 1u))) * B * S.pstride;
    D.base = S.planes;
    if (!S.mc) {
        D.flags = kDNoMC;
        return D;
    }
    const uint32_t sym = bise_get_long(S.mvs, S.mv_mode, S.mv_b, mv_index(S, T, l, a, b, c, k));
    int mvx, mvy, sign;
    decode_mv(S, sym, mvx, mvy, sign);
    const int fx = mvx & 3, fy = mvy & 3;     // X = 4x + mvx: floor(X / 4) = x + (mvx >> 2), X & 3 = mvx & 3
    D.w = (uint32_t)((4 - fx) * (4 - fy)) | ((uint32_t)(fx * (4 - fy)) << 8) | ((uint32_t)((4 - fx) * fy) << 16) |
          ((uint32_t)(fx * fy) << 24);
    D.ox = x0 + (mvx >> 2);
    D.oy = y0 + (mvy >> 2);
    const int16_t *rp = S.planes + (size_t)ref_rank(T, l, a & ~1, b & ~1, c) * plane;
    D.flags = sign < 0 ? kDNeg : 0u;
    // unclamped: every tap (x .. x + 2 of a pixel pair, y .. y + 1) of every pixel of the region lies in the plane
    if (D.ox >= 0 && D.oy >= 0 && D.ox + span + 1 <= S.cW[c] - 1 && D.oy + span <= S.cH[c] - 1) {
        D.base = rp + (size_t)D.oy * S.W + D.ox;
        if (fx == 0 && fy == 0) D.flags |= kDInt;
    } else {
        D.base = rp;
        D.flags |= kDClamp;
    }
    return D;
}

// SRV of one node-channel at a horizontally adjacent pixel pair of a block
// (Sec. 4.4, Sec. 4.8.1): p = in-block offset y * W + x of the first pixel,
// (xi, yi) its in-block position, ti its residual-tile index.  With `pair`
// the two pixels' residuals are one aligned 32-bit read at ti (even);
// without it (a sub-sampled chroma pixel shared by the pair) one value.  A
// reference node gives its resident R^; a predictive node sign * P + r^, P
// the quarter-pel bilinear of the reference's R^ with weights summing to
// 16, + 8, >> 4.
template <int BS, bool pair>
__device__ __forceinline__ void eval_pair(const DevStream &S, const NDesc &D, int c, int p, int xi, int yi, int ti,
                                          int &o0, int &o1) {
    const uint32_t f = D.flags;
#ifdef HMLFC_CHECK
    {   // the dense-plane reads below: [base + p, base + p + 2) or, unclamped, up to base + p + W + 3
        const bool near = (f & (kDRef | kDInt)) || (f & kDNoMC);
        const bool clamped = (f & kDClamp) && !(f & (kDRef | kDInt));
        if (!clamped && !(f & kDNoMC) &&
            !chk_span(S, S.planes, S.lim_planes, D.base + p, near ? 2 : (int64_t)S.W + 3)) {
            o0 = o1 = 0;
            return;
        }
        if (clamped && !chk_span(S, S.planes, S.lim_planes, D.base, (int64_t)S.cH[c] * S.W)) {
            o0 = o1 = 0;
            return;
        }
        if (!(f & kDRef) && !chk_span(S, S.ptiles, S.lim_ptiles, D.res + ti, pair ? 2 : 1)) {
            o0 = o1 = 0;
            return;
        }
    }
#endif
    if (f & kDRef) {
        o0 = __ldg(D.base + p);
        o1 = __ldg(D.base + p + 1);
        return;
    }
    // the residual, issued before the branches below so that its latency overlaps the taps'
    const uint32_t rr = pair ? __ldg(reinterpret_cast<const uint32_t *>(D.res + ti))
                             : (uint32_t)(uint16_t)__ldg(D.res + ti);
    const int r0 = (int)(int16_t)(rr & 0xFFFFu), r1 = pair ? (int)rr >> 16 : r0;
    if (f & kDNoMC) {
        o0 = r0;
        o1 = r1;
        return;
    }
    int p0, p1;
    if (f & kDInt) {
        p0 = __ldg(D.base + p);
        p1 = __ldg(D.base + p + 1);
    } else {
        int a0, a1, a2, b0, b1, b2;
        if (!(f & kDClamp)) {
            const int16_t *t = D.base + p;
            a0 = __ldg(t);
            a1 = __ldg(t + 1);
            a2 = __ldg(t + 2);
            t += S.W;
            b0 = __ldg(t);
            b1 = __ldg(t + 1);
            b2 = __ldg(t + 2);
        } else {
            const int X = D.ox + xi, Y = D.oy + yi, Wc = S.cW[c], Hc = S.cH[c];
            const int c0 = clampi(X, 0, Wc - 1), c1 = clampi(X + 1, 0, Wc - 1), c2 = clampi(X + 2, 0, Wc - 1);
            const int16_t *ra = D.base + (size_t)clampi(Y, 0, Hc - 1) * S.W;
            const int16_t *rb = D.base + (size_t)clampi(Y + 1, 0, Hc - 1) * S.W;
            a0 = __ldg(ra + c0);
            a1 = __ldg(ra + c1);
            a2 = __ldg(ra + c2);
            b0 = __ldg(rb + c0);
            b1 = __ldg(rb + c1);
            b2 = __ldg(rb + c2);
        }
        const int w00 = (int)(D.w & 0xFFu), w10 = (int)((D.w >> 8) & 0xFFu), w01 = (int)((D.w >> 16) & 0xFFu),
                  w11 = (int)(D.w >> 24);
        p0 = (w00 * a0 + w10 * a1 + w01 * b0 + w11 * b1 + 8) >> 4;
        p1 = (w00 * a1 + w10 * a2 + w01 * b1 + w11 * b2 + 8) >> 4;
    }
    o0 = (f & kDNeg) ? r0 - p0 : r0 + p0;
    o1 = (f & kDNeg) ? r1 - p1 : r1 + p1;
}

// Entry e of a decode item's descriptor list ((level-K node, block) pair,
// K = min(2, L), camera mask it.y): the shared levels L-1 .. K first, then
// level 1 of the 4 child nodes (K = 2), then level 0 of the (2^K)^2 cameras,
// channels innermost.  Returns false for the entry of a child node or camera
// that the item does not decode.
template <int BS>
__device__ __forceinline__ bool item_desc(const DevStream &S, const LevelTabs &T, const Blk<BS> &bk, const uint4 &it,
                                          int e, NDesc &D, int K) {
    const int L = S.L, cpa = 1 << K;
    const int n_sh = (L - K) * 3, n_mid = K == 2 ? 12 : 0;
    const int node = (int)(it.x / (uint32_t)S.nblocks), k = (int)(it.x - (uint32_t)node * S.nblocks);
    const int aK = node / T.gv[K], bK = node - (node / T.gv[K]) * T.gv[K];
    int l, a, b, c;
    if (e < n_sh) {
        l = K + e / 3;
        c = e - 3 * (l - K);
        a = aK >> (l - K);
        b = bK >> (l - K);
    } else if (e < n_sh + n_mid) {
        const int m = (e - n_sh) / 3;                           // child node m of level 1
        c = (e - n_sh) - 3 * m;
        l = 1;
        a = 2 * aK + (m >> 1);
        b = 2 * bK + (m & 1);
        const uint32_t under = 0x33u << (8 * (m >> 1) + 2 * (m & 1));   // its 2x2 cameras in the 4x4 mask
        if (!(it.y & under)) return false;
    } else {
        const int q = (e - n_sh - n_mid) / 3;
        c = (e - n_sh - n_mid) - 3 * q;
        l = 0;
        a = aK * cpa + q / cpa;
        b = bK * cpa + q % cpa;
        if (!((it.y >> q) & 1u)) return false;
    }
    D = make_ndesc(S, T, bk, l, a, b, c, k % S.nbx, k / S.nbx);
    return true;
}

// One pixel pair of a decode item `it` ({(level-K node, block) key, camera
// mask}, K = min(2, L)): pair pp of the block is row pp / ceil(B/2), columns
// 2 (pp % ceil(B/2)) and + 1.  Root + levels L-1 .. K once, level 1 once per
// active child node (K = 2), level 0 once per flagged camera, from the
// item's descriptors dd (item_desc order); dst_of(q) is the first pixel of
// camera q's image (nullptr: the camera has no image and is skipped).  Both
// pixels go through one evaluation site per (node, 3 channels) step.
template <int BS, bool kTile = false, class DstOf>
__device__ __forceinline__ void decode_item_pair(const DevStream &S, const LevelTabs &T, const Blk<BS> &bk,
                                                 const NDesc *__restrict__ dd, const uint4 &it, int pp,
                                                 DstOf dst_of, int K) {
    const int B = bk.size();
    const int L = S.L;
    const int n_sh = (L - K) * 3;                               // shared levels L-1 .. K
    const int n_mid = K == 2 ? 12 : 0;                          // level 1 of the 4 child nodes
    const int hp = (B + 1) >> 1;
    const int node = (int)(it.x / (uint32_t)S.nblocks), k = (int)(it.x - (uint32_t)node * S.nblocks);
    const int aK = node / T.gv[K], bK = node - (node / T.gv[K]) * T.gv[K];
    const int bx = k % S.nbx, by = k / S.nbx;
    const int yy = pp / hp, xx = 2 * (pp - yy * hp);
    const int bw = min(B, S.W - bx * B), bh = min(B, S.H - by * B);
    const bool in0 = xx < bw && yy < bh, in1 = xx + 1 < bw && yy < bh;
    const int xi = min(xx, bw - 1), yi = min(yy, bh - 1);   // pixels outside the image compute a copy
    const int p = yi * S.W + xi;
    const int ti = yy * S.pstride + xx;                 // even; rows and columns past the block read zeros
    const int gx = bx * B + xi, gy = by * B + yi;
    // sub-sampled chroma: both pixels of the pair are chroma pixel (gx >> 1, gy >> 1), at (xi >> 1,
    // yi >> 1) of the descriptors' half-size regions, inside chroma block (bx >> 1, by >> 1)
    const int xic = xi >> 1, yic = yi >> 1, pc = yic * S.W + xic;
    const int tic = ((by & 1) * (B / 2) + yic) * S.pstride + (bx & 1) * (B / 2) + xic;
    const size_t rb = ((size_t)(aK >> (L - K)) * T.gv[L] + (bK >> (L - K))) * (size_t)S.rnpx;
    int v0[3], v1[3];
    const int gx1 = in1 ? gx + 1 : gx;                 // the second pixel, when it is in the image
    v0[0] = SLD(S, roots, rb + S.roff[0] + (size_t)gy * S.W + gx);
    v1[0] = SLD(S, roots, rb + S.roff[0] + (size_t)gy * S.W + gx1);
#pragma unroll
    for (int c = 1; c < 3; c++) {
        if (S.sub) {
            v0[c] = v1[c] = SLD(S, roots, rb + S.roff[c] + (size_t)(gy >> 1) * S.cW[c] + (gx >> 1));
        } else {
            v0[c] = SLD(S, roots, rb + S.roff[c] + (size_t)gy * S.W + gx);
            v1[c] = SLD(S, roots, rb + S.roff[c] + (size_t)gy * S.W + gx1);
        }
    }
    const int lod = S.lod;                              // progressive decode: stop at level lod
    const uint32_t mask = it.y;
    const int nm = K == 2 ? 4 : 1;
    // kTile: a camera's block is a B x B slot (the serving form's resident cache), else a W x H image
    const size_t o0 = kTile ? (size_t)yy * B + xx : (size_t)gy * S.W + gx;
    // One evaluation site for every (node, 3 channels) step, so that the loop body stays small:
    // phase 0 the shared levels L-1 .. max(K, lod) into v; phase 1 the next child node m with a
    // flagged camera, its level 1 into w = v + SRV (K = 2, lod <= 1); phase 2 its flagged cameras
    // with a slot, level 0 into z = w + SRV (lod = 0), each stored to its camera image.
    int w0[3] = {0, 0, 0}, w1[3] = {0, 0, 0};
    int l = L - 1, m = -1, phase = 0, q = 0;
    uint32_t cams = 0;
    for (;;) {
        const NDesc *d = nullptr;
        if (phase == 0) {
            if (l >= max(K, lod)) {
                d = dd + (l - K) * 3;
                l--;
            } else {
                phase = 1;
                continue;
            }
        } else if (phase == 1) {
            if (++m >= nm) break;
            cams = K == 2 ? mask & (0x33u << (8 * (m >> 1) + 2 * (m & 1))) : mask;
            if (!cams) continue;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                w0[c] = v0[c];
                w1[c] = v1[c];
            }
            phase = 2;
            if (K == 2 && lod <= 1) {
                d = dd + n_sh + m * 3;
            } else {
                continue;
            }
        } else {
            if (!cams) {
                phase = 1;
                continue;
            }
            q = __ffs(cams) - 1;
            cams &= cams - 1;
            uint32_t *const img = dst_of(q);
            if (!img) continue;
            if (lod == 0) {
                d = dd + n_sh + n_mid + q * 3;
            } else {
                uint32_t *dst = img + o0;
                if (in0) dst[0] = ycocg_to_rgb8(w0[0], w0[1], w0[2]);
                if (in1) dst[1] = ycocg_to_rgb8(w1[0], w1[1], w1[2]);
                continue;
            }
        }
        int s0[3], s1[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (c > 0 && S.sub) {
                int unused;
                eval_pair<BS, false>(S, d[c], c, pc, xic, yic, tic, s0[c], unused);
                s1[c] = s0[c];
            } else {
                eval_pair<BS, true>(S, d[c], c, p, xi, yi, ti, s0[c], s1[c]);
            }
        }
        if (phase == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                v0[c] += s0[c];
                v1[c] += s1[c];
            }
        } else if (d == dd + n_sh + m * 3 && K == 2) {     // the child node's level 1
#pragma unroll
            for (int c = 0; c < 3; c++) {
                w0[c] += s0[c];
                w1[c] += s1[c];
            }
        } else {                                            // a camera's level 0
            uint32_t *dst = dst_of(q) + o0;
            const uint32_t c0 = ycocg_to_rgb8(w0[0] + s0[0], w0[1] + s0[1], w0[2] + s0[2]);
            const uint32_t c1 = ycocg_to_rgb8(w1[0] + s1[0], w1[1] + s1[1], w1[2] + s1[2]);
            if (in1 && !(reinterpret_cast<uintptr_t>(dst) & 7u)) {
                *reinterpret_cast<uint2 *>(dst) = make_uint2(c0, c1);   // both pixels, one store
            } else {
                if (in0) dst[0] = c0;
                if (in1) dst[1] = c1;
            }
        }
    }
}

// Decode the flagged blocks into the camera images, one item ((level-K node,
// block), K = min(2, L)) at a time: per pixel, the node's reconstruction
// (root + SRV levels L-1 .. K) is evaluated once, level 1 once per active
// child node (K = 2), and level 0 once per flagged camera with a slot.
// Persistent CTAs; several items per pass so that one descriptor phase
// serves more pixel work.  Each thread decodes two horizontally adjacent
// pixels, which share the descriptor reads and four of their six taps.
template <int BS>
__global__ void __launch_bounds__(256, 5) k_decode_blocks(const __grid_constant__ DevStream S,
                                                      const uint4 *__restrict__ items,
                                                      const unsigned long long *__restrict__ counters,
                                                      const uint32_t *__restrict__ camslot,
                                                      uint32_t *__restrict__ cache) {
    constexpr int kGroup = 2;                                   // items per pass
    constexpr int kDescPer = (kMaxLevels - 2) * 3 + 4 * 3 + 16 * 3;
    __shared__ LevelTabs T;
    __shared__ __align__(16) NDesc s_desc[kGroup * kDescPer];
    __shared__ uint32_t s_slot[kGroup][16];
    load_tabs(S, T);
    const Blk<BS> bk(S.B);
    const int B = bk.size();
    const int L = S.L, K = L < 2 ? L : 2, cpa = 1 << K;
    const int n_sh = (L - K) * 3;                               // shared levels L-1 .. K
    const int n_mid = K == 2 ? 12 : 0;                          // level 1 of the 4 child nodes
    const int nd = n_sh + n_mid + cpa * cpa * 3;
    const uint32_t n = (uint32_t)(__ldg(counters) >> 32);
    const size_t plane = (size_t)S.W * S.H;
    __syncthreads();
    for (uint32_t first = blockIdx.x * kGroup; first < n; first += gridDim.x * kGroup) {
        for (int d = threadIdx.x; d < kGroup * (nd + 16); d += blockDim.x) {
            const int gi = d / (nd + 16), e = d - gi * (nd + 16);
            if (first + gi >= n) continue;
            const uint4 it = __ldg(items + first + gi);
            if (e >= nd) {                                      // slots of the item's cameras
                const int q = e - nd;
                const int node = (int)(it.x / (uint32_t)S.nblocks);
                const int aK = node / T.gv[K], bK = node - (node / T.gv[K]) * T.gv[K];
                const int i = aK * cpa + q / cpa, j = bK * cpa + q % cpa;
                s_slot[gi][q] = (q < cpa * cpa && ((it.y >> q) & 1u)) ? __ldg(camslot + i * S.nv + j) : kNone;
                continue;
            }
            NDesc D;
            if (item_desc(S, T, bk, it, e, D, L < 2 ? L : 2)) s_desc[gi * kDescPer + e] = D;
        }
        __syncthreads();
        // two horizontally adjacent pixels per thread: (xx, yy) and (xx + 1, yy)
        const int hp = (B + 1) >> 1, npair = B * hp;
        for (int e = threadIdx.x; e < kGroup * npair; e += blockDim.x) {
            const int gi = e / npair, pp = e - gi * npair;
            if (first + gi >= n) continue;
            const NDesc *dd = s_desc + gi * kDescPer;
            const uint32_t *slots = s_slot[gi];
            decode_item_pair<BS>(S, T, bk, dd, __ldg(items + first + gi), pp, [&](int q) -> uint32_t * {
                const uint32_t sl = slots[q];
                return sl == kNone ? nullptr : cache + (size_t)sl * plane;
            }, K);
        }
        __syncthreads();
    }
}

// Blend of one ray whose samples are decoded directly (kept out of line so
// that the cached fast path keeps its registers; its arguments are plain
// values, so the caller keeps nothing in memory for it).
template <int BS>
__device__ __noinline__ float3 blend_direct(const DevStream &S, const hmlfc_view &V, int px, int py) {
    LevelTabs T;
    for (int t = 0; t <= kMaxLevels; t++) {
        T.gu[t] = S.gu[t];
        T.gv[t] = S.gv[t];
        if (t < kMaxLevels) {
            T.nc_base[t] = S.nc_base[t];
            T.ref_base[t] = S.ref_base[t];
            T.pred_base[t] = S.pred_base[t];
        }
    }
    const Blk<BS> bk(S.B);
    Ray r;
    ray_setup(V, S.nu, S.nv, S.W, S.H, px, py, r);
    float o[3];
    blend16(r, [&](int, int, int, int, int i, int j, int x, int y) { return sample_direct(S, T, bk, i, j, x, y); }, o);
    return make_float3(o[0], o[1], o[2]);
}

// Blend of the cached render: each ray gathers its 16 RGB8 samples from the
// decoded camera images (4 camera slots, then 4 pixels per camera at offsets
// shared by all cameras) and blends them quadrilinearly.  Each thread blends
// two rays of its tile, (px, py) and (px, py + TH / 2), which share the view
// lookup and the tile arithmetic.  kFallback: some camera may have no image
// (the call's cache could not hold every camera of the light field); a ray
// with such a camera decodes its samples directly.
// kOffsets: camslot holds each camera image's first pixel in `cache` (the
// batched form's pool of images of several sizes), not its slot index.
template <int BS, bool kFallback, bool kOffsets = false>
__device__ __forceinline__ void blend_cached_ray(const DevStream &S, const hmlfc_view &V, int px, int py,
                                                 const uint32_t *__restrict__ camslot,
                                                 const uint32_t *__restrict__ cache, float *__restrict__ out) {
    Ray r;
    ray_setup(V, S.nu, S.nv, S.W, S.H, px, py, r);
    const int sh = S.lod;                          // progressive decode: representative camera of the level-lod node
    const int i0 = (r.i0 >> sh) << sh, i1 = (r.i1 >> sh) << sh;
    const int j0 = (r.j0 >> sh) << sh, j1 = (r.j1 >> sh) << sh;
    const uint32_t s00 = __ldg(camslot + i0 * S.nv + j0), s01 = __ldg(camslot + i0 * S.nv + j1);
    const uint32_t s10 = __ldg(camslot + i1 * S.nv + j0), s11 = __ldg(camslot + i1 * S.nv + j1);
    float o[3];
    // slots are below 2^31 and kNone has the top bit set: one OR tells whether a camera has no image
    if (!kFallback || !((s00 | s01 | s10 | s11) >> 31)) {
        const uint32_t plane = (uint32_t)(S.W * S.H);
        const uint32_t p00 = (uint32_t)(r.y0 * S.W + r.x0);
        const uint32_t dx = (uint32_t)(r.x1 - r.x0), dy = (uint32_t)((r.y1 - r.y0) * S.W);
        const size_t ip = kOffsets ? 1 : plane;
        const uint32_t *c0 = cache + (size_t)s00 * ip + p00, *c1 = cache + (size_t)s01 * ip + p00;
        const uint32_t *c2 = cache + (size_t)s10 * ip + p00, *c3 = cache + (size_t)s11 * ip + p00;
        uint32_t val[16];
        // sample order of blend16: q = a*8 + b*4 + xs*2 + ys  ->  camera a*2+b, corner xs*2+ys
        val[0] = __ldg(c0); val[1] = __ldg(c0 + dy); val[2] = __ldg(c0 + dx); val[3] = __ldg(c0 + dx + dy);
        val[4] = __ldg(c1); val[5] = __ldg(c1 + dy); val[6] = __ldg(c1 + dx); val[7] = __ldg(c1 + dx + dy);
        val[8] = __ldg(c2); val[9] = __ldg(c2 + dy); val[10] = __ldg(c2 + dx); val[11] = __ldg(c2 + dx + dy);
        val[12] = __ldg(c3); val[13] = __ldg(c3 + dy); val[14] = __ldg(c3 + dx); val[15] = __ldg(c3 + dx + dy);
        blend16(r, [&](int a, int b, int xs, int ys, int, int, int, int) { return val[a * 8 + b * 4 + xs * 2 + ys]; }, o);
    } else {
        const float3 d = blend_direct<BS>(S, V, px, py);   // a camera beyond the cache capacity: decode this ray directly
        o[0] = d.x;
        o[1] = d.y;
        o[2] = d.z;
    }
    float *dst = out + V.out_offset + ((size_t)py * V.width + px) * 3;
    __stcs(dst, o[0]);
    __stcs(dst + 1, o[1]);
    __stcs(dst + 2, o[2]);
}

template <int BS, int TW, int TH, bool kFallback>
__global__ void __launch_bounds__(TW *TH / 4, 24) k_render_cached(const __grid_constant__ DevStream S,
                                                             const __grid_constant__ LaunchViews LV,
                                                             const uint32_t *__restrict__ camslot,
                                                             const uint32_t *__restrict__ cache, float *__restrict__ out) {
    int vi = 0;                                     // uniform over the CTA: one search per warp
    if ((threadIdx.x & 31) == 0) vi = find_view(LV, blockIdx.x);
    vi = __shfl_sync(0xFFFFFFFFu, vi, 0);
    const hmlfc_view &V = LV.views[vi];
    const int local = blockIdx.x - LV.tile_start[vi];
    const uint32_t mag = LV.tiles_x_magic[vi];
    const int ty = mag == 1u ? local / ((V.width + TW - 1) / TW) : qdiv(local, mag);
    const int px = (local - ty * ((V.width + TW - 1) / TW)) * TW + (int)threadIdx.x % TW;
    const int py = ty * TH + (int)threadIdx.x / TW;
    if (px >= V.width) return;
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (py + k * (TH / 4) < V.height) blend_cached_ray<BS, kFallback>(S, V, px, py + k * (TH / 4), camslot, cache, out);
}

// Blend from a decoded-block cache with one slot per (camera, block) pair
// (the serving form's resident cache): 16 slot lookups, then 16 cached RGB8
// samples.  A sample beyond the cache decodes its ray directly.
template <int BS, int TW, int TH>
__global__ void __launch_bounds__(TW *TH, 6) k_render_slots(const __grid_constant__ DevStream S,
                                                         const __grid_constant__ LaunchViews LV,
                                                         const uint32_t *__restrict__ slotmap,
                                                         const uint32_t *__restrict__ cache, float *__restrict__ out) {
    int vi = 0;                                     // uniform over the CTA: one search per warp
    if ((threadIdx.x & 31) == 0) vi = find_view(LV, blockIdx.x);
    vi = __shfl_sync(0xFFFFFFFFu, vi, 0);
    const hmlfc_view &V = LV.views[vi];
    const int local = blockIdx.x - LV.tile_start[vi];
    const uint32_t mag = LV.tiles_x_magic[vi];
    const int ty = mag == 1u ? local / ((V.width + TW - 1) / TW) : qdiv(local, mag);
    const int px = (local - ty * ((V.width + TW - 1) / TW)) * TW + (int)threadIdx.x % TW;
    const int py = ty * TH + (int)threadIdx.x / TW;
    if (px >= V.width || py >= V.height) return;
    const Blk<BS> bk(S.B);
    const int B = bk.size();
    Ray r;
    ray_setup(V, S.nu, S.nv, S.W, S.H, px, py, r);
    // slots of the 16 samples first (independent loads), then their values
    const uint32_t nv = (uint32_t)S.nv, nbl = (uint32_t)S.nblocks, nbx = (uint32_t)S.nbx;
    const int sh = S.lod;                          // progressive decode: representative camera of the level-lod node
    const uint32_t i0 = (uint32_t)((r.i0 >> sh) << sh), i1 = (uint32_t)((r.i1 >> sh) << sh);
    const uint32_t j0 = (uint32_t)((r.j0 >> sh) << sh), j1 = (uint32_t)((r.j1 >> sh) << sh);
    const uint32_t cam[4] = {i0 * nv + j0, i0 * nv + j1, i1 * nv + j0, i1 * nv + j1};
    const int bx[2] = {bk.div(r.x0), bk.div(r.x1)}, by[2] = {bk.div(r.y0), bk.div(r.y1)};
    const uint32_t blk[4] = {(uint32_t)(by[0] * S.nbx + bx[0]), (uint32_t)(by[1] * S.nbx + bx[0]),
                             (uint32_t)(by[0] * S.nbx + bx[1]), (uint32_t)(by[1] * S.nbx + bx[1])};
    const uint32_t off[4] = {(uint32_t)((r.y0 - by[0] * B) * B + (r.x0 - bx[0] * B)),
                             (uint32_t)((r.y1 - by[1] * B) * B + (r.x0 - bx[0] * B)),
                             (uint32_t)((r.y0 - by[0] * B) * B + (r.x1 - bx[1] * B)),
                             (uint32_t)((r.y1 - by[1] * B) * B + (r.x1 - bx[1] * B))};
    (void)nbx;
    uint32_t slot[16];
#pragma unroll
    for (int q = 0; q < 16; q++) slot[q] = __ldg(slotmap + (cam[q >> 2] * nbl + blk[q & 3]));
    // slots are below 2^31 and kNone has the top bit set: one OR tree tells whether any sample missed the cache
    uint32_t any_none = 0;
#pragma unroll
    for (int q = 0; q < 16; q++) any_none |= slot[q];
    float o[3];
    if (!(any_none >> 31)) {
        uint32_t val[16];
#pragma unroll
        for (int q = 0; q < 16; q++) val[q] = __ldg(cache + (slot[q] * (uint32_t)(B * B) + off[q & 3]));
        // sample order of blend16: q = a*8 + b*4 + xs*2 + ys  ->  cam a*2+b, corner xs*2+ys
        blend16(r, [&](int a, int b, int xs, int ys, int, int, int, int) { return val[a * 8 + b * 4 + xs * 2 + ys]; }, o);
    } else {
        const float3 d = blend_direct<BS>(S, V, px, py);   // a sample beyond the cache capacity: decode this ray directly
        o[0] = d.x;
        o[1] = d.y;
        o[2] = d.z;
    }
    float *dst = out + V.out_offset + ((size_t)py * V.width + px) * 3;   // write-streaming (see above)
    __stcs(dst, o[0]);
    __stcs(dst + 1, o[1]);
    __stcs(dst + 2, o[2]);
}

template <int BS>
cudaError_t render_dispatch_tw(const DevStream &ds, const LaunchViews &lv, int total_tiles, float *d_out, int mode,
                               cudaStream_t st) {
    constexpr int TW = 16, TH = 16;
    auto kern = k_render<BS, TW, TH>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kern<<<total_tiles, TW * TH, kStageSmem, st>>>(ds, lv, d_out, mode == 1 ? 1 : 0);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Batched form: many light fields and views in one pass
// ---------------------------------------------------------------------------
//
// A call's light-field descriptors, views and tile prefix live in device
// scratch (written by k_copy_blob from kernel parameters, so a captured
// graph keeps no pointer to host memory).  One launch each of mark, assign,
// decode (CTAs looping over the items of every light field) and render
// (persistent, atomic work queue over (view, tile) items) covers every light
// field of the call; the camera images of all light fields share one pool.

// Host-built image at the start of the batch scratch.
struct BatchHdr {
    int n_lf, n_views, total_tiles, tile_w, tile_h;
    int pad[3];
    int64_t n_keys, n_sk, n_cam;
};

// One light field of a batch: its stream and the first of its flags
// (super-key layout, a multiple of 16), super keys ((level-K node, block)
// pairs, K = min(2, L)) and cameras in the call's flattened arrays.
struct BatchLF {
    DevStream S;
    int64_t key_off, sk_off, cam_off;
};

struct BatchPtrs {     // device pointers into the scratch image
    const BatchHdr *hdr;
    const BatchLF *lf;
    const hmlfc_view *views;
    const int *tile_start;
};

// Copies a by-value blob of bytes into device memory.
constexpr int kBlobBytes = 30000;
struct Blob {
    int n;
    unsigned char b[kBlobBytes];
};

__global__ void k_copy_blob(const __grid_constant__ Blob blob, unsigned char *__restrict__ dst) {
    for (int k = threadIdx.x; k < blob.n; k += blockDim.x) dst[k] = blob.b[k];
}

__device__ __forceinline__ int find_view_dev(const int *__restrict__ tile_start, int n_views, int tile) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The light field of a flattened index (first index of each in off_of(lf)).
template <class OffOf>
__device__ __forceinline__ int find_lf(int n_lf, int64_t g, OffOf off_of) {
    int lf = 0;
    while (lf + 1 < n_lf && g >= off_of(lf + 1)) lf++;
    return lf;
}

// Marking of every light field's (camera, block) pairs, as k_mark: eight
// tiles per warp, one per group of 4 lanes, each with its own view and light
// field; the corner rays bound a tile's footprint (w > 0), otherwise the
// whole warp marks the tile ray by ray.
template <int BS, int TW, int TH>
__global__ void __launch_bounds__(256) k_mark_batch(const BatchPtrs P, uint8_t *__restrict__ flags) {
    const int lane = threadIdx.x & 31, q = lane & 3;
    const int total = P.hdr->total_tiles;
    const int tile = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 8) + (lane >> 2);
    const bool valid = tile < total;
    const int tc = valid ? tile : total - 1;
    const int vi = find_view_dev(P.tile_start, P.hdr->n_views, tc);
    const hmlfc_view &V = P.views[vi];
    const BatchLF &F = P.lf[V.lf];
    const DevStream &S = F.S;
    const int tiles_x = (V.width + TW - 1) / TW;
    const int local = tc - __ldg(P.tile_start + vi);
    const int x0 = (local % tiles_x) * TW, y0 = (local / tiles_x) * TH;
    const int x1 = min(x0 + TW, V.width) - 1, y1 = min(y0 + TH, V.height) - 1;
    const Blk<BS> bk(S.B);
    const float X = (float)((q & 1) ? x1 : x0) + 0.5f, Y = (float)((q & 2) ? y1 : y0) + 0.5f;
    const float *h = V.H_uv, *g = V.H_st;
    const float wu = h[6] * X + h[7] * Y + h[8], ws = g[6] * X + g[7] * Y + g[8];
    float lo[4] = {__fdividef(h[0] * X + h[1] * Y + h[2], wu), __fdividef(h[3] * X + h[4] * Y + h[5], wu),
                   __fdividef(g[0] * X + g[1] * Y + g[2], ws), __fdividef(g[3] * X + g[4] * Y + g[5], ws)};
    float hi[4] = {lo[0], lo[1], lo[2], lo[3]};
    bool ok = wu > 0.f && ws > 0.f;
#pragma unroll
    for (int k = 0; k < 4; k++) ok = ok && lo[k] == lo[k];   // NaN
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
        }
        const int ok_other = __shfl_xor_sync(0xFFFFFFFFu, (int)ok, o);   // every lane takes part
        ok = ok && ok_other != 0;
    }
    for (unsigned bad = __ballot_sync(0xFFFFFFFFu, valid && !ok) & 0x11111111u; bad; bad &= bad - 1u) {
        const int src = __ffs(bad) - 1;                    // the tile's group leader
        const int bvi = __shfl_sync(0xFFFFFFFFu, vi, src);
        const int bx0 = __shfl_sync(0xFFFFFFFFu, x0, src), by0 = __shfl_sync(0xFFFFFFFFu, y0, src);
        const int bx1 = __shfl_sync(0xFFFFFFFFu, x1, src), by1 = __shfl_sync(0xFFFFFFFFu, y1, src);
        const hmlfc_view &BV = P.views[bvi];
        const BatchLF &BF = P.lf[BV.lf];
        const DevStream &BSt = BF.S;
        const Blk<BS> bbk(BSt.B);
        const int tw = bx1 - bx0 + 1, n = tw * (by1 - by0 + 1);
        for (int e = lane; e < n; e += 32) {
            const int py = by0 + e / tw, px = bx0 + e % tw;
            Ray r;
            ray_setup(BV, BSt.nu, BSt.nv, BSt.W, BSt.H, px, py, r);
            const int ci[2] = {r.i0, r.i1}, cj[2] = {r.j0, r.j1};
            const int kb[4] = {bbk.div(r.y0) * BSt.nbx + bbk.div(r.x0), bbk.div(r.y0) * BSt.nbx + bbk.div(r.x1),
                               bbk.div(r.y1) * BSt.nbx + bbk.div(r.x0), bbk.div(r.y1) * BSt.nbx + bbk.div(r.x1)};
            for (int k = 0; k < 16; k++)
                flags[BF.key_off + flag_index<true>(BSt, ci[k >> 3], cj[(k >> 2) & 1], kb[k & 3])] = 1;
        }
    }
    if (!valid || !ok) return;                             // no warp-wide operation follows
    const int n[4] = {S.nu, S.nv, S.W, S.H};
    int bl[4], bh[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float e = k < 2 ? 1e-3f : 1e-2f;
        int a0, a1, b0, b1;
        axis_nb(lo[k] - e, n[k], a0, a1);
        axis_nb(hi[k] + e, n[k], b0, b1);
        bl[k] = a0;
        bh[k] = b1;
    }
    const int bx0 = bk.div(bl[2]), by0 = bk.div(bl[3]);
    const int nbx = bk.div(bh[2]) - bx0 + 1, by1 = bk.div(bh[3]);
    const size_t stride = (size_t)1 << (2 * (S.L < 2 ? S.L : 2));
    uint8_t *fl = flags + F.key_off;
    int e = 0;
    for (int i = bl[0]; i <= bh[0]; i++)
        for (int j = bl[1]; j <= bh[1]; j++)
            for (int by = by0; by <= by1; by++, e++) {
                if ((e & 3) != q) continue;
                uint8_t *f = fl + flag_index<true>(S, i, j, by * S.nbx + bx0);
                for (int bx = 0; bx < nbx; bx++) f[bx * stride] = 1;
            }
}

// Camera images and decode items of every light field.  The first
// item_blocks blocks: one thread per super key of the call; a super key with
// a flagged camera becomes the item {super key in its light field, camera
// mask, light field, 0}.  The rest: one warp per camera; a camera with a
// flagged block gets the offset (in pixels) of its W x H image in the call's
// image pool, or kNone beyond the pool's `capacity` pixels (its rays decode
// directly).
__global__ void __launch_bounds__(256) k_assign_batch(const BatchPtrs P, const uint8_t *__restrict__ flags,
                                                      uint32_t *__restrict__ camslot, uint4 *__restrict__ items,
                                                      unsigned long long *__restrict__ counters,
                                                      unsigned long long capacity, int item_blocks) {
    const int n_lf = P.hdr->n_lf;
    if ((int)blockIdx.x >= item_blocks) {           // camera images: one warp per camera
        const int64_t gcam = ((int64_t)blockIdx.x - item_blocks) * 8 + (threadIdx.x >> 5);
        const int lane = threadIdx.x & 31;
        if (gcam >= P.hdr->n_cam) return;
        const int lf = find_lf(n_lf, gcam, [&](int k) { return P.lf[k].cam_off; });
        const BatchLF &F = P.lf[lf];
        const DevStream &S = F.S;
        const int cam = (int)(gcam - F.cam_off);
        const int i = cam / S.nv, j = cam - (cam / S.nv) * S.nv;
        const int K = S.L < 2 ? S.L : 2;
        const uint8_t *f = flags + F.key_off + flag_index<true>(S, i, j, 0);   // block k at f[k << 2K]
        uint32_t any = 0;
        for (int k = lane; k < S.nblocks; k += 32) any |= __ldg(f + ((size_t)k << (2 * K)));
        any = __any_sync(0xFFFFFFFFu, any != 0);
        if (lane == 0) {
            uint32_t slot = kNone;
            if (any) {
                const unsigned long long px = (unsigned long long)S.W * S.H;
                const unsigned long long o = atomicAdd(counters + 1, px);
                if (o + px <= capacity) slot = (uint32_t)o;
            }
            camslot[gcam] = slot;
        }
        return;
    }
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_base;
    const int64_t gsk = (int64_t)blockIdx.x * 256 + threadIdx.x;
    uint32_t mask = 0;
    int lf = 0;
    int64_t sk = 0;
    if (gsk < P.hdr->n_sk) {
        lf = find_lf(n_lf, gsk, [&](int k) { return P.lf[k].sk_off; });
        const BatchLF &F = P.lf[lf];
        const int K = F.S.L < 2 ? F.S.L : 2, ncg = 1 << (2 * K);
        sk = gsk - F.sk_off;
        const uint8_t *f = flags + F.key_off + ((size_t)sk << (2 * K));   // the super key's camera flags
        if (K == 2) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(f));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int c = 0; c < 16; c++) mask |= ((w[c >> 2] >> (8 * (c & 3))) & 0xFFu) ? 1u << c : 0u;
        } else {
            for (int c = 0; c < ncg; c++) mask |= f[c] ? 1u << c : 0u;
        }
    }
    const uint32_t nitem = mask ? 1u : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ii = nitem;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, ii, o);
        if (lane >= o) ii += v;
    }
    if (lane == 31) s_warp[warp] = ii;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0;
        for (int w = 0; w < 8; w++) {
            const uint32_t v = s_warp[w];
            s_warp[w] = a;
            a += v;
        }
        s_base = (uint32_t)(atomicAdd(counters, (unsigned long long)a << 32) >> 32);
    }
    __syncthreads();
    if (mask) items[s_base + s_warp[warp] + ii - nitem] = make_uint4((uint32_t)sk, mask, (uint32_t)lf, 0u);
}

__device__ __forceinline__ void copy_words(void *dst, const void *src, int bytes) {
    const int n = bytes / 4;
    for (int t = threadIdx.x; t < n; t += blockDim.x)
        reinterpret_cast<uint32_t *>(dst)[t] = __ldg(reinterpret_cast<const uint32_t *>(src) + t);
}

// Block decode of every light field's items, as k_decode_blocks: G items per
// pass (G <= 4), each with its light field's stream and level tables copied
// to shared memory, its descriptors built by the whole CTA, then its pixel
// pairs decoded into its cameras' images (pool offsets in camslot).
template <int BS>
__global__ void __launch_bounds__(256, 5) k_decode_batch(const BatchPtrs P, const uint4 *__restrict__ items,
                                                        const unsigned long long *__restrict__ counters,
                                                        const uint32_t *__restrict__ camslot,
                                                        uint32_t *__restrict__ cache, int G) {
    constexpr int kMaxGroup = 4;
    constexpr int kDescPer = (kMaxLevels - 2) * 3 + 4 * 3 + 16 * 3;
    __shared__ __align__(16) DevStream s_S[kMaxGroup];
    __shared__ LevelTabs s_T[kMaxGroup];
    __shared__ __align__(16) NDesc s_desc[kMaxGroup * kDescPer];
    __shared__ uint32_t s_img[kMaxGroup][16];
    __shared__ uint4 s_it[kMaxGroup];
    const uint32_t n = (uint32_t)(__ldg(counters) >> 32);
    G = max(1, min(G, kMaxGroup));
    for (uint32_t first = blockIdx.x * G; first < n; first += gridDim.x * G) {
        __syncthreads();                                        // the previous pass is done with the slices
        for (int gi = 0; gi < G; gi++) {
            if (first + gi >= n) break;
            const uint4 it = __ldg(items + first + gi);
            if (threadIdx.x == 0) s_it[gi] = it;
            copy_words(&s_S[gi], &P.lf[it.z].S, (int)sizeof(DevStream));
        }
        __syncthreads();
        for (int gi = 0; gi < G; gi++)
            if (first + gi < n) load_tabs(s_S[gi], s_T[gi]);
        __syncthreads();
        for (int d = threadIdx.x; d < G * (kDescPer + 16); d += blockDim.x) {
            const int gi = d / (kDescPer + 16), e = d - gi * (kDescPer + 16);
            if (first + gi >= n) continue;
            const DevStream &S = s_S[gi];
            const LevelTabs &T = s_T[gi];
            const uint4 it = s_it[gi];
            const int L = S.L, K = L < 2 ? L : 2, cpa = 1 << K;
            const int nd = (L - K) * 3 + (K == 2 ? 12 : 0) + cpa * cpa * 3;
            if (e >= kDescPer) {                                // pool offsets of the item's cameras
                const int q = e - kDescPer;
                const int node = (int)(it.x / (uint32_t)S.nblocks);
                const int aK = node / T.gv[K], bK = node - (node / T.gv[K]) * T.gv[K];
                const int i = aK * cpa + q / cpa, j = bK * cpa + q % cpa;
                s_img[gi][q] = (q < cpa * cpa && ((it.y >> q) & 1u))
                                   ? __ldg(camslot + P.lf[it.z].cam_off + (int64_t)i * S.nv + j) : kNone;
                continue;
            }
            if (e >= nd) continue;
            const Blk<BS> bk(S.B);
            NDesc D;
            if (item_desc(S, T, bk, it, e, D, L < 2 ? L : 2)) s_desc[gi * kDescPer + e] = D;
        }
        __syncthreads();
        // two horizontally adjacent pixels per thread; an item's block size may differ from another's (BS = 0)
        int npair = 0;
        for (int gi = 0; gi < G && first + gi < n; gi++) {
            const int B = s_S[gi].B;
            npair = max(npair, B * ((B + 1) >> 1));
        }
        for (int e = threadIdx.x; e < G * npair; e += blockDim.x) {
            const int gi = e / npair, pp = e - gi * npair;
            if (first + gi >= n) continue;
            const DevStream &S = s_S[gi];
            const Blk<BS> bk(S.B);
            if (pp >= bk.size() * ((bk.size() + 1) >> 1)) continue;
            const uint32_t *img = s_img[gi];
            decode_item_pair<BS>(S, s_T[gi], bk, s_desc + gi * kDescPer, s_it[gi], pp, [&](int q) -> uint32_t * {
                const uint32_t o = img[q];
                return o == kNone ? nullptr : cache + o;
            }, S.L < 2 ? S.L : 2);
        }
    }
}

// Blend of every light field's views: persistent CTAs take (view, tile)
// items in order from a counter; each tile as k_render_cached, RPT rays per
// thread, from the cameras' images at their pool offsets (a camera without
// an image sends its rays to the direct decode).
template <int BS, int TW, int TH, int RPT>
__global__ void __launch_bounds__(TW *TH / RPT, 16) k_render_batch(const BatchPtrs P, const uint32_t *__restrict__ camslot,
                                                              const uint32_t *__restrict__ cache,
                                                              unsigned int *__restrict__ work, float *__restrict__ out) {
    __shared__ int s_tile;
    const int total = P.hdr->total_tiles, n_views = P.hdr->n_views;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int tile = s_tile;
        __syncthreads();                                        // every thread has read it before the next write
        if (tile >= total) break;
        int vi = 0;
        if ((threadIdx.x & 31) == 0) vi = find_view_dev(P.tile_start, n_views, tile);
        vi = __shfl_sync(0xFFFFFFFFu, vi, 0);
        const hmlfc_view &V = P.views[vi];
        const BatchLF &F = P.lf[V.lf];
        const int tiles_x = (V.width + TW - 1) / TW;
        const int local = tile - __ldg(P.tile_start + vi);
        const int ty = local / tiles_x;
        const int px = (local - ty * tiles_x) * TW + (int)threadIdx.x % TW;
        const int py = ty * TH + (int)threadIdx.x / TW;
        if (px >= V.width) continue;
#pragma unroll
        for (int k = 0; k < RPT; k++)
            if (py + k * (TH / RPT) < V.height)
                blend_cached_ray<BS, true, true>(F.S, V, px, py + k * (TH / RPT), camslot + F.cam_off, cache, out);
    }
}


// ---------------------------------------------------------------------------
// Serving form: a decoded-block cache that stays resident across calls
// ---------------------------------------------------------------------------
//
// Per slot: the (camera, block) key it holds (owner) and the call that last
// used it (epoch).  A call marks its blocks, stamps the resident ones with
// its epoch (hits), then claims slots for the rest by clock order (misses),
// taking only slots not stamped by this call -- so nothing the call uses is
// evicted -- and decodes the claimed blocks cluster by cluster.

// Hits: every flagged key that already has a slot stamps it.
__global__ void __launch_bounds__(256) k_resident_hits(const uint8_t *__restrict__ flags, int64_t n_keys,
                                                       const uint32_t *__restrict__ slotmap,
                                                       uint32_t *__restrict__ epoch, uint32_t cur) {
    for (int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; key < n_keys;
         key += (int64_t)gridDim.x * blockDim.x) {
        if (!flags[key]) continue;
        const uint32_t s = slotmap[key];
        if (s != kNone) epoch[s] = cur;
    }
}

// Misses, one thread per (level-1 node, block): claim a slot for every
// flagged camera without one; one decode item {cluster key, mask, -, -},
// {slot of camera 0..3} per cluster with a claimed camera.
__global__ void __launch_bounds__(256) k_resident_misses(const __grid_constant__ DevStream S,
                                                         const uint8_t *__restrict__ flags,
                                                         uint32_t *__restrict__ slotmap, uint32_t *__restrict__ owner,
                                                         uint32_t *__restrict__ epoch, uint32_t *__restrict__ clock,
                                                         uint32_t capacity, uint32_t cur, uint4 *__restrict__ items,
                                                         unsigned long long *__restrict__ counters) {
    const int64_t n_ck = (int64_t)S.gu[1] * S.gv[1] * S.nblocks;
    const int64_t ck = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ck >= n_ck) return;
    const int node = (int)(ck / S.nblocks), k = (int)(ck - (int64_t)node * S.nblocks);
    const int a1 = node / S.gv[1], b1 = node - (node / S.gv[1]) * S.gv[1];
    uint32_t mask = 0, slots[4] = {kNone, kNone, kNone, kNone};
    for (int q = 0; q < 4; q++) {
        const int i = 2 * a1 + (q >> 1), j = 2 * b1 + (q & 1);
        if (i >= S.nu || j >= S.nv) continue;
        const int64_t key = ((int64_t)i * S.nv + j) * S.nblocks + k;
        if (!flags[key] || slotmap[key] != kNone) continue;
        for (uint32_t tries = 0; tries < capacity; tries++) {
            const uint32_t s = atomicAdd(clock, 1u) % capacity;
            const uint32_t old = epoch[s];
            if (old == cur || atomicCAS(&epoch[s], old, cur) != old) continue;
            const uint32_t prev = owner[s];
            if (prev != kNone) slotmap[prev] = kNone;      // not used by this call (its epoch was older)
            owner[s] = (uint32_t)key;
            slotmap[key] = s;
            slots[q] = s;
            mask |= 1u << q;
            break;
        }
    }
    if (!mask) return;
    const unsigned long long old = atomicAdd(counters, (1ull << 32) | (unsigned long long)__popc(mask));
    const uint32_t item = (uint32_t)(old >> 32);
    items[2 * (size_t)item] = make_uint4((uint32_t)ck, mask, 0u, 0u);
    items[2 * (size_t)item + 1] = make_uint4(slots[0], slots[1], slots[2], slots[3]);
}

// Decode the claimed blocks (as k_decode_blocks) into their B x B slots:
// items are (level-1 node, block) pairs with a mask over the node's 2 x 2
// cameras and one slot per camera, decoded by the same pixel-pair
// evaluation over the dense reference planes and residual tiles.
template <int BS>
__global__ void __launch_bounds__(256, 5) k_decode_resident(const __grid_constant__ DevStream S,
                                                           const uint4 *__restrict__ items,
                                                           const unsigned long long *__restrict__ counters,
                                                           uint32_t *__restrict__ cache) {
    constexpr int kGroup = 4;
    constexpr int kDescPer = (kMaxLevels - 1) * 3 + 4 * 3;
    __shared__ LevelTabs T;
    __shared__ __align__(16) NDesc s_desc[kGroup * kDescPer];
    __shared__ uint4 s_it[kGroup][2];
    load_tabs(S, T);
    const Blk<BS> bk(S.B);
    const int B = bk.size(), B2 = B * B;
    const int L = S.L, K = L < 1 ? L : 1;
    const uint32_t n = (uint32_t)(__ldg(counters) >> 32);
    const int nd = (L - K) * 3 + 4 * 3;
    for (uint32_t first = blockIdx.x * kGroup; first < n; first += gridDim.x * kGroup) {
        __syncthreads();                                        // the previous pass is done with the slices
        if (threadIdx.x < 2 * kGroup && first + (threadIdx.x >> 1) < n)
            s_it[threadIdx.x >> 1][threadIdx.x & 1] = __ldg(items + 2 * (size_t)first + threadIdx.x);
        __syncthreads();
        for (int d = threadIdx.x; d < kGroup * nd; d += blockDim.x) {
            const int gi = d / nd, e = d - gi * nd;
            if (first + gi >= n) continue;
            NDesc D;
            if (item_desc(S, T, bk, s_it[gi][0], e, D, K)) s_desc[gi * kDescPer + e] = D;
        }
        __syncthreads();
        const int npair = B * ((B + 1) >> 1);
        for (int e = threadIdx.x; e < kGroup * npair; e += blockDim.x) {
            const int gi = e / npair, pp = e - gi * npair;
            if (first + gi >= n) continue;
            const uint4 sl = s_it[gi][1];
            decode_item_pair<BS, true>(S, T, bk, s_desc + gi * kDescPer, s_it[gi][0], pp, [&](int q) -> uint32_t * {
                const uint32_t slot = q == 0 ? sl.x : q == 1 ? sl.y : q == 2 ? sl.z : sl.w;
                return slot == kNone ? nullptr : cache + (size_t)slot * B2;
            }, K);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_decode_tiles(const DevStream &ds, const uint32_t *d_src, int n_tiles, int16_t *d_tiles,
                                int stride, int first, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    k_decode_tiles<<<n_tiles, 256, 0, st>>>(ds, reinterpret_cast<const uint4 *>(d_src), n_tiles, d_tiles, stride,
                                            first);
    return cudaGetLastError();
}

cudaError_t launch_build_planes(const DevStream &ds, int64_t n_ref, int16_t *d_planes, cudaStream_t st) {
    if (n_ref <= 0 || ds.nblocks <= 0) return cudaSuccess;
    dim3 grid((unsigned)ds.nblocks, (unsigned)(n_ref < 65535 ? n_ref : 65535));
    k_build_planes<<<grid, 256, 0, st>>>(ds, (int)n_ref, d_planes);
    return cudaGetLastError();
}

#define HMLFC_DISPATCH_B(B, CALL) \
    switch (B) {                  \
        case 4: { constexpr int BS = 4; CALL; } break;   \
        case 8: { constexpr int BS = 8; CALL; } break;   \
        case 16: { constexpr int BS = 16; CALL; } break; \
        case 32: { constexpr int BS = 32; CALL; } break; \
        default: { constexpr int BS = 0; CALL; } break;  \
    }

cudaError_t launch_decode_pixels(const DevStream &ds, const int32_t *d_coords, int64_t n, uint8_t *d_rgb,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < 152 * 64 ? want : 152 * 64);
    HMLFC_DISPATCH_B(ds.B, (k_decode_pixels<BS><<<grid, 256, 0, st>>>(ds, reinterpret_cast<const int4 *>(d_coords), n,
                                                                       d_rgb)));
    return cudaGetLastError();
}

cudaError_t launch_render(const DevStream &ds, const LaunchViews &lv, int total_tiles, float *d_out, int mode,
                          cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    HMLFC_DISPATCH_B(ds.B, (e = render_dispatch_tw<BS>(ds, lv, total_tiles, d_out, mode, st)));
    return e;
}

cudaError_t launch_mark(const DevStream &ds, const LaunchViews &lv, int total_tiles, uint8_t *flags, bool super_layout,
                        cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((total_tiles + 63) / 64);   // 8 warps of 8 tiles
    if (super_layout) {
        HMLFC_DISPATCH_B(ds.B, (k_mark<BS, 16, 16, true><<<grid, 256, 0, st>>>(ds, lv, total_tiles, flags)));
    } else {
        HMLFC_DISPATCH_B(ds.B, (k_mark<BS, 16, 16, false><<<grid, 256, 0, st>>>(ds, lv, total_tiles, flags)));
    }
    return cudaGetLastError();
}

cudaError_t launch_assign(const DevStream &ds, const uint8_t *flags, uint32_t *camslot, uint4 *items,
                          unsigned long long *counters, uint32_t capacity, cudaStream_t st) {
    const int K = ds.L < 2 ? ds.L : 2;
    const int64_t n_sk = (int64_t)ds.gu[K] * ds.gv[K] * ds.nblocks;
    const int64_t item_blocks = (n_sk + 255) / 256, cam_blocks = ((int64_t)ds.nu * ds.nv + 7) / 8;
    k_assign<<<(unsigned)(item_blocks + cam_blocks), 256, 0, st>>>(ds, flags, camslot, items, counters, capacity,
                                                                    (int)item_blocks);
    return cudaGetLastError();
}

cudaError_t launch_decode_blocks(const DevStream &ds, const uint4 *items, const unsigned long long *counters,
                                 const uint32_t *camslot, uint32_t *cache, int grid, cudaStream_t st) {
    HMLFC_DISPATCH_B(ds.B, (k_decode_blocks<BS><<<grid, 256, 0, st>>>(ds, items, counters, camslot, cache)));
    return cudaGetLastError();
}

cudaError_t launch_render_cached(const DevStream &ds, const LaunchViews &lv, int total_tiles, const uint32_t *camslot,
                                 const uint32_t *cache, bool all_cameras, float *d_out, cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    if (all_cameras) {
        HMLFC_DISPATCH_B(ds.B, (k_render_cached<BS, 16, 16, false><<<total_tiles, 64, 0, st>>>(ds, lv, camslot, cache,
                                                                                                 d_out)));
    } else {
        HMLFC_DISPATCH_B(ds.B, (k_render_cached<BS, 16, 16, true><<<total_tiles, 64, 0, st>>>(ds, lv, camslot, cache,
                                                                                                d_out)));
    }
    return cudaGetLastError();
}

cudaError_t launch_render_slots(const DevStream &ds, const LaunchViews &lv, int total_tiles, const uint32_t *slotmap,
                                const uint32_t *cache, float *d_out, cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    HMLFC_DISPATCH_B(ds.B, (k_render_slots<BS, 16, 16><<<total_tiles, 256, 0, st>>>(ds, lv, slotmap, cache, d_out)));
    return cudaGetLastError();
}

cudaError_t launch_copy_blob(const void *src, int n, void *dst, cudaStream_t st) {
    for (int o = 0; o < n; o += kBlobBytes) {
        Blob b;
        b.n = n - o < kBlobBytes ? n - o : kBlobBytes;
        memcpy(b.b, static_cast<const unsigned char *>(src) + o, (size_t)b.n);
        k_copy_blob<<<1, 256, 0, st>>>(b, static_cast<unsigned char *>(dst) + o);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t batch_lf_bytes() { return sizeof(BatchLF); }
size_t batch_hdr_bytes() { return sizeof(BatchHdr); }

void batch_fill_lf(void *dst, const DevStream &ds, int64_t key_off, int64_t sk_off, int64_t cam_off) {
    BatchLF f;
    memset(&f, 0, sizeof f);
    f.S = ds;
    f.key_off = key_off;
    f.sk_off = sk_off;
    f.cam_off = cam_off;
    memcpy(dst, &f, sizeof f);
}

void batch_fill_hdr(void *dst, int n_lf, int n_views, int total_tiles, int tile_w, int tile_h, int64_t n_keys,
                    int64_t n_sk, int64_t n_cam) {
    BatchHdr h;
    memset(&h, 0, sizeof h);
    h.n_lf = n_lf;
    h.n_views = n_views;
    h.total_tiles = total_tiles;
    h.tile_w = tile_w;
    h.tile_h = tile_h;
    h.n_keys = n_keys;
    h.n_sk = n_sk;
    h.n_cam = n_cam;
    memcpy(dst, &h, sizeof h);
}

namespace {

constexpr int kBatchRenderCtasPerSm = 16;   // the blend's resident CTAs of 64 threads (64 registers)

template <int BS, int TW, int TH, int RPT>
cudaError_t batch_kernels(const BatchPtrs &P, const BatchLaunch &L, cudaEvent_t const *phase, cudaStream_t st) {
    if (phase && phase[0]) cudaEventRecord(phase[0], st);
    k_mark_batch<BS, TW, TH><<<(unsigned)((L.total_tiles + 63) / 64), 256, 0, st>>>(P, L.flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int item_blocks = (int)((L.n_sk + 255) / 256), cam_blocks = (int)((L.n_cam + 7) / 8);
    k_assign_batch<<<(unsigned)(item_blocks + cam_blocks), 256, 0, st>>>(P, L.flags, L.camslot, L.items, L.counters,
                                                                       L.capacity, item_blocks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (phase && phase[1]) cudaEventRecord(phase[1], st);
    k_decode_batch<BS><<<L.decode_ctas, 256, 0, st>>>(P, L.items, L.counters, L.camslot, L.cache, L.group);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (phase && phase[2]) cudaEventRecord(phase[2], st);
    k_render_batch<BS, TW, TH, RPT><<<L.sm_count * kBatchRenderCtasPerSm, TW * TH / RPT, 0, st>>>(
        P, L.camslot, L.cache, L.work, L.d_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (phase && phase[3]) cudaEventRecord(phase[3], st);
    return cudaSuccess;
}

template <int BS>
cudaError_t batch_tiles(int tile_shape, const BatchPtrs &P, const BatchLaunch &L, cudaEvent_t const *phase,
                        cudaStream_t st) {
    switch (tile_shape) {
        case 1: return batch_kernels<BS, 32, 8, 4>(P, L, phase, st);
        case 2: return batch_kernels<BS, 8, 8, 1>(P, L, phase, st);
        default: return batch_kernels<BS, 16, 16, 4>(P, L, phase, st);
    }
}

}  // namespace

cudaError_t launch_batch(int B, int tile_shape, const void *image, const int *ptr_offsets, const BatchLaunch &L,
                         cudaEvent_t const *phase, cudaStream_t st) {
    BatchPtrs P;
    const unsigned char *base = static_cast<const unsigned char *>(image);
    P.hdr = reinterpret_cast<const BatchHdr *>(base + ptr_offsets[0]);
    P.lf = reinterpret_cast<const BatchLF *>(base + ptr_offsets[1]);
    P.views = reinterpret_cast<const hmlfc_view *>(base + ptr_offsets[2]);
    P.tile_start = reinterpret_cast<const int *>(base + ptr_offsets[3]);
    cudaError_t e = cudaSuccess;
    HMLFC_DISPATCH_B(B, (e = batch_tiles<BS>(tile_shape, P, L, phase, st)));
    return e;
}

__global__ void k_accumulate(const unsigned long long *__restrict__ counters, unsigned long long *__restrict__ totals) {
    const unsigned long long c = counters[0];
    totals[0] += c & 0xFFFFFFFFull;   // blocks decoded
    totals[1] += c >> 32;             // decode items
}

cudaError_t launch_accumulate(const unsigned long long *counters, unsigned long long *totals, cudaStream_t st) {
    k_accumulate<<<1, 1, 0, st>>>(counters, totals);
    return cudaGetLastError();
}

cudaError_t launch_resident(const DevStream &ds, const uint8_t *flags, int64_t n_keys, uint32_t *slotmap,
                            uint32_t *owner, uint32_t *epoch, uint32_t *clock, uint32_t capacity, uint32_t cur,
                            uint4 *items, unsigned long long *counters, uint32_t *cache, int decode_grid,
                            cudaStream_t st) {
    const int64_t gk = (n_keys + 255) / 256;
    k_resident_hits<<<(unsigned)(gk < 4096 ? gk : 4096), 256, 0, st>>>(flags, n_keys, slotmap, epoch, cur);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n_ck = (int64_t)ds.gu[1] * ds.gv[1] * ds.nblocks;
    k_resident_misses<<<(unsigned)((n_ck + 255) / 256), 256, 0, st>>>(ds, flags, slotmap, owner, epoch, clock,
                                                                       capacity, cur, items, counters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    HMLFC_DISPATCH_B(ds.B, (k_decode_resident<BS><<<decode_grid, 256, 0, st>>>(ds, items, counters, cache)));
    return cudaGetLastError();
}

cudaError_t launch_render_relaxed(const DevStream &ds, const LaunchViews &lv, int total_tiles, const float *coeff,
                                  const float *root, float *d_out, bool bias, cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    HMLFC_DISPATCH_B(ds.B, (k_relax<BS, false><<<total_tiles, 256, 0, st>>>(ds, lv, coeff, root, d_out, nullptr,
                                                                            nullptr, nullptr, bias ? 1 : 0)));
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const DevStream &ds, const LaunchViews &lv, int total_tiles,
                                   const float *grad_out, float *grad_coeff, float *grad_root, cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    HMLFC_DISPATCH_B(ds.B, (k_relax<BS, true><<<total_tiles, 256, 0, st>>>(ds, lv, nullptr, nullptr, nullptr,
                                                                           grad_out, grad_coeff, grad_root, 0)));
    return cudaGetLastError();
}

cudaError_t launch_dequant(const DevStream &ds, int64_t n_nc, float *coeff, float *root, cudaStream_t st) {
    const int64_t plane = (int64_t)ds.W * ds.H;
    const int64_t n_roots = (int64_t)ds.gu[ds.L] * ds.gv[ds.L];
    const int64_t gx = (plane + 255) / 256;
    dim3 grid((unsigned)(gx < 4096 ? gx : 4096), (unsigned)(n_nc + n_roots * 3));
    HMLFC_DISPATCH_B(ds.B, (k_dequant<BS><<<grid, 256, 0, st>>>(ds, n_nc, coeff, root)));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed scratch of the allocation-free render entry point
// ---------------------------------------------------------------------------
//
// The decoded-block cache of hmlfc_render_views_noalloc lives in this
// file-scope device array instead of memory allocated per call.  Every GPU
// that loads the library holds it until the process exits.  In host code the
// name is only a host-side stand-in for the symbol; the device address of
// each device's copy is looked up once, with that device current, by
// fixed_scratch() below and then passed to the kernels.

static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

namespace {
std::mutex g_fixed_mu;
void *g_fixed_ptr[kMaxDevices] = {};
}  // namespace

cudaError_t fixed_scratch(int device, void **ptr) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_fixed_mu);
    if (!g_fixed_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fixed_scratch);
        if (e != cudaSuccess) return e;
        g_fixed_ptr[device] = p;
    }
    *ptr = g_fixed_ptr[device];
    return cudaSuccess;
}

}  // namespace hmlfc
