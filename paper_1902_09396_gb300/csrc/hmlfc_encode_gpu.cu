// HMLFC encoder on the GPU: the same stream, byte for byte, as the host
// encoder.  Hierarchy of rounded 2x2 means (Sec. 4.3), closed-loop coding top
// down with the phase-shifted block search of Sec. 4.4 (Eq. 1-2 and the
// argmin displays; quarter-pel refinement around each sign's integer winner),
// the quantiser and block thresholds (Sec. 4.5), BISE records (Sec. 4.6) and
// the breadth-first stream (Sec. 4.7).
//
// Within one level all blocks of the reference members are independent, and
// so are all blocks of the predictive members once the references are
// reconstructed: each pass is one grid with a CTA per (node-channel, block).
// Every choice follows the host encoder's fixed keys (cost, |mv|_1, raster
// order, integer before fractional, subtractive sign on ties), reduced as
// 64-bit lexicographic keys, so the output does not depend on the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hmlfc.h"
#include "hmlfc_host.h"

using namespace hmlfc;

namespace {

constexpr int kEncThreads = 128;
constexpr int kMaxEncSearch = 32;           // window (2 Ws + 1)^2 candidates kept in shared memory
constexpr int kMaxPlaneBlock = 32;          // largest block whose refinement phase planes fit in shared memory

struct EncGeo {
    int W, H, B, nbx, nblocks, Ws, q, thr, side;
    int gv, pv;                              // node-grid widths of this level and of its parent level
    int planes;                              // refinement through precomputed phase planes (B <= 32)
};

// One node-channel of a pass: e = (a * gv + b) * 3 + c within the level, its
// breadth-first index and (predictive members) its rank among the
// motion-compensated node-channels.
struct EncItem {
    int e, nc, prank, pad;
};

enum EncErr : int { kErrRange = 1, kErrGroup = 2 };

constexpr int kCounters = 64;               // spread work counters over this many words

// Events recorded around the predictive (block-search) pass of each level,
// from the top level down: events[2 i] before and events[2 i + 1] after.
cudaEvent_t g_enc_events[2 * kMaxLevels];
int g_n_enc_events = 0;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ int quant(int r, int q) {
    const int m = (abs(r) + (q >> 1)) / q;
    return r < 0 ? -m : m;
}

__device__ __forceinline__ void dev_bise_choose(uint32_t range, int &mode, int &b) {
    int bp = 0, bt = 0, bq = 0;
    while ((1ull << bp) < range) bp++;
    while ((3ull << bt) < range) bt++;
    while ((5ull << bq) < range) bq++;
    const uint64_t np = 1ull << bp, nt = 3ull << bt, nq = 5ull << bq;
    if (np <= nt && np <= nq) { mode = 0; b = bp; }
    else if (nt <= nq) { mode = 1; b = bt; }
    else { mode = 2; b = bq; }
}

__device__ __forceinline__ uint64_t dev_bise_bits(int mode, int b, uint64_t n) {
    if (mode == 0) return n * (uint64_t)b;
    if (mode == 1) return ((n + 4) / 5) * (uint64_t)(8 + 5 * b);
    return ((n + 2) / 3) * (uint64_t)(7 + 3 * b);
}

__device__ __forceinline__ unsigned long long min_u64(unsigned long long a, unsigned long long b) {
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min_u64(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Quarter-pel bilinear prediction (weights sum to 16, +8 >> 4) at block pixel
// (lx, ly) for motion (mx, my) in quarter units, from a window whose (0, 0)
// is the clamped reference pixel (x0 - Ws - 1, y0 - Ws - 1).
__device__ __forceinline__ int qpel_win(const int16_t *win, int ww, int Ws, int lx, int ly, int mx, int my) {
    const int xi = lx + (mx >> 2) + Ws + 1, yi = ly + (my >> 2) + Ws + 1;
    const int fx = mx & 3, fy = my & 3;
    const int16_t *w = win + yi * ww + xi;
    const int s = (4 - fx) * (4 - fy) * (int)w[0] + fx * (4 - fy) * (int)w[1] + (4 - fx) * fy * (int)w[ww] +
                  fx * fy * (int)w[ww + 1];
    return (s + 8) >> 4;
}

// YCoCg-R of every view: RGB8 [views][H][W][3] -> int16 [views][3][H][W].
__global__ void k_enc_ycocg(const uint8_t *__restrict__ lf, int16_t *__restrict__ lev0, int64_t plane, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / plane, px = i - v * plane;
        const uint8_t *src = lf + 3 * i;
        const int R = src[0], G = src[1], Bc = src[2];
        const int co = R - Bc;
        const int t = Bc + (co >> 1);
        const int cg = G - t;
        int16_t *dst = lev0 + v * 3 * plane + px;
        dst[0] = (int16_t)(t + (cg >> 1));
        dst[plane] = (int16_t)co;
        dst[2 * plane] = (int16_t)cg;
    }
}

// Reference key views of the next level: rounded mean of each 2x2 cluster of
// the level's grid (1, 2 or 4 members at the edges), per pixel and channel.
__global__ void k_enc_rkv(const int16_t *__restrict__ lo, int16_t *__restrict__ hi, int gu, int gv, int pv,
                          int64_t plane, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / plane, px = i - e * plane;
        const int c = (int)(e % 3), node = (int)(e / 3), A = node / pv, Bn = node - (node / pv) * pv;
        int s = 0, k = 0;
        for (int da = 0; da < 2; da++)
            for (int db = 0; db < 2; db++) {
                const int a = 2 * A + da, b = 2 * Bn + db;
                if (a < gu && b < gv) {
                    s += lo[(((int64_t)a * gv + b) * 3 + c) * plane + px];
                    k++;
                }
            }
        const int m = k == 4 ? (s + 2) >> 2 : k == 2 ? (s + 1) >> 1 : s;   // floor((s + k/2) / k), k in {1, 2, 4}
        hi[i] = (int16_t)m;
    }
}

// One block of one node-channel of a pass.  SEARCH: 0 none, 1 integer
// stage, 2 integer stage + quarter-pel refinement.  PRED: predictive member
// (prediction from the reference member's dequantised SRV), else reference
// member.  ZMV: predictive with motion forced to (0, 0), sign +.
template <bool PRED, int SEARCH, bool ZMV>
__global__ void __launch_bounds__(kEncThreads, 12) k_enc_block(
    const EncGeo G, const EncItem *__restrict__ items, const int16_t *__restrict__ child_lev,
    const int16_t *__restrict__ par_recon, const int16_t *__restrict__ rhat_in, int16_t *__restrict__ recon_out,
    int16_t *__restrict__ rhat_out, int16_t *__restrict__ lvbuf, uint32_t *__restrict__ hdr,
    unsigned long long *__restrict__ val, uint32_t *__restrict__ mvsym, int *__restrict__ err,
    unsigned long long *__restrict__ frac_terms) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_key[2];
    __shared__ int s_mv[3];
    __shared__ int s_red[4][kEncThreads / 32];
    __shared__ short s_valid[98];
    __shared__ int s_nvalid;

    const int B = G.B, B2 = B * B;
    const int item = (int)(blockIdx.x / (unsigned)G.nblocks);
    const int k = (int)(blockIdx.x - (unsigned)item * (unsigned)G.nblocks);
    const EncItem it = items[item];
    const int c = it.e % 3, node = it.e / 3, a = node / G.gv, b = node - (node / G.gv) * G.gv;
    const int x0 = (k % G.nbx) * B, y0 = (k / G.nbx) * B;
    const int bw = min(B, G.W - x0), bh = min(B, G.H - y0), n = bw * bh;
    const int64_t plane = (int64_t)G.W * G.H;
    const int16_t *child = child_lev + (int64_t)it.e * plane;
    const int16_t *par = par_recon + ((int64_t)((a >> 1) * G.pv + (b >> 1)) * 3 + c) * plane;
    const int16_t *R = PRED ? rhat_in + ((int64_t)((a & ~1) * G.gv + (b & ~1)) * 3 + c) * plane : nullptr;

    const int Ws = G.Ws, nside = 2 * Ws + 1, ncand = nside * nside;
    const int ww = B + 2 * Ws + 3;                              // window pitch (one spare pixel each side)
    const int HW = B + 1, psz = HW * HW;                        // phase planes: (B+1)^2 positions from -1
    int *s_S = reinterpret_cast<int *>(smem);                  // S = child - parent, [n]
    uint32_t *s_cost = reinterpret_cast<uint32_t *>(s_S + B2);    // [2][ncand] integer, then [2][49] refinement
    int16_t *s_P = reinterpret_cast<int16_t *>(s_cost + 2 * max(ncand, 49));   // [2][16][psz] (planes only)
    int *s_pr = reinterpret_cast<int *>(s_P);                   // prediction [n], after the search (same space)
    int16_t *s_win = s_P + max(G.planes ? 2 * 16 * psz : 0, 2 * B2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ly = i / bw, lx = i - ly * bw;
        const int64_t o = (int64_t)(y0 + ly) * G.W + x0 + lx;
        s_S[i] = (int)child[o] - (int)par[o];
    }
    if (SEARCH > 0) {
        for (int i = threadIdx.x; i < ww * ww; i += blockDim.x) {
            const int ly = i / ww, lx = i - ly * ww;
            const int X = clampi(x0 - Ws - 1 + lx, 0, G.W - 1), Y = clampi(y0 - Ws - 1 + ly, 0, G.H - 1);
            s_win[i] = R[(int64_t)Y * G.W + X];
        }
        for (int i = threadIdx.x; i < 2 * ncand; i += blockDim.x) s_cost[i] = 0u;
        if (threadIdx.x == 0) s_nvalid = 0;
    }
    __syncthreads();

    int mvx = 0, mvy = 0, sign = 1;
    if (SEARCH > 0) {
        // integer stage: costs of every (dx, dy) for both signs.  A work item is
        // (row pair, dy, three consecutive dx): the three candidates slide over
        // one window row held in registers.
        {
            const int ngx = (nside + 2) / 3, nrg = (bh + 1) >> 1;
            for (int t = threadIdx.x; t < nrg * nside * ngx; t += blockDim.x) {
                const int gx = t % ngx, rest = t / ngx, dyi = rest % nside, rg = rest / nside;
                const int dy = dyi - Ws, dx0 = 3 * gx - Ws;
                int cp0 = 0, cm0 = 0, cp1 = 0, cm1 = 0, cp2 = 0, cm2 = 0;
                for (int row = 2 * rg; row < min(2 * rg + 2, bh); row++) {
                    const int *srow = s_S + row * bw;
                    const int16_t *wrow = s_win + (row + dy + Ws + 1) * ww + dx0 + Ws + 1;
                    int w0 = wrow[0], w1 = wrow[1];
                    for (int x = 0; x < bw; x++) {
                        const int w2 = wrow[x + 2], sv = srow[x];
                        cp0 += abs(sv - w0);
                        cm0 += abs(sv + w0);
                        cp1 += abs(sv - w1);
                        cm1 += abs(sv + w1);
                        cp2 += abs(sv - w2);
                        cm2 += abs(sv + w2);
                        w0 = w1;
                        w1 = w2;
                    }
                }
                const int c0 = dyi * nside + 3 * gx;
                atomicAdd(&s_cost[c0], (uint32_t)cp0);
                atomicAdd(&s_cost[ncand + c0], (uint32_t)cm0);
                if (3 * gx + 1 < nside) {
                    atomicAdd(&s_cost[c0 + 1], (uint32_t)cp1);
                    atomicAdd(&s_cost[ncand + c0 + 1], (uint32_t)cm1);
                }
                if (3 * gx + 2 < nside) {
                    atomicAdd(&s_cost[c0 + 2], (uint32_t)cp2);
                    atomicAdd(&s_cost[ncand + c0 + 2], (uint32_t)cm2);
                }
            }
        }
        __syncthreads();
        // per sign: minimum of (cost, |dx| + |dy|, raster index)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp < 2) {
            unsigned long long best = ~0ull;
            for (int cand = lane; cand < ncand; cand += 32) {
                const int dy = cand / nside - Ws, dx = cand - (cand / nside) * nside - Ws;
                const unsigned long long key = ((unsigned long long)s_cost[warp * ncand + cand] << 32) |
                                               ((unsigned long long)(abs(dx) + abs(dy)) << 16) | (unsigned)cand;
                best = min_u64(best, key);
            }
            best = warp_min_u64(best);
            if (lane == 0) s_key[warp] = best;
        }
        __syncthreads();
        if (SEARCH == 2) {
            // quarter-pel refinement: the 7x7 quarter offsets around each sign's integer winner
            const int cs0 = (int)(s_key[0] & 0xFFFFu), cs1 = (int)(s_key[1] & 0xFFFFu);
            for (int i = threadIdx.x; i < 2 * 49; i += blockDim.x) s_cost[i] = 0u;
            if (G.planes) {
                // Offsets (ox, oy) in [-3, 3]^2 around (4 dx, 4 dy) use phase (ox & 3, oy & 3) at integer
                // base (dx + (ox >> 2), dy + (oy >> 2)): the 16 phase planes of the (B+1)^2 positions from
                // -1 cover every candidate.  Separable and exact: H = (4 - fx) a + fx b per row, then
                // P = ((4 - fy) H + fy H' + 8) >> 4.
                const int nps = cs0 == cs1 ? 1 : 2;
                for (int t = threadIdx.x; t < nps * 16 * HW; t += blockDim.x) {      // one plane row per thread
                    const int ps = t / (16 * HW), r = t - ps * 16 * HW, f = r / HW, v = r - f * HW;
                    const int fx = f & 3, fy = f >> 2;
                    const int cc = ps ? cs1 : cs0;
                    const int dx = cc % nside - Ws, dy = cc / nside - Ws;
                    const int16_t *top = s_win + (v + dy + Ws) * ww + dx + Ws, *bot = top + ww;
                    const int w00 = (4 - fx) * (4 - fy), w01 = fx * (4 - fy), w10 = (4 - fx) * fy, w11 = fx * fy;
                    int16_t *pp = s_P + (ps * 16 + f) * psz + v * HW;
                    int a0 = top[0], c0 = bot[0];
                    for (int u = 0; u < HW; u++) {
                        const int a1 = top[u + 1], c1 = bot[u + 1];
                        pp[u] = (int16_t)((w00 * a0 + w01 * a1 + w10 * c0 + w11 * c1 + 8) >> 4);
                        a0 = a1;
                        c0 = c1;
                    }
                }
            }
            if (threadIdx.x < 98) {
                const int sg = threadIdx.x / 49, o = threadIdx.x - sg * 49;
                const int cc = sg ? cs1 : cs0;
                const int mx = 4 * (cc % nside - Ws) + o % 7 - 3, my = 4 * (cc / nside - Ws) + o / 7 - 3;
                if (o != 24 && abs(mx) <= 4 * Ws && abs(my) <= 4 * Ws) s_valid[atomicAdd(&s_nvalid, 1)] = (short)threadIdx.x;
            }
            __syncthreads();
            const int nvalid = s_nvalid;
            const bool same = cs0 == cs1;
            const int rpg = (bh + 3) >> 2;                      // rows per work item (4 items per candidate)
            for (int t = threadIdx.x; t < 4 * nvalid; t += blockDim.x) {
                const int so = s_valid[t >> 2], r0 = (t & 3) * rpg, r1 = min(bh, r0 + rpg);
                const int sg = so >= 49, o = so - 49 * sg;
                const int ox = o % 7 - 3, oy = o / 7 - 3;
                int acc = 0;
                if (G.planes) {
                    const int f = (oy & 3) * 4 + (ox & 3);
                    const int16_t *pl = s_P + ((same ? 0 : sg) * 16 + f) * psz + (1 + (oy >> 2)) * HW + 1 + (ox >> 2);
                    for (int row = r0; row < r1; row++) {
                        const int *srow = s_S + row * bw;
                        const int16_t *prow = pl + row * HW;
                        if (sg == 0)
                            for (int x = 0; x < bw; x++) acc += abs(srow[x] - (int)prow[x]);
                        else
                            for (int x = 0; x < bw; x++) acc += abs(srow[x] + (int)prow[x]);
                    }
                } else {
                    const int cc = sg ? cs1 : cs0;
                    const int mx = 4 * (cc % nside - Ws) + ox, my = 4 * (cc / nside - Ws) + oy;
                    const int m = sg ? -1 : 1;
                    for (int row = r0; row < r1; row++) {
                        const int *srow = s_S + row * bw;
                        for (int x = 0; x < bw; x++) acc += abs(srow[x] - m * qpel_win(s_win, ww, Ws, x, row, mx, my));
                    }
                }
                atomicAdd(&s_cost[so], (uint32_t)acc);
            }
            __syncthreads();
            if (warp < 2) {
                // a fractional candidate replaces the integer winner only at a strictly lower cost;
                // among fractional candidates: (cost, |mv|_1 in quarter units, raster order)
                const int cand = warp ? cs1 : cs0;
                const int cx = 4 * (cand % nside - Ws), cy = 4 * (cand / nside - Ws);
                unsigned long long best = ~0ull;
                for (int o = lane; o < 49; o += 32) {
                    const int mx = cx + o % 7 - 3, my = cy + o / 7 - 3;
                    if (o == 24 || abs(mx) > 4 * Ws || abs(my) > 4 * Ws) continue;
                    best = min_u64(best, ((unsigned long long)s_cost[warp * 49 + o] << 32) |
                                             ((unsigned long long)(abs(mx) + abs(my)) << 16) | (unsigned)o);
                }
                best = warp_min_u64(best);
                if (lane == 0) {
                    // refinement terms evaluated for this sign (work counter)
                    int vx = 0, vy = 0;
                    for (int o = -3; o <= 3; o++) {
                        vx += abs(cx + o) <= 4 * Ws;
                        vy += abs(cy + o) <= 4 * Ws;
                    }
                    atomicAdd(frac_terms + (blockIdx.x & (kCounters - 1)), (unsigned long long)(vx * vy - 1) * n);
                    const uint32_t ic = (uint32_t)(s_key[warp] >> 32);
                    int rx = cx, ry = cy;
                    uint32_t bc = ic;
                    if (best != ~0ull && (uint32_t)(best >> 32) < ic) {
                        const int o = (int)(best & 0xFFFFu);
                        rx = cx + o % 7 - 3;
                        ry = cy + o / 7 - 3;
                        bc = (uint32_t)(best >> 32);
                    }
                    s_red[0][warp] = (int)bc;                 // cost of this sign's winner
                    s_red[1][warp] = rx;
                    s_red[2][warp] = ry;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const int pick = (uint32_t)s_red[0][0] <= (uint32_t)s_red[0][1] ? 0 : 1;
                s_mv[0] = s_red[1][pick];
                s_mv[1] = s_red[2][pick];
                s_mv[2] = pick == 0 ? 1 : -1;
            }
        } else if (threadIdx.x == 0) {
            const int pick = (uint32_t)(s_key[0] >> 32) <= (uint32_t)(s_key[1] >> 32) ? 0 : 1;
            const int cand = (int)(s_key[pick] & 0xFFFFu);
            s_mv[0] = 4 * (cand % nside - Ws);
            s_mv[1] = 4 * (cand / nside - Ws);
            s_mv[2] = pick == 0 ? 1 : -1;
        }
        __syncthreads();
        mvx = s_mv[0];
        mvy = s_mv[1];
        sign = s_mv[2];
    }

    // residual, quantiser, energy and level range
    int energy = 0, any = 0, lmin = 0x7FFFFFFF, lmax = -0x7FFFFFFF - 1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ly = i / bw, lx = i - ly * bw;
        int pr = 0;
        if (PRED && SEARCH > 0) pr = sign * qpel_win(s_win, ww, Ws, lx, ly, mvx, mvy);
        if (PRED && ZMV) pr = R[(int64_t)(y0 + ly) * G.W + x0 + lx];
        const int res = s_S[i] - pr;
        const int lv = quant(res, G.q);
        energy += abs(res);
        any |= lv != 0;
        lmin = min(lmin, lv);
        lmax = max(lmax, lv);
        s_pr[i] = pr;
        s_S[i] = lv;                                            // S is not needed any more
    }
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        energy = warp_sum(energy);
        any = __any_sync(0xFFFFFFFFu, any);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            lmin = min(lmin, __shfl_xor_sync(0xFFFFFFFFu, lmin, o));
            lmax = max(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, o));
        }
        if (lane == 0) {
            s_red[0][warp] = energy;
            s_red[1][warp] = any;
            s_red[2][warp] = lmin;
            s_red[3][warp] = lmax;
        }
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    energy = 0;
    any = 0;
    lmin = 0x7FFFFFFF;
    lmax = -0x7FFFFFFF - 1;
    for (int w = 0; w < nw; w++) {
        energy += s_red[0][w];
        any |= s_red[1][w];
        lmin = min(lmin, s_red[2][w]);
        lmax = max(lmax, s_red[3][w]);
    }
    const bool sig = any && energy >= G.thr;
    const int64_t bi = (int64_t)it.nc * G.nblocks + k;
    if (threadIdx.x == 0) {
        uint64_t words = 0;
        uint32_t h = 0;
        if (sig) {
            int mode, bb;
            dev_bise_choose((uint32_t)(lmax - lmin + 1), mode, bb);
            words = 1 + (dev_bise_bits(mode, bb, (uint64_t)n) + 31) / 32;
            h = (uint32_t)(uint16_t)(int16_t)lmin | ((uint32_t)bb << 16) | ((uint32_t)mode << 21);
            if (lmin < -32768 || lmax > 32767) atomicOr(err, kErrRange);
        }
        hdr[bi] = h;
        val[bi] = (words << 32) | (sig ? 1ull : 0ull);
        if (PRED && (SEARCH > 0 || ZMV))
            mvsym[(int64_t)it.prank * G.nblocks + k] =
                ((uint32_t)(mvx + 4 * Ws) * (uint32_t)G.side + (uint32_t)(mvy + 4 * Ws)) * 2u + (sign < 0 ? 1u : 0u);
    }
    // reconstruction (closed loop) and the levels of a significant block
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ly = i / bw, lx = i - ly * bw;
        const int64_t o = (int64_t)(y0 + ly) * G.W + x0 + lx;
        const int lv = s_S[i];
        const int shat = s_pr[i] + (sig ? G.q * lv : 0);
        const int v = (int)par[o] + shat;
        bad |= v < -32768 || v > 32767 || shat < -32768 || shat > 32767;
        recon_out[(int64_t)it.e * plane + o] = (int16_t)v;
        if (!PRED) rhat_out[(int64_t)it.e * plane + o] = (int16_t)shat;
        if (sig) lvbuf[bi * B2 + i] = (int16_t)lv;
    }
    if (bad) atomicOr(err, kErrRange);
}

// Exclusive scan of 64-bit values (record words << 32 | significance), three
// phases with 1024 values per CTA.
constexpr int kScanPer = 1024;

__global__ void k_scan_reduce(const unsigned long long *__restrict__ v, int64_t n,
                              unsigned long long *__restrict__ part) {
    __shared__ unsigned long long s[kEncThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanPer;
    unsigned long long acc = 0;
    for (int i = threadIdx.x; i < kScanPer; i += blockDim.x)
        if (base + i < n) acc += v[base + i];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s[w];
        part[blockIdx.x] = t;
    }
}

// Exclusive scan of the partials in place, one CTA; part[np] = total.
__global__ void k_scan_partials(unsigned long long *part, int64_t np) {
    __shared__ unsigned long long s[kEncThreads];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < np; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long x = i < np ? part[i] : 0ull;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const unsigned long long y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
            __syncthreads();
            s[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < np) part[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[np] = carry;
}

__global__ void k_scan_apply(const unsigned long long *__restrict__ v, int64_t n,
                             const unsigned long long *__restrict__ part, unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s[kEncThreads];
    constexpr int per = kScanPer / kEncThreads;
    const int64_t base = (int64_t)blockIdx.x * kScanPer + (int64_t)threadIdx.x * per;
    unsigned long long loc[per], acc = 0;
#pragma unroll
    for (int r = 0; r < per; r++) {
        loc[r] = base + r < n ? v[base + r] : 0ull;
        acc += loc[r];
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kEncThreads; o <<= 1) {
        const unsigned long long y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned long long run = part[blockIdx.x] + s[threadIdx.x] - acc;
#pragma unroll
    for (int r = 0; r < per; r++) {
        if (base + r < n) out[base + r] = run;
        run += loc[r];
    }
}

// Group entries {bitmap, first record word, first offset, 0} and the 16-bit
// offsets of the significant blocks, one thread per (node-channel, group).
__global__ void k_ser_groups(const unsigned long long *__restrict__ val, const unsigned long long *__restrict__ pre,
                             int64_t n_nc, int nblocks, int ngroups, uint4 *__restrict__ groups,
                             uint16_t *__restrict__ offs, int *__restrict__ err) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_nc * ngroups) return;
    const int64_t nc = t / ngroups;
    const int gi = (int)(t - nc * ngroups);
    const int64_t first = nc * nblocks + (int64_t)gi * 32;
    const unsigned long long p0 = pre[first];
    const uint32_t gbase = (uint32_t)(p0 >> 32), obase = (uint32_t)p0;
    uint32_t bitmap = 0;
    for (int r = 0; r < 32 && gi * 32 + r < nblocks; r++) {
        if (!(val[first + r] & 1ull)) continue;
        bitmap |= 1u << r;
        const unsigned long long p = pre[first + r];
        const uint32_t rel = (uint32_t)(p >> 32) - gbase;
        if (rel > 0xFFFFu) atomicOr(err, kErrGroup);
        offs[(uint32_t)p] = (uint16_t)rel;
    }
    groups[t] = make_uint4(bitmap, gbase, obase, 0u);
}

__device__ __forceinline__ void bits_or(uint32_t *buf, uint64_t pos, uint32_t v, int w) {
    if (w == 0) return;
    const uint64_t k = pos >> 5;
    const int sh = (int)(pos & 31u);
    const uint64_t wide = (uint64_t)(v & (w >= 32 ? 0xFFFFFFFFu : ((1u << w) - 1u))) << sh;
    atomicOr(buf + k, (uint32_t)wide);
    if (sh + w > 32) atomicOr(buf + k + 1, (uint32_t)(wide >> 32));
}

// BISE field of value group g of n values (mode, b) at bit 0 of buf; values
// are v(i) for i < n, 0 past the end.
template <class F>
__device__ __forceinline__ void bise_group(uint32_t *buf, int mode, int b, uint64_t g, uint64_t n, F v) {
    if (mode == 0) {
        bits_or(buf, g * (uint64_t)b, v(g), b);
        return;
    }
    const int per = mode == 1 ? 5 : 3, radix = mode == 1 ? 3 : 5, hw = mode == 1 ? 8 : 7;
    const uint64_t base = g * (uint64_t)(hw + per * b);
    const uint32_t mask = (1u << b) - 1u;
    uint32_t packed = 0, mul = 1;
    for (int r = 0; r < per; r++) {
        const uint64_t i = g * per + r;
        const uint32_t x = i < n ? v(i) : 0u;
        packed += (x >> b) * mul;
        mul *= (uint32_t)radix;
        bits_or(buf, base + hw + (uint64_t)r * b, x & mask, b);
    }
    bits_or(buf, base, packed, hw);
}

// Block records: header word + BISE payload, one warp per (node-channel,
// block); the payload is assembled in shared memory.
__global__ void k_ser_records(const unsigned long long *__restrict__ val, const unsigned long long *__restrict__ pre,
                              const uint32_t *__restrict__ hdr, const int16_t *__restrict__ lvbuf, int64_t nkeys,
                              int W, int H, int B, int nbx, int nblocks, int max_words, uint32_t *__restrict__ recs) {
    extern __shared__ uint32_t s_words[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t key = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (key >= nkeys) return;
    const unsigned long long v = val[key];
    if (!(v & 1ull)) return;
    const int words = (int)(v >> 32);
    uint32_t *buf = s_words + warp * max_words;
    for (int i = lane; i < words; i += 32) buf[i] = 0u;
    __syncwarp();
    const uint32_t h = hdr[key];
    const int m = (int)(int16_t)(h & 0xFFFFu), b = (int)((h >> 16) & 31u), mode = (int)((h >> 21) & 3u);
    const int k = (int)(key % nblocks);
    const int x0 = (k % nbx) * B, y0 = (k / nbx) * B;
    const uint64_t n = (uint64_t)min(B, W - x0) * (uint64_t)min(B, H - y0);
    const int16_t *lv = lvbuf + key * (int64_t)B * B;
    const uint64_t ng = mode == 0 ? n : mode == 1 ? (n + 4) / 5 : (n + 2) / 3;
    for (uint64_t g = lane; g < ng; g += 32)
        bise_group(buf + 1, mode, b, g, n, [&](uint64_t i) { return (uint32_t)((int)lv[i] - m); });
    __syncwarp();
    uint32_t *dst = recs + (uint32_t)(pre[key] >> 32);
    for (int i = lane; i < words; i += 32) dst[i] = i == 0 ? h : buf[i];
}

// Motion-vector symbols of every motion-compensated node-channel in
// breadth-first order, one thread per BISE group, into zeroed words.
__global__ void k_ser_mvs(const uint32_t *__restrict__ sym, uint64_t n, int mode, int b, uint32_t *__restrict__ out) {
    const uint64_t ng = mode == 0 ? n : mode == 1 ? (n + 4) / 5 : (n + 2) / 3;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < ng;
         g += (uint64_t)gridDim.x * blockDim.x)
        bise_group(out, mode, b, g, n, [&](uint64_t i) { return sym[i]; });
}

int grid_for(int64_t n, int per_block) {
    return (int)std::min<int64_t>((n + per_block - 1) / per_block, 152 * 64);
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

int enc_fail(cudaError_t e, const char *what) {
    return fail(HMLFC_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <bool PRED, int SEARCH, bool ZMV>
cudaError_t launch_pass(const EncGeo &G, int n_items, const EncItem *items, const int16_t *child, const int16_t *par,
                        const int16_t *rhat_in, int16_t *recon, int16_t *rhat_out, int16_t *lvbuf, uint32_t *hdr,
                        unsigned long long *val, uint32_t *mvsym, int *err, unsigned long long *frac,
                        size_t smem, cudaStream_t st) {
    auto kern = k_enc_block<PRED, SEARCH, ZMV>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)((int64_t)n_items * G.nblocks), kEncThreads, smem, st>>>(G, items, child, par, rhat_in, recon,
                                                                            rhat_out, lvbuf, hdr, val, mvsym, err,
                                                                            frac);
    return cudaGetLastError();
}

}  // namespace

extern "C" int hmlfc_set_encode_events(void *const *events, int n) {
    if (n < 0 || n > 2 * kMaxLevels || (n > 0 && !events)) return fail(HMLFC_E_INVALID_ARG, "encode events");
    for (int i = 0; i < n; i++) g_enc_events[i] = static_cast<cudaEvent_t>(events[i]);
    g_n_enc_events = n;
    return HMLFC_OK;
}

extern "C" int hmlfc_encode_device(const uint8_t *d_lf, int nu, int nv, int W, int H, const hmlfc_encode_params *p,
                                   void *cuda_stream, void **h_out, size_t *nbytes, hmlfc_encode_stats *stats) {
    if (!d_lf || !p || !h_out || !nbytes) return fail(HMLFC_E_INVALID_ARG, "NULL argument");
    if (nu < 1 || nv < 1 || W < 1 || H < 1 || nu > 65536 || nv > 65536 || W > 65536 || H > 65536)
        return fail(HMLFC_E_INVALID_ARG, "light-field size");
    if (p->levels < 1 || p->levels > kMaxLevels || p->block < 1 || p->block > kMaxBlock || p->search < 0 ||
        p->search > 64 || p->qstep < 1 || p->qstep > kCoefLimit || p->t_ref < 0 || p->t_pred < 0 || p->mc < 0 ||
        p->mc > 3)
        return fail(HMLFC_E_INVALID_ARG, "encoder parameters");
    if ((p->mc == 1 || p->mc == 3) && p->search > kMaxEncSearch)
        return fail(HMLFC_E_UNSUPPORTED, "device search window above %d", kMaxEncSearch);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Geometry g;
    if (p->chroma != 0) return fail(HMLFC_E_UNSUPPORTED, "the device encoder codes full-resolution chroma only");
    fill_geometry(g, nu, nv, W, H, p->levels, p->block, p->search, p->qstep, p->t_ref, p->t_pred, p->mc != 0);
    const int L = g.L, B = g.B;
    const int64_t plane = (int64_t)W * H, n_views = (int64_t)nu * nv;
    const int64_t nkeys = g.n_nc * g.nblocks;
    if ((int64_t)3 * n_views * g.nblocks > 0x7FFFFFFFll) return fail(HMLFC_E_UNSUPPORTED, "too many blocks per level");

    // per (level, pass) node-channel lists, and the motion-compensated ranks
    std::vector<EncItem> items;
    std::vector<int64_t> item_first[kMaxLevels][2];
    int64_t n_pred_mc = 0;
    {
        std::vector<int64_t> prank((size_t)g.n_nc, -1);
        for (int l = L - 1; l >= 0; l--)
            for (int a = 0; a < g.gu[l]; a++)
                for (int b = 0; b < g.gv[l]; b++)
                    for (int c = 0; c < 3; c++) {
                        const bool ref = (a % 2 == 0) && (b % 2 == 0);
                        const int64_t nc = g.nc_base[l] + ((int64_t)a * g.gv[l] + b) * 3 + c;
                        if (!ref && p->mc != 0) prank[(size_t)nc] = n_pred_mc++;
                    }
        for (int l = L - 1; l >= 0; l--)
            for (int pass = 0; pass < 2; pass++) {
                item_first[l][pass].push_back((int64_t)items.size());
                for (int a = 0; a < g.gu[l]; a++)
                    for (int b = 0; b < g.gv[l]; b++) {
                        const bool ref = (a % 2 == 0) && (b % 2 == 0);
                        if ((pass == 0) != ref) continue;
                        for (int c = 0; c < 3; c++) {
                            const int e = (a * g.gv[l] + b) * 3 + c;
                            const int64_t nc = g.nc_base[l] + e;
                            items.push_back(EncItem{e, (int)nc, (int)std::max<int64_t>(prank[(size_t)nc], 0), 0});
                        }
                    }
                item_first[l][pass].push_back((int64_t)items.size());
            }
    }

    // device memory: levels I_0..I_L, two reconstructions, the reference SRVs,
    // levels of every block, per-block header / scan values, MV symbols
    std::vector<int64_t> lev_off(L + 2, 0);
    for (int l = 0; l <= L; l++) lev_off[l + 1] = lev_off[l] + (int64_t)g.gu[l] * g.gv[l] * 3 * plane;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t lvl0 = (size_t)n_views * 3 * plane * 2;
    const int64_t nparts = (nkeys + kScanPer - 1) / kScanPer;
    const size_t o_lev = 0, o_rec0 = up(o_lev + (size_t)lev_off[L + 1] * 2), o_rec1 = up(o_rec0 + lvl0),
                 o_rhat = up(o_rec1 + lvl0), o_lvb = up(o_rhat + lvl0),
                 o_hdr = up(o_lvb + (size_t)nkeys * B * B * 2), o_val = up(o_hdr + (size_t)nkeys * 4),
                 o_pre = up(o_val + (size_t)nkeys * 8), o_part = up(o_pre + (size_t)nkeys * 8),
                 o_mv = up(o_part + (size_t)(nparts + 1) * 8), o_items = up(o_mv + (size_t)n_pred_mc * g.nblocks * 4),
                 o_err = up(o_items + items.size() * sizeof(EncItem)), o_cnt = up(o_err + 16),
                 total_scratch = up(o_cnt + kCounters * 8);
    DevBuf scratch;
    cudaError_t e = cudaMalloc(&scratch.p, total_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HMLFC_E_OOM, "device encoder scratch (%zu bytes)", total_scratch);
    }
    uint8_t *base = static_cast<uint8_t *>(scratch.p);
    int16_t *lev = reinterpret_cast<int16_t *>(base + o_lev);
    int16_t *rec[2] = {reinterpret_cast<int16_t *>(base + o_rec0), reinterpret_cast<int16_t *>(base + o_rec1)};
    int16_t *rhat = reinterpret_cast<int16_t *>(base + o_rhat);
    int16_t *lvbuf = reinterpret_cast<int16_t *>(base + o_lvb);
    uint32_t *hdr = reinterpret_cast<uint32_t *>(base + o_hdr);
    unsigned long long *val = reinterpret_cast<unsigned long long *>(base + o_val);
    unsigned long long *pre = reinterpret_cast<unsigned long long *>(base + o_pre);
    unsigned long long *part = reinterpret_cast<unsigned long long *>(base + o_part);
    uint32_t *mvsym = reinterpret_cast<uint32_t *>(base + o_mv);
    EncItem *d_items = reinterpret_cast<EncItem *>(base + o_items);
    int *d_err = reinterpret_cast<int *>(base + o_err);
    unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(base + o_cnt);

    e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(EncItem), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, kCounters * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rhat, 0, lvl0, st);
    if (e == cudaSuccess) {
        const int64_t n = n_views * plane;
        k_enc_ycocg<<<grid_for(n, kEncThreads), kEncThreads, 0, st>>>(d_lf, lev, plane, n);
        e = cudaGetLastError();
    }
    for (int l = 0; l < L && e == cudaSuccess; l++) {
        const int64_t n = (int64_t)g.gu[l + 1] * g.gv[l + 1] * 3 * plane;
        k_enc_rkv<<<grid_for(n, kEncThreads), kEncThreads, 0, st>>>(lev + lev_off[l], lev + lev_off[l + 1], g.gu[l],
                                                                     g.gv[l], g.gv[l + 1], plane, n);
        e = cudaGetLastError();
    }
    // closed loop, top down; the parent reconstruction of level L-1 is the roots
    const int16_t *par = lev + lev_off[L];
    const int Ws = p->search, nside = 2 * Ws + 1;
    const int search_mode = p->mc == 1 ? 2 : p->mc == 3 ? 1 : 0;
    // shared memory: S [B^2] int, costs, planes [2][16][(B+1)^2] int16 sharing their space with the
    // prediction [B^2] int, window [(B + 2 Ws + 3)^2] int16
    const int planes = B <= kMaxPlaneBlock ? 1 : 0;
    const size_t smem_base = (size_t)B * B * 4 + (size_t)2 * std::max(nside * nside, 49) * 4 + (size_t)B * B * 4;
    const size_t smem_search =
        (size_t)B * B * 4 + (size_t)2 * std::max(nside * nside, 49) * 4 +
        std::max<size_t>(planes ? (size_t)2 * 16 * (B + 1) * (B + 1) * 2 : 0, (size_t)B * B * 4) +
        (size_t)(B + 2 * Ws + 3) * (B + 2 * Ws + 3) * 2;
    for (int l = L - 1; l >= 0 && e == cudaSuccess; l--) {
        EncGeo G{W, H, B, g.nbx, g.nblocks, Ws, g.q, 0, g.side, g.gv[l], g.gv[l + 1], planes};
        int16_t *out = rec[l & 1];
        const int16_t *child = lev + lev_off[l];
        // pass 0: reference members; their dequantised SRVs go to rhat
        {
            G.thr = g.t_ref;
            const int64_t i0 = item_first[l][0][0], ni = item_first[l][0][1] - i0;
            if (ni > 0)
                e = launch_pass<false, 0, false>(G, (int)ni, d_items + i0, child, par, nullptr, out, rhat, lvbuf, hdr,
                                                 val, mvsym, d_err, d_cnt, smem_base, st);
        }
        // pass 1: predictive members against the reference member's dequantised SRV
        const int ev = 2 * (L - 1 - l);
        if (e == cudaSuccess && ev + 1 < g_n_enc_events) e = cudaEventRecord(g_enc_events[ev], st);
        if (e == cudaSuccess) {
            G.thr = g.t_pred;
            const int64_t i0 = item_first[l][1][0], ni = item_first[l][1][1] - i0;
            if (ni > 0) {
                if (p->mc == 0)
                    e = launch_pass<true, 0, false>(G, (int)ni, d_items + i0, child, par, rhat, out, nullptr, lvbuf,
                                                    hdr, val, mvsym, d_err, d_cnt, smem_base, st);
                else if (p->mc == 2)
                    e = launch_pass<true, 0, true>(G, (int)ni, d_items + i0, child, par, rhat, out, nullptr, lvbuf,
                                                   hdr, val, mvsym, d_err, d_cnt, smem_base, st);
                else if (search_mode == 1)
                    e = launch_pass<true, 1, false>(G, (int)ni, d_items + i0, child, par, rhat, out, nullptr, lvbuf,
                                                    hdr, val, mvsym, d_err, d_cnt, smem_search, st);
                else
                    e = launch_pass<true, 2, false>(G, (int)ni, d_items + i0, child, par, rhat, out, nullptr, lvbuf,
                                                    hdr, val, mvsym, d_err, d_cnt, smem_search, st);
            }
        }
        if (e == cudaSuccess && ev + 1 < g_n_enc_events) e = cudaEventRecord(g_enc_events[ev + 1], st);
        par = out;
    }
    // exclusive scan of (record words, significance) over the breadth-first blocks
    if (e == cudaSuccess) {
        k_scan_reduce<<<(unsigned)nparts, kEncThreads, 0, st>>>(val, nkeys, part);
        k_scan_partials<<<1, kEncThreads, 0, st>>>(part, nparts);
        k_scan_apply<<<(unsigned)nparts, kEncThreads, 0, st>>>(val, nkeys, part, pre);
        e = cudaGetLastError();
    }
    unsigned long long tot = 0, cnt[kCounters] = {0};
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, part + nparts, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return enc_fail(e, "device encoder");
    if (herr & kErrRange) return fail(HMLFC_E_UNSUPPORTED, "values outside the int16 range while encoding");

    // stream layout (as the host encoder's)
    const uint64_t nsig = tot & 0xFFFFFFFFull, nrecw = tot >> 32;
    const uint64_t nmv = (uint64_t)n_pred_mc * g.nblocks;
    int mv_mode = 0, mv_b = 0;
    if (g.mc) bise_choose(2ull * g.side * g.side, mv_mode, mv_b);
    const uint64_t nmvw = g.mc ? (bise_bits(mv_mode, mv_b, nmv) + 31) / 32 : 0;
    auto a16 = [](uint64_t v) { return (v + 15) & ~(uint64_t)15; };
    const uint64_t n_root_vals = (uint64_t)g.n_roots * 3 * plane;
    const uint64_t o_roots = (uint64_t)kHeaderWords * 4;
    const uint64_t o_groups = a16(o_roots + n_root_vals * 2);
    const uint64_t o_offs = a16(o_groups + (uint64_t)g.n_nc * g.ngroups * 16);
    const uint64_t o_recs = a16(o_offs + nsig * 2);
    const uint64_t o_mvs = a16(o_recs + nrecw * 4);
    const uint64_t total = a16(o_mvs + nmvw * 4);
    if (total > 0xFFFFFFF0ull) return fail(HMLFC_E_UNSUPPORTED, "stream larger than 4 GB");
    DevBuf dstream;
    e = cudaMalloc(&dstream.p, (size_t)total + 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HMLFC_E_OOM, "device stream buffer");
    }
    uint8_t *ds = static_cast<uint8_t *>(dstream.p);
    int max_words = 2;
    {
        int mode, bb;
        bise_choose(65536, mode, bb);    // the widest alphabet a block can need (int16 levels)
        max_words = 2 + (int)((bise_bits(mode, bb, (uint64_t)B * B) + 31) / 32);
    }
    e = cudaMemsetAsync(ds, 0, (size_t)total + 8, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ds + o_roots, lev + lev_off[L], n_root_vals * 2, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        const int64_t ng = g.n_nc * g.ngroups;
        k_ser_groups<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(val, pre, g.n_nc, g.nblocks, g.ngroups,
                                                                  reinterpret_cast<uint4 *>(ds + o_groups),
                                                                  reinterpret_cast<uint16_t *>(ds + o_offs), d_err);
        const int wpb = 8;
        const size_t sm = (size_t)wpb * max_words * 4;
        if (sm > 48 * 1024)
            e = cudaFuncSetAttribute(k_ser_records, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            k_ser_records<<<(unsigned)((nkeys + wpb - 1) / wpb), wpb * 32, sm, st>>>(
                val, pre, hdr, lvbuf, nkeys, W, H, B, g.nbx, g.nblocks, max_words,
                reinterpret_cast<uint32_t *>(ds + o_recs));
        if (e == cudaSuccess && nmv)
            k_ser_mvs<<<grid_for((int64_t)nmv, 256), 256, 0, st>>>(mvsym, nmv, mv_mode, mv_b,
                                                                   reinterpret_cast<uint32_t *>(ds + o_mvs));
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    uint8_t *hs = static_cast<uint8_t *>(std::malloc((size_t)total));
    if (!hs) return fail(HMLFC_E_OOM, "stream allocation");
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, ds, (size_t)total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        std::free(hs);
        return enc_fail(e, "device stream assembly");
    }
    if (herr & kErrGroup) {
        std::free(hs);
        return fail(HMLFC_E_UNSUPPORTED, "block group larger than 64 K words");
    }
    uint32_t h[kHeaderWords] = {0};
    h[0] = kMagic; h[1] = kVersion; h[2] = (uint32_t)g.nu; h[3] = (uint32_t)g.nv; h[4] = (uint32_t)g.W;
    h[5] = (uint32_t)g.H; h[6] = (uint32_t)g.L; h[7] = (uint32_t)g.B; h[8] = (uint32_t)g.Ws; h[9] = (uint32_t)g.q;
    h[10] = (uint32_t)g.t_ref; h[11] = (uint32_t)g.t_pred; h[12] = g.mc ? 1u : 0u; h[13] = (uint32_t)mv_mode;
    h[14] = (uint32_t)mv_b; h[15] = (uint32_t)g.n_nc; h[16] = (uint32_t)g.ngroups; h[17] = (uint32_t)nsig;
    h[18] = (uint32_t)nrecw; h[19] = (uint32_t)nmv; h[20] = (uint32_t)nmvw; h[21] = (uint32_t)o_roots;
    h[22] = (uint32_t)o_groups; h[23] = (uint32_t)o_offs; h[24] = (uint32_t)o_recs; h[25] = (uint32_t)o_mvs;
    h[26] = (uint32_t)total;
    std::memcpy(hs, h, sizeof h);
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        const bool searched = p->mc == 1 || p->mc == 3;
        int64_t n_pred_items = 0;
        for (int l = 0; l < L; l++) n_pred_items += item_first[l][1][1] - item_first[l][1][0];
        stats->blocks_searched = searched ? (uint64_t)n_pred_items * g.nblocks : 0;
        stats->int_terms = searched ? (uint64_t)n_pred_items * 2ull * nside * nside * (uint64_t)plane : 0;
        for (int i = 0; i < kCounters; i++) stats->frac_terms += cnt[i];
        stats->sig_blocks = nsig;
        stats->blocks = (uint64_t)nkeys;
    }
    *h_out = hs;
    *nbytes = (size_t)total;
    return HMLFC_OK;
}
