// Internal definitions shared by the host code and the CUDA kernels of the
// product library (never by the CPU oracle).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "hmlfc.h"

namespace hmlfc {

constexpr int kMaxLevels = 16;      // tree height limit (grid up to 65536 per axis)
constexpr int kMaxBlock = 64;       // block size limit
constexpr int kCoefLimit = 16384;   // |dequantised coefficient| bound enforced at load
constexpr uint32_t kMagic = 0x464C4D48u;
constexpr uint32_t kVersion = 1u;
constexpr int kHeaderWords = 32;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int64_t kMaxSlots = 0x7FFFFFFF;   // cache slots stay below 2^31, so kNone is the only value with bit 31 set
constexpr int kDecodeCtasPerSm = 32;        // CTAs per SM launched for the cached block decode (5 resident; from sweeps)

// Everything a kernel needs to decode samples of one stream.  Passed by value
// as a kernel parameter (it lives in the constant bank while the kernel runs).
struct DevStream {
    int nu, nv, W, H, L, B, Ws, q, mc, mv_mode, mv_b;
    int nbx, nby, nblocks, ngroups;
    int side;                       // 8 * Ws + 1
    int gu[kMaxLevels + 1], gv[kMaxLevels + 1];
    int nc_base[kMaxLevels];        // breadth-first index of level l's first node-channel
    int ref_base[kMaxLevels];       // rank of level l's first reference node-channel
    int pred_base[kMaxLevels];      // rank of level l's first predictive node-channel
    const int16_t *roots;           // [roots][3][H][W]
    const uint4 *groups;            // [n_nc][ngroups] {bitmap, record base, offset base, residual rank}
    const uint16_t *offs;           // [n_sig]
    const uint32_t *recs;           // [n_rec_words + 2]
    const uint32_t *mvs;            // [n_mv_words + 2]
    const uint32_t *ref_tab;        // [n_ref_nc][nblocks] tile index, 0 = the zero tile
    const int16_t *tiles;           // [n_tiles + 1][B * B]
    const int16_t *planes;          // [n_ref_nc][H][W] the same reference SRVs as dense planes (+ padding)
    // the dequantised residual r^ of every significant predictive block, decoded at load: tile t at
    // ptiles + t * B * pstride, row stride pstride = B rounded up to even (4-byte aligned pixel pairs),
    // zero outside the block's valid pixels; tile 0 is all zeros; a predictive group's first tile is 1 +
    // word 3 of its entry
    const int16_t *ptiles;
    int pstride;
    uint32_t *status;               // bit 0: an out-of-range coordinate was seen
    int lod;                        // progressive decode: levels below lod are left out (0 = full decode)
    // chroma sub-sampling (Sec. 4.5): sub = 1 codes Co and Cg at ceil(W/2) x ceil(H/2).  Per channel c:
    // plane size, block grid, the offset of its plane in a root's planes (rnpx values per root), and the
    // offset of its blocks' MV symbols in a predictive node's (mv_node symbols per node).  The dense
    // reference planes keep row stride W for every channel (chroma in their top-left ceil(H/2) x ceil(W/2)).
    int sub;
    int cW[3], cH[3], cnbx[3], cnb[3], roff[3], mv_coff[3];
    int mv_node;
    int64_t rnpx;
    // element counts of the arrays above (the bounds a HMLFC_CHECK build checks every read against) and of
    // the motion-vector symbols
    int64_t lim_roots, lim_groups, lim_offs, lim_recs, lim_mvs, lim_ref_tab, lim_tiles, lim_planes, lim_mv;
    int64_t lim_ptiles;
};

// Status bits of a stream object: kStatusCoord, a decode_pixels coordinate
// outside the light field; kStatusBounds, a read that a HMLFC_CHECK build
// found outside its array (the read was skipped).
constexpr uint32_t kStatusCoord = 1u, kStatusBounds = 2u;

// Views of one launch, by value (kernel parameter space).
constexpr int kMaxViewsPerLaunch = 128;

struct LaunchViews {
    int n_views;
    int tile_w, tile_h;
    int tile_start[kMaxViewsPerLaunch + 1];
    uint32_t tiles_x_magic[kMaxViewsPerLaunch];   // quotient multiplier of each view's tiles per row
    hmlfc_view views[kMaxViewsPerLaunch];
};

// Size of the fixed device array behind hmlfc_render_views_noalloc.
constexpr size_t kFixedScratchBytes = (size_t)32 << 20;
static_assert(kFixedScratchBytes == HMLFC_FIXED_SCRATCH_BYTES, "fixed scratch size of the public header");
constexpr int kMaxDevices = 64;

// Device address of the fixed scratch array on `device`, which must be the
// current device; looked up on the first call per device.
cudaError_t fixed_scratch(int device, void **ptr);

// Launchers implemented in hmlfc_kernels.cu.
// Decode n_tiles records into B-row tiles of row stride `stride`, tile t of
// the list at d_tiles + (t + first) * B * stride.
cudaError_t launch_decode_tiles(const DevStream &ds, const uint32_t *d_src, int n_tiles, int16_t *d_tiles,
                                int stride, int first, cudaStream_t st);
cudaError_t launch_build_planes(const DevStream &ds, int64_t n_ref, int16_t *d_planes, cudaStream_t st);
cudaError_t launch_decode_pixels(const DevStream &ds, const int32_t *d_coords, int64_t n, uint8_t *d_rgb,
                                 cudaStream_t st);
cudaError_t launch_render(const DevStream &ds, const LaunchViews &lv, int total_tiles, float *d_out, int mode,
                          cudaStream_t st);
// Flags of the (camera, block) pairs the views reach: super_layout groups the
// cameras of each (level-min(2, L) node, block) pair (the cached render),
// otherwise camera-major (the serving form's keys).
cudaError_t launch_mark(const DevStream &ds, const LaunchViews &lv, int total_tiles, uint8_t *flags, bool super_layout,
                        cudaStream_t st);
// Camera slots (counters[1]) and decode items (counters[0] >> 32).
cudaError_t launch_assign(const DevStream &ds, const uint8_t *flags, uint32_t *camslot, uint4 *items,
                          unsigned long long *counters, uint32_t capacity, cudaStream_t st);
cudaError_t launch_decode_blocks(const DevStream &ds, const uint4 *items, const unsigned long long *counters,
                                 const uint32_t *camslot, uint32_t *cache, int grid, cudaStream_t st);
// all_cameras: the cache holds an image for every camera of the light field,
// so no ray needs the direct-decode fallback.
cudaError_t launch_render_cached(const DevStream &ds, const LaunchViews &lv, int total_tiles, const uint32_t *camslot,
                                 const uint32_t *cache, bool all_cameras, float *d_out, cudaStream_t st);
// Blend from a cache with one B x B slot per (camera, block) pair (slotmap).
cudaError_t launch_render_slots(const DevStream &ds, const LaunchViews &lv, int total_tiles, const uint32_t *slotmap,
                                const uint32_t *cache, float *d_out, cudaStream_t st);
// Serving form: resident decoded-block cache (hits, misses with eviction, decode).
cudaError_t launch_resident(const DevStream &ds, const uint8_t *flags, int64_t n_keys, uint32_t *slotmap,
                            uint32_t *owner, uint32_t *epoch, uint32_t *clock, uint32_t capacity, uint32_t cur,
                            uint4 *items, unsigned long long *counters, uint32_t *cache, int decode_grid,
                            cudaStream_t st);

cudaError_t launch_accumulate(const unsigned long long *counters, unsigned long long *totals, cudaStream_t st);

// Batched form (one pass over many light fields).
cudaError_t launch_copy_blob(const void *src, int n, void *dst, cudaStream_t st);
size_t batch_lf_bytes();
size_t batch_hdr_bytes();
// key_off: the light field's first flag (a multiple of 16), sk_off its first
// super key, cam_off its first camera in the call's flattened arrays.
void batch_fill_lf(void *dst, const DevStream &ds, int64_t key_off, int64_t sk_off, int64_t cam_off);
void batch_fill_hdr(void *dst, int n_lf, int n_views, int total_tiles, int tile_w, int tile_h, int64_t n_keys,
                    int64_t n_sk, int64_t n_cam);
// Scratch and sizes of one batched pass: flags (n_keys), camera image
// offsets (n_cam), items (n_sk), counters {items << 32, image pixels
// allocated}, the blend's tile counter, the image pool (capacity pixels,
// below 2^31), items per decode pass and the decode's CTA count.
struct BatchLaunch {
    int total_tiles = 0;
    uint8_t *flags = nullptr;
    uint32_t *camslot = nullptr;
    uint4 *items = nullptr;
    unsigned long long *counters = nullptr;
    unsigned int *work = nullptr;
    uint32_t *cache = nullptr;
    unsigned long long capacity = 0;
    int64_t n_sk = 0, n_cam = 0;
    int group = 2, decode_ctas = 0, sm_count = 0;
    float *d_out = nullptr;
};
cudaError_t launch_batch(int B, int tile_shape, const void *image, const int *ptr_offsets, const BatchLaunch &L,
                         cudaEvent_t const *phase, cudaStream_t st);
// bias: the forward carries the expected rounding of the integer decode.
cudaError_t launch_render_relaxed(const DevStream &ds, const LaunchViews &lv, int total_tiles, const float *coeff,
                                  const float *root, float *d_out, bool bias, cudaStream_t st);
cudaError_t launch_render_backward(const DevStream &ds, const LaunchViews &lv, int total_tiles,
                                   const float *grad_out, float *grad_coeff, float *grad_root, cudaStream_t st);
cudaError_t launch_dequant(const DevStream &ds, int64_t n_nc, float *coeff, float *root, cudaStream_t st);

}  // namespace hmlfc
