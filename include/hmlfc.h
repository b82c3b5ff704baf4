/*
 * hmlfc.h -- C ABI of the GB300 HMLFC library: random-access decoding of a
 * hierarchical motion-compensated light-field stream fused with two-plane
 * novel-view rendering (Pratapa & Manocha, "HMLFC: Hierarchical
 * Motion-Compensated Light Field Compression for Interactive Rendering",
 * arXiv 1902.09396).
 *
 * Conventions
 * -----------
 * - Every entry point returns HMLFC_OK (0) or a negative HMLFC_E_* code;
 *   hmlfc_last_error() gives a thread-local message for the last failure.
 * - Arguments named d_* are device pointers owned by the caller; h_* are host
 *   pointers owned by the caller.  The library never frees caller memory.
 * - Calls that take a `cuda_stream` (a cudaStream_t passed as void*; NULL =
 *   the legacy default stream) enqueue their work on it and return without
 *   synchronising, except hmlfc_load_stream, hmlfc_encode_device and
 *   hmlfc_check_status, which synchronise it.  hmlfc_encode,
 *   hmlfc_requantize and the hmlfc_touched_bytes* counters are host-only.
 * - Render scratch (decoded camera images, their index, the host-output
 *   staging) is allocated stream-ordered from a library-owned pool per
 *   device that keeps the memory it has mapped for later calls.
 * - The hmlfc_set_* switches are process-wide and not thread-safe.
 * - A stream object may be used from several CUDA streams at once for
 *   reading (render, decode, backward); it must not be freed while work
 *   that uses it is in flight.
 *
 * Stream format (little-endian; all offsets in bytes; sections 16-byte
 * aligned).  The paper fixes the tree, the BISE coding and the breadth-first
 * order (Sec. 4.3-4.7) but not the bit layout, the block index or the
 * cluster shape; the readings fixed here are:
 *
 *   header: 32 x u32
 *     [0] magic 0x464C4D48 ("HMLF")  [1] version 1
 *     [2] nu  [3] nv   camera grid (u, v)      [4] W  [5] H   view size
 *     [6] L   SRV levels (tree height; roots are the level-L RKVs)
 *     [7] B   block size  [8] Ws search window (px)  [9] q quantiser step
 *     [10] T_ref [11] T_pred block thresholds  [12] flags (bit 0: MC, bit 1:
 *     chroma sub-sampled 4:2:0)
 *     [13] mv_mode [14] mv_b  BISE alphabet of the motion-vector symbols
 *     [15] n_nc node-channels  [16] groups per node-channel
 *     [17] n_sig significant blocks  [18] record words  [19] MV symbols
 *     [20] MV words  [21..25] offsets of roots, groups, block offsets,
 *     records, MV words  [26] total bytes  [27..31] zero
 *   tree: level l has ceil(nu/2^l) x ceil(nv/2^l) nodes; node (a, b) of
 *     level l+1 is the RKV of the 2x2 cluster {2a, 2a+1} x {2b, 2b+1} of
 *     level l (Sec. 4.3).  The cluster member with both coordinates even is
 *     its reference SRV, the others are predictive SRVs (Sec. 4.4).  Camera
 *     (i, j) lies under node (i >> l, j >> l) at level l.
 *   node-channels: breadth-first from the top (Sec. 4.7): l = L-1 .. 0,
 *     nodes row-major (a major), channels Y, Co, Cg (YCoCg-R, Sec. 4.5).
 *   channel planes: Y is W x H; Co and Cg are W x H too, or, with flag bit
 *     1, ceil(W/2) x ceil(H/2) (Sec. 4.5 sub-sampled chroma: the rounded mean
 *     of each 2x2 pixel group; sample (x, y) reads chroma pixel
 *     (x >> 1, y >> 1)).  Every plane of a channel has that channel's size
 *     and its own B x B block grid.
 *   roots: int16, per root (row-major) its Y, Co, Cg planes in turn.
 *   blocks: B x B raster blocks of each node-channel, k = by * nbx + bx;
 *     edge blocks are partial (bw x bh valid pixels, in-block index
 *     (y - y0) * bw + (x - x0)).
 *   groups: per node-channel ceil(luma blocks / 32) groups (a sub-sampled
 *     chroma node-channel leaves its last ones empty); per run of 32 blocks
 *     of the node-channel's plane a {bitmap, record base
 *     word, block-offset base, 0} quadruple; bit r marks block 32g+r
 *     significant (Sec. 4.5 thresholds); its record starts at record word
 *     base + offsets[offset base + popcount(bitmap & ((1 << r) - 1))]
 *     (u16 offsets).  Insignificant blocks are zero.
 *   records: u32 header (bits 0-15 int16 min level m, 16-20 b, 21-22
 *     mode) followed by the BISE payload of the block's levels minus m
 *     (Sec. 4.6): mode 0 = b bits per value; mode 1 = groups of 5 values
 *     with an 8-bit trit byte t0+3t1+9t2+27t3+81t4 then 5 x b low bits;
 *     mode 2 = groups of 3 values with a 7-bit field q0+5q1+25q2 then 3 x b
 *     low bits; value = hi * 2^b + low; bit k is bit k%32 of word k/32.
 *     The dequantised coefficient is q * (m + value).
 *   motion vectors: one BISE sequence (mode, b of the header) with one
 *     symbol per block (of its channel's grid) of every predictive
 *     node-channel, in breadth-first order: ((mvx + 4Ws)(8Ws + 1) + (mvy + 4Ws)) * 2 + (sign < 0), mv in
 *     quarter pixels within [-4Ws, 4Ws].
 *
 * Decoding one sample (Sec. 4.8.1): value_c = root_c(x, y) + sum over l of
 * SRV_l,c(x, y); a reference SRV is its dequantised coefficient R^; a
 * predictive SRV is sign * P + r^ where r^ is its dequantised residual and
 * P = (sum of 4 bilinear taps of its reference's R^ at (4x + mvx, 4y + mvy)
 * quarter-pel, weights summing to 16, + 8) >> 4 with taps clamped to the
 * image (Sec. 4.4; quarter-pel after the sub-pel extension of Sec. 6).  The
 * inverse YCoCg-R then gives RGB, each clamped to [0, 255].
 */
#ifndef HMLFC_H
#define HMLFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HMLFC_OK 0
#define HMLFC_E_INVALID_ARG -1
#define HMLFC_E_CORRUPT -2
#define HMLFC_E_OOM -3
#define HMLFC_E_CUDA -4
#define HMLFC_E_TIMEOUT -5
#define HMLFC_E_UNSUPPORTED -6

/* Largest number of views one render call takes, and of distinct streams. */
#define HMLFC_MAX_VIEWS 1048576
#define HMLFC_MAX_STREAMS 16

typedef struct hmlfc_stream hmlfc_stream;

/*
 * One novel view (96 bytes).  Output pixel (px, py) is the ray whose
 * two-plane coordinates (Sec. 2.1) are (u, v) = H_uv (px + .5, py + .5, 1)
 * and (s, t) = H_st (px + .5, py + .5, 1) (projective, row-major 3x3).
 * (u, v) is in camera-grid units (camera (i, j) at (u, v) = (i, j)); (s, t)
 * is in pixels (sample x at s = x).  The 16 neighbouring samples
 * (floor/ceil of each coordinate, clamped to the grid and image) are blended
 * quadrilinearly.  The view's FP32 RGB output, in [0, 1] (= RGB8 / 255), is
 * written as [height][width][3] starting at element out_offset of d_out.
 * `lf` indexes the streams array of the call.
 */
typedef struct {
    int32_t lf;
    int32_t width;
    int32_t height;
    float H_uv[9];
    float H_st[9];
    int32_t reserved;
    int64_t out_offset;
} hmlfc_view;

typedef struct {
    int32_t nu, nv, width, height, levels, block, search, qstep, mc;
    int32_t n_roots;
    int32_t chroma;         /* 1: chroma sub-sampled 4:2:0 */
    int64_t n_nc, n_blocks, n_sig, n_ref_tiles;
    int64_t stream_bytes;   /* size of the compressed stream */
    int64_t device_bytes;   /* device memory held by the stream object */
} hmlfc_stream_info_t;

/*
 * Parse and validate a compressed stream (format above), copy it to device
 * `device` and decode, once, its roots and every reference SRV into resident
 * block-sparse tiles (Sec. 4.8.2: all reference SRVs are decoded at the start
 * of decompression and kept in a sparse form).  The bytes are copied; the
 * caller may free them on return.  Synchronous.  Errors: HMLFC_E_CORRUPT (the
 * header, an index entry or a record points outside the stream),
 * HMLFC_E_INVALID_ARG, HMLFC_E_OOM, HMLFC_E_CUDA.
 */
int hmlfc_load_stream(const void *h_bytes, size_t nbytes, int device, void *cuda_stream, hmlfc_stream **out);

/* Release the stream object and its device memory (NULL is ignored). */
void hmlfc_free_stream(hmlfc_stream *s);

int hmlfc_stream_info(const hmlfc_stream *s, hmlfc_stream_info_t *out);

/*
 * Random-access decoding (Sec. 4.8.1, Sec. 4.8.4) of n samples.
 * d_coords: int32 [n][4] = (i, j, x, y): camera (i, j), pixel (x, y).
 * d_rgb: uint8 [n][3] output.  A coordinate outside the light field decodes
 * to (0, 0, 0) and sets the stream's status word, which hmlfc_check_status
 * reports as HMLFC_E_INVALID_ARG.  n = 0 is a no-op.
 */
int hmlfc_decode_pixels(const hmlfc_stream *s, const int32_t *d_coords, int64_t n, uint8_t *d_rgb,
                        void *cuda_stream);

/*
 * Progressive decoding (Sec. 1 and Sec. 4: the tree's upper levels hold what
 * the views share, the lower levels their detail, and the breadth-first
 * stream orders them top down): as hmlfc_decode_pixels, but the sum of
 * Sec. 4.8.1 stops at `level` (0 <= level <= L): sample (i, j, x, y) is the
 * reconstruction of the level-`level` node (i >> level, j >> level), i.e.
 * root + SRV levels L-1 .. level, through the inverse YCoCg-R and clamp.
 * level 0 is hmlfc_decode_pixels; level L gives the stored roots.  Errors: as
 * hmlfc_decode_pixels; HMLFC_E_INVALID_ARG for a level outside 0..L.
 */
int hmlfc_decode_pixels_lod(const hmlfc_stream *s, const int32_t *d_coords, int64_t n, int level, uint8_t *d_rgb,
                            void *cuda_stream);

/*
 * Synchronise `cuda_stream` and report (then clear) the stream object's
 * status word: HMLFC_OK, or HMLFC_E_INVALID_ARG if a decode on it met an
 * out-of-range coordinate since the last check.
 */
int hmlfc_check_status(const hmlfc_stream *s, void *cuda_stream);

/*
 * Render n_views novel views (Sec. 5: ray-traced views decoded on the fly):
 * per output ray, (u,v,s,t) from the view's homographies, the 16 neighbouring
 * light-field samples decoded by random access from streams[view.lf], and
 * their quadrilinear blend.  h_views is host memory.  Views of different
 * sizes and streams may be mixed.  Coordinates outside the grid or image
 * clamp to the edge.
 */
int hmlfc_render_views(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                       float *d_out, void *cuda_stream);

/*
 * Render into host memory: as hmlfc_render_views, with the output in h_out
 * (host memory, the same packed layout; page-locked for full speed).  The
 * library stages the output in device memory allocated from cuda_stream's
 * pool; the decode runs once for all views, then the blend runs in groups
 * of 8 views, each group's views copied to the host on a library-owned copy
 * stream while the next group blends.  Asynchronous: h_out holds the views
 * once cuda_stream has synchronised (cuda_stream waits for the copies).
 * Calls on different CUDA streams overlap: one call's decode runs while an
 * earlier call's copies drain (all copies run in order on one copy stream
 * per device).  Errors: as hmlfc_render_views; HMLFC_E_OOM for the staging.
 */
int hmlfc_render_views_host(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                            float *h_out, void *cuda_stream);

/*
 * Level-of-detail render: as hmlfc_render_views with every sample decoded
 * progressively to `level` (see hmlfc_decode_pixels_lod): the 16 samples of
 * a ray come from the level-`level` reconstructions of its cameras' nodes,
 * so the work per call falls with the level (fewer SRV levels and one
 * decoded block per node instead of per camera).  level must lie in 0..L of
 * every stream (HMLFC_E_INVALID_ARG otherwise).  The per-tile staging of
 * hmlfc_set_render_path(2) is replaced by the per-ray path for level > 0.
 */
int hmlfc_render_views_lod(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                           int level, float *d_out, void *cuda_stream);

/*
 * hmlfc_render_views without any memory allocation (the paper has no
 * counterpart: this is an interface for callers of this library).
 *
 * Some callers cannot allocate device memory at the time they render: a
 * frame loop with a hard deadline that must not stall on the allocator or
 * fail on fragmentation midway, code running under a caching allocator that
 * has to account for every byte, or code capturing work into a CUDA graph
 * in a capture mode that forbids cudaMalloc.  (It makes CUDA calls, so it
 * cannot run inside a host function enqueued on a stream.)  This
 * entry point gives them the cached render of hmlfc_render_views, with the
 * same results, using only memory the library reserved when it was loaded:
 * a fixed device array of 32 MiB (HMLFC_FIXED_SCRATCH_BYTES), which every GPU
 * that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * - Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 * - Limit: the block index of a stream (1 byte per (camera, block) pair, 16
 *   bytes per (level-2 node, block) pair, 4 bytes per camera) must fit the
 *   array; a larger stream is rejected with HMLFC_E_UNSUPPORTED and a
 *   message, and hmlfc_render_views should be used instead.  The rest of the
 *   array holds decoded camera images (W * H * 4 bytes each); the rays of
 *   cameras beyond it decode their samples directly (same results, slower).
 * - Sharing: every call uses the same array and leaves its contents behind;
 *   each call clears what must start at zero.  Calls whose GPU work overlaps
 *   (on different CUDA streams, or from several host threads without
 *   ordering) race on the array and must be serialised by the caller.
 */
#define HMLFC_FIXED_SCRATCH_BYTES (32u << 20)
int hmlfc_render_views_noalloc(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views,
                               int n_views, float *d_out, void *cuda_stream);

/*
 * Batched form of hmlfc_render_views (same results): all views of all
 * streams in one pass -- one launch each of footprint marking, camera-image
 * and item assignment, a block decode over every stream's items and a
 * persistent blend whose CTAs take (view, tile) items from an atomic
 * counter.  The camera images of all streams share one pool (cameras beyond
 * it decode their rays directly).  The call's view records and stream
 * descriptors are copied into stream-ordered scratch by kernels whose
 * parameters carry them, so the call can be captured in a CUDA graph and
 * replayed without touching host memory.  Streams may differ in block size
 * and chroma mode.
 */
int hmlfc_render_batch(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                       float *d_out, void *cuda_stream);

/* Tunables of hmlfc_render_batch (process-wide): rays per tile (0: 16x16,
 * 1: 32x8, 2: 8x8), decode items per pass (1-8; above 4 act as 4), decode
 * CTAs launched per SM (1-32), camera-image pool bytes (0 keeps the current
 * value; default 2 GiB).  Chosen per workload by the package's autotuner. */
int hmlfc_set_batch_tuning(int tile_shape, int group, int ctas_per_sm, size_t cache_bytes);

/*
 * Serving form.  A server keeps a decoded-block cache of one stream resident
 * on the device across render calls (cache_bytes of B * B * 4-byte slots, plus
 * a slot map of 4 bytes per (camera, block) pair).  Each call marks the
 * blocks its views reach, reuses the resident ones, decodes the others into
 * slots not used by the call (oldest first), and blends every ray from the
 * cache; results equal hmlfc_render_views.  Calls on one server must be
 * ordered on one CUDA stream (they share its cache).  create and free are
 * synchronous; render is asynchronous.  hmlfc_server_stats synchronises and
 * writes {blocks decoded since creation, decode items, cache slots}.
 */
typedef struct hmlfc_server hmlfc_server;
int hmlfc_server_create(const hmlfc_stream *s, size_t cache_bytes, void *cuda_stream, hmlfc_server **out);
int hmlfc_server_render(hmlfc_server *sv, const hmlfc_view *h_views, int n_views, float *d_out, void *cuda_stream);
int hmlfc_server_stats(const hmlfc_server *sv, void *cuda_stream, int64_t *out3);
void hmlfc_server_free(hmlfc_server *sv);

/*
 * Differentiable relaxation (for gradient-based refinement of the residuals):
 * the same render with real-valued coefficients -- exact bilinear weights
 * instead of the >> 4 rounding, YCoCg-R inverse with /2 instead of >> 1, no
 * clamp.  It is linear in the coefficients for the stream's fixed motion
 * vectors and signs.
 * d_coeff[k]: float [n_nc][H][W] per stream (breadth-first node-channel
 * order; references hold R^, predictive nodes r^); d_root[k]: float
 * [n_roots][3][H][W].
 */
int hmlfc_render_views_relaxed(const hmlfc_stream *const *streams, int n_streams, const float *const *d_coeff,
                               const float *const *d_root, const hmlfc_view *h_views, int n_views, float *d_out,
                               void *cuda_stream);

/*
 * hmlfc_render_views_relaxed with flags.  HMLFC_RELAX_BIAS: every rounding
 * the relaxation drops carries its expected value, so that at the stream's
 * own coefficients the relaxed render has no mean offset from the integer
 * render.  A predictor with quarter-pel phase (fx, fy) = (mvx & 3, mvy & 3)
 * adds g / 32, g = gcd(4 - fx, fx) * gcd(4 - fy, fy) (the mean of
 * floor((S + 8) / 16) - S / 16 when S is equally likely in each residue
 * class its weights allow; 0 for integer motion), times its sign; each >> 1
 * of the YCoCg-R inverse becomes v / 2 - 1/4, which adds (1/2, 1/4, 1/2)
 * levels to (R, G, B).  The terms are constants, so hmlfc_render_backward
 * is the adjoint of both forms.  Other flag bits: HMLFC_E_INVALID_ARG.
 */
#define HMLFC_RELAX_BIAS 1u
int hmlfc_render_views_relaxed_ex(const hmlfc_stream *const *streams, int n_streams, const float *const *d_coeff,
                                  const float *const *d_root, const hmlfc_view *h_views, int n_views, uint32_t flags,
                                  float *d_out, void *cuda_stream);

/*
 * Adjoint of hmlfc_render_views_relaxed: ACCUMULATES d(<out, grad_out>) into
 * d_grad_coeff[k] (float [n_nc][H][W]) and d_grad_root[k] (float
 * [n_roots][3][H][W]) for every stream k.  Decoded tiles are recomputed,
 * nothing is stored between the passes.  Accumulation uses FP32 atomics, so
 * the summation order (and the last bits) may vary between runs.
 */
int hmlfc_render_backward(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                          const float *d_grad_out, float *const *d_grad_coeff, float *const *d_grad_root,
                          void *cuda_stream);

/*
 * Write the stream's dequantised coefficients (float [n_nc][H][W]) and roots
 * (float [n_roots][3][H][W]) to device memory: the starting point of the
 * relaxation.
 */
int hmlfc_dequant(const hmlfc_stream *s, float *d_coeff, float *d_root, void *cuda_stream);

/* Encoder parameters (Sec. 4.5: tree height, block size, two block
 * thresholds, search window) plus the quantiser step and the MC mode
 * (0 = none, 1 = phase-shifted with quarter-pel refinement, 2 = zero
 * motion, 3 = phase-shifted integer-pel as in the paper).  chroma: 0 = Co and
 * Cg at full resolution; 1 = sub-sampled 4:2:0 (Sec. 4.5: Co and Cg coded at
 * ceil(W/2) x ceil(H/2), each the rounded mean of a 2x2 pixel group, decoded
 * by nearest-pixel reconstruction; needs an even block size). */
typedef struct {
    int32_t levels, block, search, qstep, t_ref, t_pred, mc, threads, chroma;
} hmlfc_encode_params;

/*
 * Encode h_lf (uint8 [nu][nv][H][W][3], RGB) into a stream of the format
 * above (Sec. 4.3-4.7).  *h_out is allocated by the library; release it with
 * hmlfc_free_host.  Synchronous, host threads only.
 */
int hmlfc_encode(const uint8_t *h_lf, int nu, int nv, int width, int height, const hmlfc_encode_params *p,
                 void **h_out, size_t *nbytes);

/* Work done by one device encode (all counts over the whole light field). */
typedef struct {
    uint64_t blocks;            /* (node-channel, block) pairs coded */
    uint64_t sig_blocks;        /* of which significant (a record in the stream) */
    uint64_t blocks_searched;   /* predictive blocks run through the block search (mc 1 or 3) */
    uint64_t int_terms;         /* |S - R| and |S + R| terms of the integer stage (Eq. 1-2), both signs */
    uint64_t frac_terms;        /* |S -+ P| terms of the quarter-pel refinement, P bilinear (mc 1) */
} hmlfc_encode_stats;

/*
 * Encode on the GPU: the same stream, byte for byte, as hmlfc_encode with the
 * same arguments (Sec. 4.3-4.7).  The closed loop runs top down, one grid per
 * level and member class (references first, then the predictive members
 * against them); the block search of Sec. 4.4 (Eq. 1-2, both signs, integer
 * stage then quarter-pel refinement) runs one CTA per block.
 * d_lf: device memory, uint8 [nu][nv][H][W][3] RGB, caller-owned, read only.
 * The library allocates its device scratch (about 11x the light field's
 * bytes) and frees it before returning; *h_out is host memory, released with
 * hmlfc_free_host.  p->threads is ignored.  Work runs on cuda_stream, which is
 * synchronised before the call returns.  Errors: as hmlfc_encode;
 * HMLFC_E_UNSUPPORTED also for a search window above 32 with mc 1 or 3;
 * HMLFC_E_OOM when the scratch cannot be allocated; HMLFC_E_CUDA.
 * stats (may be NULL) receives the work counts of this call.
 */
int hmlfc_encode_device(const uint8_t *d_lf, int nu, int nv, int width, int height, const hmlfc_encode_params *p,
                        void *cuda_stream, void **h_out, size_t *nbytes, hmlfc_encode_stats *stats);

/*
 * Events (cudaEvent_t, caller-owned) that hmlfc_encode_device records on its
 * stream around the block-search pass of each level, top level first:
 * events[2 i] before and events[2 i + 1] after the pass of level L-1-i.
 * n = 0 (events may be NULL) turns the recording off; n <= 32.  Process-wide
 * setting, not thread-safe.
 */
int hmlfc_set_encode_events(void *const *events, int n);

/*
 * Re-encode a stream with new coefficients (float [n_nc][H][W], host) and
 * roots (float [n_roots][3][H][W], host) at the same quantiser step, motion
 * vectors and signs: coefficients are rounded to the nearest multiple of q,
 * roots to integers, and blocks whose levels are all zero become
 * insignificant.  Synchronous.
 */
int hmlfc_requantize(const hmlfc_stream *s, const float *h_coeff, const float *h_root, void **h_out, size_t *nbytes);

void hmlfc_free_host(void *p);

/*
 * Bytes that rendering the views must move at least once: the FP32 output
 * plus every distinct root pixel (6 B), predictive block (group entry,
 * offset, record, motion-vector bits) and significant reference tile
 * (B * B * 2 + 4 B) the views' samples reach.  One value per view into
 * h_bytes.  Synchronous, host threads only (a measurement aid).
 */
int hmlfc_touched_bytes(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views, int n_views,
                        double *h_bytes);

/* The same count over the whole call: every distinct item once, however
 * many views reach it, plus every view's output (one total into h_total);
 * h_cam_blocks (may be NULL) receives the number of distinct (camera, block)
 * pairs that hold a reached sample. */
int hmlfc_touched_bytes_union(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views,
                              int n_views, double *h_total, double *h_cam_blocks);

/* The same count for a level-of-detail render at `level` (0..L): samples
 * are keyed by their level-`level` node, only levels L-1 .. level are reached,
 * and h_cam_blocks counts (node, block) pairs. */
int hmlfc_touched_bytes_union_lod(const hmlfc_stream *const *streams, int n_streams, const hmlfc_view *h_views,
                                  int n_views, int level, double *h_total, double *h_cam_blocks);

/*
 * Render strategy (process-wide).  0 (default): decode every (camera, block)
 * pair the call's views reach once, into per-camera RGB8 images held in
 * stream-ordered scratch memory (allocated on the call's stream from the
 * library pool, released on it when the call's work ends), then blend each
 * ray from the images; the rays of cameras beyond the scratch capacity decode
 * their samples directly, and if not even one image fits or the scratch
 * cannot be allocated, each tile stages its own footprint instead.  1: every
 * ray decodes its own 16 samples.  2: each 16 x 16 tile stages its footprint
 * in shared memory.  All give bit-identical output.
 */
int hmlfc_set_render_path(int path);

/* Scratch budget of one cached render call, in bytes: the block index plus
 * the decoded camera images (W * H * 4 bytes each).  A call allocates an
 * image for every camera of the stream, or as many as the budget holds
 * (cameras beyond it decode their rays directly, much more slowly).
 * Default 8 GiB (a 32x32 grid of 1024^2 cameras takes 4 GiB); 0 disables
 * the cache. */
int hmlfc_set_block_cache_bytes(size_t bytes);

/*
 * Measurement aid (process-wide): four caller-created CUDA events that the
 * cached render records on the call's stream before marking, before the
 * block decode, before the blend and at the end, so that each phase can be
 * timed with cudaEventElapsedTime; NULL stops the recording.
 */
int hmlfc_set_phase_events(void *const *events);

const char *hmlfc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HMLFC_H */
