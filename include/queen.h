/*
 * queen.h -- C ABI of the GB300 (sm_103a) implementation of QUEEN's per-frame
 * residual-training hot path (arXiv 2412.04469).
 *
 * Conventions shared by every entry point
 *   - Pointers named *_host point to host memory; every other pointer is a
 *     device pointer owned by the caller.  The library never allocates or
 *     frees device memory and keeps no state between calls except the
 *     thread-local error string.
 *   - Every call enqueues its kernels on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and returns without synchronising, unless its
 *     comment says otherwise.
 *   - Per-Gaussian arrays are structure-of-arrays planes: plane k of an array
 *     with stride S starts at element k * S.  S (n_stride) must be >= n and a
 *     multiple of 4.
 *   - Return value: QN_OK or a negative QN_ERR_* code; qn_last_error() gives a
 *     message for the calling thread.  Argument checks happen before any
 *     launch, so an error return never leaves partial output behind, except
 *     QN_ERR_CUDA, which reports a failed launch.
 *
 * Raw Gaussian attributes A ([n_attr][n_stride] float32, n_attr = 11 + 3 K,
 * K = (sh_degree + 1)^2; Sec. 3.1):
 *   planes 0-2 position p, 3-6 quaternion (w, x, y, z; need not be unit),
 *   7-9 log-scale, 10 logit-opacity, 11 + 3 k + ch SH coefficient k
 *   (k = l^2 + l + m, real SH without the Condon-Shortley phase) of channel ch.
 */
#ifndef QUEEN_H
#define QUEEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    QN_OK = 0,
    QN_ERR_INVALID_ARG = -1,
    QN_ERR_CUDA = -2,
    QN_ERR_CAPACITY = -3,
    QN_ERR_TIMEOUT = -4,
    QN_ERR_UNSUPPORTED = -5
};

#define QN_TILE 16            /* 16 x 16 pixel tiles */
#define QN_MAX_CATEGORIES 8   /* residual decoder categories */
#define QN_MAX_LATENT 16      /* latent width per category */
#define QN_MAX_TILES_X 256    /* image width  <= 4096 */
#define QN_MAX_TILES_Y 256    /* image height <= 4096 */
#define QN_DECODE_BWD_BLOCKS 1216 /* per-block partials of the decoder gradient */
#define QN_MLP_BWD_BLOCKS 256     /* per-block partials of the MLP gradient */
#define QN_LOSS_BLOCKS 2048       /* per-block partials of the image loss */

typedef void *qn_stream_t;    /* cudaStream_t */

/* Pinhole camera (host struct, passed by pointer, copied at launch).
 * World -> camera: t_cam = R p + t with R row-major; camera x right, y down,
 * z forward.  Pixel (u, v) samples the image plane at (u + 0.5, v + 0.5);
 * p' = (fx x / z + cx, fy y / z + cy).  campos is the camera centre, used
 * for the SH view direction. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_plane;
    float campos[3];
    int32_t width, height;
} qn_camera;

/* Residual categories (Sec. 3.4): category c decodes lat_dim[c] latents into
 * attribute planes attr_begin[c] .. attr_begin[c] + attr_count[c] - 1; the
 * planes must lie in 3 .. n_attr - 1 and not overlap.  Latent planes and
 * decoder blocks (row-major attr_count x lat_dim) follow category order. */
typedef struct {
    int32_t n_cat;
    int32_t attr_begin[QN_MAX_CATEGORIES];
    int32_t attr_count[QN_MAX_CATEGORIES];
    int32_t lat_dim[QN_MAX_CATEGORIES];
} qn_decoder_layout;

/* Hard-concrete gate hyper-parameters (Eq. 6-8): temperature tau, stretch
 * interval (gamma0, gamma1) with gamma0 < 0 < 1 < gamma1.  noise (nullable,
 * device [n] f32, u in (0, 1), e.g. from qn_gate_uniform): the stochastic
 * hard-concrete sample of the cited gate formulation, g-hat =
 * sigmoid((log alpha + log u - log(1 - u)) / tau), for training; NULL gives
 * Eq. 6 as written.  L_reg (Eq. 8) does not depend on the noise. */
typedef struct {
    float tau, gamma0, gamma1;
    const float *noise;
} qn_gate_params;

/* Message of the last error on this host thread ("" if none). */
const char *qn_last_error(void);
/* Library version string. */
const char *qn_version(void);

/* ------------------------------------------------------------------------ */
/* Residual decode and gate -- Sec. 3.2, Eq. 4-8.                            */
/* ------------------------------------------------------------------------ */

/*
 * A_t = A_{t-1} + R_t (Eq. 4).  For each category c and Gaussian i:
 *   l = clamp(round_half_even(lat), -128, 127)          (Eq. 5, STE forward)
 *   r_c = D_c float(l)   (bf16 decoder, FP32 accumulation) added to its planes
 * and for the position (Eq. 6-7, deterministic hard-concrete gate):
 *   g = min(1, max(0, sigmoid(log_alpha / tau) (gamma1 - gamma0) + gamma0))
 *   p_t = p_{t-1} + g lp
 * L_reg = sum_i sigmoid(log_alpha_i - tau log(-gamma0 / gamma1))  (Eq. 8).
 *
 *   prev  [n_attr][n_stride] f32  A_{t-1}             (read)
 *   lat   [sum lat_dim][n_stride] f32  continuous latents (read)
 *   dec   bf16 bits, concatenated row-major D_c blocks  (read)
 *   lp    [3][n_stride] f32  pre-gated position residual (read)
 *   log_alpha [n] f32                                   (read)
 *   skip  [n] u8 (nullable): Gaussians with skip != 0 are frozen -- their
 *         out columns and gate entries are left as they are and they add
 *         nothing to lreg.  A Gaussian whose residual parameters do not
 *         change keeps its A_t, so after one call without skip the frozen
 *         columns already hold it.
 *   out   [n_attr][n_stride] f32  A_t                   (written; may not alias prev)
 *   gate  [n] f32 g_i                                    (written; nullable)
 *   lreg  [1] f32 L_reg over the Gaussians not skipped   (written; nullable)
 * Errors: QN_ERR_INVALID_ARG for n < 0, bad stride, null required pointers,
 * a layout outside the limits above.
 */
int qn_decode_residuals(int32_t n, int32_t n_stride, int32_t n_attr, const float *prev,
                        const float *lat, const uint16_t *dec, const qn_decoder_layout *layout_host,
                        const float *lp, const float *log_alpha, const qn_gate_params *gate_host,
                        const uint8_t *skip, float *out, float *gate, float *lreg, qn_stream_t stream);

/*
 * Adjoint of qn_decode_residuals for dL/dA_t = d_out and dL/dL_reg = d_lreg:
 *   d_lat   = D_c^T d_out[c planes]              (straight-through estimator)
 *   d_dec   = sum_i d_out[c planes]_i float(l_i)^T   (FP32, overwritten)
 *   d_lp    = g d_out[0..2]
 *   d_log_alpha = (d_out[0..2] . lp) dg/dlog_alpha + d_lreg p (1 - p),
 *     dg/dlog_alpha = (gamma1 - gamma0) ghat (1 - ghat) / tau inside the clamp, 0 outside.
 * skip (nullable, [n] u8): Gaussians with skip != 0 get zero d_lat, d_lp,
 * d_log_alpha and add nothing to d_dec.
 *   d_lat [sum lat_dim][n_stride], d_dec [sum attr_count*lat_dim], d_lp [3][n_stride],
 *   d_log_alpha [n]: written.
 *   partials [QN_DECODE_BWD_BLOCKS * sum attr_count*lat_dim] f32: scratch for
 *     per-block partial sums of d_dec, added in block order (reproducible).
 */
int qn_decode_residuals_bwd(int32_t n, int32_t n_stride, int32_t n_attr, const float *lat,
                            const uint16_t *dec, const qn_decoder_layout *layout_host,
                            const float *lp, const float *log_alpha,
                            const qn_gate_params *gate_host, const float *d_out, float d_lreg,
                            const uint8_t *skip, float *d_lat, float *d_dec, float *d_lp,
                            float *d_log_alpha, float *partials, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* EWA projection and SH colour -- Sec. 3.1, Eq. 1.                          */
/* ------------------------------------------------------------------------ */

/*
 * Projected record of one Gaussian ("splat"), 48 bytes, 16-byte aligned:
 *   s[0] = (mean2d x, mean2d y, opacity, depth t_z)
 *   s[1] = (conic a, conic b, conic c, 0)   power = -0.5 (a dx^2 + c dy^2) - b dx dy
 *   s[2] = (r, g, b, 0)                      colour = max(0, 0.5 + sum_k h_k Y_k(dir))
 * Its gradient record has the same layout: (d mean2d x, d mean2d y,
 * d opacity, 0), (d a, d b, d c, 0), (d r, d g, d b, 0).
 * rect = (x0, y0, x1, y1): half-open tile range; (0,0,0,0) when culled.
 */
typedef struct {
    float s[12];
} qn_splat;

/*
 * Sigma = R(q) S S^T R(q)^T, S = diag(exp(log-scale)); t = W p;
 * Sigma' = J W Sigma W^T J^T + blur I with J the affine Jacobian at t (x/z and
 * y/z clamped to +-1.3 half-extent / focal inside J); conic = Sigma'^-1;
 * radius = ceil(3 sqrt(mid + sqrt(max(0.1, mid^2 - det))));
 * rect = [floor((p' - r)/16), floor((p' + r + 15)/16)) clamped to the grid.
 * With tight_rects != 0 the rect is further intersected with the tiles
 * [floor((p' - h)/16), floor((p' + h)/16) + 1) where h = sqrt(1.01 k Sigma'_xx)
 * + 0.01 (likewise y), k = 2 ln(255 o) + 0.01: a slightly widened bounding box
 * of the ellipse outside which o exp(power) < 1/255.  Every dropped
 * (tile, Gaussian) pair is skipped by every pixel of its tile, so images and
 * gradients are unchanged; only the pair lists shrink.  A Gaussian with k <= 0
 * (o < 0.995/255, never visible) gets an empty rect.
 * Culled (rect zero): t_z <= near_plane, det <= 0, or an empty rect.
 *   attrs [n_attr][n_stride] f32 A_t (read); splats [n] qn_splat, rects [n] int4
 *   (written).  sh_degree in 0..3, n_attr == 11 + 3 (sh_degree+1)^2.
 */
int qn_project(int32_t n, int32_t n_stride, int32_t sh_degree, const float *attrs,
               const qn_camera *cam_host, float blur, int32_t tight_rects, qn_splat *splats,
               int32_t *rects, qn_stream_t stream);

/*
 * Adjoint of qn_project: d_attrs[n_attr][n_stride] (overwritten) from the
 * gradient records d_splats[n]; culled Gaussians get zero.  The colour clamp
 * and the Jacobian clamp pass zero gradient.  skip (nullable, [n] u8): the
 * columns of Gaussians with skip != 0 are left unwritten (the decode adjoint
 * ignores them under the same mask).
 */
int qn_project_bwd(int32_t n, int32_t n_stride, int32_t sh_degree, const float *attrs,
                   const qn_camera *cam_host, float blur, const qn_splat *d_splats,
                   const uint8_t *skip, float *d_attrs, qn_stream_t stream);

/*
 * qn_decode_residuals then qn_project in one pass (Eq. 4-8, then Eq. 1): each
 * block stages a tile of 64 Gaussians' columns of prev, lat and lp in shared
 * memory, adds the residuals there with the same operations in the same
 * order as qn_decode_residuals, and projects the result as qn_project does,
 * so gate, lreg, out, splats and rects equal those of the two calls bit for
 * bit (lreg up to the order of its float sum).  A_t is not read back: the
 * projection reads the staged tile.
 *   Arguments as for qn_decode_residuals and qn_project (n_attr ==
 *   11 + 3 (sh_degree + 1)^2).  out [n_attr][n_stride] (nullable) receives
 *   A_t for the projection adjoint; it may not alias prev.
 *   skip (nullable): skipped Gaussians keep their gate entries and add
 *   nothing to lreg, but unlike qn_decode_residuals they are decoded,
 *   projected and written to out like the rest (their residual parameters
 *   are frozen, so they reproduce the A_t of the last call that trained them).
 * prev, lat, lp, splats and rects must be 16-byte aligned (the staging copies
 * 16-byte chunks); n_stride is a multiple of 4 as everywhere.
 * Errors: QN_ERR_INVALID_ARG as for the two calls, and for misaligned pointers.
 */
int qn_decode_project(int32_t n, int32_t n_stride, int32_t n_attr, int32_t sh_degree, const float *prev,
                      const float *lat, const uint16_t *dec, const qn_decoder_layout *layout_host,
                      const float *lp, const float *log_alpha, const qn_gate_params *gate_host,
                      const uint8_t *skip, const qn_camera *cam_host, float blur, int32_t tight_rects,
                      float *gate, float *lreg, float *out, qn_splat *splats, int32_t *rects,
                      qn_stream_t stream);

/*
 * qn_project_bwd then qn_decode_residuals_bwd in one pass, without A_t or
 * dL/dA_t in memory: each block stages a tile of 64 Gaussians' columns of
 * prev (A_{t-1}), lat and lp in shared memory, rebuilds A_t there with the
 * operations of qn_decode_project (Eq. 4-8), runs the projection adjoint
 * (Eq. 1) on it into a staged dL/dA_t, then the gate and decoder adjoints.
 * d_lat, d_lp and d_log_alpha equal those of the two calls bit for bit (fed
 * the A_t that qn_decode_project or qn_decode_residuals gives); d_dec is the
 * same sum in another order (per-block partials of the tiles, then summed in
 * block order: reproducible).
 *   Arguments as for qn_decode_project and qn_decode_residuals_bwd:
 *   d_splats [n] gradient records (read), d_lreg dL/dL_reg,
 *   d_lat [sum lat_dim][n_stride], d_dec [sum attr_count*lat_dim],
 *   d_lp [3][n_stride], d_log_alpha [n] (written),
 *   partials [QN_DECODE_BWD_BLOCKS * sum attr_count*lat_dim] f32 scratch.
 *   skip (nullable): skipped Gaussians get zero d_lat, d_lp, d_log_alpha and
 *   add nothing to d_dec.
 * prev, lat, lp and d_splats must be 16-byte aligned.
 * Errors: QN_ERR_INVALID_ARG as for the calls it replaces, and for
 * misaligned pointers.
 */
int qn_decode_project_bwd(int32_t n, int32_t n_stride, int32_t n_attr, int32_t sh_degree, const float *prev,
                          const float *lat, const uint16_t *dec, const qn_decoder_layout *layout_host,
                          const float *lp, const float *log_alpha, const qn_gate_params *gate_host,
                          const uint8_t *skip, const qn_camera *cam_host, float blur, const qn_splat *d_splats,
                          float d_lreg, float *d_lat, float *d_dec, float *d_lp, float *d_log_alpha,
                          float *partials, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Tile binning -- the tile-based rasterizer the paper builds on (Sec. 4).    */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace qn_bin_sort needs for n Gaussians on a
 * tiles_x x tiles_y grid. */
size_t qn_bin_sort_workspace_size(int32_t n, int32_t tiles_x, int32_t tiles_y);

/*
 * Emits one (tile, Gaussian) pair per tile of every non-empty rect and sorts
 * the pairs by the 64-bit key (tile << 32) | bits(float depth) -- stable, so
 * equal keys keep Gaussian index order.  Implemented as an LSD radix sort of
 * the 32 depth bits over the n Gaussians followed by one stable counting pass
 * on the tile digit over the pairs; the result equals the stable sort.
 *   depth [n] f32 (read; > 0 for every Gaussian with a non-empty rect),
 *     it may be a strided view: element i at depth[i * depth_stride]
 *   rects [n] int4 (read)
 *   vals  [pair_capacity] u32 Gaussian index per sorted pair (written)
 *   keys  [pair_capacity] u64 sorted keys (written; nullable)
 *   ranges [tiles_x * tiles_y][2] u32: (#pairs with tile < t, #pairs with tile <= t)
 *   n_pairs [1] i64 device: the pair count P (written)
 *   n_pairs_host (nullable): if given, the call synchronises `stream`, stores
 *     P there and returns QN_ERR_CAPACITY when P > pair_capacity.
 * When P > pair_capacity no pair is written and every range is (0, 0).  Pair
 * positions are 32-bit, so a capacity above 2^32 - 1 counts as 2^32 - 1.
 */
int qn_bin_sort(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects,
                int32_t tiles_x, int32_t tiles_y, void *workspace, size_t workspace_bytes,
                int64_t pair_capacity, uint32_t *vals, uint64_t *keys, uint32_t *ranges,
                int64_t *n_pairs, int64_t *n_pairs_host, qn_stream_t stream);

/*
 * qn_bin_sort that writes only the lists of the tiles holding at most
 * list_max pairs (none for 0, all for 0xffffffff) and no keys; ranges,
 * n_pairs, n_pairs_host and the workspace as qn_bin_sort leaves them.  The
 * other lists are formed by qn_render_fwd_binned as it composites, which
 * writes the part of each it walks.  The point: most pairs belong to long
 * lists, of which compositing visits a short prefix, while a short list is
 * often walked to its end.  Arguments, results and errors as qn_bin_sort.
 */
int qn_bin_sort_partial(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects,
                        int32_t tiles_x, int32_t tiles_y, void *workspace, size_t workspace_bytes,
                        int64_t pair_capacity, uint32_t list_max, uint32_t *vals, uint32_t *ranges,
                        int64_t *n_pairs, int64_t *n_pairs_host, qn_stream_t stream);

/* Size of the device array that qn_bin_sort_noalloc uses as its workspace. */
#define QN_BIN_SORT_STATIC_BYTES (40u << 20)

/*
 * qn_bin_sort without a caller-provided workspace, for callers that cannot
 * allocate device memory while binning -- code running inside a memory pool
 * or allocator hook, a plugin that must not touch the host application's
 * allocator, or a real-time loop that forbids allocation.  The paper has no
 * counterpart; this is a convenience of this library.
 *
 * Arguments, results and errors are those of qn_bin_sort, minus `workspace`
 * and `workspace_bytes`.  The scratch space is a fixed file-scope device
 * array of QN_BIN_SORT_STATIC_BYTES (40 MiB), which every GPU that loads this
 * library keeps until the process exits.  A problem whose
 * qn_bin_sort_workspace_size exceeds that is rejected with
 * QN_ERR_INVALID_ARG before any launch (40 MiB covers 300,000 Gaussians on a
 * 1352 x 1014 image).
 * The first call on each device looks up the array's device address (with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture.  The kept address assumes the
 * device's primary context lives as long: after cudaDeviceReset it is stale.
 * No call allocates or frees memory.  All calls share the one array, and each
 * call re-initialises what it reads: calls that overlap on the GPU (another
 * stream, another host thread) race on it and must be serialised by the caller.
 * The binning state (sorted values, per-chunk counts, tile offsets, masks)
 * stays in that private array, so this call feeds the forward compositing
 * only: the compositing adjoint's per-Gaussian sum (qn_render_bwd) needs the
 * workspace of a qn_bin_sort call.
 */
int qn_bin_sort_noalloc(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects,
                        int32_t tiles_x, int32_t tiles_y, int64_t pair_capacity, uint32_t *vals,
                        uint64_t *keys, uint32_t *ranges, int64_t *n_pairs, int64_t *n_pairs_host,
                        qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Compositing -- Sec. 3.1, Eq. 2, and its adjoint.                          */
/* ------------------------------------------------------------------------ */

/*
 * Per pixel (u, v) at (u + 0.5, v + 0.5), front to back over its tile's list:
 *   alpha = min(0.99, o exp(power)); skipped when alpha < 1/255 (no test of
 *   power > 0: for a positive definite conic it only fires on rounding);
 *   stop before a Gaussian that would leave T < 1e-4;
 *   C += c alpha T; T *= 1 - alpha.   img = C + T bg.
 *   img [3][H][W] f32, T_final [H][W] f32, last [H][W] u32 = 1 + list position
 *   (within the tile) of the last contributor, 0 if none (all written).
 *   n_contrib [H][W] u32 (nullable): number of contributors of each pixel.
 *   composited [n] u8 (nullable): set to 1 for every Gaussian that some pixel
 *     composites (never cleared -- zero it before the call).
 *   tile_order [n_tiles] u32 (nullable): a permutation of the tiles, the
 *     order in which the tiles are started (e.g. qn_tile_order's, heaviest
 *     first); it changes no result.
 *   tile_cost [n_tiles] u32 (nullable): written with each tile's largest
 *     `last`, the length of the list prefix its pixels visit.
 *   bg_host: 3 floats in host memory.
 */
int qn_render_fwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                  const qn_splat *splats, const float *bg_host, float *img, float *T_final,
                  uint32_t *last, uint32_t *n_contrib, uint8_t *composited, const uint32_t *tile_order,
                  uint32_t *tile_cost, qn_stream_t stream);

/*
 * qn_render_fwd after qn_bin_sort_partial (n, workspace, workspace_bytes and
 * vals those of that call, the workspace unchanged since): a tile whose list
 * was written reads it from vals; a longer one is formed from the workspace
 * -- the same list, in the same order -- as the tile composites, and every
 * list position a pixel of the tile walks (at least every position below the
 * tile's largest `last`, which is all qn_render_bwd reads) is written to
 * vals[ranges[2 t] + position]; the rest of vals is left as it is.  Every
 * output equals qn_render_fwd's on fully written lists, bit for bit.  ranges
 * may be the binning's or qn_mask_ranges' output (its empty tiles walk
 * nothing).  vals [pair_capacity of the binning] u32 (read, written in part).
 * The call also writes into the workspace, for qn_render_bwd's gather, the
 * first list position of each chunk of Gaussians it walks in each tile (with
 * list_max 0 the binning leaves those to it).
 * Errors: those of qn_render_fwd, and QN_ERR_INVALID_ARG for a missing,
 * misaligned or too small workspace.
 */
int qn_render_fwd_binned(const qn_camera *cam_host, int32_t n, void *workspace, size_t workspace_bytes,
                         const uint32_t *ranges, uint32_t *vals, const qn_splat *splats, const float *bg_host,
                         float *img, float *T_final, uint32_t *last, uint32_t *n_contrib, uint8_t *composited,
                         const uint32_t *tile_order, uint32_t *tile_cost, qn_stream_t stream);

/*
 * tile_order = the tiles by descending tile_cost (costs above 1023 count as
 * 1023; the order among equal costs is unspecified).  The compositing
 * kernels start their tiles in index order, so a deep tile that starts late
 * sets the end of the launch; started first, it overlaps the rest.  Not part
 * of the paper: a scheduling aid.  tile_cost, tile_order [n_tiles] u32.
 */
int qn_tile_order(int32_t n_tiles, const uint32_t *tile_cost, uint32_t *tile_order, qn_stream_t stream);

/*
 * Adjoint of qn_render_fwd for d_img [3][H][W]: the per-Gaussian gradient
 * records d_splats [n] (qn_splat layout: d mean2d, d opacity, d conic,
 * d rgb; overwritten; zero for culled and skipped Gaussians).  Each pixel's
 * list is walked from its last contributor back to the front, T rebuilt by
 * division by (1 - alpha) and the colour behind each Gaussian carried along:
 *   dC/dc_k = alpha_k T_k, dC/dalpha_k = T_k (c_k - B_k), B_last = bg,
 *   B_{k-1} = alpha_k c_k + (1 - alpha_k) B_k; the 0.99 cap passes zero
 *   gradient to opacity, conic and mean; alpha = o G gives dalpha/do = G.
 * Two passes, both without float atomics (every sum has a fixed order, so the
 * result is reproducible bit for bit): per tile, each Gaussian's gradients are
 * summed over the tile's pixels into one record per visited list position of
 * pair_scratch; then each Gaussian's records are summed over the tiles of its
 * rect in row-major order.
 *   n, rects: the Gaussians and int4 rects given to qn_bin_sort; ranges, vals:
 *     its output (ranges may have tiles emptied, e.g. a training mask's).
 *   workspace: the qn_bin_sort workspace that produced the pairs (same n,
 *     rects and tile grid); the call also keeps its own state there.
 *   pair_scratch [pair_capacity] qn_splat: scratch, pair_capacity as given to
 *     that qn_bin_sort call.
 *   skip (nullable, [n] u8): Gaussians with skip != 0 get zero gradient.  A
 *     skipped Gaussian that some pixel composites still enters the others'
 *     gradients (through T and the colour behind).
 *   composited (nullable, [n] u8): qn_render_fwd's marks of the same
 *     forward pass.  A Gaussian without one changes no pixel, so the walk
 *     drops it before any arithmetic; the result is the same.  (Learned skip:
 *     clearing the skip of the composited Gaussians first -- qn_clear_marked
 *     -- drops every still-skipped Gaussian from the walk.)
 *   tile_order (nullable): as for qn_render_fwd (e.g. qn_tile_order of the
 *     forward's tile_cost).
 * Errors: QN_ERR_INVALID_ARG for a null required pointer, a misaligned
 * pointer or a workspace smaller than qn_bin_sort_workspace_size.
 */
int qn_render_bwd(const qn_camera *cam_host, int32_t n, const int32_t *rects, const uint32_t *ranges,
                  const uint32_t *vals, const qn_splat *splats, const float *bg_host, const float *T_final,
                  const uint32_t *last, const float *d_img, const uint8_t *skip, const uint8_t *composited,
                  const uint32_t *tile_order, void *workspace, size_t workspace_bytes, qn_splat *pair_scratch,
                  qn_splat *d_splats, qn_stream_t stream);

/*
 * The two passes of qn_render_bwd as separate calls (for stage timing);
 * qn_render_bwd_pairs followed by qn_render_bwd_gather with the same
 * arguments is qn_render_bwd.  The first writes pair_scratch and the
 * visited prefix of every tile into the workspace; the second reads them.
 */
int qn_render_bwd_pairs(const qn_camera *cam_host, int32_t n, const uint32_t *ranges, const uint32_t *vals,
                        const qn_splat *splats, const float *bg_host, const float *T_final, const uint32_t *last,
                        const float *d_img, const uint8_t *skip, const uint8_t *composited,
                        const uint32_t *tile_order, void *workspace, size_t workspace_bytes, qn_splat *pair_scratch,
                        qn_stream_t stream);
int qn_render_bwd_gather(const qn_camera *cam_host, int32_t n, const int32_t *rects, const uint8_t *skip,
                         const void *workspace, size_t workspace_bytes, const qn_splat *pair_scratch,
                         qn_splat *d_splats, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Loss and optimiser steps of the training iteration (Eq. 3, Eq. 11).       */
/* ------------------------------------------------------------------------ */

/*
 * L1 term of Eq. 3 over count values, weighted by w:
 *   loss[0] = w mean |img - target|, d_img = w sign(img - target) / count
 * (both written; sign(0) = 0).  With mse != 0 the squared error is used
 * instead (loss[0] = w mean (img - target)^2, d_img = 2 w (img - target) / count),
 * the loss of Eq. 9.  img, target, d_img: count floats.  partials
 * [QN_LOSS_BLOCKS] f32: scratch for per-block sums, added in block order (the
 * loss is reproducible bit for bit).
 */
int qn_image_loss(int64_t count, const float *img, const float *target, float w, int32_t mse,
                  float *loss, float *d_img, float *partials, qn_stream_t stream);

/*
 * Adam (Kingma & Ba) on `rows` planes of n elements with stride `stride`:
 *   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * skip (nullable, [n] u8): columns with skip != 0 keep param, m and v.
 * param_bf16 (nullable): also writes the updated values rounded to bf16
 * (round to nearest even), stride as param.
 */
int qn_adam(int32_t rows, int32_t n, int32_t stride, float *param, const float *grad, float *m,
            float *v, int32_t step, float lr, float beta1, float beta2, float eps,
            const uint8_t *skip, uint16_t *param_bf16, qn_stream_t stream);

#define QN_ADAM_MAX_GROUPS 16

/* One parameter group of qn_adam_groups: `rows` planes of n elements with
 * stride `stride` (device pointers; param_bf16 nullable as in qn_adam), its
 * learning rate, and whether the skip mask applies (use_skip != 0). */
typedef struct {
    float *param;
    const float *grad;
    float *m;
    float *v;
    uint16_t *param_bf16;
    int32_t rows, n, stride;
    float lr;
    int32_t use_skip;
} qn_adam_group;

/*
 * One Adam step (as qn_adam) over n_groups <= QN_ADAM_MAX_GROUPS parameter
 * groups in a single launch, with the step count on the device: *step
 * (device int32) is incremented first and the bias corrections use the new
 * value, so repeated calls -- also replays of a captured CUDA graph -- count
 * steps without the host.  groups_host is read during the call only.
 * skip ([n] u8, nullable) applies to the groups with use_skip.
 */
int qn_adam_groups(int32_t n_groups, const qn_adam_group *groups_host, int32_t *step, float beta1, float beta2,
                   float eps, const uint8_t *skip, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Viewspace gradient difference and gate initialisation -- Sec. 3.3.        */
/* ------------------------------------------------------------------------ */

/*
 * Eq. 9: score[0..1][i] += scale * (d mean2d x, d mean2d y) of d_splats[i].
 * With d_splats the compositing adjoint of the upstream image
 * 2 (I_{t-1} - I_t) / (3 H W) at the rendering of A_{t-1} (qn_image_loss with
 * mse, then qn_render_bwd) and scale = 1 / V, summing over the V views gives
 * d_t: the MSE is linear in the target, so this single adjoint per view equals
 * the difference of the two gradients Eq. 9 writes.
 *   score [2][n_stride] f32 (read-modify-write; zero it before the first view)
 */
int qn_viewspace_accum(int32_t n, int32_t n_stride, const qn_splat *d_splats, float scale, float *score,
                       qn_stream_t stream);

/*
 * Eq. 10 and Eq. 8 solved for log alpha:
 *   norms[i] = |d_t,i|, median[0] = lower median of the norms (element
 *   (m-1)/2 of the m sorted values); with nonzero_median != 0 only the m
 *   non-zero norms count (median 0 if none), so that Gaussians no view sees do
 *   not pull the median to 0.  p_i = norms_i / (norms_i + median) (1 or 0 for
 *   a zero median), clamped to [1e-6, 1 - 1e-6];
 *   log_alpha[i] = log(p_i / (1 - p_i)) + tau log(-gamma0 / gamma1), so that
 *   sigmoid(log_alpha_i - tau log(-gamma0/gamma1)) = p_i.
 *   score [2][n_stride] (read); norms [n], median [1], log_alpha [n] (written).
 */
int qn_gate_init(int32_t n, int32_t n_stride, const float *score, const qn_gate_params *gate_host,
                 int32_t nonzero_median, float *norms, float *median, float *log_alpha, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Learned static-skip MLP.  Not part of the paper: a per-Gaussian classifier */
/* trained on the gates that earlier frames of the method produce, whose      */
/* "static" predictions let the adjoints and the Adam step skip Gaussians.   */
/* ------------------------------------------------------------------------ */

#define QN_MLP_FEATURES 16
#define QN_MLP_PARAMS 5313   /* W1[64][16] b1[64] W2[64][64] b2[64] W3[64] b3 */

/*
 * Features X [16][n_stride] f32 (written) of each Gaussian:
 *   0 p_i of Eq. 10 (|d| / (|d| + median); 1 or 0 for a zero median)
 *   1 clip(log(|d| / median + 1e-6), -8, 8) / 4 (0 for a zero median)
 *   2, 3 direction d / (|d| + 1e-20) of the score d_t (Eq. 9)
 *   4-6 position of A_{t-1};  7 previous gate g_{t-1} (0 if prev_gate is NULL)
 *   8 sigmoid(log_alpha_{t-1} - tau log(-gamma0/gamma1)) (Eq. 8; log_alpha 0 if NULL)
 *   9 opacity;  10-12 (log-scale + 3) / 2
 *   13 clip(100 |g_{t-1} lp_{t-1}|, 0, 8) (0 if prev_lp is NULL)
 *   14 the previous frame's label of qn_skip_labels (prev_static != 0), or
 *      [g_{t-1} == 0] when prev_static is NULL;  15 1
 *   score [2][n_stride], median [1] (from qn_gate_init), prev [n_attr][n_stride],
 *   prev_gate [n], prev_log_alpha [n], prev_lp [3][n_stride], prev_static [n] u8
 *   (last four nullable).
 */
int qn_skip_features(int32_t n, int32_t n_stride, int32_t n_attr, const float *score, const float *median,
                     const float *prev, const float *prev_gate, const float *prev_log_alpha,
                     const float *prev_lp, const uint8_t *prev_static, const qn_gate_params *gate_host,
                     float *X, qn_stream_t stream);

/*
 * logit = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per Gaussian, with the
 * parameters in bf16 (params, QN_MLP_PARAMS values) and FP32 accumulation.
 * logits [n] (nullable) and skip [n] u8 = [sigmoid(logit) > threshold]
 * (nullable; one of the two required).  threshold in (0, 1).
 */
int qn_skip_mlp_fwd(int32_t n, int32_t n_stride, const float *X, const uint16_t *params, float threshold,
                    float *logits, uint8_t *skip, qn_stream_t stream);

/*
 * Training labels: labels[i] = 1 (static) when Gaussian i's residual of the
 * finished frame is exactly zero -- gate[i] == 0 and every latent of
 * lat [n_latent][n_stride] rounds to 0 -- and, with hit [n] u8 (nullable),
 * hit[i] == 0: no pixel composited it during the frame (qn_or_marks over the
 * iterations' qn_render_fwd composited marks), so it received no image
 * gradient; else 0.
 */
int qn_skip_labels(int32_t n, int32_t n_stride, int32_t n_latent, const float *gate, const float *lat,
                   const uint8_t *hit, uint8_t *labels, qn_stream_t stream);

/* dst[i] |= (src[i] != 0) for i < n (u8 marks): accumulates qn_render_fwd's
 * per-iteration composited marks over a frame. */
int qn_or_marks(int32_t n, const uint8_t *src, uint8_t *dst, qn_stream_t stream);

/* flags[i] = 0 where marks[i] != 0, for i < n (u8): clears the skip flag of
 * every skipped Gaussian that qn_render_fwd found composited, so that the
 * adjoint of the same iteration gives it its gradient and it trains from then
 * on. */
int qn_clear_marked(int32_t n, const uint8_t *marks, uint8_t *flags, qn_stream_t stream);

/*
 * Gradient of the mean binary cross-entropy between sigmoid(logit) and
 * labels [n] u8 (1 = static) over the n rows of X: d_params [QN_MLP_PARAMS]
 * f32 and loss [1] (nullable) are overwritten.  A row range [r0, r0 + n) of a
 * larger X is passed as X + r0 with the same n_stride, labels + r0.
 * partials [QN_MLP_BWD_BLOCKS * (QN_MLP_PARAMS + 1)] f32: scratch for per-block
 * partial sums, added in block order (reproducible).
 */
int qn_skip_mlp_bwd(int32_t n, int32_t n_stride, const float *X, const uint8_t *labels, const uint16_t *params,
                    float *d_params, float *loss, float *partials, qn_stream_t stream);

/*
 * Gate noise for the stochastic hard-concrete sample: u[i] for i < n from
 * Philox4x32-10 (Salmon et al., SC 2011; 10 rounds, multipliers 0xD2511F53,
 * 0xCD9E8D57, key increments 0x9E3779B9, 0xBB67AE85) with counter
 * (i, *step, 0, 0) and key (seed mod 2^32, seed >> 32): the first output
 * word x, as u = ((x >> 9) + 1/2) / 2^23 in (0, 1).  step (device i32) is
 * read on the device, so a captured graph draws fresh noise whenever the
 * step advances (e.g. the Adam step of qn_adam_groups).  u [n] f32.
 */
int qn_gate_uniform(int32_t n, uint64_t seed, const int32_t *step, float *u, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Adaptive masked training -- Sec. 3.3; App. B (t_d = 0.001, 48 x 48).      */
/* ------------------------------------------------------------------------ */

/*
 * rects_out[i] = rects[i] for a dynamic Gaussian, else an empty rect:
 * dynamic when |(ndc_x score[0][i], ndc_y score[1][i])| > t_d, the score
 * being d_t of Eq. 9 in pixel units (qn_viewspace_accum) and ndc_x, ndc_y
 * the factors to the units t_d is stated in (W/2 and H/2 for normalised
 * device coordinates; 1 for pixels).  Binning and compositing with rects_out
 * render the dynamic Gaussians alone.  rects, rects_out [n] int4 (16-byte
 * aligned), score [2][n_stride] f32.
 */
int qn_select_rects(int32_t n, int32_t n_stride, const int32_t *rects, const float *score, float ndc_x,
                    float ndc_y, float t_d, int32_t *rects_out, qn_stream_t stream);

/*
 * The mask of one view from the dynamic-only rendering: a pixel is dynamic
 * when its last contributor is > 0 (last [H][W] u32 of qn_render_fwd; the
 * first Gaussian passing the alpha test always contributes, so these are the
 * pixels some dynamic Gaussian covers with alpha >= 1/255).  Dilated with a
 * k x k box (k even): pixel_mask[y][x] = 1 when a dynamic pixel lies in
 * [x - k/2 + 1, x + k/2] x [y - k/2 + 1, y + k/2].  tile_mask [tiles] u8
 * marks the 16 x 16 tiles holding a masked pixel; *n_masked (device i32) =
 * number of masked pixels.  tmp [H][W] u8 scratch.  All outputs written.
 */
int qn_dilate_mask(int32_t width, int32_t height, const uint32_t *last, int32_t k, uint8_t *tmp,
                   uint8_t *pixel_mask, uint8_t *tile_mask, int32_t *n_masked, qn_stream_t stream);

/*
 * ranges_out[t] = ranges[t] for tiles with tile_mask[t] != 0, else the empty
 * range [ranges[t][0], ranges[t][0]): qn_render_fwd and qn_render_bwd given
 * ranges_out skip the unmasked tiles.
 */
int qn_mask_ranges(int32_t n_tiles, const uint32_t *ranges, const uint8_t *tile_mask, uint32_t *ranges_out,
                   qn_stream_t stream);

/*
 * The loss of qn_image_loss restricted to the masked pixels: over the
 * channels x *n_masked values with pixel_mask[p] != 0 (pixel p of each
 * channel plane of hw pixels), loss[0] = w mean |img - target| (or the mean
 * square with mse != 0); d_img = w sign(img - target) / (channels n_masked)
 * (or 2 w (img - target) / ...) on masked values and 0 elsewhere; both 0 when
 * *n_masked == 0.  n_masked is read on the device (as qn_dilate_mask leaves
 * it), so the call can be captured in a CUDA graph.  partials
 * [QN_LOSS_BLOCKS] f32 scratch, summed in block order.
 */
int qn_masked_image_loss(int64_t hw, int32_t channels, const float *img, const float *target,
                         const uint8_t *pixel_mask, const int32_t *n_masked, float w, int32_t mse, float *loss,
                         float *d_img, float *partials, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* D-SSIM term of Eq. 3 (Sec. 3.1).                                          */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace qn_dssim_loss needs (0 for sizes it rejects). */
size_t qn_dssim_workspace_size(int32_t width, int32_t height, int32_t channels);

/*
 * Adds the D-SSIM term of Eq. 3 with weight w to a loss and its image
 * gradient:  loss[0] += w (1 - mean SSIM),  d_img += w dD-SSIM/d img.
 * SSIM per channel and pixel from the local means, variances and covariance
 * of img and target under an 11 x 11 Gaussian window (sigma 1.5; taps outside
 * the image read zero), C1 = 0.01^2, C2 = 0.03^2 (values in [0, 1]).  With
 * pixel_mask [H][W] u8 and n_masked (device i32, the number of non-zero mask
 * entries, as qn_dilate_mask leaves it) the mean runs over the masked pixels
 * only (the windows still read every pixel) and both additions are 0 when
 * *n_masked == 0; pass both NULL for the whole image.  img, target, d_img
 * [channels][H][W] f32 planes; d_img may not alias img or target; loss and
 * d_img must hold values already (e.g. qn_image_loss's L1 term weighted
 * 1 - w).  workspace: >= qn_dssim_workspace_size bytes, 16-byte aligned.
 * The loss is summed in a fixed order (reproducible).
 */
int qn_dssim_loss(int32_t width, int32_t height, int32_t channels, const float *img, const float *target,
                  const uint8_t *pixel_mask, const int32_t *n_masked, float w, float *loss, float *d_img,
                  void *workspace, size_t workspace_bytes, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Compressed per-frame packet -- Sec. 3.2.1 and App. B (storage).           */
/* ------------------------------------------------------------------------ */

#define QN_PACKET_STREAM_SYMBOLS 8192   /* symbols per independently coded rANS stream */
#define QN_PACKET_SCALE_BITS 12         /* model frequencies sum to 2^12 */

/* Bytes of device workspace qn_pack_frame needs (0 for a bad layout). */
size_t qn_pack_workspace_size(int32_t n, const qn_decoder_layout *layout);
/* Upper bound on the size of a packet for n Gaussians and this layout. */
size_t qn_packet_max_bytes(int32_t n, const qn_decoder_layout *layout);

/*
 * The packet of one frame's residual R_t, written to packet (device) with its
 * size in *packet_bytes (host).  Contents (little-endian):
 *   header: u32 magic 0x46504E51, version 1, n, n_cat, 8192, 12; per category
 *     u32 lat_dim, attr_count, n_streams, payload bytes; per category u16
 *     freq[256]; per category u32 stream_bytes[n_streams];
 *   per category the rANS streams (zero-padded to 4 bytes): the integer
 *     latents (Eq. 5: round half to even, saturate to int8) + 128 of the
 *     category, flattened latent-major (dimension k, then Gaussian i) and
 *     cut into streams of 8192 symbols, each coded on its own under the
 *     category's frequencies (counts quantised to sum 2^12: f = max(1,
 *     floor(count 2^12 / total)); a shortfall goes to the most frequent
 *     symbol, smallest on ties; an excess is taken back in one pass by
 *     decreasing f, then increasing symbol, each giving up to f - 1).  rANS
 *     with a 32-bit state in [2^23, 2^31), byte renormalisation, coding the
 *     symbols last to first; a stream is the final state (4 bytes) followed
 *     by the emitted bytes in reverse order of emission;
 *   per category the decoder's bf16 bits, row-major (zero-padded to 4);
 *   u32 n_coo, u32 index[n_coo] (increasing) of the Gaussians with
 *     gate != 0, f32 lp[3][n_coo] their pre-gated position residuals: the
 *     gate is binarised for storage (taken as 1 where it is not 0).
 * lat [sum lat_dim][n_stride] f32 continuous latents; dec the concatenated
 * bf16 decoder blocks (as for qn_decode_residuals); lp [3][n_stride] f32;
 * gate [n] f32 (qn_decode_residuals' gate output).  workspace (256-byte
 * aligned) >= qn_pack_workspace_size; packet (4-byte aligned) >= the packet's
 * size (qn_packet_max_bytes bounds it; QN_ERR_INVALID_ARG if too small).
 * Synchronises the stream (the frequency tables and the layout are built on
 * the host from device counts).
 */
int qn_pack_frame(int32_t n, int32_t n_stride, const qn_decoder_layout *layout, const float *lat,
                  const uint16_t *dec, const float *lp, const float *gate, void *workspace, size_t workspace_bytes,
                  uint8_t *packet, size_t packet_capacity, size_t *packet_bytes, qn_stream_t stream);

/* Bytes of device workspace qn_unpack_frame needs for a packet of that size. */
size_t qn_unpack_workspace_size(int32_t n, int32_t n_stride, const qn_decoder_layout *layout,
                                size_t packet_bytes);

/*
 * A_t = A_{t-1} + R_t from a packet (host memory): the streams decoded on
 * the GPU into latents, the decoders and the COO position residuals (gate 1
 * on the listed Gaussians, 0 elsewhere) through qn_decode_residuals, so the
 * result is what that call gives for the same integer latents, decoders and
 * binarised gates.  prev, out [n_attr][n_stride] f32 (device).  The header is
 * checked against n and the layout, and the sections against the size;
 * stream bytes read past their end or out-of-range COO indices are detected
 * on the device: QN_ERR_INVALID_ARG ("corrupt packet") in every such case.
 * Synchronises the stream.
 */
int qn_unpack_frame(const uint8_t *packet_host, size_t packet_bytes, int32_t n, int32_t n_stride, int32_t n_attr,
                    const qn_decoder_layout *layout, const float *prev, float *out, void *workspace,
                    size_t workspace_bytes, qn_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Data layout for the learned static skip.                                  */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace qn_partition needs for n flags (0 for n < 0). */
size_t qn_partition_workspace_size(int32_t n);

/*
 * Stable partition of 0..n-1 by flags [n] u8: perm [n] i32 (device) lists
 * the indices with flags == 0 in increasing order, then the others in
 * increasing order; *n_first (device i32) = number of zero flags.
 * Reordering every per-Gaussian plane by perm (qn_gather_columns) puts the
 * skipped Gaussians (flag != 0) in one contiguous run at the end, which is
 * what lets the skip save memory traffic in the adjoint and Adam kernels.
 * workspace: >= qn_partition_workspace_size(n) bytes of device memory.
 */
int qn_partition(int32_t n, const uint8_t *flags, int32_t *perm, int32_t *n_first, void *workspace,
                 size_t workspace_bytes, qn_stream_t stream);

/*
 * dst[r][i] = src[r][perm[i]] for r < rows, i < n; elements of elem_bytes
 * (1, 2, 4 or 8) bytes, row strides in elements.  perm [n] i32 (device) must
 * hold column indices of src (not checked); dst may not alias src.
 */
int qn_gather_columns(int32_t rows, int32_t n, int32_t elem_bytes, const void *src, int64_t src_stride,
                      const int32_t *perm, void *dst, int64_t dst_stride, qn_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* QUEEN_H */
