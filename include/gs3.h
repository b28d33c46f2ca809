/*
 * gs3.h -- C ABI of libgs3, the GB300 (sm_103a) kernels of one Stage-1
 * training step of 3DGStream (arXiv 2403.01444): Neural Transformation Cache
 * query (hash-grid encoding + tiny MLP, Section 4.1), transformation of the
 * previous frame's Gaussians (Section 4.1), EWA projection with SH colour
 * (Section 3.2, Eq. 2-3), tile binning + key sort, front-to-back alpha
 * compositing (Section 3.2, Eq. 4), the L1 + D-SSIM loss (Eq. 6), the
 * hand-written backward of all of them, and Adam (Suppl. A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns a gs_status (0 = GS_OK).  Invalid host arguments
 *    return GS_ERR_INVALID_ARG before anything is launched; a failed launch
 *    returns GS_ERR_CUDA (gs_last_error() gives the message).
 *  - Array arguments are DEVICE pointers owned by the caller (allocated by
 *    e.g. PyTorch).  The library never allocates or frees device memory;
 *    scratch comes from a caller buffer sized by the matching *_workspace_size.
 *    Struct arguments (gs_gaussians, gs_hashgrid, ...) are HOST structs whose
 *    pointer fields are device pointers; they are read before the call returns.
 *  - Every call is asynchronous on the given stream (a cudaStream_t; NULL is
 *    the legacy default stream), takes no host synchronisation, and is safe to
 *    capture in a CUDA graph.  Errors found on the device are written to a
 *    caller-provided device word (d_err) and read at the caller's sync point.
 *  - Layouts are row-major, FP32 unless stated.  N = number of Gaussians,
 *    V = views in one launch, K = (sh_deg + 1)^2.  Images are planar
 *    [V][3][H][W].  Per-(view, Gaussian) arrays are [V][N][...].
 *  - Pixel (x, y) has its centre at (x + 0.5, y + 0.5).  Tiles are 16 x 16.
 */
#ifndef GS3_H
#define GS3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

typedef int gs_status;
enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1,
    GS_ERR_CAPACITY = -2,   /* more tile intersections than the caller's buffers hold */
    GS_ERR_CUDA = -3,
    GS_ERR_TIMEOUT = -4,    /* a bounded device wait gave up */
    GS_ERR_NONFINITE = -5
};

/* element types of typeless (void*) buffers */
enum { GS_F32 = 0, GS_F16 = 1, GS_BF16 = 2, GS_NONE = 3 };

typedef void *gs_stream; /* cudaStream_t */

#define GS_TILE 16
#define GS_MAX_VIEWS 64

/* Gaussian set (Section 3.1, Eq. 1-2).  Device pointers. */
typedef struct {
    const float *mean;          /* [N][3] */
    const float *quat;          /* [N][4] (w, x, y, z); normalised inside the projection */
    const float *scale;         /* [N][3] positive scales (activation applied) */
    const float *opacity_logit; /* [N]; opacity = sigmoid(logit) */
    const float *sh;            /* [N][K][3] SH coefficients, degree sh_deg <= 3 */
    int64_t n;
    int32_t sh_deg;
} gs_gaussians;

/* Pinhole camera (OpenCV frame: +z forward, +y down). Passed as a DEVICE
 * array [V] so that a captured graph reads the current views at replay. */
typedef struct {
    float viewmat[12]; /* world -> camera [R | t], row-major 3x4 */
    float fx, fy, cx, cy;
    int32_t width, height;
    float campos[3];   /* camera centre in world coordinates */
} gs_camera;

/* Per-(view, Gaussian) projected records, device pointers, each [V][N][...]. */
typedef struct {
    float *mean2d;         /* [V][N][2] pixel coordinates */
    float *conic_opacity;  /* [V][N][4] (A, B, C, opacity): inverse 2D covariance [[A,B],[B,C]] */
    float *rgb;            /* [V][N][3] SH colour + 0.5, clamped at 0 */
    float *depth;          /* [V][N] camera-space z */
    int32_t *radius;       /* [V][N] ceil(3 sqrt(lambda_max)); 0 = culled */
    int32_t *tiles_touched;/* [V][N] number of 16x16 tiles in the footprint rectangle */
} gs_projected;

/* Multi-resolution hash grid (Section 4.1; Suppl. A).  Level resolutions
 * N_l = floor(n_min * b^l + 1e-6), b = exp((ln n_max - ln n_min) / (levels - 1)).
 * Level l is a dense (N_l+1)^3 grid when that fits in 2^log2_table entries,
 * else the I-NGP spatial hash.  Coordinates are normalised by the box aabb
 * (min xyz, max xyz) and clamped to it.  Table layout: [entries][features]. */
typedef struct {
    int32_t levels;      /* L <= 16 */
    int32_t features;    /* F == 2 */
    int32_t log2_table;  /* log2 T */
    int32_t n_min, n_max;
    float aabb[6];
} gs_hashgrid;

/* MLP 32 -> 64 -> 64 -> 7, ReLU, no biases (Section 4.1 Eq. 5; Suppl. A).
 * Weights are [out][in] row-major, concatenated W1 | W2 | W3 (6592 values). */
enum { GS_MLP_FP32 = 0, GS_MLP_BF16 = 1 };
typedef struct {
    int32_t precision;   /* GS_MLP_FP32: SIMT FP32; GS_MLP_BF16: tcgen05 BF16 x BF16 -> FP32
                            for the two hidden layers, FP32 output layer (64 -> 7) */
    const float *w_f32;  /* FP32 master weights (device); required for both precisions */
    const void *w_bf16;  /* BF16 copy of the same layout (device), used when precision == BF16 */
} gs_mlp;

#define GS_MLP_IN 32
#define GS_MLP_HIDDEN 64
#define GS_MLP_OUT 7
#define GS_MLP_PARAMS (64 * 32 + 64 * 64 + 7 * 64)

/* Adam hyper-parameters (Suppl. A: rate 0.002).  The update with step number
 * t (d_state->step: 0 for the first applied update) uses the rate
 *   lr * lr_final_ratio ^ (min(t, decay_steps - 1) / (decay_steps - 1))
 * when decay_steps > 1, an exponential decay to lr * lr_final_ratio over
 * decay_steps updates (held there after), and lr when decay_steps <= 1.  The
 * rate is derived on the device from the step counter, so a captured CUDA
 * graph follows the schedule. */
typedef struct {
    float lr, beta1, beta2, eps;
    float lr_final_ratio;
    int32_t decay_steps;
} gs_adam;

/* Training state kept in DEVICE memory, read and advanced by the kernels so a
 * whole step needs no host round trip: dynamic loss scale, non-finite flag,
 * number of applied Adam steps, clean steps since the last scale change. */
typedef struct {
    float loss_scale;
    int32_t found_inf;
    int32_t step;
    int32_t clean_steps;
} gs_train_state;

/* ------------------------------------------------------------------ misc */

/* Message of the last failing call in this thread ("" if none). */
GS_API const char *gs_last_error(void);
/* Library version, (major << 16) | minor. */
GS_API int gs_version(void);
/* Number of CUDA kernels this library has launched since it was loaded. */
GS_API uint64_t gs_launch_count(void);
/* Number of tensor-core MLP blocks that gave up a bounded wait on their MMA
 * completion barrier (0 in normal operation; reads device memory, syncs). */
GS_API int gs_tc_timeouts(void);
/* Failure-detection self-test (the paper has no counterpart): one block waits,
 * with the tensor-core kernels' bounded mbarrier wait, on a barrier that
 * nothing arrives on, giving up after `tries` attempts (1 .. 2^20); writes
 * GS_ERR_TIMEOUT to *d_status (device int32) when the wait ran out (always,
 * by construction) and GS_OK otherwise.  The context stays usable. */
GS_API gs_status gs_tc_wait_selftest(uint32_t tries, int32_t *d_status, gs_stream stream);
/* Failure-detection control (the paper has no counterpart): the number of
 * polls after which the tensor-core MLP kernels (ntc_mlp_fwd / ntc_mlp_bwd
 * with BF16 weights, ntc_fused_fwd / ntc_fused_bwd) give up waiting for an
 * MMA batch.  GS_TC_WAIT_TRIES_DEFAULT is the default; 0 makes every such
 * wait give up at once, which tests use to run the timeout path.  A kernel
 * that gives up still waits, bounded by the default, for the MMA batch in
 * flight, releases its tensor memory, counts the event (gs_tc_timeouts) and
 * marks what it did not finish as non-finite: the rows of raw7 (and of the
 * fused forward's transformed mean and rotation) become NaN, the reverse's
 * weight gradient becomes NaN.  A Stage-1 step then skips its Adam update
 * through gs_check_finite, and gs_project culls and reports the Gaussians.
 * Process-wide; applies to kernels launched or captured after the call. */
#define GS_TC_WAIT_TRIES_DEFAULT 4194304u
GS_API gs_status gs_tc_set_wait_limit(uint32_t tries);

/* ------------------------------------------------------------ projection */

/* EWA projection and SH colour of every Gaussian into V views
 * (Section 3.2, Eq. 2-3; colour Section 3.1).  Per (view, Gaussian):
 *   t = R mu + t_w; cull if t_z <= 0.2
 *   Sigma = R(q) diag(s)^2 R(q)^T; J = perspective Jacobian at t with
 *   t_x/t_z, t_y/t_z clamped to 1.3x the half field of view
 *   Sigma2d = J W Sigma W^T J^T + 0.3 I, det(Sigma2d) > 0 for finite input
 *   conic = Sigma2d^-1, its determinant summed from non-negative terms
 *   (Cauchy-Binet on P = J W R(q) diag(s)) so that needles keep FP32 accuracy
 *   radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det))
 *   mean2d = (fx t_x / t_z + cx, fy t_y / t_z + cy)
 *   tile rect x in [floor((u - r)/16), floor((u + r + 15)/16)) clamped to the
 *   image's tiles (same in y); an empty rect culls (radius = tiles_touched = 0)
 *   rgb = max(0, sum_k Y_k(dir) sh_k + 0.5), dir = (mu - campos)/|mu - campos|
 *   opacity = sigmoid(logit)
 * All V views share width W and height H.  Overwrites every field of out.
 * A Gaussian whose mean, rotation, scale or opacity is not finite, or whose
 * record would not be (a non-finite SH coefficient), is culled in every view
 * and, when d_err (device int32, may be NULL) is non-NULL and still 0, sets
 * *d_err = GS_ERR_NONFINITE; the caller reads the word at its sync point. */
GS_API gs_status gs_project(const gs_gaussians *g, const gs_camera *d_cams, int V, int W, int H,
                            const gs_projected *out, int32_t *d_err, gs_stream stream);

/* Reverse of gs_project for mean and rotation (Section 4.1: in Stage 1 only
 * the transformed mean and rotation receive gradients).  grads[V][N][8] holds
 * dL/d(u, v, A, B, C, r, g, b) per (view, Gaussian) as written by
 * gs_raster_bwd.  Overwrites d_mean[N][3] and d_quat[N][4] (gradient wrt the
 * un-normalised input quaternion), summed over the V views. */
GS_API gs_status gs_project_bwd(const gs_gaussians *g, const gs_camera *d_cams, int V, int W, int H,
                         const float *grads, float *d_mean, float *d_quat, gs_stream stream);

/* Reverse of gs_project wrt every parameter, for the Gaussians
 * [first, first + count) of g (Stage 2 of Section 4.2 trains every attribute
 * of the added Gaussians while the transformed ones stay fixed).  grads is
 * gs_raster_bwd's [V][g->n][8] array and d_opacity its [V][g->n] opacity
 * gradient (NULL = 0).  Overwrites, for j < count, d_mean[j][3],
 * d_quat[j][4] (wrt the un-normalised quaternion), d_scale[j][3] (wrt the
 * scales s, not log s), d_opacity_logit[j] (opacity = sigmoid(logit)) and
 * d_sh[j][K][3], summed over the V views.  GS_ERR_INVALID_ARG if the range
 * leaves [0, g->n). */
GS_API gs_status gs_project_bwd_full(const gs_gaussians *g, const gs_camera *d_cams, int V, int W,
                                     int H, const float *grads, const float *d_opacity,
                                     int64_t first, int64_t count, float *d_mean, float *d_quat,
                                     float *d_scale, float *d_opacity_logit, float *d_sh,
                                     gs_stream stream);

/* --------------------------------------------------------- binning + sort */

/* Scratch bytes gs_bin_sort needs for n Gaussians, V views of W x H and room
 * for `capacity` (Gaussian, tile) pairs; 0 for arguments gs_bin_sort rejects
 * (n < 0, V < 1, capacity < 0, n * V >= 2^32 - 1). */
GS_API size_t gs_bin_sort_workspace_size(int64_t n, int V, int W, int H, int64_t capacity);

/* Tile binning and key sort (the tile pipeline of Section 3.2).  Tiles are
 * grouped in bins of bin x bin tiles (bin = 1: one tile per bin).  Every
 * (view, Gaussian, bin touched by its tile rect) pair gets key =
 * (view * bins + bin_id) << 32 | IEEE bits of its FP32 depth and value =
 * Gaussian index, bin_id = (tile_y / bin) * bins_x + tile_x / bin; pairs are
 * ordered by (key, value).  Writes vals[count] (sorted values),
 * ranges[V * bins][2] ([first, last+1) per bin, zeros when empty), *d_count
 * (device int64) and, when keys != NULL, keys[count] (for checking).
 * Bit-exact and deterministic.  With bin > 1 each tile's list is the ordered
 * subsequence of its bin's list whose tile rectangles hold the tile, which the
 * compositing kernels select on the fly (same records, same order).
 * If count > capacity, *d_err is set to GS_ERR_CAPACITY, nothing is written
 * past capacity, and every range is empty; the caller regrows and reruns.
 * ws: scratch of gs_bin_sort_workspace_size bytes, 256-byte aligned. */
GS_API gs_status gs_bin_sort(const gs_projected *proj, int64_t n, int V, int W, int H, int bin,
                      int64_t capacity,
                      uint32_t *vals, uint32_t *ranges, uint64_t *keys, int64_t *d_count,
                      int32_t *d_err, void *ws, size_t ws_bytes, gs_stream stream);

/* gs_bin_sort without a caller workspace, for callers that cannot allocate
 * device memory when they bin (allocators that forbid new device allocations
 * after start-up, render loops that must not stall or fail on an allocation,
 * plug-ins handed only pre-sized buffers).  The paper has no counterpart: it
 * is a deployment variant of gs_bin_sort, with the same arguments, outputs,
 * capacity protocol and bit-exact results, minus ws / ws_bytes.
 * Scratch is a 20 MiB static device array inside the library, held by every
 * GPU that loads it until exit.  Limits: n * V <= 131072, capacity <= 1048576,
 * and gs_bin_sort_workspace_size() of the call <= 20 MiB; larger calls return
 * GS_ERR_INVALID_ARG without launching.  All calls share the array: calls that
 * overlap on the GPU race and must be serialised.  The first call on a device
 * looks up the array's address; make it before any stream capture.  That
 * address is kept for the lifetime of the device's primary context: do not
 * call this function on a device again after cudaDeviceReset.
 * Allocates nothing (no cudaMalloc / cudaFree, no allocating library call). */
GS_API gs_status gs_bin_sort_noalloc(const gs_projected *proj, int64_t n, int V, int W, int H,
                                     int bin, int64_t capacity, uint32_t *vals, uint32_t *ranges,
                                     uint64_t *keys, int64_t *d_count, int32_t *d_err,
                                     gs_stream stream);

/* ------------------------------------------------------------ compositing */

/* The records a compositing forward staged for each tile, in list order (the
 * per-tile lists of Section 3.2 after the footprint tests, up to where the
 * tile's pixels stopped): for tile t of view v (i = v * tiles + t, tiles =
 * ceil(W/16) * ceil(H/16), t = tile_y * ceil(W/16) + tile_x),
 * rec[2 * (i * cap + j)] is the Gaussian index and rec[2 * (i * cap + j) + 1]
 * the position in the bin's list of its j-th staged record, j < count[i];
 * the list ends at the last staged record that some pixel of the tile went
 * through before it stopped (the records after it took part at no pixel);
 * count[i] = -1 when that is more than cap records.  Device memory
 * owned by the caller: rec uint32[V * tiles * cap * 2] (8-byte aligned),
 * count int32[V * tiles]; 1 <= cap <= 2^20. */
typedef struct {
    uint32_t *rec;
    int32_t *count;
    int32_t cap;
} gs_tile_lists;

/* Front-to-back alpha compositing (Section 3.2, Eq. 4), one 16x16 tile per
 * block.  Per pixel, over its tile's sorted list: power = -(A dx^2 + C dy^2)/2
 * - B dx dy with (dx, dy) = pixel centre - mean2d; skip if power > 0;
 * alpha = min(0.99, opacity exp(power)); skip if alpha < 1/255; stop before a
 * Gaussian that would take T below 1e-4; C += rgb alpha T; T *= 1 - alpha.
 * Writes img[V][3][H][W] = C + T bg, T_final[V][H][W] and last[V][H][W] (1 +
 * position in the bin's list of the last Gaussian added, 0 if none).  vals /
 * ranges are gs_bin_sort's output for the same bin.  A record whose
 * alpha-ellipse cannot reach 1/255 at any pixel centre of a tile (a margin
 * of 0.01 in the quadratic form) is not staged for that tile: every pixel
 * would skip it, so results are unchanged.  d_stats (device uint64[2], or
 * NULL) accumulates the (pixel, Gaussian) pairs evaluated and added.  lists
 * (or NULL) receives each tile's staged records for gs_raster_bwd. */
GS_API gs_status gs_raster_fwd(const gs_projected *proj, int64_t n, int V, int W, int H, int bin,
                        const float *bg, const uint32_t *vals, const uint32_t *ranges, float *img,
                        float *T_final, int32_t *last, uint64_t *d_stats, const gs_tile_lists *lists,
                        gs_stream stream);

/* Reverse of gs_raster_fwd: walks each pixel's list back to front from
 * `last`, recomputing T_i = T_{i+1} / (1 - alpha_i) from T_final (no per-pair
 * state is stored).  Per-(view, Gaussian) gradients are reduced across each
 * warp and each tile before one vector atomic per (Gaussian, tile).
 * Overwrites grads[V][N][8] = dL/d(u, v, A, B, C, r, g, b) and, when non-NULL,
 * d_opacity[V][N].  bg is a host array of 3 floats.  d_stats (device
 * uint64[2], or NULL) accumulates the pairs walked and the pairs that had
 * contributed.  lists (or NULL): written by the gs_raster_fwd call on the same
 * proj, n, V, W, H, bin, vals and ranges; the reverse then stages a tile's
 * records from its list instead of testing its bin's list again (a tile with
 * count -1 is tested as without lists).  Results are the same either way. */
GS_API gs_status gs_raster_bwd(const gs_projected *proj, int64_t n, int V, int W, int H, int bin,
                        const float *bg, const uint32_t *vals, const uint32_t *ranges,
                        const float *T_final, const int32_t *last, const float *d_img,
                        float *grads, float *d_opacity, uint64_t *d_stats,
                        const gs_tile_lists *lists, gs_stream stream);

/* ------------------------------------------------------------------- loss */

GS_API size_t gs_loss_workspace_size(int planes, int H, int W);

/* L = (1 - lambda) mean|I - I*| + lambda (1 - SSIM(I, I*)) (Eq. 6, lambda =
 * 0.2), SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2,
 * C2 = 0.03^2, zero padding, mean over all planes and pixels.  img and target
 * are [planes][H][W].  Writes d_img = dL/dI, *d_loss and, if non-NULL,
 * *d_ssim (device floats). */
GS_API gs_status gs_loss_l1_dssim(const float *img, const float *target, int planes, int H, int W,
                           float lambda, float *d_img, float *d_loss, float *d_ssim, void *ws,
                           size_t ws_bytes, gs_stream stream);

/* ---------------------------------------------------- transformation cache */

/* Number of table entries (rows) of the grid; < 0 on invalid arguments. */
GS_API int64_t ntc_hashgrid_entries(const gs_hashgrid *grid);

/* The order in which the encoding kernels visit the Gaussians, for locality
 * in the table: order[n] = the Gaussians sorted by the Morton code (10 bits
 * an axis) of their mean within the grid's box, ties by index.  Any
 * permutation of 0..n-1 gives the same encodings; this one makes the 32
 * Gaussians of a warp neighbours, so at the coarse levels their corners fall
 * in few table rows.  ws: scratch of ntc_spatial_order_workspace_size(n)
 * bytes, 256-byte aligned; order is device uint32[n]. */
GS_API size_t ntc_spatial_order_workspace_size(int64_t n);
GS_API gs_status ntc_spatial_order(const float *mean, int64_t n, const gs_hashgrid *grid, uint32_t *order,
                                   void *ws, size_t ws_bytes, gs_stream stream);

/* enc[n][L*F] = per level, trilinear interpolation of the 8 corner features
 * around the normalised mean (Section 4.1).  table_dtype: GS_F16 or GS_F32;
 * enc_dtype: GS_F32 or GS_BF16.  order (device uint32[n], or NULL for 0..n-1):
 * a permutation of the Gaussians giving the order of the work (for example
 * ntc_spatial_order's); the results are the same for any. */
GS_API gs_status ntc_encode_fwd(const float *mean, int64_t n, const gs_hashgrid *grid, const void *table,
                         int table_dtype, void *enc, int enc_dtype, const uint32_t *order, gs_stream stream);

/* d_table[entries][F] += trilinear-weighted scatter of d_enc[n][L*F]
 * (FP32 atomics; the caller zeroes d_table between steps -- adam_step does).
 * order: as for ntc_encode_fwd (the sums differ only in the order of the
 * atomic additions).  d_count (device int64, or NULL): only the rows
 * order[0 .. *d_count) are scattered -- a row list such as ntc_active_rows'
 * (needs order). */
GS_API gs_status ntc_encode_bwd(const float *mean, int64_t n, const gs_hashgrid *grid, const float *d_enc,
                         float *d_table, const uint32_t *order, const int64_t *d_count, gs_stream stream);

/* raw7[n][7] = W3 relu(W2 relu(W1 enc)) (Section 4.1 Eq. 5).  enc_dtype
 * GS_F32 or GS_BF16. */
GS_API gs_status ntc_mlp_fwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w, float *raw7,
                      gs_stream stream);

/* Reverse of ntc_mlp_fwd with d_raw7 multiplied by *d_scale (device float;
 * NULL = 1): dW[6592] += sum over rows (FP32), d_enc[n][32] = dL/d enc
 * (written when non-NULL).  rows / d_rows (both or neither): only the rows
 * rows[0 .. *d_rows) are worked on and only their d_enc rows written (a row
 * whose d_raw7 is zero adds nothing to dW and has a zero d_enc);
 * ntc_active_rows gives such a list. */
GS_API gs_status ntc_mlp_bwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w,
                      const float *d_raw7, const float *d_scale, float *dW, float *d_enc,
                      const uint32_t *rows, const int64_t *d_rows, gs_stream stream);

/* The rows of d_raw7[n][7] with a nonzero (or non-finite) value: writes
 * rows[0 .. *d_count) (device uint32[n]) in no particular order and *d_count
 * (device int64). */
GS_API gs_status ntc_active_rows(const float *d_raw7, int64_t n, uint32_t *rows, int64_t *d_count,
                                 gs_stream stream);

/* Transformation (Section 4.1): mean_out = mean + raw7[0:3];
 * quat_out = norm(quat) x norm(raw7[3:7]) (order 0, the paper's product) or
 * norm(raw7[3:7]) x norm(quat) (order 1); Hamilton product, (w, x, y, z);
 * norm(v) = v / max(|v|, 1e-12).  Means outside grid->aabb are not moved and
 * their rotation is only normalised (Suppl. A discards them). */
GS_API gs_status ntc_apply(const float *mean, const float *quat, const float *raw7, int64_t n,
                    const float *aabb, int order, float *mean_out, float *quat_out,
                    gs_stream stream);

/* Reverse of ntc_apply wrt raw7: overwrites d_raw7[n][7]. */
GS_API gs_status ntc_apply_bwd(const float *mean, const float *quat, const float *raw7, int64_t n,
                        const float *aabb, int order, const float *d_mean_out,
                        const float *d_quat_out, float *d_raw7, gs_stream stream);

/* Fused cache forward (Section 4.1, Eq. 5): hash encoding of every mean from
 * the FP16 table, the BF16 tcgen05 MLP and the transformation in one kernel.
 * Same arithmetic as ntc_encode_fwd (FP16 table, BF16 encoding) +
 * ntc_mlp_fwd (GS_MLP_BF16) + ntc_apply.  Writes mean_out[n][3],
 * quat_out[n][4], raw7[n][7] and enc_save (BF16 [n][32], the encodings the
 * backward reads).  w->precision must be GS_MLP_BF16. */
GS_API gs_status ntc_fused_fwd(const float *mean, const float *quat, int64_t n,
                               const gs_hashgrid *grid, const void *table_f16, const gs_mlp *w,
                               int order, float *mean_out, float *quat_out, float *raw7,
                               void *enc_save, gs_stream stream);

/* Fused cache backward: ntc_apply_bwd + ntc_mlp_bwd + ntc_encode_bwd in one
 * kernel, from the gradients wrt the transformed means and rotations.
 * d_raw7 is scaled by *d_scale (device float; NULL = 1) as in ntc_mlp_bwd;
 * dW[6592] and d_table[entries][2] are accumulated (scaled). */
GS_API gs_status ntc_fused_bwd(const float *mean, const float *quat, const float *raw7,
                               const void *enc_save, int64_t n, const gs_hashgrid *grid,
                               const gs_mlp *w, int order, const float *d_mean_out,
                               const float *d_quat_out, const float *d_scale, float *dW,
                               float *d_table, gs_stream stream);

/* Warm-up loss (Section 4.1 Eq. 7): mean over rows of |dmu|_1 - cos^2(norm(dq), (1,0,0,0)).
 * Writes *d_loss (device float) and d_raw7[n][7] = dL/d raw7. */
GS_API gs_status ntc_warmup_loss(const float *raw7, int64_t n, float *d_raw7, float *d_loss,
                          gs_stream stream);

/* ------------------------------------------------------------- optimiser */

/* Sets d_state->found_inf = 1 if any of g[n] is not finite.  g must be
 * 16-byte aligned (GS_ERR_INVALID_ARG otherwise). */
GS_API gs_status gs_check_finite(const float *g, int64_t n, gs_train_state *d_state, gs_stream stream);

/* Bias-corrected Adam (Suppl. A) on p[n] with gradient g * (1 / loss_scale)
 * and step number d_state->step + 1, skipped when d_state->found_inf is set;
 * the rate follows gs_adam's schedule (lr_final_ratio > 0 when decay_steps > 1,
 * GS_ERR_INVALID_ARG otherwise).
 * Zeroes g afterwards (ready for the next step's accumulation).  If shadow is
 * non-NULL, writes the updated parameters converted to shadow_dtype (GS_F16 or
 * GS_BF16).  All state (m, v) FP32, in place.  p, g, m, v 16-byte aligned,
 * shadow 8-byte aligned (GS_ERR_INVALID_ARG otherwise). */
GS_API gs_status adam_step(float *p, float *g, float *m, float *v, int64_t n, const gs_adam *hp,
                    const gs_train_state *d_state, void *shadow, int shadow_dtype,
                    gs_stream stream);

/* End of a step: on a non-finite gradient halve the loss scale and clear the
 * flag; else count the step and double the scale after growth_interval clean
 * steps (growth_interval <= 0 keeps the scale fixed). */
GS_API gs_status gs_train_state_advance(gs_train_state *d_state, int growth_interval, gs_stream stream);

/* SH rotation (Suppl. B): rotates the SH coefficients of n Gaussians whose
 * orientation changed from quat_from to quat_to (both [n][4], w x y z, not
 * necessarily unit; 16-byte aligned), i.e. by the world rotation
 * Rw = R(quat_to) R(quat_from)^T, so that the colour seen from direction d
 * afterwards is the colour seen from Rw^T d before.  Each band l >= 1 is
 * multiplied by M_l = [P_l(Rw N_k)]_k A_l^-1 over 2l + 1 fixed directions N_k
 * (the coordinate axes for band 1); band 0 is copied.  sh_in, sh_out
 * [n][K][3] (K = (sh_deg + 1)^2) may be the same array. */
GS_API gs_status gs_sh_rotate(const float *quat_from, const float *quat_to, const float *sh_in,
                              int64_t n, int sh_deg, float *sh_out, gs_stream stream);

/* ----------------------------------------- Stage 2: adaptive 3DG addition */

/* The added, frame-specific Gaussians of Stage 2 (Section 4.2) as rows of
 * their trainable parameters, row = [mean 3 | quat 4 | log scale 3 |
 * opacity logit 1 | SH K x 3] (GS_ADDED_COLS(K) floats, K = (sh_deg + 1)^2),
 * with their Adam moments in the same layout.  All device arrays of
 * capacity rows, owned by the caller. */
#define GS_ADDED_COLS(K) (11 + 3 * (K))
typedef struct {
    float *rows;
    float *m, *v;
    int64_t capacity;
    int32_t sh_deg;
} gs_added;

/* View-space positional gradient statistics (Section 4.2, after 3DG-S): for
 * j < count and each view v where record (v, first + j) is visible
 * (radius > 0), accum[j] += grad_scale * |(dL/du * W / 2, dL/dv * H / 2)|
 * (the gradient wrt the normalised device coordinates of the 2D mean) and
 * denom[j] += 1.  grads [V][n][8] and radius [V][n] as written by
 * gs_raster_bwd / gs_project for n Gaussians. */
GS_API gs_status gs_viewspace_grad_accum(const float *grads, const int32_t *radius, int V, int64_t n,
                                         int64_t first, int64_t count, int W, int H,
                                         float grad_scale, float *accum, int32_t *denom,
                                         gs_stream stream);

/* idx[0 .. *d_nsel) = the j < count, in increasing order, with denom[j] > 0
 * and accum[j] / denom[j] > tau (FP32).  One block; no workspace. */
GS_API gs_status gs_select_above(const float *accum, const int32_t *denom, int64_t count, float tau,
                                 int32_t *idx, int64_t *d_nsel, gs_stream stream);

/* Spawn (Section 4.2): for k < *d_nsel, source Gaussian i = idx[k] of src
 * gives the added row *d_nadd + k: mean = mu_i + sqrt(2) R_i diag(s_i) z[k]
 * (a draw from N(mu_i, 2 Sigma_i); z [*d_nsel][3] standard normal draws
 * supplied by the caller), rotation (1, 0, 0, 0), log scale = log s_i,
 * opacity logit = log(opacity_init / (1 - opacity_init)), SH copied.  Rows
 * beyond dst->capacity are dropped and *d_err set to GS_ERR_CAPACITY;
 * *d_nadd becomes min(capacity, *d_nadd + *d_nsel).  Moments of new rows
 * are zeroed. */
GS_API gs_status gs_added_spawn(const gs_gaussians *src, const int32_t *idx, const int64_t *d_nsel,
                                const float *z, float opacity_init, gs_added *dst,
                                int64_t *d_nadd, int32_t *d_err, gs_stream stream);

/* Quantity control at the end of a Stage-2 epoch (Section 4.2): of the n_src
 * rows of src, those with sigmoid(opacity logit) >= tau_opacity are kept, in
 * order (with their moments); then every kept row j with denom[j] > 0 and
 * accum[j] / denom[j] > tau_grad adds, in order, a row with mean =
 * mu_j + R_j diag(s_j) z[j] (a draw from N(mu_j, Sigma_j); z [n_src][3]),
 * log scale + log(split_scale), rotation and SH of row j, opacity
 * opacity_init (as a spawned Gaussian), moments zero.  Writes dst (a
 * different buffer) and *d_ndst; rows beyond dst->capacity are dropped with
 * *d_err = GS_ERR_CAPACITY.  One block. */
GS_API gs_status gs_added_densify_prune(const gs_added *src, int64_t n_src, const float *accum,
                                        const int32_t *denom, float tau_grad, float tau_opacity,
                                        float split_scale, float opacity_init, const float *z,
                                        gs_added *dst, int64_t *d_ndst, int32_t *d_err,
                                        gs_stream stream);

/* Bias-corrected Adam on the n rows of a: gradients from
 * gs_project_bwd_full's arrays (d_scale wrt s is turned into the gradient wrt
 * log s), per-group learning rates lr[6] = {mean, rotation, log scale,
 * opacity logit, SH band 0, SH bands >= 1}, step d_state->step + 1 (loss
 * scale 1; skipped when d_state->found_inf is set); then writes the rendered
 * attributes of each row into out's arrays (mean, quat, scale =
 * exp(log scale), opacity_logit, sh; written through out's pointers) at
 * Gaussian index out_first + row. */
GS_API gs_status gs_added_adam(gs_added *a, int64_t n, const float *d_mean, const float *d_quat,
                               const float *d_scale, const float *d_opacity_logit,
                               const float *d_sh, const float *lr, float beta1, float beta2,
                               float eps, const gs_train_state *d_state, const gs_gaussians *out,
                               int64_t out_first, gs_stream stream);

/* Writes the rendered attributes of rows [0, n) of a into out at Gaussian
 * index out_first + row (as the tail of gs_added_adam). */
GS_API gs_status gs_added_to_render(const gs_added *a, int64_t n, const gs_gaussians *out,
                                    int64_t out_first, gs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GS3_H */
