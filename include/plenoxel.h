/*
 * plenoxel.h -- C ABI of libplenoxel, a CUDA (sm_103a) implementation of the
 * Plenoxels differentiable volume renderer (Yu, Fridovich-Keil et al.,
 * "Plenoxels: Radiance Fields without Neural Networks", arXiv 2112.05131).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns a plx_status.  PLX_OK is 0.  On failure,
 *   plx_last_error() returns a message for the calling thread.  No C++
 *   exception crosses this boundary.
 * - Arguments are validated on the host before anything is launched; a bad
 *   argument returns PLX_EINVAL and launches nothing.
 * - Device pointers ("d_" prefix) are owned by the caller, who allocates and
 *   frees them.  The library never allocates device memory: the derived
 *   structures a grid needs live in a caller-provided workspace whose size
 *   plx_grid_workspace_bytes() returns.  Host pointers ("h_" prefix, or
 *   plain output integers) are only read or written during the call.
 * - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *   void*, NULL = the legacy default stream) unless a call says it
 *   synchronises.  Inputs must stay valid until the stream reaches the work.
 * - Kernels that meet corrupt data (an index volume entry >= n_rows) record
 *   a code in the grid's device status word, skip the access and go on;
 *   plx_check() reports it.  No kernel traps or waits on another kernel.
 *
 * Grid layout (Sec. 3.2; Supp. B.1)
 * ---------------------------------------------------------
 * - The grid is a dense R x R x R lattice of nodes, the voxel corners that
 *   hold the values (Sec. 3).  Node (i,j,k) has linear id
 *   n = (i*R + j)*R + k (k fastest, i along x) and sits at world position
 *   aabb_min + (i,j,k) * h, h = (aabb_max - aabb_min) / (R - 1).
 * - d_idx: int32 [R^3]; -1 marks an empty (NULL) node, otherwise the row of
 *   the node in the data table.  NULL nodes count as all-zero values.
 * - F32 rows: float [n_rows][32] = [sigma, R0..R8, G0..G8, B0..B8, 4 x pad]
 *   (28 values padded to 128 bytes; the pad is never read).  The base
 *   pointer must be 16-byte aligned.
 * - BF16-SH rows: uint16 [n_rows][32] = [sigma as FP32 in slots 0-1,
 *   SH[0..26] as bfloat16 in slots 2..28, 3 x pad] (64 bytes per row).
 *   Density stays FP32; the SH coefficients are rounded to nearest-even
 *   from the F32 rows by plx_pack_bf16().  Compositing and all accumulation
 *   are FP32 in both forms.
 * - Gradient and RMSProp-state rows (d_grad_rows, d_v) use the F32 row
 *   layout [n_rows][32].
 *
 * Rays and rendering (Eq. 1, Sec. 3.1)
 * ------------------------------------
 * - Rays: d_origins, d_dirs float [n][3]; directions must be unit length and
 *   are used as given (no renormalisation); they are also the SH argument.
 * - The ray is clipped to the box [aabb_min, aabb_max] (slab test,
 *   t_near = max(t_in, 0)); samples sit at t_s = t_near + s * delta for
 *   s = 0, 1, ... while t_s < t_far, with delta = step_vox * min_a h_a in
 *   world units, and every sample has delta_s = delta.
 * - Each sample interpolates all 28 values trilinearly from the 8 nodes of
 *   its cell (Sec. 3.3): g = clamp((x - aabb_min)/h, 0, R-1),
 *   base = min(floor(g), R-2), f = g - base.
 * - sigma_s = max(0, interpolated sigma); colour c_ch = max(0, sum_l Y_l(d)
 *   k_{ch,l}) with real degree-2 SH Y_0..Y_8 (Sec. 3.2; ReLU per Supp. B.1).
 * - Compositing: T_0 = 1, alpha_s = 1 - exp(-sigma_s delta), w_s = T_s
 *   alpha_s, T_{s+1} = T_s (1 - alpha_s); before sample s the march stops if
 *   T_s < stop_thresh; C = sum_s w_s c_s + T_end * bg.
 */
#ifndef PLENOXEL_H
#define PLENOXEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLX_OK = 0,
    PLX_EINVAL = 1,       /* invalid argument; nothing was launched            */
    PLX_ENOMEM = 2,       /* a caller-provided buffer is too small             */
    PLX_ECUDA = 3,        /* the CUDA runtime reported an error                */
    PLX_ETIMEOUT = 4,     /* a host-side wait reached its deadline             */
    PLX_EBUSY = 5,        /* the object is in use by another call              */
    PLX_EUNSUPPORTED = 6, /* valid but outside what this build supports        */
    PLX_EDEVICE = 7       /* a kernel recorded corrupt data (see plx_check)    */
} plx_status;

enum { PLX_SH_F32 = 0, PLX_SH_BF16 = 1 };

/* Descriptor of a sparse grid. */
typedef struct {
    int32_t reso;        /* R, nodes per axis, 2 <= R <= 2048                   */
    float aabb_min[3];   /* world box; aabb_max > aabb_min on every axis        */
    float aabb_max[3];
    int64_t n_rows;      /* number of occupied nodes (rows), 0 <= n_rows < 2^31 */
    int32_t sh_form;     /* which rows the renderer reads: PLX_SH_F32/PLX_SH_BF16 */
} plx_grid_desc;

/* Rendering options. */
typedef struct {
    float step_vox;      /* sample spacing in units of the smallest cell size (> 0) */
    float bg[3];         /* background colour composited with T_end            */
    float stop_thresh;   /* early termination threshold on T (0 = march to t_far) */
} plx_render_opts;

/* Opaque grid handle: the descriptor plus caller-owned device pointers. */
typedef struct plx_grid plx_grid;

/* ---------------------------------------------------------------- status */

const char *plx_status_str(plx_status s);
/* Message of the last failing call on this thread ("" if none). */
const char *plx_last_error(void);
/* Library version string. */
const char *plx_version(void);

/* ---------------------------------------------------------------- grid */

/* Bytes of device workspace a grid with this descriptor needs (device status
 * word, the per-cell occupancy bitmask of R^3 bits used for empty-space
 * skipping, and the per-row "touched" bitmask that the sparse RMSProp reads).
 * Returns 0 for an invalid descriptor. */
size_t plx_grid_workspace_bytes(const plx_grid_desc *desc);

/* Create a grid handle over caller-owned buffers and build its derived
 * structures into d_workspace (asynchronously on `stream`).
 *   d_idx        int32 [R^3] index volume (read-only to the library)
 *   d_rows_f32   F32 rows [n_rows][32]; required for PLX_SH_F32, and for any
 *                call that reads or updates the master values (TV, RMSProp,
 *                prune, upsample, plx_pack_bf16); may be NULL for a
 *                render-only BF16 grid
 *   d_rows_bf16  BF16-SH rows [n_rows][32] uint16; required for PLX_SH_BF16,
 *                must be NULL for PLX_SH_F32
 *   d_workspace  plx_grid_workspace_bytes(desc) bytes, 256-byte aligned,
 *                owned by the caller and reserved for this grid until destroy
 * The handle itself is host memory freed by plx_grid_destroy. */
plx_status plx_grid_create(const plx_grid_desc *desc, const int32_t *d_idx, float *d_rows_f32,
                           uint16_t *d_rows_bf16, void *d_workspace, void *stream,
                           plx_grid **out);
plx_status plx_grid_destroy(plx_grid *grid);
/* Copy the descriptor of a grid. */
plx_status plx_grid_get_desc(const plx_grid *grid, plx_grid_desc *out);

/* Round the SH of every F32 row to bfloat16 (nearest-even) into the BF16-SH
 * rows, copying density as FP32 (the storage form of the grid's BF16 rows). */
plx_status plx_pack_bf16(plx_grid *grid, void *stream);

/* Synchronise `stream`, then read and clear the grid's device status word.
 * Returns PLX_EDEVICE if a kernel recorded corrupt data since the last check. */
plx_status plx_check(const plx_grid *grid, void *stream);

/* ---------------------------------------------------------------- rays */

/* Pinhole rays through pixel centres (Sec. 4.1; the centred-pixel convention
 * of Supp. D), camera looking down -z with y up.
 *   d_cams   float [n_cams][18] = c2w (3x4 row-major), fx, fy, cx, cy, W, H;
 *            all cameras share W and H
 *   d_pix    int64 [n] pixel ids view*H*W + v*W + u, 0 <= id < n_cams*W*H
 *   d_origins, d_dirs  float [n][3] outputs
 * W, H     the shared image size (must equal the cameras' W and H entries)
 * With pixel centre (u+0.5, v+0.5): d = normalise(R (((u+0.5)-cx)/fx,
 * -((v+0.5)-cy)/fy, -1)), o = camera centre.  d is evaluated in double-float
 * arithmetic and rounded once, i.e. it is the FP32 rounding of the exact
 * direction except within ~1e-14 of a rounding midpoint.  An id outside
 * [0, n_cams*W*H) yields a zero origin and direction. */
plx_status plx_gen_rays(const float *d_cams, int32_t n_cams, int32_t W, int32_t H,
                        const int64_t *d_pix, int64_t n, float *d_origins, float *d_dirs,
                        void *stream);

/* ---------------------------------------------------------------- render */

/* Forward render of n rays (Eq. 1) into d_rgb float [n][3] and, if d_T_end is
 * not NULL, the final transmittance float [n].  Reads the grid's F32 or
 * BF16-SH rows according to its sh_form. */
plx_status plx_render(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                      const plx_render_opts *opts, float *d_rgb, float *d_T_end, void *stream);

/* Adjoint of plx_render (Sec. 3.5: the renderer is differentiated end to end;
 * Supp. B.1, on its gradient kernels).  d_grad_rgb float [n][3] = dL/dC.  Adds
 * dL/d(row values) into d_grad_rows F32 [n_rows][32] (+=; padding columns
 * untouched) and marks the rows it touches in the grid's touched bitmask.
 * The march is recomputed (no per-sample state is stored).  Per sample:
 *   dL/dc_ch = g_ch w_s;  dL/dk_{ch,l} = dL/dc_ch [pre_ch > 0] Y_l;
 *   dL/dsigma_s = delta sum_ch g_ch (T_{s+1} c_ch - R_ch) [sigma_pre > 0],
 *   R = sum_{j>s} w_j c_j + T_end bg,
 * scattered to the 8 corners with their trilinear weights (NULL corners skip).
 * Rows are accumulated with float atomics, so the summation order (and the
 * last bits) can vary between runs.
 * lambda_sparsity (>= 0, finite) adds the Cauchy sparsity prior of Sec. 3.7
 * (Eq. 4), lambda_sparsity sum log(1 + 2 sigma_s^2) over every sample the
 * rays take (sigma_s the activated density): its density gradient
 * lambda_sparsity 4 sigma_s / (1 + 2 sigma_s^2) joins dL/dsigma_s above, and
 * its value is added to *d_loss_sparsity (device float, may be NULL; one
 * atomic per 32 samples).  0 leaves the prior out. */
plx_status plx_render_backward(const plx_grid *grid, const float *d_origins, const float *d_dirs,
                               int64_t n, const plx_render_opts *opts, const float *d_grad_rgb,
                               float *d_grad_rows, float lambda_sparsity, float *d_loss_sparsity,
                               void *stream);

/* ---------------------------------------------------------------- training march
 *
 * The forward/adjoint pair of the optimisation step (Sec. 3.5; Supp. B.1:
 * batches of 5000 rays), computing exactly what plx_render and
 * plx_render_backward compute (up to FP32 summation order), but splitting
 * every ray into chunks of 32 compacted samples that run as independent work
 * items, so that the few rays with hundreds of non-empty samples do not set
 * the time of a small batch.  plx_render_train leaves a march state in a
 * caller buffer (per chunk: where its samples start, its transmittance before
 * it and the colour that arrives after it); plx_render_backward_train reads it
 * instead of re-marching the rays.
 *
 * With stop_thresh > 0 both calls use the one-warp-per-ray kernels of
 * plx_render / plx_render_backward (the state then only records that). */

/* Bytes of march state for n rays on this grid with these options (0 for
 * invalid arguments or n >= 2^31).  The layout is private to the library. */
size_t plx_march_state_bytes(const plx_grid *grid, int64_t n, const plx_render_opts *opts);

/* As plx_render, and writes the march state of these rays into d_state
 * (device, 16-byte aligned, at least plx_march_state_bytes(grid, n, opts)
 * bytes, caller-owned).  Requires n x (chunks per ray) < 2^31, where chunks
 * per ray = ceil((longest chord / delta + 2) / 32) + 1. */
plx_status plx_render_train(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                            const plx_render_opts *opts, float *d_rgb, float *d_T_end, void *d_state,
                            size_t state_bytes, void *stream);

/* plx_render_train in two calls: plx_march_plan writes the plan of these rays
 * into d_state (reading only the index volume and the occupancy mask, never
 * the rows, so it may run concurrently with calls that change rows, such as
 * plx_rmsprop_step); plx_render_planned then marches the planned chunks and
 * writes the colours.  plx_render_planned checks on the device that d_state
 * holds a plan of these rays, this grid and these options; otherwise it writes
 * nothing and plx_check then returns PLX_EDEVICE. */
plx_status plx_march_plan(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                          const plx_render_opts *opts, void *d_state, size_t state_bytes, void *stream);
plx_status plx_render_planned(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                              const plx_render_opts *opts, float *d_rgb, float *d_T_end, void *d_state,
                              size_t state_bytes, void *stream);

/* plx_render_planned followed by plx_mse_grad in the same kernel (Sec. 3.5: the
 * reconstruction loss of the batch): writes the colours d_rgb, the gradient
 * d_grad_rgb = 2 (C - target) / n and adds L = sum |C - target|^2 / n to
 * *d_loss (if not NULL).  d_target float [n][3]; d_grad_rgb may alias neither
 * d_rgb nor d_target. */
plx_status plx_render_planned_mse(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                                  const plx_render_opts *opts, const float *d_target, float *d_rgb,
                                  float *d_grad_rgb, float *d_loss, void *d_state, size_t state_bytes, void *stream);

/* As plx_render_backward, for the rays, grid and options of the last
 * plx_render_train (or plx_render_planned) that used d_state, enqueued after
 * it, before the grid's rows change.  The kernel checks the state's header (ray buffers, grid rows,
 * sizes, options) on the device; on a mismatch it adds nothing and plx_check
 * then returns PLX_EDEVICE.  lambda_sparsity and d_loss_sparsity: the Cauchy
 * sparsity prior, as in plx_render_backward. */
plx_status plx_render_backward_train(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                                     const plx_render_opts *opts, const float *d_grad_rgb, const void *d_state,
                                     size_t state_bytes, float *d_grad_rows, float lambda_sparsity,
                                     float *d_loss_sparsity, void *stream);

/* ---------------------------------------------------------------- serving
 *
 * Rendering image requests of several resident scenes in one launch (Sec. 3:
 * a trained grid renders novel views directly, with no network).  A request
 * is cut into 16x16-pixel tiles; a launch takes any list of tiles, from any
 * requests and scenes, which lets a scheduler batch requests continuously.
 * Each pixel's ray is generated as plx_gen_rays does and marched as plx_render
 * does, so its colour does not depend on the rest of the launch. */
#define PLX_TILE_W 16
#define PLX_TILE_H 16
#define PLX_TILES_MAX_SCENES 8

typedef struct {
    int32_t scene;   /* index into the call's grids[] */
    int32_t camera;  /* index into d_cams (float [18] each, the layout of plx_gen_rays) */
    int32_t x0, y0;  /* top-left pixel of the tile */
    int32_t W, H;    /* size of the request's image; the tile's pixels outside it are skipped */
    float *d_rgb;    /* the request's image, float [H][W][3] row-major, device, caller-owned */
} plx_tile;

/* Renders n_tiles tiles (d_tiles: device array) with the background and
 * step of *opts.  grids: host array of 1..PLX_TILES_MAX_SCENES grid handles,
 * all of the same sh_form, each with the rows its form renders from.  A tile
 * whose scene or camera index is out of range, or whose d_rgb is NULL, is
 * skipped and recorded in grids[0]'s status (plx_check on grids[0] then
 * returns PLX_EDEVICE).  Tiles must not overlap. */
plx_status plx_render_tiles(const plx_grid *const *grids, int32_t n_grids, const float *d_cams, int32_t n_cams,
                            const plx_tile *d_tiles, int64_t n_tiles, const plx_render_opts *opts, void *stream);

/* Traffic accounting (a measurement aid, not part of the method): for each
 * ray, d_counts int64 [n][3] receives (a) the number of distinct lattice
 * nodes that are corners of the ray's sampled cells having at least one
 * occupied corner, (b) how many of those nodes are occupied, and (c) how many
 * samples are marched (those in such cells), following the same samples and
 * early termination as plx_render.  (a) x 4 bytes of index reads plus (b) x
 * row bytes is the least a forward march must move. */
plx_status plx_count_nodes(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                           const plx_render_opts *opts, int64_t *d_counts, void *stream);

/* Key of the weight-threshold prune (Sec. 3.4 "Coarse to Fine": a voxel is
 * dropped when its weight T_s (1 - exp(-sigma_s delta)) is small on every
 * training ray).  Marches the n rays exactly as plx_render and, for every
 * taken sample with a positive weight, raises d_wmax[r] to that weight for
 * each occupied corner node (row r) of the sample's cell -- all 8 corners,
 * whatever their trilinear weights.
 *   d_origins, d_dirs  float [n][3] device
 *   d_wmax             float [M] device, updated in place (max); it must hold
 *                      non-negative values (zeros to start), and calls over
 *                      further rays continue the maximum
 * Either SH form (the density is what matters).  Stream-ordered; nothing is
 * allocated. */
plx_status plx_max_weight(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                          const plx_render_opts *opts, float *d_wmax, void *stream);

/* Reconstruction loss of a ray batch (Sec. 3.5, the MSE term of the loss):
 *   L = 1/n sum_r ||C_r - Chat_r||^2  and  dL/dChat_r = 2 (Chat_r - C_r) / n.
 *   d_rgb, d_target  float [n][3]: rendered and target colours
 *   d_grad_rgb       float [n][3] output (may alias neither input)
 *   d_loss           float [1] or NULL: L is added to it (atomically) */
plx_status plx_mse_grad(const float *d_rgb, const float *d_target, int64_t n, float *d_grad_rgb, float *d_loss,
                        void *stream);

/* ---------------------------------------------------------------- regulariser / optimiser */

/* Total-variation gradient (Sec. 3.5 loss; Supp. B.1: stochastic contiguous
 * segments, differences scaled by R/256, missing density neighbour = 0,
 * missing SH neighbour = own value).  For each selected node v (empty nodes
 * may be selected) and value d:
 *   D_a = (V_d(v + e_a) - V_d(v)) * R/256,  t = sqrt(D_x^2 + D_y^2 + D_z^2),
 *   L += lambda_d / n_selected * t,
 * lambda_0 = lambda_sigma, lambda_{d>0} = lambda_sh; t = 0 gives no gradient.
 *   d_seg_start, d_seg_len  int64 [n_seg]: runs of linear node ids, each
 *                           inside [0, R^3); runs must not overlap
 *   n_selected              sum of d_seg_len (the host knows it)
 *   d_grad_rows             F32 [n_rows][32], += (occupied rows only; marks them touched)
 *   d_loss                  float [1] or NULL: L is added to it (atomically)
 * Reads the F32 rows (d_rows_f32 must be set). */
plx_status plx_tv_grad(const plx_grid *grid, const int64_t *d_seg_start, const int64_t *d_seg_len,
                       int64_t n_seg, int64_t n_selected, float lambda_sigma, float lambda_sh,
                       float *d_grad_rows, float *d_loss, void *stream);

/* RMSProp (Sec. 3.5) on every entry with a non-zero gradient:
 *   v <- beta v + (1 - beta) g^2;  x <- x - lr g / (sqrt(v) + eps);  g <- 0,
 * lr = lr_sigma for the density column, lr_sh for the SH columns.  Entries
 * with g == 0 keep x and v unchanged.  Updates the F32 rows in place and,
 * for a BF16-SH grid, re-packs the updated rows.
 *   sparse = 0: sweep every row.
 *   sparse = 1: visit only rows marked in the grid's touched bitmask (by
 *               plx_render_backward / plx_tv_grad since the last step), which
 *               is exact whenever every non-zero gradient came from those calls.
 * Both modes clear the touched bitmask.  Successive calls on one grid must be
 * ordered on the device (one stream, or events between streams): a sparse
 * call builds its row list in the grid's workspace and resets the list
 * length that the grid's next sparse call uses. */
plx_status plx_rmsprop_step(plx_grid *grid, float *d_grad_rows, float *d_v, float lr_sigma,
                            float lr_sh, float beta, float eps, int32_t sparse, void *stream);

/* Gradient sparsity (Sec. 3.8 and its figure: after the first minutes of
 * optimisation few voxels receive a gradient): writes to *d_count (device
 * int64) the number of rows marked in the grid's touched bitmask, i.e. the
 * rows that the adjoints and TV have added to since the last
 * plx_rmsprop_step -- call it before that step.  One small launch; reads
 * n_rows / 8 bytes. */
plx_status plx_count_touched(const plx_grid *grid, int64_t *d_count, void *stream);

/* ---------------------------------------------------------------- prune / upsample */

/* Density-threshold pruning with dilation (Sec. 3.4 "Coarse to Fine"):
 * hot(n) = occupied and sigma >= tau; a node is kept if it is occupied and
 * (dilate ? some node of its 3x3x3 neighbourhood, clipped to the grid, is hot
 * : it is hot).  Kept nodes get new rows in ascending node id.
 * Two phases around one caller allocation:
 *   plx_grid_prune_count  computes the keep map into d_ws
 *                         (plx_prune_workspace_bytes(R) bytes, 256-aligned),
 *                         synchronises `stream` and returns the count
 *   plx_grid_prune_apply  writes d_idx_new int32 [R^3] and d_rows_new F32
 *                         [n_keep][32] (NULL allowed when n_keep is 0); d_ws
 *                         must still hold the count's result and n_keep must
 *                         be the count it returned (rows beyond it are never
 *                         written; a mismatch is recorded for plx_check) */
size_t plx_prune_workspace_bytes(int32_t reso);
plx_status plx_grid_prune_count(const plx_grid *grid, float tau, int32_t dilate, void *d_ws,
                                int64_t *n_keep, void *stream);
plx_status plx_grid_prune_apply(const plx_grid *grid, const void *d_ws, int64_t n_keep, int32_t *d_idx_new,
                                float *d_rows_new, void *stream);

/* Weight-threshold pruning (Sec. 3.4 "Coarse to Fine"; the paper's synthetic
 * and 360-degree scenes use it): as plx_grid_prune_count, but hot(n) =
 * occupied and d_key[row of n] >= tau, with d_key float [M] on the device
 * (normally the rows' maximum weights from plx_max_weight; the paper's
 * synthetic threshold is 0.256).  Follow it with plx_grid_prune_apply. */
plx_status plx_grid_prune_count_key(const plx_grid *grid, const float *d_key, float tau, int32_t dilate, void *d_ws,
                                    int64_t *n_keep, void *stream);

/* Trilinear resampling to a new resolution (Sec. 3.4: subdivide and
 * initialise by trilinear interpolation; any resolution).  New node i' along
 * an axis sits at old grid coordinate i'(R-1)/(R'-1): base = floor of it
 * (integer division), rem = i'(R-1) mod (R'-1), frac = rem/(R'-1); the +1
 * node has weight frac and takes part only if rem != 0.  A new node is
 * occupied iff one of its taking-part old nodes is; values interpolate with
 * NULL = 0.  Two phases as for pruning, with
 * plx_upsample_workspace_bytes(R') bytes of d_ws; n_rows_new is the count
 * plx_grid_upsample_count returned. */
size_t plx_upsample_workspace_bytes(int32_t new_reso);
plx_status plx_grid_upsample_count(const plx_grid *grid, int32_t new_reso, void *d_ws,
                                   int64_t *n_rows_new, void *stream);
plx_status plx_grid_upsample_apply(const plx_grid *grid, int32_t new_reso, const void *d_ws, int64_t n_rows_new,
                                   int32_t *d_idx_new, float *d_rows_new, void *stream);

/* ---------------------------------------------------------------- pruning without allocation */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while they run (an embedder with a fixed memory
 * budget and no allocator to lend, or a real-time loop that cannot afford the
 * device-wide synchronisation an allocation may cause).
 *
 * plx_grid_prune_noalloc performs plx_grid_prune_count followed by
 * plx_grid_prune_apply in one call, with the same result, but keeps its scratch
 * in a fixed device array inside the library instead of a caller workspace:
 *   d_idx_new   int32 [R^3] output index volume
 *   d_rows_new  F32 rows output with room for the grid's n_rows rows (pruning
 *               never adds rows); may be NULL only when n_rows is 0
 *   n_keep      host output: the number of rows written
 * It allocates nothing and synchronises `stream` (it needs the count on the
 * host).  Limits and sharing rules of the fixed array:
 *   - grids of at most PLX_PRUNE_NOALLOC_MAX_RESO nodes per axis; larger grids
 *     return PLX_EUNSUPPORTED without launching anything;
 *   - every GPU that loads the library holds PLX_PRUNE_NOALLOC_SCRATCH_BYTES
 *     of device memory for it until the process exits;
 *   - every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing); the first call on a
 *     device may load the library's device code there, so make that first
 *     call before any stream capture;
 *   - all calls share the array, which keeps the last call's contents; calls
 *     whose work overlaps on the GPU (other streams or host threads on the same
 *     device) race on it and must be serialised by the caller. */
#define PLX_PRUNE_NOALLOC_MAX_RESO 256
#define PLX_PRUNE_NOALLOC_SCRATCH_BYTES 4325632 /* the prune workspace of a 256^3 grid */
plx_status plx_grid_prune_noalloc(const plx_grid *grid, float tau, int32_t dilate, int32_t *d_idx_new,
                                  float *d_rows_new, int64_t *n_keep, void *stream);
/* ---------------------------------------------------------------- optimisation step
 *
 * One step of the optimisation (Sec. 3.5; Supp. B.1) in one call: rays for
 * the batch's pixels (plx_gen_rays), plan and forward with the MSE gradient
 * (plx_march_plan, plx_render_planned_mse), adjoint with the Cauchy prior
 * when lambda_sparsity > 0 (plx_render_backward_train), TV on the given
 * segments (plx_tv_grad) and RMSProp (plx_rmsprop_step), ordered on three
 * streams the trainer owns (the march and the plan at the device's highest
 * priority, TV at its lowest).  Each step's RMSProp update is deferred to the
 * start of the next call (or to plx_trainer_finish), beside that batch's
 * plan; TV runs beside the forward and adjoint.  The result equals the serial
 * order of those calls up to the order of FP32 atomic additions.
 *
 * Rays and march state are kept in two sets in a caller workspace; passing
 * the next call's pixel array as d_next_pix has that batch generated and
 * planned during this step's march.  The next call uses that plan when it
 * passes the same d_pix pointer and n with pix_is_ahead = 1, which asserts
 * that the pixel ids there have not changed since; otherwise it plans again.
 *
 * Ordering with the caller's stream: the step starts after the work already
 * enqueued on `stream` and `stream` waits for the step's end (colours, loss,
 * gradient complete) and for the plan of d_next_pix (which has then read the
 * pixel ids).  The deferred update is not included: call plx_trainer_finish
 * before reading rows or v.  On an error the trainer must be destroyed. */
typedef struct plx_trainer plx_trainer;
typedef struct {
    int32_t batch;            /* most rays in one step */
    plx_render_opts opts;     /* stop_thresh > 0 makes the march recompute the adjoint's samples */
    float lambda_tv_sigma;    /* TV weights (Sec. 3.5) */
    float lambda_tv_sh;
    float lambda_sparsity;    /* Cauchy prior weight (Sec. 3.7, Eq. 4); 0: none */
    float beta;               /* RMSProp (Sec. 3.5) */
    float eps;
    int32_t sparse_rmsprop;   /* 1: update only rows marked touched (plx_rmsprop_step) */
    int32_t max_segments;     /* most TV segments of a host-fed step (plx_trainer_step_host); 0: none */
} plx_trainer_desc;

/* Device workspace of a trainer for this grid and descriptor (0 for
 * invalid arguments): two sets of rays and march state, colours and dL/dC. */
size_t plx_trainer_workspace_bytes(const plx_grid *grid, const plx_trainer_desc *desc);

/* d_cams: float [n_cams][18] cameras (plx_gen_rays), images W x H; pixel ids
 * are view*H*W + v*W + u.  d_grad_rows, d_v: F32 [n_rows][32] gradient
 * (zero) and RMSProp state, caller-owned, used by every step.  d_workspace:
 * 256-byte aligned, at least plx_trainer_workspace_bytes bytes. */
plx_status plx_trainer_create(plx_grid *grid, const plx_trainer_desc *desc, const float *d_cams, int32_t n_cams,
                              int32_t W, int32_t H, float *d_grad_rows, float *d_v, void *d_workspace,
                              size_t workspace_bytes, plx_trainer **out);
plx_status plx_trainer_destroy(plx_trainer *trainer);

/* One step on n (<= batch) pixels d_pix int64 [n] with targets d_target
 * float [n][3]; TV on n_seg segments (d_seg_start/d_seg_len int64, n_selected
 * nodes in all; NULL or 0 for none); lr_sigma/lr_sh for this step's update.
 * d_loss (float [1], nullable) accumulates the MSE; d_loss_sparsity (nullable)
 * the Cauchy prior; d_touched (int64 [1], nullable) receives the number of
 * rows with a gradient this step (plx_count_touched, before the update).
 * events: NULL, or 8 CUDA events recorded on the march stream around the
 * stages (update, plan wait, forward, adjoint, TV wait), for timing.
 * set_out (host, nullable) receives the set of rays and state the step used
 * (see plx_trainer_buffers). */
plx_status plx_trainer_step(plx_trainer *trainer, const int64_t *d_pix, int64_t n, const float *d_target,
                            const int64_t *d_seg_start, const int64_t *d_seg_len, int64_t n_seg, int64_t n_selected,
                            float lr_sigma, float lr_sh, const int64_t *d_next_pix, int32_t pix_is_ahead,
                            float *d_loss, float *d_loss_sparsity, int64_t *d_touched, void *const *events,
                            int32_t *set_out, void *stream);

/* A batch in host memory for plx_trainer_step_host: pixel ids int64 [n],
 * targets float [n][3] and TV segments int64 [n_seg] (NULL or n_seg = 0 for
 * none; n_selected nodes in all).  The buffers should be page-locked
 * (cudaHostAlloc or registered) so that the copies are asynchronous; they are
 * the caller's and must stay unchanged until the step that reads them has
 * completed. */
typedef struct {
    const int64_t *pix;
    const float *target;
    const int64_t *seg_start;
    const int64_t *seg_len;
    int64_t n, n_seg, n_selected;
} plx_host_batch;

/* One step of plx_trainer_step fed from host memory, for callers whose
 * batches are produced on the host: the batch's inputs are copied into the
 * trainer's own device buffers (two sets) and the step's MSE is copied back
 * to *h_loss (page-locked; nullable).  With `next` (nullable) the following
 * batch's inputs are copied and planned during this step's march, so that the
 * next call, passing the same host arrays (the same pix pointer and n) as
 * `batch`, starts with them on the device; otherwise its inputs are copied at
 * its start.  The copies run on the trainer's streams beside the march: the
 * next batch's upload before its plan, the loss download once the forward has
 * produced it, beside the adjoint.  n <= batch and n_seg <= max_segments of
 * the descriptor.  `stream` is ordered as for plx_trainer_step and also waits
 * for the loss download, so that *h_loss is complete once `stream` is. */
plx_status plx_trainer_step_host(plx_trainer *trainer, const plx_host_batch *batch, const plx_host_batch *next,
                                 float lr_sigma, float lr_sh, float *h_loss, void *stream);

/* Applies the pending update on `stream`. */
plx_status plx_trainer_finish(plx_trainer *trainer, void *stream);

/* Device buffers of set 0 or 1: rays float [batch][3], the colours of the
 * last step float [batch][3], the march state and its size (any output may
 * be NULL). */
plx_status plx_trainer_buffers(const plx_trainer *trainer, int32_t set, float **d_origins, float **d_dirs,
                               float **d_rgb, void **d_state, size_t *state_bytes);

#ifdef __cplusplus
}
#endif

#endif /* PLENOXEL_H */
