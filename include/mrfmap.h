/*
 * mrfmap.h -- C ABI of the GB300 (sm_103a) ray-MRF occupancy mapper.
 *
 * The library implements the inference path of MRFMap (Shankar & Michael,
 * arXiv 2006.03512): every valid depth pixel becomes a ray factor over the
 * voxels a 3D-DDA walk visits (Section III-A, Eq. 1; Section IV-A), and loopy
 * sum-product belief propagation (Section III-B) runs with the closed-form
 * ray->voxel messages of Eqs. "pos"/"neg" and the voxel->ray cavity messages
 * of Eq. "node_to_factor", giving per-voxel occupancy marginals.
 *
 * Conventions for every entry point:
 *  - Return value: MRF_OK (0) or a negative MRF_E* code.  After a failure the
 *    context is "sticky": later calls return the same code without doing work
 *    until mrf_last_error() has been called, which returns the message and
 *    clears the state.  No C++ exception crosses this boundary.
 *  - "_dev" pointers are CUDA device pointers on the context's device; "_host"
 *    pointers are host memory.  The caller owns every buffer it passes; the
 *    library owns everything it allocates (stream-ordered, on the context's
 *    stream) and frees it in mrf_destroy().
 *  - Work is enqueued on the context's CUDA stream and is asynchronous unless
 *    the entry point says it synchronises.  A device buffer passed in must stay
 *    valid until the work enqueued by that call has completed.
 *  - Voxel (x, y, z) has linear index x + nx * (y + ny * z) ("x fastest"); its
 *    min corner is origin + res * (x, y, z), in metres.
 */
#ifndef MRFMAP_H
#define MRFMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRF_OK 0
#define MRF_EINVAL (-1)   /* an argument is out of range or inconsistent          */
#define MRF_ENOMEM (-2)   /* device or host allocation failed                       */
#define MRF_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed            */
#define MRF_ETIMEOUT (-4) /* a bounded device-side wait gave up                     */
#define MRF_ESTATE (-5)   /* call not valid in the context's current state          */
#define MRF_ERANGE (-6)   /* a size exceeds what the library supports (e.g. >= 2^32 edges) */

#define MRF_PREC_F32 0    /* FP32 messages (default)                                */
#define MRF_PREC_F64 1    /* plain FP64 form: thread per ray, FP64 messages          */
#define MRF_PREC_BF16 2   /* FP32 arithmetic, per-edge messages stored as bf16       */
#define MRF_PREC_F32_LOG 3 /* ablation: the paper's log-domain form in FP32         */

/* mrf_options.variants: the paper implementation's departures from exact BP */
#define MRF_VAR_LENGTH_WEIGHT 1   /* messages weighted by the traversed length       */
#define MRF_VAR_KEYFRAME_AVG 2    /* one average message per (keyframe, voxel)       */

typedef struct mrf_ctx mrf_ctx; /* opaque; created by mrf_create, owned by the library */

/* Dense voxel grid.  nx, ny, nz >= 1 with nx*ny*nz < 2^32; res > 0 metres. */
typedef struct {
    int32_t nx, ny, nz;
    float res;
    float origin[3];
} mrf_grid;

/* Pinhole intrinsics; pixel (u, v) has its centre at integer (u, v); the camera
 * looks along +z with x right and y down (the OpenCV convention). */
typedef struct {
    float fx, fy, cx, cy;
} mrf_intrinsics;

/*
 * Forward sensor model (Eq. "noise"; Section IV-C): the likelihood of the
 * measured range Z given a surface at range d along the ray is
 *     nu(d) = (1 - outlier_w) * N(Z; d + b(d), sigma(d)) + outlier_w / d_hi,
 * with log sigma(d) and b(d) tabulated at the centres d_lo + (k + 1/2) * delta,
 * delta = (d_hi - d_lo) / n_bins, and interpolated linearly (clamped at the
 * ends).  log_sigma and bias are HOST pointers of n_bins floats, read during
 * the call; bias may be NULL (b = 0).  n_bins >= 2, d_hi > d_lo,
 * 0 <= outlier_w < 1.
 */
typedef struct {
    int32_t n_bins;
    float d_lo, d_hi;
    const float *log_sigma;
    float outlier_w;
    const float *bias;
} mrf_noise_lut;

/*
 * precision: MRF_PREC_F32, MRF_PREC_F64, MRF_PREC_BF16 or MRF_PREC_F32_LOG.  BF16 keeps the FP32
 *            arithmetic and rounds each stored ray -> voxel message to bf16
 *            (nearest even; 2 bytes per edge instead of 4); the voxel totals
 *            sum the rounded values.  It runs on the pipelined ray kernel
 *            only: mrf_infer returns MRF_ERANGE if a ray is longer than it
 *            takes (4088 edges).  Not in the paper, which stores FP32.
 *            MRF_PREC_F32_LOG is an ablation of the default's arithmetic: the
 *            messages of Eqs. "pos"/"neg" in the log domain, as the paper
 *            evaluates them (Section IV-A), in FP32 with one thread per ray:
 *            log P_i = sum_{k<i} log(1 - mu_k) as a Kahan-compensated prefix sum,
 *            log A_i and log B_i by log-add-exp recurrences, lambda_i = log pos_i -
 *            log neg_i; then the per-edge voxel totals.  Slow (several FP32
 *            transcendentals per edge); for accuracy comparisons.
 * nu_bg:     likelihood of the all-empty configuration of a ray (the ray leaves
 *            the grid or passes its truncation point without meeting an
 *            occupied voxel).  < 0 selects outlier_w / d_hi of the first frame's
 *            table; 0 is the paper's potential taken literally (then a one-voxel
 *            ray sends an infinite message, clamped to +-64 in log-odds).
 * init_p:    mu_{o -> psi}(o = 1) sent on every edge in the first pass
 *            (Section IV-A uses 0.1); <= 0 selects the prior.
 * debug_checks: nonzero enables host-side structure checks after each build.
 * variants:  0 (exact flooding BP) or a combination of the implementation
 *            variants of the paper's Section "Belief Propagation":
 *            MRF_VAR_LENGTH_WEIGHT: a ray's log-odds message lambda enters the
 *              voxel's belief as w lambda, w = min(1, l / h) with l the length
 *              the ray travels in the voxel and h the voxel edge; the message
 *              back to the ray leaves out its own w lambda
 *              (T = logit gamma + sum w lambda, cavity T - w lambda).  The
 *              stored per-edge value is w lambda.  Runs the tile-per-CTA ray
 *              kernel (mrf_set_plan is overridden).
 *            MRF_VAR_KEYFRAME_AVG: after each pass, every stored message of a
 *              (keyframe, voxel) pair is replaced by the pair's mean, so each
 *              ray's cavity leaves out its keyframe's average message; the
 *              belief (the sum) is unchanged.  Keyframes are the frames in the
 *              order they were added.
 *            Variants need MRF_PREC_F32 (MRF_EINVAL otherwise) and make
 *            mrf_grad return MRF_ESTATE (its adjoint is that of exact BP).
 * long_ray_f64: 0 (off), or a ray length in edges: FP32 contexts then compute
 *            the messages of every longer ray with FP64 prefix and suffix
 *            accumulations (from the same FP32 cavities; stored as FP32), the
 *            rest as usual; the voxel totals then sum per-edge messages (no
 *            per-group pre-aggregation).  Needs MRF_PREC_F32 and no variants.
 */
typedef struct {
    int32_t precision;
    float nu_bg;
    float init_p;
    int32_t debug_checks;
    int32_t variants;
    int32_t long_ray_f64;
} mrf_options;

/* Per-kernel-class device time accumulated while profiling is on. */
typedef struct {
    double ms_ray_messages;    /* ray -> voxel message kernel (Eqs. pos/neg)       */
    double ms_voxel_reduce;    /* voxel totals / cavity source (Eq. node_to_factor) */
    double ms_other_infer;     /* init, marginals and fix-up kernels during infer   */
    double ms_build;           /* transpose (sort) and plan kernels                 */
    double ms_traverse;        /* ray set-up, offsets and 3D-DDA walk               */
    int64_t n_ray_messages, n_voxel_reduce, n_other_infer, n_build, n_traverse;
} mrf_profile_times;

/* Fill *opt with the defaults (FP32, nu_bg from the table, init_p = prior). */
void mrf_default_options(mrf_options *opt);

/*
 * Create a map over grid g with Bernoulli voxel prior gamma = prior
 * (Eq. "prior_potential"), 0 < prior < 1.  cuda_stream is a cudaStream_t (NULL
 * = the legacy default stream) on the current device.  opt may be NULL
 * (defaults).  Errors: MRF_EINVAL, MRF_ENOMEM, MRF_ECUDA.
 */
int mrf_create(mrf_ctx **out, const mrf_grid *g, float prior, const mrf_options *opt, void *cuda_stream);

/* Free everything the context owns (after synchronising its stream).  NULL is a no-op. */
void mrf_destroy(mrf_ctx *ctx);

/* Drop every frame but keep allocations for reuse.  Errors: as mrf_create. */
int mrf_reset(mrf_ctx *ctx);

/* Change the stream later work is enqueued on. */
int mrf_set_stream(mrf_ctx *ctx, void *cuda_stream);

/*
 * Add one depth frame: W x H z-depths in metres, row-major (pixel (u, v) at
 * v * W + u), 0 or non-finite = no measurement.  cam_to_world is a HOST 3x4
 * row-major [R | c] camera-to-world pose.  Every valid pixel becomes one ray
 * (Section III-A: rays are independent measurements); the ray starts at the
 * camera centre or where it enters the grid and stops 3 sigma(Z) past the
 * measured range or where it leaves the grid (Section IV-B).  The walk is a
 * 3D-DDA (Section IV-A) that records, per visited voxel, its index and the
 * sensor likelihood nu(d) at the midpoint range d of the ray's segment in that
 * voxel.  The noise table is copied; depth_dev is read asynchronously.
 * Synchronises once (to size the new edges).
 * Errors: MRF_EINVAL (W, H <= 0, bad table), MRF_ENOMEM, MRF_ERANGE, MRF_ECUDA.
 */
int mrf_add_frame(mrf_ctx *ctx, const float *depth_dev, int32_t W, int32_t H, const double cam_to_world[12],
                  const mrf_intrinsics *K, const mrf_noise_lut *lut);

/* As mrf_add_frame with depth in HOST memory (copied to the device inside). */
int mrf_add_frame_host(mrf_ctx *ctx, const float *depth_host, int32_t W, int32_t H,
                       const double cam_to_world[12], const mrf_intrinsics *K, const mrf_noise_lut *lut);

/*
 * Run `iters` flooding passes of loopy BP (Section IV-A's up and down passes)
 * from the initial messages: pass 1 sends mu(o = 1) = init_p on every edge;
 * each pass computes every ray->voxel message from the previous pass's
 * cavities (Eqs. "pos"/"neg", evaluated by per-ray prefix and suffix scans),
 * then every voxel's total log-odds T_v = logit(prior) + sum of its incoming
 * ray messages (the marginal equation; cavities for the next pass are
 * T_v - lambda, Eq. "node_to_factor").  The result depends only on the frames
 * added and iters.  Builds the voxel-sorted transpose first if frames were
 * added since the last call.  iters >= 0; with no frames every p = prior.
 * Asynchronous.  Errors: MRF_EINVAL, MRF_ENOMEM, MRF_ECUDA.
 */
int mrf_infer(mrf_ctx *ctx, int32_t iters);

/* Write p_v = sigmoid(T_v) for all nx*ny*nz voxels (x fastest) into out_dev
 * (floats).  A batched context writes every scene's voxels, scenes in order. */
int mrf_marginals(mrf_ctx *ctx, float *out_dev);

/* As mrf_marginals into HOST memory; synchronises. */
int mrf_marginals_host(mrf_ctx *ctx, float *out_host);

/* ---- batches of scenes, kernel plans, CUDA graphs -------------------------
 * Not in the paper: many independent maps inferred as one.                  */

/* A context holding n_scenes independent maps (grids[n_scenes], one prior):
 * their voxels get consecutive keys and their edges one CSR, so every pass
 * runs over all scenes at once.  The total voxel count (and its brick-padded
 * key space) must stay below 2^32 and the total edge count below 2^32 -
 * 8192; larger collections are run in several contexts.  mrf_add_frame adds
 * to scene 0; marginals come out scene after scene.  Voxel-indexed exports,
 * held-out frames and mrf_grad need a single-scene context (MRF_ESTATE). */
int mrf_create_batch(mrf_ctx **out, int32_t n_scenes, const mrf_grid *grids, float prior, const mrf_options *opt,
                     void *cuda_stream);

/* Number of scenes and of voxels over all scenes.  Either pointer may be NULL. */
int mrf_scene_count(mrf_ctx *ctx, int32_t *n_scenes, int64_t *n_voxels);

/* mrf_add_frame for scene `scene` of a batched context (0 <= scene < n_scenes). */
int mrf_add_frame_to(mrf_ctx *ctx, int32_t scene, const float *depth_dev, int32_t W, int32_t H,
                     const double cam_to_world[12], const mrf_intrinsics *K, const mrf_noise_lut *lut);

/* Kernel plan for the next transpose build (it marks the context for a
 * rebuild): ray_items = edges per thread of the ray kernel (0: the library's
 * choice from the longest ray; 4, 8, 16 or 32); threads = 0 (choice), 128,
 * 256 or 512 for the pipelined kernel, -1 for the tile-per-CTA kernel;
 * groups = -1 (choice), 0 (per-edge voxel totals) or 1 (per-(tile, voxel)
 * partial sums, pipelined kernel only).  The pipelined shapes are 256 x 8,
 * 256 x 16, 128 x 16 and 512 x 4 (threads x edges); a choice the rays do
 * not allow (a window too short for the longest ray, another pairing)
 * falls back to the library's.  Results do not depend on the plan beyond FP32
 * rounding order.  Errors: MRF_EINVAL for values outside these sets. */
int mrf_set_plan(mrf_ctx *ctx, int32_t ray_items, int32_t threads, int32_t groups);

/* mrf_infer through a CUDA graph: the first call for a given iters runs the
 * passes normally and records them (on a stream of the context's own,
 * ordered after earlier work on the context's stream); later calls replay
 * the recording with one graph launch, ordered the same way.  Adding frames,
 * mrf_reset or mrf_set_plan drop the recording.  Same results and errors as
 * mrf_infer. */
int mrf_infer_graph(mrf_ctx *ctx, int32_t iters);

/* ---- learning the noise table: gradient of a held-out depth likelihood ---
 * Not in the paper, which fits the table offline (Section IV-C).           */

/* A held-out depth frame: traversed like mrf_add_frame (lut sets the 3-sigma
 * truncation of its rays) but kept out of the map; mrf_grad scores the map
 * with it.  Same arguments and errors as mrf_add_frame.  mrf_reset drops
 * held-out frames too. */
int mrf_add_heldout(mrf_ctx *ctx, const float *depth_dev, int32_t W, int32_t H, const double cam_to_world[12],
                    const mrf_intrinsics *K, const mrf_noise_lut *lut);

/* The accuracy metric of the paper's Section "Evaluation Metric for
 * Probabilistic Occupancy Maps" for the current marginals on one depth frame.
 * Every valid pixel's ray is walked from the near plane to the grid exit (no
 * 3-sigma truncation), over voxels v_1..v_N with entry and exit ranges
 * [s_i, e_i).  With p_i the marginal as mrf_marginals writes it (FP32),
 * alpha_i = -log(1 - p_i) / h (a whole voxel crossed keeps visibility
 * 1 - p_i), vis_1 = 1 and vis_{i+1} = vis_i exp(-alpha_i (e_i - s_i)), the
 * most likely surface is the voxel with the largest alpha_i vis_i (the first
 * on ties); it is put beyond the map instead when vis_{N+1} exceeds that
 * voxel's mass vis_i - vis_{i+1}, or when the ray crosses no voxel.  The ray is
 * accurate when its range Z lies in [s_i, e_i) of the chosen voxel, or, beyond
 * the map, when Z > e_N.  depth_dev, W, H, cam_to_world, K and lut are as for
 * mrf_add_frame (the table only decides which pixels are valid).  result_dev
 * (device, W*H int8, nullable) gets 1 / 0 per evaluated pixel and -1 for
 * pixels without a ray (invalid depth or a ray missing the grid).  Writes the
 * counts of accurate and evaluated rays.  Single-scene contexts after
 * mrf_infer (MRF_ESTATE otherwise); synchronises the context's stream. */
int mrf_accuracy(mrf_ctx *ctx, const float *depth_dev, int32_t W, int32_t H, const double cam_to_world[12],
                 const mrf_intrinsics *K, const mrf_noise_lut *lut, int8_t *result_dev, int64_t *n_accurate,
                 int64_t *n_evaluated);

/* Loss and gradient with respect to the noise table theta = (log_sigma[n_bins],
 * outlier_w) of
 *   loss = -sum_r log( sum_i nu_i p_{v_i} prod_{k<i}(1 - p_{v_k}) + nu_bg prod_k (1 - p_{v_k}) )
 * over the held-out rays r (voxels v_1..v_N in range order), where p are the
 * marginals after `iters` passes of BP on the map's frames and every nu (map
 * and held-out edges) is the likelihood of Eq. "noise" under theta: the
 * probability of the held-out depths when each voxel's occupancy is drawn
 * from its marginal (Eq. "depth_message" summed over the first occupied
 * voxel).  The edges (voxels, ranges) stay as the frames were traversed;
 * nu_bg = outlier_w / d_hi unless the context fixed it.  Every edge's
 * likelihood becomes theta's and the map is left inferred with it, so a
 * fitting loop can call this repeatedly.  The reverse pass keeps each pass's
 * messages and voxel totals (4 bytes per edge and per voxel key per pass)
 * and recomputes the ray scans from them in FP64; the result is bitwise
 * reproducible.  loss, grad_log_sigma[n_bins] and grad_outlier_w are host
 * pointers; synchronous.  Errors: MRF_EINVAL (table out of range, iters < 0,
 * null pointer), MRF_ESTATE (not an FP32 context, no frames or no held-out
 * frames), MRF_ENOMEM, MRF_ECUDA. */
int mrf_grad(mrf_ctx *ctx, int32_t iters, const mrf_noise_lut *theta, double *loss, double *grad_log_sigma,
             double *grad_outlier_w);

/* Number of rays (pixels of all frames, including invalid ones) and edges. */
int mrf_stats(mrf_ctx *ctx, int64_t *n_rays, int64_t *n_edges);

/* Longest ray (edges) and number of non-empty voxels (valid after mrf_infer). */
int mrf_stats2(mrf_ctx *ctx, int32_t *max_ray_len, int64_t *n_touched_voxels);

/* How the edges are planned for the kernels (valid after mrf_infer; -1 while
 * frames have been added since): ray_items = edges per thread of the ray
 * kernel; n_ray_tiles = its tiles (runs of whole rays); n_groups = the
 * (tile, voxel) groups whose messages the ray kernel sums before the voxel
 * totals, or 0 when it writes per-edge messages only (FP64, or tiles of 32
 * edges per thread).  Any pointer may be NULL.  The paper has no counterpart:
 * this reports the library's own data layout. */
int mrf_plan_info(mrf_ctx *ctx, int32_t *ray_items, int64_t *n_ray_tiles, int64_t *n_groups);

/* Block until the context's stream has finished.  Returns MRF_ETIMEOUT (and
 * clears the condition) when a bounded device-side wait gave up since the last
 * check: the ray kernel's waits for its bulk copies give up after one second. */
int mrf_synchronize(mrf_ctx *ctx);

/* Failure injection for tests; the paper has no counterpart.
 * mrf_debug_fail_alloc: the nth device allocation the context makes from now
 *   on (1 = the next) fails with MRF_ENOMEM and the message "...: injected";
 *   0 turns it off.  The context keeps its earlier buffers and stays usable
 *   once the error has been read (mrf_last_error).
 * mrf_debug_wait_probe: enqueues one CTA that waits on a shared-memory
 *   barrier nothing arrives on; its bounded wait gives up after one second
 *   and the next mrf_synchronize returns MRF_ETIMEOUT.  Nothing faults, traps
 *   or hangs; the context stays usable. */
int mrf_debug_fail_alloc(mrf_ctx *ctx, int64_t nth);
int mrf_debug_wait_probe(mrf_ctx *ctx);

/* Message of the last failure ("" if none); clears the sticky error state. */
const char *mrf_last_error(mrf_ctx *ctx);

/* ---- inspection: copies into caller-owned device buffers ---------------- */

/* ray_off_dev: n_rays+1 int64 edge offsets; vox_dev: n_edges voxel indices;
 * d_dev (nullable): n_edges midpoint ranges; Z_dev (nullable): n_rays ranges. */
int mrf_export_rays(mrf_ctx *ctx, int64_t *ray_off_dev, uint32_t *vox_dev, float *d_dev, float *Z_dev);

/* Per-edge likelihoods nu(d) as used by the FP32 path (n_edges floats). */
int mrf_export_nu(mrf_ctx *ctx, float *nu_dev);

/* Last ray->voxel log-odds messages (n_edges) and voxel log-odds T (nx*ny*nz),
 * FP32 or BF16 contexts (bf16 messages are widened to FP32 exactly); either
 * pointer may be NULL.  MRF_ESTATE on an FP64 context. */
int mrf_export_messages(mrf_ctx *ctx, float *lam_dev, float *T_dev);

/* Same for the FP64 path. */
int mrf_export_messages_f64(mrf_ctx *ctx, double *lam_dev, double *T_dev);

/* Voxel-sorted transpose, in the library's internal voxel order (the grid cut
 * into 8x8x8 bricks numbered x-fastest, Morton order inside a brick):
 * perm_dev (n_edges edge ids, sorted by voxel, by edge id within a voxel);
 * seg_off_dev (n_seg+1 offsets into perm) and seg_vox_dev (n_seg linear voxel
 * indices x + nx (y + ny z)) for the non-empty voxels in that order.  Pass NULL
 * pointers to query *n_seg only. */
int mrf_export_transpose(mrf_ctx *ctx, uint32_t *perm_dev, uint32_t *seg_off_dev, uint32_t *seg_vox_dev,
                         int64_t *n_seg);

/* Per-tile voxel groups of the pre-aggregating ray kernel, exported for
 * inspection (the paper has no counterpart: they only reorder the sums of
 * Eq. "T" so that each (ray tile, voxel) pair is summed once in shared memory).
 * The FP32 edge array (ray after ray, frame after frame) is cut into tiles of
 * whole rays; tile t holds edges [tile_E[t], tile_E[t+1]) and its window
 * starts at tile_E[t] rounded down to 8.  A group is one voxel of one tile.
 *   tile_E_dev  n_tiles+1 int64;
 *   tg_off_dev  n_tiles+1 int64: tile t's groups are slots [tg_off[t], tg_off[t+1]);
 *   lidx_dev    n_edges uint16: tile t's edges in tile-major order at positions
 *               [tile_E[t], tile_E[t+1]): voxel order (the internal voxel keys
 *               of mrf_export_transpose), edge order within a voxel; each entry
 *               the edge's index in the tile's window;
 *   gid_dev     n_edges uint16: each edge's group index within its tile (groups
 *               numbered in voxel order);
 *   ends_dev    ceil(n_edges/32) uint32: bit q of word q/32 set where tile-major
 *               position q ends a group;
 *   gkey_dev    n_groups uint32: each group slot's internal voxel key.
 * Device buffers owned by the caller; any may be NULL (n_tiles / n_groups,
 * nullable host pointers, receive the sizes).  Builds the tables first if
 * frames were added since the last build.  MRF_ESTATE when the context's plan
 * has no groups (FP64 or BF16-free ungrouped plans, rays too long for the
 * pipelined kernel, mrf_set_plan without groups). */
int mrf_export_groups(mrf_ctx *ctx, int64_t *tile_E_dev, int64_t *tg_off_dev, uint16_t *lidx_dev, uint16_t *gid_dev,
                      uint32_t *ends_dev, uint32_t *gkey_dev, int64_t *n_tiles, int64_t *n_groups);

/* ---- profiling ----------------------------------------------------------- */

/* Nonzero: record CUDA events around every kernel class on the context's stream. */
int mrf_profile_enable(mrf_ctx *ctx, int32_t on);

/* Synchronise, then return and reset the accumulated times. */
int mrf_profile_read(mrf_ctx *ctx, mrf_profile_times *out);

/* Kernel launches issued by this context since creation (all kernel classes). */
int64_t mrf_launch_count(const mrf_ctx *ctx);

/* ---- standalone kernels on caller buffers (no context) ------------------ */

/*
 * Ray->voxel messages for R rays in CSR form (Eqs. "pos"/"neg" with the
 * all-empty term nu_bg): for edge e of a ray, with cavity log-odds
 * L_e = T[vox[e]] - lam[e] (or L_e = L0 when first != 0), writes the new
 * log-odds message into lam[e] in place.  ray_off_dev: R+1 non-decreasing
 * int64 offsets starting at 0; vox_dev, nu_dev, lam_dev: ray_off[R] entries;
 * T_dev: indexed by vox.  workspace_dev: mrf_ray_messages_workspace() bytes,
 * 16-byte aligned, caller-owned.  Rays longer than 8000 edges: MRF_ERANGE.
 * Asynchronous on stream.  Errors: MRF_EINVAL, MRF_ERANGE, MRF_ECUDA.
 */
size_t mrf_ray_messages_workspace(int64_t n_rays, int64_t n_edges, int32_t max_ray_len);
int mrf_ray_messages(const int64_t *ray_off_dev, int64_t n_rays, int32_t max_ray_len, const uint32_t *vox_dev,
                     const float *nu_dev, const float *T_dev, float *lam_dev, float nu_bg, int32_t first, float L0,
                     void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * Voxel totals (the marginal equation in log-odds):
 * T[seg_vox[s]] = logit_prior + sum_{k in [seg_off[s], seg_off[s+1])} lam[perm[k]]
 * for s < n_seg, summed in a fixed order (deterministic).  Voxels not listed
 * are not written.  workspace_dev: mrf_voxel_reduce_workspace() bytes.
 */
size_t mrf_voxel_reduce_workspace(int64_t n_edges);
int mrf_voxel_reduce(const uint32_t *perm_dev, const uint32_t *seg_off_dev, const uint32_t *seg_vox_dev,
                     int64_t n_seg, int64_t n_edges, const float *lam_dev, float logit_prior, float *T_dev,
                     void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * mrf_voxel_reduce without any allocation.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory during a call (a mapping
 * loop under a fixed, preallocated memory budget; code running inside a
 * memory allocator's callbacks).  Same inputs, outputs and summation order as
 * mrf_voxel_reduce; the scratch is a device array of 1.25 MiB defined by the
 * library, which every device that loads the library keeps until the process
 * exits.  n_edges must not exceed MRF_NOALLOC_MAX_EDGES (MRF_ERANGE otherwise).
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current, and keeps it with the
 * current context's id; make that first call before any stream capture.  After
 * cudaDeviceReset (or with another context current on the device) the next call
 * looks the address up again, so make that call before any capture as well.  All calls share the one array, so calls that overlap on
 * the GPU (different streams, or host threads without ordering between them)
 * race and must not be issued.  Asynchronous on stream.
 * Errors: MRF_EINVAL, MRF_ERANGE, MRF_ECUDA.
 */
#define MRF_NOALLOC_MAX_EDGES ((int64_t)1 << 28)
int mrf_voxel_reduce_noalloc(const uint32_t *perm_dev, const uint32_t *seg_off_dev, const uint32_t *seg_vox_dev,
                             int64_t n_seg, int64_t n_edges, const float *lam_dev, float logit_prior, float *T_dev,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MRFMAP_H */
