/*
 * dgs.h -- C ABI of the B300 delivery-state renderer for dynamic Gaussian scenes.
 *
 * The library renders a dynamic Gaussian scene as it stands in an incomplete
 * delivery state and scores that state against the complete render, for one
 * state or for many states in one batch, forward and backward.  It follows the
 * paper "Renderable Partial Representations for Dynamic Gaussian Splatting
 * under Incomplete Delivery":
 *   - Section 3: N fixed-identity Gaussians in clusters; per cluster one base
 *     completion group and refinement groups; every attribute is base plus
 *     additive refinements; every dependency-closed subset is renderable.
 *   - Eq. 1: mu_i(t) = mubar_i + sum_r b_r(t) q_{i,r} + refinement residuals,
 *     with the shared basis b_{2j-1}(t) = cos(2 pi j t), b_{2j}(t) = sin(2 pi j t)
 *     and the cluster affine taken as the identity.
 *   - Sections 4 and 7.4: dependencies are enforced after delivery; a layer is
 *     usable only when all layers below it in its cluster are usable.
 *   - Section 6: many delivery states of one scene rasterized in one batch;
 *     the batched result equals serial (one state at a time) evaluation.
 *   - Eq. 3: the distortion D of a state against the reference render, taken
 *     here as the per-state MSE (accumulated in FP64) and its PSNR.
 * Rasterization is EWA splatting of the 3D Gaussians, tile-binned on 16x16
 * pixel tiles with a stable 64-bit (tile | depth) order, composited front to
 * back in FP32 (the readings of every unstated constant are listed in the
 * project's design notes and match the FP64 oracle used by the tests).
 *
 * Conventions for every entry point:
 *   - Pointers marked [device] are CUDA device pointers on the context's
 *     device, [host] are host pointers.  The caller owns every buffer it
 *     passes; the library owns only the workspace inside a dgs_ctx.
 *   - Calls are asynchronous on the given stream, except that a call may
 *     synchronize that stream once or twice to size its workspace (the number
 *     of projected records and of tile entries); it never synchronizes other
 *     streams.  A context must not be used by two host threads at once.
 *   - Return 0 on success or a negative DGS_E_* code; dgs_last_error() then
 *     describes the failure.  Arguments are validated before any launch; an
 *     invalid call launches nothing and leaves outputs untouched.
 *   - Mask bits at positions >= n_clusters * n_layers are ignored.
 */
#ifndef DGS_H
#define DGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGS_VERSION 1

#if defined(__GNUC__)
#define DGS_API __attribute__((visibility("default")))
#else
#define DGS_API
#endif

enum {
    DGS_OK = 0,
    DGS_E_INVALID_ARG = -1,   /* null pointer, bad count, mismatched sizes */
    DGS_E_UNSUPPORTED = -2,   /* e.g. sh_degree not in {0, 3}, > 1024 clusters */
    DGS_E_OOM = -3,           /* workspace allocation failed */
    DGS_E_CUDA = -4,          /* a CUDA runtime call or launch failed */
    DGS_E_CAPACITY = -5,      /* a count exceeds 32-bit indexing */
    DGS_E_SCRATCH = -6,       /* dgs_image_mse_noalloc: sizes exceed its fixed scratch */
    DGS_E_STALE = -7          /* dgs_render_backward: the masks changed after the forward whose images were passed */
};

/* Doubles of fixed device scratch held by dgs_image_mse_noalloc (512 KiB per GPU). */
#define DGS_NOALLOC_MAX_PARTS 65536

typedef struct dgs_ctx dgs_ctx;
typedef void *dgs_stream;     /* a cudaStream_t; NULL = the legacy default stream */

/*
 * One scene (Section 3, Eq. 1).  Gaussians are stored cluster-contiguous:
 * Gaussians cluster_offsets[c] .. cluster_offsets[c+1]-1 form cluster c.
 * n_layers L counts the base layer: layer 0 = base, layers 1..L-1 = refinements.
 * All arrays [device], FP32, row-major:
 *   mu0 [n][3]          canonical mean (mubar of Eq. 1)
 *   u [R][n][3]         temporal coefficients q_{i,r} of Eq. 1 (R = temporal_rank)
 *   log_scale [n][3]    log of the three axis scales
 *   quat [n][4]         rotation quaternion (w, x, y, z), normalised on use
 *   opacity_logit [n]   opacity o = sigmoid(logit)
 *   colour [n][NC]      NC = 3 (sh_degree 0: RGB) or 48 (sh_degree 3: 16 real
 *                       SH coefficients x 3 channels, channel innermost)
 *   res [L-1][n][K]     refinement l (1..L-1) of Gaussian i, K = 11 + NC:
 *                       dmu[3], dlog_scale[3], dquat[4], dlogit[1], dcolour[NC]
 *   affine [C][T][12]   optional cluster affine A_{c,t} of Eq. 1 (NULL = the
 *                       identity): keyframe k of cluster c, row-major 3x4
 *                       (linear part | translation), holds A at time k / T
 *                       (T = affine_T >= 1); between keyframes the twelve
 *                       entries are interpolated linearly, periodically in t
 *                       with period 1
 *   res_mode            how refinements are read (Section 3: refinements are
 *                       quantized with learned steps):
 *                       0  res as given (float);
 *                       1  res_q [L-1][n][K] int16 symbols times res_step
 *                          [L-1][K] (one step per layer and component); res
 *                          unused; no refinement gradient;
 *                       2  res quantized on the fly: symbol v = round(res /
 *                          res_step) (FP32 quotient, ties to even) clipped to
 *                          [-32768, 32767], value v * step; gradients pass
 *                          straight through the rounding (zero where clipped)
 *                          and the step receives sum g (v - res / step), or
 *                          g v where clipped
 * A Gaussian of cluster c at delivered depth d >= 1 renders with every
 * attribute = base + res[0] + ... + res[d-2]; at depth 0 it is absent.  Its
 * mean at time t is A_{c,t} mu0 + (position residuals) + sum_r b_r(t) u_r.
 */
typedef struct {
    int32_t n, n_clusters, n_layers, sh_degree, temporal_rank;
    const int32_t *cluster_offsets;   /* [device] [n_clusters + 1] */
    const float *mu0;
    const float *u;
    const float *log_scale;
    const float *quat;
    const float *opacity_logit;
    const float *colour;
    const float *res;
    const float *affine;              /* [device] [n_clusters][affine_T][12] or NULL */
    int32_t affine_T;
    const int16_t *res_q;             /* [device] [L-1][n][K] (res_mode 1) */
    const float *res_step;            /* [device] [L-1][K] (res_mode 1 and 2) */
    int32_t res_mode;
} dgs_scene;

/* Gradients in the scene's layout, [device], ACCUMULATED (+=) by the backward. */
typedef struct {
    float *mu0, *u, *log_scale, *quat, *opacity_logit, *colour, *res;
    float *affine;                    /* [n_clusters][affine_T][12]; needed when the scene has an affine */
    float *res_step;                  /* [L-1][K]; needed with res_mode 2 */
} dgs_scene_grad;

/* OpenCV pinhole: p_cam = R_wc p_world + t_wc; x right, y down, z forward;
 * pixel (x, y) has its centre at (x + 0.5, y + 0.5).  [host] */
typedef struct {
    float R_wc[9];
    float t_wc[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} dgs_camera;

/*
 * A batch of delivery states.  masks [device] [n_states][W32] uint32,
 * W32 = ceil(n_clusters * n_layers / 32); bit b = c * n_layers + l (word b/32,
 * bit b%32) is set when packet (cluster c, layer l) arrived.  t [host] [n_states]
 * is each state's time, cam [host] [n_states] its index into the camera array.
 * States with equal (cam, t) form a view group and share decoded and projected
 * Gaussians and tile lists.
 */
typedef struct {
    const uint32_t *masks;
    const float *t;
    const int32_t *cam;
    int32_t n_states;
} dgs_states;

/* Create a context on CUDA device `device`.  Returns DGS_OK and *out. */
DGS_API int dgs_create(dgs_ctx **out, int device);
/* Free the context and its workspace (device memory); NULL is accepted. */
DGS_API void dgs_destroy(dgs_ctx *ctx);
/* Message of the last failed call on this context ("" if none). [host] */
DGS_API const char *dgs_last_error(const dgs_ctx *ctx);
/* DGS_VERSION of the loaded library. */
DGS_API int dgs_version(void);

/*
 * Render one delivery state (Section 3 + closure of Sections 4 / 7.4):
 * mask [device] [W32], time t, camera [host], background bg [host][3].
 * image [device] [H][W][3] FP32 receives C + T_final * bg per pixel.
 * Bit-equal to that state's image from dgs_render_states_batched.
 */
DGS_API int dgs_render_state(dgs_ctx *ctx, const dgs_scene *scene, const uint32_t *mask, float t,
                     const dgs_camera *cam, const float *bg, float *image, dgs_stream stream);

/*
 * Render every state of a batch in one pass (Section 6): shared decode and
 * projection per (view group, Gaussian, delivered depth), one stable tile
 * sort for the batch, per-state filtered compositing.  cams [host] [n_cams];
 * all cameras must have the same width and height.  images [device]
 * [n_states][H][W][3].  The call records its projection and tile lists in the
 * context for a following dgs_render_backward with the same arguments.
 */
DGS_API int dgs_render_states_batched(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states,
                              const dgs_camera *cams, int n_cams, const float *bg,
                              float *images, dgs_stream stream);

/*
 * Adjoint of dgs_render_states_batched (Section 4 training, Eq. 2): given
 * dL/dimages [device] [n_states][H][W][3], accumulate (+=) dL/d(parameters)
 * into grads (every pointer [device], scene layout).  images [device]
 * [n_states][H][W][3] is the forward's output for the same arguments, or NULL:
 * with it the adjoint walks each tile once, without it a first walk recomputes
 * each pixel's final value (same gradients up to float atomic order; images
 * that are not this forward's output give wrong gradients, undetected).  Either
 * way transmittance is recomputed per tile, not stored.  Refinement layers a
 * state did not deliver get exactly zero from that state.  If the context's
 * last forward call had the same arguments (same pointers, counts, times and
 * cameras) its projection and tile lists are reused, provided the masks still
 * hold the bits that forward rendered: the library keeps a device copy of them
 * and compares (one stream synchronization).  If they changed, the call fails
 * with DGS_E_STALE when images were passed (they belong to the old masks), and
 * without images it renders lists for the current masks.  The scene's
 * attribute values are not compared: they must not change between a forward
 * and its backward.
 */
DGS_API int dgs_render_backward(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states,
                        const dgs_camera *cams, int n_cams, const float *bg, const float *images,
                        const float *dL_dimages, const dgs_scene_grad *grads, dgs_stream stream);

/*
 * Several scenes in one call (the serving mix: many scenes, each with its own
 * states, cameras and image size).  Job k renders jobs[k].states of
 * jobs[k].scene into jobs[k].images exactly as dgs_render_states_batched would
 * (bit for bit).  Every scene gets a workspace of its own inside the context
 * (kept between calls, so job k of the next call reuses the memory of job k of
 * this one), its records and tile lists are prepared scene by scene, and one
 * persistent forward raster launch works through the (scene, tile, state)
 * items of all jobs from one queue.  All jobs use one sort tile size: the one
 * fixed by dgs_set_tile_size, else 32 px.  No batch splitting under a memory
 * budget: every scene's workspace is held at once.  jobs [host] [n_jobs];
 * returns DGS_E_INVALID_ARG (message names the scene) for a bad job.
 */
typedef struct {
    const dgs_scene *scene;        /* [host] */
    dgs_states states;             /* masks [device], t / cam [host] */
    const dgs_camera *cams;        /* [host] [n_cams] */
    int32_t n_cams;
    float bg[3];
    float *images;                 /* [device] [n_states][H][W][3] */
} dgs_scene_job;
DGS_API int dgs_render_scenes_batched(dgs_ctx *ctx, const dgs_scene_job *jobs, int n_jobs, dgs_stream stream);

/* Adjoint of the last dgs_render_scenes_batched call, for the same jobs (the
 * same scenes, states, cameras and images): dL_dimages [host] [n_jobs] of
 * [device] [n_states][H][W][3], grads [host] [n_jobs] accumulated (+=) as by
 * dgs_render_backward.  One adjoint raster launch covers every job; the
 * projection adjoint runs per scene.  Returns DGS_E_INVALID_ARG when a job is
 * not the one its workspace last rendered, and DGS_E_STALE when a job's masks
 * changed since that forward. */
DGS_API int dgs_render_scenes_backward(dgs_ctx *ctx, const dgs_scene_job *jobs, int n_jobs,
                                       const float *const *dL_dimages, const dgs_scene_grad *grads,
                                       dgs_stream stream);

/*
 * Eq. 3 distortion of every state against the complete render of its view:
 * renders the full-delivery image of each view group and each state, without
 * writing state images, and writes mse [device] [n_states] (FP64 sum of
 * squared FP32 differences over 3*H*W values, divided by 3*H*W) and
 * psnr [device] [n_states] = 10 log10(1 / mse) (+inf when mse == 0).
 */
DGS_API int dgs_state_utility(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states,
                      const dgs_camera *cams, int n_cams, const float *bg,
                      double *mse, double *psnr, dgs_stream stream);

/*
 * Tile reuse in the distortion passes (dgs_state_utility, dgs_group_utility;
 * on by default).  Whether a state's walk over a tile's sorted Gaussians
 * includes an entry depends only on the state's delivered depth of that
 * entry's cluster (Sections 3-4), so two states of one view (same camera and
 * time) whose delivered depths agree on every cluster the walk reaches before
 * all of the tile's pixels stop render that tile identically.  With reuse on,
 * views with at least 8 states render one state of each such group per tile
 * and give the others its FP64 squared-error partial: every output is
 * bit-identical to rendering each state (the groups are exact, not
 * approximate).  enable: 0 renders every (state, tile); nonzero reuses.  The
 * reuse pass synchronizes the stream once per grouping round (at most 17).
 * Returns DGS_E_INVALID_ARG for a null ctx.
 */
DGS_API int dgs_set_tile_reuse(dgs_ctx *ctx, int enable);

/* Side of the square sort tiles that binning, the tile sort and the tile
 * ranges use (an acceleration structure: images, squared errors and
 * gradients are bit-identical for every size, because a Gaussian's footprint
 * is a per-pixel test and every sum runs over fixed 16 x 16 pixel blocks).
 * Larger tiles give fewer (tile, Gaussian) entries to sort; raster warps then
 * walk the longer run of their tile for their own 16-pixel-wide region.
 * size: 16 or 32, or 0 to let the library choose per batch shape.  Applies to
 * the calls and plans made after it.  Returns DGS_E_INVALID_ARG for a null
 * ctx or another size. */
DGS_API int dgs_set_tile_size(dgs_ctx *ctx, int size);

/* Cap on the context's workspace (records, tile entries, sort and raster
 * buffers), in bytes; 0 leaves only the device's free memory as the limit.
 * A context call (dgs_render_states_batched, dgs_render_backward,
 * dgs_state_utility, dgs_group_utility) whose workspace would exceed the cap,
 * or fail to allocate, runs its batch of states in halves, recursively, until
 * each part fits (the paper's probe for the largest batch that fits a memory
 * budget, recovering from a failed allocation).  Every state renders the same
 * bits in any batch, so images and squared errors do not change; gradients
 * accumulate over the parts (the same up to the order of float additions).
 * A single state that does not fit fails with DGS_E_OOM.  Plans are sized at
 * creation and do not split.  Returns DGS_E_INVALID_ARG for a null ctx. */
DGS_API int dgs_set_memory_budget(dgs_ctx *ctx, uint64_t bytes);

/* The context's workspace bytes now, and how many times a batch was split
 * because its workspace did not fit (since creation).  Either pointer may be
 * NULL.  Returns DGS_E_INVALID_ARG for a null ctx. */
DGS_API int dgs_memory_stats(const dgs_ctx *ctx, uint64_t *workspace_bytes, int64_t *batch_splits);

/* Sort tile side in pixels (16 or 32) that the context's last prepared batch
 * used: the fixed size of dgs_set_tile_size, else the autotuner's choice for
 * that call shape; 0 before the first call.  tile_px [host].  Returns
 * DGS_E_INVALID_ARG for a null pointer. */
DGS_API int dgs_last_tile_size(const dgs_ctx *ctx, int32_t *tile_px);

/*
 * Work of the context's last distortion pass: pairs [host] = (state, tile)
 * pairs it scored, rendered [host] = pairs it rendered (the rest took a
 * rendered pair's partial; equal to pairs without reuse), rounds [host] =
 * grouping rounds (0 without reuse).  Any pointer may be NULL.  Returns
 * DGS_E_INVALID_ARG for a null ctx.
 */
DGS_API int dgs_tile_reuse_stats(const dgs_ctx *ctx, int64_t *pairs, int64_t *rendered, int32_t *rounds);

/*
 * Counterfactual render utility of completion groups (Section 5, Eq. 3 and
 * Eq. 4).  A completion group g is one packet (cluster, layer): groups [host]
 * [n_groups][2].  contexts holds n_groups * n_contexts states (masks [device],
 * t and cam [host]); state g * n_contexts + j is context j of group g, which
 * should be a valid partial receiver state that lacks g (a context that
 * already holds g, or lacks a prerequisite of g, gives Delta = 0).  For each
 * context m the call renders m and m u g (one batch of 2 n_groups n_contexts
 * states, all sharing decode and projection per view) and forms
 *   Delta_g(m) = D(I, R(m)) - D(I, R(m u g)),
 * D = the MSE of dgs_state_utility against the complete render I of the
 * state's view.  delta [device] [n_groups * n_contexts] (may be NULL) receives
 * every Delta; stats [device] [n_groups][4] receives per group
 *   mean   = E_m[Delta_g]                (over its n_contexts contexts)
 *   Q      = Q_q(Delta_g)                (linear interpolation between order
 *                                         statistics, position q (n - 1))
 *   std    = Std_m(Delta_g)              (population standard deviation)
 *   utility = ((1 - alpha) mean + alpha Q) / (1 + beta std)
 * (the paper's setting: alpha = 0.25, beta = 0.05, q = 0.10).  All in FP64.
 * Needs 1 <= n_contexts <= DGS_UTILITY_MAX_CONTEXTS, 0 <= q <= 1, beta >= 0.
 */
#define DGS_UTILITY_MAX_CONTEXTS 4096
DGS_API int dgs_group_utility(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *contexts,
                              const int32_t *groups, int n_groups, int n_contexts, const dgs_camera *cams,
                              int n_cams, const float *bg, double alpha, double beta, double q, double *delta,
                              double *stats, dgs_stream stream);

/*
 * The packet-conditioned training objective of Section 4 (Eq. 2) over a batch
 * of rendered states, with its gradient.  For state s with reference image
 * refs[ref_index[s]]:
 *   D_s = MSE(I_s, ref) + ssim_weight (1 - SSIM(I_s, ref))
 * SSIM: 11x11 Gaussian window (sigma 1.5), zero-padded same-size filtering,
 * C1 = 0.01^2, C2 = 0.03^2, mean over pixels and channels.  Then
 *   L = mean_s D_s + lambda_c CVaR_q(D) + lambda_t F + lambda_m M
 *       + anchor_weight mean_{s in anchors} D_s
 * CVaR_q(D) = the mean of the ceil(q S) largest D (ties: lower state index);
 * F = mean over temporal pairs (i, j) of the MSE between the rendered change
 * I_j - I_i and the reference change; M = mean over prefix pairs (i, j), state
 * j extending state i, of max(0, D_j - D_i).  The rate term is absent (its
 * weight is 0 in the paper's setting).  params NULL = the paper's weights:
 * 0.20, 0.30, 0.05, 0.10, 2.0, 0.50.
 * images [device] [S][H][W][3], refs [device] [n_refs][H][W][3], ref_index
 * [host] [S], pairs_t / pairs_m [host] [n][2] state indices, anchors [host]
 * [n_anchors]; loss [device] [1] (required), D [device] [S] (may be NULL),
 * dL_dimages [device] [S][H][W][3] (may be NULL: no gradient).  1 <= S <=
 * DGS_OBJECTIVE_MAX_STATES.  Sums over pixels, states and pairs are FP64.
 */
typedef struct dgs_objective_params {
    double ssim_weight, lambda_c, cvar_q, lambda_t, lambda_m, anchor_weight;
} dgs_objective_params;
#define DGS_OBJECTIVE_MAX_STATES 16384
DGS_API int dgs_objective(dgs_ctx *ctx, const float *images, const float *refs, const int32_t *ref_index, int S,
                          int n_refs, int H, int W, const int32_t *pairs_t, int n_pairs_t, const int32_t *pairs_m,
                          int n_pairs_m, const int32_t *anchors, int n_anchors, const dgs_objective_params *params,
                          double *loss, double *D, float *dL_dimages, dgs_stream stream);

/*
 * Per-image MSE (FP64 accumulation) and PSNR of images [device] [S][H][W][3]
 * against refs [device] [n_refs][H][W][3], image s against refs[ref_index[s]]
 * (ref_index [host] [S]).  mse, psnr [device] [S] (psnr may be NULL).  If
 * dL_dimages [device] [S][H][W][3] is not NULL it receives the gradient of
 * L = sum_s weight * mse_s, i.e. weight * 2 (image - ref) / (3 H W).
 */
DGS_API int dgs_image_mse(dgs_ctx *ctx, const float *images, const float *refs, const int32_t *ref_index,
                  int S, int n_refs, int H, int W, float weight, double *mse, double *psnr,
                  float *dL_dimages, dgs_stream stream);

/*
 * Plans: capture-safe execution of a fixed batch (Section 6 batching, run as a
 * CUDA-graph-friendly sequence).  A plan fixes the scene (its pointers; the
 * values may change between calls), the states' times and camera indices, the
 * cameras, the background and -- for mode DGS_PLAN_RENDER with ref_index --
 * the reference image of each state for dgs_plan_image_mse.  dgs_plan_create
 * runs once, synchronously, on the given masks: it plans the view groups,
 * sizes a private workspace (records exactly: at most one depth per state and
 * cluster; tile entries as the masks' count times entry_headroom (>= 1, 0 =
 * 1.25) plus 65536), tunes the states-per-block of the forward raster and
 * uploads every table.  Afterwards dgs_plan_render / _backward / _utility /
 * _image_mse only launch kernels on `stream`: no allocation, no host copy,
 * no synchronisation, launch sizes fixed by the plan, counts kept on the
 * device -- so they can be captured in a CUDA graph and replayed with other
 * masks of the same shape ([n_states][W32], device).  If some masks need more
 * tile entries than reserved, the surplus entries are dropped and
 * dgs_plan_status reports DGS_E_CAPACITY (re-create the plan with more
 * headroom).  A plan is used by one stream at a time; dgs_plan_backward uses
 * the lists of the plan's last dgs_plan_render.  Results equal the
 * corresponding context calls bit for bit (images, MSE) or up to float atomic
 * order (gradients).
 */
typedef struct dgs_plan dgs_plan;
enum { DGS_PLAN_RENDER = 1, DGS_PLAN_UTILITY = 2 };

/*
 * Arenas: one scratch workspace (records, keys, tile entries, sort and raster
 * buffers) shared by every plan created in it, for batches of plans that run
 * one after another on one stream, e.g. many scenes in one CUDA graph (the
 * scratch is sized to the largest plan, not the sum).  Each plan keeps its
 * own small tables.  Rules: create every plan of an arena before capturing
 * any of them (a later creation may reallocate the scratch); a plan's
 * dgs_plan_backward must follow its own dgs_plan_render with no other plan of
 * the arena run in between (checked on the host: DGS_E_INVALID_ARG);
 * destroy the plans before the arena (dgs_arena_destroy returns
 * DGS_E_INVALID_ARG while plans remain).  Error messages of the arena's plans
 * share one string.
 */
typedef struct dgs_arena dgs_arena;
DGS_API int dgs_arena_create(dgs_ctx *ctx, dgs_arena **out);
DGS_API int dgs_arena_destroy(dgs_arena *arena);

/* arena: NULL for a private workspace. */
DGS_API int dgs_plan_create(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                            int n_cams, const float *bg, int mode, const int32_t *ref_index /*[host] [n_states] or NULL*/,
                            int n_refs, float entry_headroom, dgs_arena *arena, dgs_plan **out);
DGS_API void dgs_plan_destroy(dgs_plan *plan);
DGS_API const char *dgs_plan_last_error(const dgs_plan *plan);
/* images [device] [n_states][H][W][3]: as dgs_render_states_batched. */
DGS_API int dgs_plan_render(dgs_plan *plan, const uint32_t *masks, float *images, dgs_stream stream);
/* dgs_plan_render and dgs_plan_image_mse in one pass: the forward raster
 * writes each pixel, its squared error against refs[ref_index[s]] and
 * dL/dimage = weight * 2 (image - ref) / (3 H W) (dL_dimages [device]
 * [n_states][H][W][3], or NULL) as it composites it.  Images and dL/dimages
 * are bit-identical to the two calls; mse / psnr [device] [n_states] sum the
 * same FP32 squared errors in FP64 per 16 x 16 pixel block, so they equal the
 * two calls' up to the order of the FP64 additions.  refs [device]
 * [n_refs][H][W][3].  Needs a plan made with ref_index; counts as the
 * render a dgs_plan_backward follows. */
DGS_API int dgs_plan_render_mse(dgs_plan *plan, const uint32_t *masks, float *images, const float *refs, float weight,
                                double *mse, double *psnr, float *dL_dimages, dgs_stream stream);
/* images (the last dgs_plan_render's output, or NULL) and dL/dimages [device]:
 * accumulates into grads as dgs_render_backward. */
DGS_API int dgs_plan_backward(dgs_plan *plan, const float *images, const float *dL_dimages,
                              const dgs_scene_grad *grads, dgs_stream stream);
/* mse, psnr [device] [n_states]: as dgs_state_utility (mode DGS_PLAN_UTILITY). */
DGS_API int dgs_plan_utility(dgs_plan *plan, const uint32_t *masks, double *mse, double *psnr, dgs_stream stream);
/* As dgs_image_mse with the plan's ref_index; refs [device] [n_refs][H][W][3]. */
DGS_API int dgs_plan_image_mse(dgs_plan *plan, const float *images, const float *refs, float weight, double *mse,
                               double *psnr, float *dL_dimages, dgs_stream stream);
/* Synchronizes `stream`; the last call's record and tile-entry counts [host];
 * DGS_E_CAPACITY (and clears the flag) when entries overflowed since the last check. */
/* Sort tile side in pixels (16 or 32) fixed at the plan's creation.  tile_px [host].
 * Returns DGS_E_INVALID_ARG for a null pointer. */
DGS_API int dgs_plan_tile_size(const dgs_plan *plan, int32_t *tile_px);
DGS_API int dgs_plan_status(dgs_plan *plan, int64_t *n_records, int64_t *n_entries, dgs_stream stream);

/* The Eq. 2 objective of dgs_objective for a plan made with ref_index, in
 * two steps so that the per-step call can be captured in a CUDA graph.
 * dgs_plan_set_objective (not during a capture) fixes the pair and anchor
 * lists [host] (as dgs_objective's, states of the plan) and the weights
 * (NULL: the paper's), validates them, allocates the plan's objective
 * buffers and uploads the tables.  dgs_plan_objective then only launches
 * kernels: images, refs [device] as dgs_objective's; loss [device] [1],
 * D [device] [n_states] or NULL, dL_dimages [device] or NULL; the same bits
 * as dgs_objective with the same arguments.  Returns DGS_E_INVALID_ARG when
 * the objective was not set. */
DGS_API int dgs_plan_set_objective(dgs_plan *plan, const int32_t *pairs_t, int n_pairs_t, const int32_t *pairs_m,
                                   int n_pairs_m, const int32_t *anchors, int n_anchors,
                                   const dgs_objective_params *params);
DGS_API int dgs_plan_objective(dgs_plan *plan, const float *images, const float *refs, double *loss, double *D,
                               float *dL_dimages, dgs_stream stream);

/*
 * Test and inspection access to the projected records and tile lists of the
 * context's last dgs_render_states_batched / dgs_render_state call (or of a
 * backward that re-prepared).  Sizes go to the [host] out-parameters (any may
 * be NULL); each [device] buffer that is not NULL receives a device-to-device
 * copy on `stream`:
 *   recs        [n_rec][12] u32 -- the 48-byte records: mx, my, a2, b2, c2, o,
 *               r, g, b (floats; the conic scaled for base-2 exponents:
 *               a2 = -log2(e)/2 A, b2 = -log2(e) B, c2 = -log2(e)/2 C),
 *               box x = xlo | xhi << 16, box y = ylo | yhi << 16,
 *               cluster | clamp << 11 | depth << 12 | view group << 16 |
 *               boxed << 31 (cluster: 10 bits; depth 0 = culled; boxed: the
 *               3-sigma box is narrower than the alpha >= 1/255 box on some
 *               axis; clamp: alpha may reach the 0.99 clamp, set unless
 *               o <= 0.98 and the conic's condition number is <= 1e4)
 *   depth_keys  [n_rec]  float bits of camera depth of the live records, sorted
 *               stably by (view group, depth): each view group's records in
 *               ascending depth, view groups in order; the sort drops culled
 *               records, so the array ends with 0xFFFFFFFF, one per culled record
 *   depth_slots [n_rec]  the record slot of each sorted depth key (0xFFFFFFFF
 *               in the dropped tail)
 *   entry_keys  [n_ent]  view group * tiles + tile, ascending (stable)
 *   entry_vals  [n_ent]  record slot of each entry
 *   ranges      [n_view_groups * tiles][2]  [start, end) of each tile's run
 * Record slots are laid out view group, cluster, Gaussian, depth (ascending).
 * Fails with DGS_E_INVALID_ARG when there is no such call to export.
 */
DGS_API int dgs_debug_tile_lists(dgs_ctx *ctx, uint32_t *n_rec, uint32_t *n_ent, int32_t *n_view_groups,
                                 uint32_t *tiles, uint32_t *recs, uint32_t *depth_keys, uint32_t *depth_slots,
                                 uint32_t *entry_keys, uint32_t *entry_vals, uint32_t *ranges, dgs_stream stream);

/*
 * dgs_image_mse without allocation, for callers that cannot allocate: code that
 * runs inside a memory pool or arena it does not own, real-time loops where an
 * allocation (and the device synchronisation a free implies) is not allowed, or
 * hosts that forbid a library from touching the allocator.  The paper has no
 * counterpart; this is a deployment variant of the per-image MSE above.
 *   - No context: runs on the calling thread's current device and stream.
 *   - ref_index is [device] [S] (not host); an out-of-range index makes that
 *     image's mse (and its dL_dimages values) NaN instead of reading past refs.
 *     All other arguments as for dgs_image_mse.
 *   - Allocates nothing: no cudaMalloc / cudaFree / allocating library call.
 *     Its only scratch is a fixed file-scope device array of
 *     DGS_NOALLOC_MAX_PARTS doubles (512 KiB) that every GPU which loads the
 *     library holds until the process exits.  The call fails with
 *     DGS_E_SCRATCH, launching nothing, when S * ceil(H W / 1024) exceeds
 *     DGS_NOALLOC_MAX_PARTS, and with DGS_E_INVALID_ARG when S > 65535.
 *   - The first call on each device looks up the scratch array's device
 *     address (cudaGetSymbolAddress) with that device current and keeps it for
 *     the process; make that first call before any stream capture on the
 *     device.  The kept address belongs to the device's primary context, which
 *     the CUDA runtime uses: after cudaDeviceReset, or with another context
 *     current, the address is stale, so do not call this entry point then.
 *   - Every call on a device shares the one scratch array (each call rewrites
 *     all the partial sums it reads, so nothing needs clearing; the array keeps
 *     the last call's values).  Calls that overlap on the GPU, e.g. on two
 *     streams at once, race on it: serialise them.
 * Returns DGS_OK, DGS_E_INVALID_ARG, DGS_E_SCRATCH or DGS_E_CUDA (no message:
 * there is no context).
 */
DGS_API int dgs_image_mse_noalloc(const float *images, const float *refs, const int32_t *ref_index, int S,
                                  int n_refs, int H, int W, float weight, double *mse, double *psnr,
                                  float *dL_dimages, dgs_stream stream);

/*
 * Launch counters (host side).  The library counts every kernel it launches in
 * one process-wide counter; dgs_kernel_launches returns how many launches
 * (from any context, plan or the context-free entry point) happened since
 * this context was created or last reset.  Take the difference around a call
 * to count that call's launches, with no other library call in between.
 */
DGS_API int64_t dgs_kernel_launches(const dgs_ctx *ctx);
DGS_API void dgs_reset_kernel_launches(dgs_ctx *ctx);

/*
 * Launch profiler (library-wide).  While enabled, every named kernel launch is
 * bracketed by CUDA events recorded on its own stream.  dgs_profile_read
 * synchronizes the device, writes up to max_names aggregated rows -- name
 * (names + 32*k, NUL-terminated, 32 bytes each), total milliseconds and launch
 * count -- clears the records, and returns the number of rows (or < 0 on
 * error).  Enabling (or disabling) also clears.  Host pointers.
 */
DGS_API void dgs_profile_enable(dgs_ctx *ctx, int on);
DGS_API int dgs_profile_read(dgs_ctx *ctx, int max_names, char *names, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* DGS_H */
