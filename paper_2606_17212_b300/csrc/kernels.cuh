// Host-side launchers of the library's kernels (one translation unit each).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dgs_internal.cuh"

namespace dgs {

void launch_closure(const uint32_t *masks, int S, int words, int C, int L, const int32_t *vg_of_state,
                    uint8_t *depth, uint32_t *need, int force_full, int sms, cudaStream_t st);
void launch_layout_counts(const uint32_t *need, const int32_t *offs, int V, int C, uint32_t *counts, int sms,
                          cudaStream_t st);
void launch_project(const SceneDev &s, const ViewGroup *vgs, int V, const uint32_t *need, const uint32_t *recBase,
                    Rec *recs, uint32_t *keys, uint32_t *vals, int sms, cudaStream_t st);
// n_dev (optional): live count on the device, n is then the capacity.
// counts [n] tiles per depth-ordered record; bins [n] its tile rectangle
// (radix_sort_entries)
void launch_tile_count(const Rec *recs, const uint32_t *order, uint32_t n, int tiles_x, uint32_t tiles,
                       int tile_shift, uint32_t *counts, uint4 *bins, int sms, cudaStream_t st,
                       const uint32_t *n_dev = nullptr);
void launch_clamp_count(const uint32_t *total, uint32_t cap, uint32_t *out, uint32_t *flags, cudaStream_t st);
void launch_ranges(const uint32_t *keys, uint32_t n, uint2 *ranges, int sms, cudaStream_t st,
                   const uint32_t *n_dev = nullptr);
// *flag |= 1 when the n words of a and b differ anywhere (flag zeroed by the caller)
void launch_words_differ(const uint32_t *a, const uint32_t *b, size_t n, uint32_t *flag, int sms, cudaStream_t st);

struct RasterArgs {
    const Rec *recs;
    const uint32_t *evals;        // entry -> record slot, tile-major
    const uint2 *ranges;          // [V * tiles]
    const uint8_t *depth;         // [S][C]
    const int32_t *vg_of_state;   // [S]
    int S, C, W, H, tiles_x;
    uint32_t tiles;
    int tile_shift;               // sort tiles are 2^tile_shift pixels square
    int blocks_x;                 // 16 x 16 pixel blocks per image row (squared-error partials)
    uint32_t blocks;              // blocks per image
    float bg0, bg1, bg2;
    float *images;                // [S][H][W][3] or null
    const float *refs;            // [n_refs][H][W][3] or null (MSE epilogue)
    const int32_t *ref_of_state;  // [S]
    double *partial;              // [S][blocks] FP64 squared-error partial sums per 16 x 16 pixel block
    int img_s0;                   // images hold states img_s0, img_s0 + 1, ...
    uint32_t *stop;               // [S][tiles] or null: run prefix staged while the state had a live pixel
    float *dL;                    // [S][H][W][3] or null: with refs, dL/dimage = gscale (image - ref)
    float gscale;
};
// Work queue of the persistent forward raster: (view group, tile) pairs in
// descending cost order, each expanded into that view group's state groups.
struct WorkQueue {
    const uint32_t *tile_order;    // [V * tiles] view group * tiles + tile, costliest first
    const uint32_t *item_offsets;  // [V * tiles + 1] first work item of each tile_order entry
    uint32_t n_vt;                 // V * tiles
    uint32_t n_items;
    const int32_t *group_first;    // [n_groups] first index into state_order
    const int32_t *group_count;    // [n_groups] states in the group (<= G)
    const int32_t *vg_group_base;  // [V] first group of each view group
    const int32_t *state_order;    // [S] states sorted by view group
    uint32_t *counter;             // zeroed before the launch
    // Explicit work list (tile reuse), used when item_first is set: item k
    // renders states list_state[item_first[k] .. + item_count[k]) on the
    // view-group tile list_vt[item_first[k]]; the item count is *n_items_dev.
    const uint32_t *item_first = nullptr;
    const uint32_t *item_count = nullptr;
    const uint32_t *list_vt = nullptr;
    const uint32_t *list_state = nullptr;
    const uint32_t *n_items_dev = nullptr;
};
// G = states composited per staged batch (1, 2, 4 or 8); blocks = persistent grid.
// persistent grid: sms x the resident blocks per SM of the instantiation launched
void launch_raster_fwd(const RasterArgs &a, const WorkQueue &q, int G, int sms, cudaStream_t st);
// query (once) the resident blocks per SM of every forward instantiation, so
// that no launch inside a stream capture needs a runtime query
void raster_fwd_query_occupancy();
void launch_tile_costs(const uint2 *ranges, uint32_t n, uint32_t *keys, uint32_t *vals, int sms, cudaStream_t st);
void launch_item_counts(const uint32_t *tile_order, uint32_t n, uint32_t tiles, const int32_t *vg_ngroups,
                        uint32_t *counts, int sms, cudaStream_t st);

struct RasterBwdArgs {
    RasterArgs f;
    const float *dL_dimg;         // [S][H][W][3]
    const float *img_fwd;         // [S][H][W][3] the forward's images, or null (recomputed)
    float4 *rec_grad;             // [nRec][3] pixel moments of dL/dpower (d = m - pixel centre) and colour:
                                  // (S dx, S dy, S dx^2, S dx dy), (S dy^2, S 1, dL/dr, dL/dg), (dL/db, -, -, -)
};
void launch_raster_bwd(const RasterBwdArgs &a, int sms, cudaStream_t st);
// Several scenes in one launch (device arrays of per-job arguments).  Forward:
// queues[k] as launch_raster_fwd's, job k's items [item_off[k], item_off[k + 1])
// of one shared zeroed counter, every job with images, no MSE, tile shift
// tile_shift.  Adjoint: job k's items [item_off[k], item_off[k + 1]) with
// item_off[k + 1] - item_off[k] = raster_bwd_items(jobs[k].f), forward images given.
void launch_raster_fwd_multi(const RasterArgs *args, const WorkQueue *queues, const uint32_t *item_off, int n_jobs,
                             uint32_t *counter, int tile_shift, int sms, cudaStream_t st);
size_t raster_bwd_items(const RasterArgs &a);
void launch_raster_bwd_multi(const RasterBwdArgs *jobs, const size_t *item_off, int n_jobs, size_t total_items,
                             cudaStream_t st);

void launch_mse_reduce(const double *partial, int S, int parts, double inv_count, double *mse, double *psnr,
                       cudaStream_t st);
// parts = mse_parts(H, W) partial sums per image
void launch_image_mse(const float *images, const float *refs, const int32_t *ref_index, int S, int H, int W,
                      float weight, double *partial, int parts, float *dL, cudaStream_t st);

// Counterfactual utility (Eq. 3 / Eq. 4): paired masks, per-group statistics.
void launch_pair_masks(const uint32_t *ctx_masks, const int2 *groups, int G, int M, int words, int L,
                       uint32_t *out, int sms, cudaStream_t st);
void launch_group_stats(const double *mse, int G, int M, double alpha, double beta, double q, double *delta,
                        double *stats, cudaStream_t st);

// Eq. 2 objective (objective.cu).
typedef dgs_objective_params ObjectiveParams;
int objective_tiles(int H, int W, int *tiles_x);
size_t objective_smem(int S);
void launch_ssim_fwd(const float *images, const float *refs, const int32_t *ref_index, int S, int H, int W,
                     float *d_mx, float *d_exx, float *d_exy, double *part, cudaStream_t st);
void launch_temporal(const float *images, const float *refs, const int32_t *ref_index, const int2 *pairs,
                     int n_pairs, int H, int W, double *tpart, int chunks, cudaStream_t st);
int objective_prepare();   // 0 on success
int launch_objective(const double *part, int n_tiles, const double *tpart, int chunks, int n_t, const int2 *pm,
                     int n_m, const int32_t *anchors, int n_a, int S, double inv_vals, const ObjectiveParams &prm,
                     double *D, double *weight, double *loss, cudaStream_t st);
void launch_objective_grad(const float *images, const float *refs, const int32_t *ref_index, int S, int H, int W,
                           const float *d_mx, const float *d_exx, const float *d_exy, const double *weight,
                           float ssim_weight, float tscale, const int32_t *toff, const int2 *tlist, float *dL,
                           cudaStream_t st);

// Tile reuse across states (share.cu).
void launch_first_clusters(const Rec *recs, const uint32_t *evals, const uint2 *ranges, uint32_t n_vt, int C,
                           uint32_t *ord_c, uint32_t *ord_fp, int sms, cudaStream_t st);
void launch_pairs_init(const uint32_t *vt_off, uint32_t n_vt, uint32_t n_pairs, uint32_t tiles,
                       const int32_t *vg_first, const int32_t *state_order, uint32_t *pvt, uint32_t *pst,
                       uint8_t *pk, int sms, cudaStream_t st);
void launch_segments(const uint32_t *keys, const uint32_t *n_dev, size_t n_cap, uint2 *seg, int sms,
                     cudaStream_t st);
// keys: [n_cap] u64 scratch
void launch_share_group(const uint2 *seg, uint32_t n_vt, const uint32_t *pvt, const uint32_t *pst,
                        const uint8_t *pk, const uint32_t *n_dev, size_t n_cap, const uint32_t *ord_c,
                        const uint8_t *depth, int C, unsigned long long *keys, uint32_t *prep, int sms,
                        cudaStream_t st);
void launch_rep_flags(const uint32_t *pst, const uint32_t *prep, const uint32_t *n_dev, size_t n_cap,
                      uint32_t *flag, int sms, cudaStream_t st);
void launch_compact_pairs(const uint32_t *flag, const uint32_t *pos, const uint32_t *n_dev, size_t n_cap,
                          const uint32_t *pvt, const uint32_t *pst, const uint8_t *pk, uint32_t *ovt,
                          uint32_t *ost, uint8_t *ok, int sms, cudaStream_t st);
void launch_item_lists(const uint32_t *lvt, const uint2 *seg, const uint32_t *n_dev, size_t n_cap, int G,
                       uint32_t *flag, uint32_t *pos, uint32_t *n_items_dev, void *scan_ws, uint32_t *item_first,
                       uint32_t *item_count, int sms, cudaStream_t st);
void launch_share_resolve(const uint32_t *pvt, const uint32_t *pst, uint8_t *pk, const uint32_t *prep,
                          const uint32_t *n_dev, size_t n_cap, const TileGeom &geo, const uint32_t *ord_c,
                          const uint32_t *ord_fp, const uint8_t *depth, int C, const uint32_t *stop,
                          double *partial, uint32_t *pending, int sms, cudaStream_t st);

// rec_cap: record slots of rec_grad (the per-record mean gradients of the
// affine, g.rec_gmu, are cleared over it)
// rec_grad: read, then cleared record by record (every record of [0, rec_cap) is zero afterwards)
void launch_project_bwd(const SceneDev &s, const ViewGroup *vgs, int V, const uint32_t *need,
                        const uint32_t *recBase, float4 *rec_grad, const GradDev &g, size_t rec_cap,
                        int sms, cudaStream_t st);

}  // namespace dgs
