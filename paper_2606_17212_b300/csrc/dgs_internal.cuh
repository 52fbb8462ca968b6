// Internal declarations shared by the library's CUDA translation units.
//
// Data layout in HBM (all produced and consumed by the kernels of this library):
//   depth   [S][C]  u8     delivered depth of cluster c in state s (closure)
//   need    [V][C]  u32    bit d set when some state of view group v renders
//                          cluster c at depth d (d = 1..L); bit 0 unused
//   recBase [V*C+1] u32    first record slot of (v, c); records of (v, c) are
//                          laid out Gaussian-major, depth-minor
//   Rec     [nRec]  48 B   one projected variant (view group, Gaussian, depth)
//   recKey  [nRec]  u32    float bits of camera depth (0xFFFFFFFF = culled)
//   bins    [nRec]  uint4  tile rectangle of each record in depth order (first
//                          tile key, tile columns, slot): the entries' source
//   entries [nEnt]  u32 key (v * tiles + tile), u32 value (record slot)
//   ranges  [V*T]   uint2  [start, end) of each (view group, tile) run
//   partial [S][B]  f64    squared-error partial of each state and 16x16 pixel block
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dgs.h"

namespace dgs {

// Sort tiles (the unit of binning, sorting and tile ranges) are 2^tile_shift
// pixels square, tile_shift 4 or 5 (16 or 32 px), chosen per batch.  Raster
// warps work on 16-pixel-wide regions inside a tile, and per-state squared-
// error partials are kept per BLOCK x BLOCK pixel block of the image whatever
// the tile size, so every tile size gives the same bits.
constexpr int BLOCK = 16;                // pixel block of the squared-error partials; raster region width
constexpr int MIN_TILE_SHIFT = 4, MAX_TILE_SHIFT = 5;

// Tile and block grids of one image size.
struct TileGeom {
    int tiles_x, tiles_y, tile_shift;    // sort tiles of 2^tile_shift pixels
    int blocks_x, blocks_y;              // 16 x 16 pixel blocks
    uint32_t tiles, blocks;
};
// The 16 x 16 pixel blocks of sort tile `tile`: columns [bx0, bx1), rows [by0, by1).
__host__ __device__ inline void tile_blocks(const TileGeom &g, uint32_t tile, int &bx0, int &bx1, int &by0, int &by1)
{
    const int r = 1 << (g.tile_shift - 4), tx = (int)(tile % (uint32_t)g.tiles_x), ty = (int)(tile / (uint32_t)g.tiles_x);
    bx0 = tx * r; by0 = ty * r;
    bx1 = bx0 + r < g.blocks_x ? bx0 + r : g.blocks_x;
    by1 = by0 + r < g.blocks_y ? by0 + r : g.blocks_y;
}
constexpr int MAX_CLUSTERS = 1024;
constexpr int MAX_LAYERS = 8;

// Tile reuse across states (share.cu): group keys hold the delivered depths
// (4 bits each, MAX_LAYERS <= 15) of up to SHARE_MAX_K clusters; the first
// SHARE_ORDER = SHARE_MAX_K + 1 clusters of each run are kept; one block's
// hash table has SHARE_TABLE slots.
constexpr int SHARE_MAX_K = 15;
constexpr int SHARE_ORDER = SHARE_MAX_K + 1;
constexpr int SHARE_TABLE = 8192;
static_assert(MAX_LAYERS <= 15, "depths are packed in 4 bits");

// Records hold the conic (A = xx, B = xy, C = yy) pre-scaled for base-2
// exponents: a2 = K_AC A, b2 = K_B B, c2 = K_AC C, so that a pixel's
// log2(e) * power = a2 dx^2 + b2 dx dy + c2 dy^2 and alpha = o 2^(that)
// (e^power == 2^(log2(e) power)); the raster stages records by plain copies.
constexpr float LOG2E = 1.4426950408889634f;
constexpr float K_AC = -0.5f * LOG2E;
constexpr float K_B = -LOG2E;
constexpr float INV_K_AC = 1.0f / K_AC, INV_K_B = 1.0f / K_B;

// One projected Gaussian variant, 48 bytes, read as three float4.
struct __align__(16) Rec {
    float mx, my, A, B;        // mean2d, scaled conic a2 (xx), b2 (xy)
    float C, o, r, g;          // scaled conic c2 (yy), opacity, colour r, g
    float b;                   // colour b
    uint32_t bx;               // xlo | xhi << 16   (inclusive pixel range)
    uint32_t by;               // ylo | yhi << 16
    uint32_t cd;               // cluster | clamp << 11 | depth << 12 | view group << 16 | boxed << 31
                               // (depth 0 = culled; boxed: pixels need the box test, the 3-sigma box
                               // clips the alpha box; clamp: alpha can reach the 0.99 clamp)
};
static_assert(sizeof(Rec) == 48, "record layout");
constexpr uint32_t REC_CLUSTER = 0x3ffu;     // cluster field of Rec::cd (MAX_CLUSTERS = 1024)
constexpr uint32_t REC_CLAMP = 1u << 11;     // Rec::cd flag: o 2^p2 can reach the 0.99 clamp
static_assert(MAX_CLUSTERS <= 1024, "cluster field");

// Per view group (camera, time) parameters, uploaded by the planner.
struct ViewGroup {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float time;
    float campos[3];
    int32_t width, height;
    int32_t cam;
    int32_t pad;
};

struct SceneDev {
    int n, C, L, sh, R, nc, K;
    const int32_t *offs;
    const float *mu0, *u, *ls, *quat, *logit, *colour, *res;
    const float *affine;       // [C][aT][12] cluster affine keyframes, or null (identity)
    int aT;
    const int16_t *res_q;      // [L-1][n][K] refinement symbols (res_mode 1)
    const float *res_step;     // [L-1][K] quantization steps (res_mode 1, 2)
    int res_mode;              // 0 float refinements, 1 symbols x step, 2 quantized on the fly
};

struct GradDev {
    float *mu0, *u, *ls, *quat, *logit, *colour, *res, *affine;
    float *rec_gmu;            // [nRec][3] per-record mean gradient (only with an affine)
    float *res_step;           // [L-1][K] step gradients (res_mode 2)
    float *gq;                 // [L-1][n][K] gradients of the decoded refinements (res_mode 2 workspace)
};

// ------------------------------------------------------------------ MSE
// Per-image squared error (Eq. 3's D = MSE): each pixel's squared RGB error is
// formed in FP32 with fixed rounding and the sum over pixels is accumulated in
// FP64, in partial sums of MSE_CHUNK_PIX pixels.  B300 issues FP64 at a small
// fraction of its FP32 rate, so FP64 is spent only where precision needs it:
// on the sum of up to millions of terms, not on three differences per pixel
// (relative error of one pixel's term below 5 * 2^-24 to first order: one
// rounding in each difference, squared, plus the multiply and two fused adds).
constexpr int MSE_CHUNK_PIX = 1024;
__host__ __device__ inline int mse_parts(int H, int W)
{
    return (int)(((size_t)H * (size_t)W + MSE_CHUNK_PIX - 1) / MSE_CHUNK_PIX);
}
__device__ __forceinline__ float pixel_sq_err(float x0, float x1, float x2, float y0, float y1, float y2)
{
    const float d0 = __fsub_rn(x0, y0), d1 = __fsub_rn(x1, y1), d2 = __fsub_rn(x2, y2);
    return __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
}

// ------------------------------------------------------------------ launches
// Every kernel launch of the library goes through this counter so that the
// number of device launches per call can be reported.
void count_launch();
// Optional per-kernel timing: when profiling is on, prof_begin/prof_end record
// CUDA events on the launching stream around a named launch.
void prof_begin(const char *name, cudaStream_t st);
void prof_end(cudaStream_t st);
struct ProfScope {
    cudaStream_t st;
    ProfScope(const char *name, cudaStream_t s) : st(s) { prof_begin(name, s); }
    ~ProfScope() { prof_end(st); }
};

// Exclusive scan of n u32 values (in place allowed: out may equal in).
// total_out [device] receives the sum when not null.  Uses ws_bytes of scratch
// from `ws` (query with scan_workspace_bytes).
size_t scan_workspace_bytes(size_t n);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total_out,
                               void *ws, cudaStream_t st);

// Stable LSD radix sort of (key, value) u32 pairs on key bits [0, bits).
// Ping-pongs between (k0, v0) and (k1, v1); returns in *result_in_alt whether
// the sorted data ended in (k1, v1).  ws from radix_workspace_bytes(n, V)
// (V = 0 for the plain sort).  With n_dev the live count is read on the
// device (n is then the capacity), so the launch sequence does not depend on
// it (capture-safe).
size_t radix_workspace_bytes(size_t n, int V = 0);
// prof: the profiler name of the passes (one name per kind of sort)
cudaError_t radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, size_t n,
                             int bits, void *ws, cudaStream_t st, bool *result_in_alt,
                             const uint32_t *n_dev = nullptr, const char *prof = "radix_pass");

// The same, segment by segment: items [start(v), start(v + 1)) with start(v) =
// seg_start[v * stride] (device, non-decreasing, v = 0 .. V; start(V) is the
// live count) are sorted stably among themselves and stay in their segment.
// Records segmented by view group come out in (view group, key) order.
// With kept (device [V + 1]) the items whose key is 0xFFFFFFFF (culled
// records) are dropped: kept receives the compacted segment starts, kept[V]
// the number of items left, and only that many sorted items are written.
cudaError_t radix_sort_pairs_seg(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, size_t n_cap,
                                 const uint32_t *seg_start, uint32_t stride, int V, int bits, void *ws,
                                 cudaStream_t st, bool *result_in_alt, const char *prof, uint32_t *kept = nullptr);

// Tile entries of records sorted by (view group, depth), sorted stably by
// (view group, tile), without an unsorted copy.  The records of view group v
// are [rec_start[v * rec_stride], rec_start[(v + 1) * rec_stride]), so their
// entries form one segment and only the tile index (bits [0, bits) of key -
// v * tiles) needs sorting.  The first pass generates every entry from the
// record's tile rectangle, bins[j] = (key of its first tile = view group *
// tiles + ty0 * tiles_x + tx0, tile columns tw, record slot, 0), record j
// owning entries [toffs[j], toffs[j] + counts[j]).  Entries at or past e_cap
// (or *nent_dev) are dropped; nrec_dev / nent_dev as n_dev above.  The
// (k0, v0) / (k1, v1) convention is radix_sort_pairs'; ws from
// radix_workspace_bytes(e_cap, V).  When one pass sorts the tiles (bits <= 8)
// and ranges ([V * tiles], device) is given, the [start, end) of every
// (view group, tile) run is written from that pass's digit table and
// *ranges_done is set.
cudaError_t radix_sort_entries(const uint4 *bins, const uint32_t *toffs, const uint32_t *counts, uint32_t n_rec,
                               const uint32_t *nrec_dev, const uint32_t *rec_start, uint32_t rec_stride, int V,
                               int tiles_x, uint32_t tiles, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                               size_t e_cap, const uint32_t *nent_dev, int bits, void *ws, cudaStream_t st,
                               bool *result_in_alt, int sms, uint2 *ranges = nullptr, bool *ranges_done = nullptr);

}  // namespace dgs
