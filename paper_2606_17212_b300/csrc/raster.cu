// Tile rasterization of delivery states: forward compositing with an optional
// fused FP64 squared-error epilogue, and the adjoint compositing kernel.
//
// One 128-thread block renders one 16x16 tile of one state; every thread owns
// two vertically adjacent pixels, every warp an 8x8 quadrant of the tile.  The tile's run of
// the batch-wide sorted entry list holds every depth variant any state of the
// view group needs; each batch of 256 entries is staged in shared memory
// keeping only the variants this state renders (variant depth == the state's
// delivered depth of the Gaussian's cluster), compacted in order, and each
// warp then walks only the staged Gaussians whose pixel box and alpha >= 1/255
// ellipse reach its quadrant.
// Filtering a sorted run keeps it sorted, so every pixel sees exactly the
// (depth, Gaussian) order it would see alone: batched == per-state, bit for bit.
//
// Per pixel and Gaussian the work is a handful of FP32 ops and one MUFU exp:
// these kernels are ALU/issue bound, not HBM bound.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr int RT = 128;               // threads per raster block
constexpr int RW = RT / 32;           // warps per block; warp w owns rows 4w..4w+3 of the tile
constexpr int BATCH = 256;            // entries staged per batch (two per thread)

// Records hold the conic pre-scaled (a2 = K_AC A, b2 = K_B B, c2 = K_AC C), so
// one pixel's exponent in base 2, p2 = log2(e) * power = a2 dx^2 + b2 dx dy +
// c2 dy^2, costs two fused multiply-adds per pixel on top of two per-entry
// products shared by the thread's two pixels, and alpha = o 2^p2.

// 2^x on the MUFU unit (ex2.approx.ftz: relative error ~2^-22, tiny results flush to 0)
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// p2 at vertical offset dy, given the entry's per-column terms u = a2 dx^2 and v = b2 dx
__device__ __forceinline__ float log2_power(float u, float v, float c2, float dy)
{
    return __fmaf_rn(__fmaf_rn(c2, dy, v), dy, u);
}

struct Staged {
    float4 r0[BATCH];                 // mx, my, a2, b2 (scaled conic)
    float4 r1[BATCH];                 // c2, o, r, g
    float4 r2[BATCH];                 // b, box x, box y, cd
    int4 box[BATCH];                  // xlo, xhi - xlo, ylo, yhi - ylo
    uint32_t slot[BATCH];
    uint8_t list[RW][BATCH];          // per-warp indices of staged entries reaching its rows
    int cnt[RW];
    int wcnt[2][RW];
};

__device__ __forceinline__ int4 unpack_box(const float4 &r2)
{
    const uint32_t bx = __float_as_uint(r2.y), by = __float_as_uint(r2.z);
    const int x0 = (int)(bx & 0xffffu), y0 = (int)(by & 0xffffu);
    return make_int4(x0, (int)(bx >> 16) - x0, y0, (int)(by >> 16) - y0);
}

// Can Gaussian (mx, my, conic A B C, opacity o) reach alpha >= 1/255 at some
// pixel centre of the rectangle [x0, x1] x [y0, y1]?  alpha >= 1/255 needs
// q(d) = A dx^2 + 2 B dx dy + C dy^2 <= rho = 2 ln(255 o) with d = p - m.  The
// minimum of the convex q over the rectangle is 0 when it holds the mean, else
// it lies on an edge (1-D quadratic, clamped vertex).  rho is inflated by
// 1e-3 relative + 1e-3 so FP32 rounding never drops a pixel that composites
// (the 1e-3 also covers undoing the records' scaling of the conic);
// skipping a Gaussian that stays below 1/255 on the whole strip changes nothing.
__device__ __forceinline__ bool ellipse_meets_rect(const float4 &r0, const float4 &r1, float x0, float x1,
                                                   float y0, float y1)
{
    const float A = r0.z * INV_K_AC, B = r0.w * INV_K_B, C = r1.x * INV_K_AC, o = r1.y;   // records: scaled
    const float rho = fmaf(2.0f * __logf(255.0f * o), 1.001f, 1e-3f);
    const float X0 = x0 - r0.x, X1 = x1 - r0.x, Y0 = y0 - r0.y, Y1 = y1 - r0.y;
    if (X0 <= 0.0f && X1 >= 0.0f && Y0 <= 0.0f && Y1 >= 0.0f) return true;
    float best = 3.4e38f;
    // vertical edges dx = X: minimise over dy in [Y0, Y1]
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float X = e ? X1 : X0;
        const float dy = fminf(fmaxf(__fdividef(-B * X, C), Y0), Y1);
        best = fminf(best, A * X * X + 2.0f * B * X * dy + C * dy * dy);
    }
    // horizontal edges dy = Y: minimise over dx in [X0, X1]
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float Y = e ? Y1 : Y0;
        const float dx = fminf(fmaxf(__fdividef(-B * Y, A), X0), X1);
        best = fminf(best, A * dx * dx + 2.0f * B * dx * Y + C * Y * Y);
    }
    return best <= rho;
}

// pixel coordinate v lies in [lo, lo + w] (w >= 0): one subtract, one unsigned compare
__device__ __forceinline__ bool in_range(int v, int lo, int w) { return (unsigned)(v - lo) <= (unsigned)w; }

// Warp w of a tile block owns the 8x8 quadrant (w & 1, w >> 1) of the tile;
// lane l owns column l & 7 and rows 2 (l >> 3), 2 (l >> 3) + 1 of it.  Over the
// workloads' Gaussians an 8x8 quadrant meets ~8% fewer (pixel, Gaussian) pairs
// than a 16x4 strip after culling (less perimeter for the same 64 pixels).
struct Quad {
    int c0, r0;                       // first column and row of the warp's quadrant
    int px, py0;                      // this lane's column and first row
};
__device__ __forceinline__ Quad quad_of(int tx, int ty, int w, int lane)
{
    Quad q;
    q.c0 = tx * TILE + (w & 1) * 8;
    q.r0 = ty * TILE + (w >> 1) * 8;
    q.px = q.c0 + (lane & 7);
    q.py0 = q.r0 + 2 * (lane >> 3);
    return q;
}

// Does the staged entry j reach quadrant (c0, r0): box overlap, then the ellipse test.
__device__ __forceinline__ bool reaches_quad(const int4 &bx, const float4 &r0, const float4 &r1, int c0, int r0q)
{
    return bx.x <= c0 + 7 && bx.x + bx.y >= c0 && bx.z <= r0q + 7 && bx.z + bx.w >= r0q &&
           ellipse_meets_rect(r0, r1, (float)c0 + 0.5f, (float)c0 + 7.5f, (float)r0q + 0.5f, (float)r0q + 7.5f);
}

// Stage entries [start, min(start + BATCH, end)) of the tile run, keeping the
// variants this state renders, compacted in order; then build each warp's list
// of kept entries whose box reaches the warp's rows.  Returns the kept count.
__device__ __forceinline__ int stage_batch(const Rec *__restrict__ recs, const uint32_t *__restrict__ evals,
                                           const uint8_t *sdep, uint32_t start, uint32_t end, const Quad &wq,
                                           Staged &sm)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    bool keep[2];
    float4 x0[2], x1[2], x2[2];
    uint32_t slot[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t e = start + (uint32_t)(h * RT + t);
        keep[h] = false;
        x0[h] = x1[h] = x2[h] = make_float4(0, 0, 0, 0);
        slot[h] = 0;
        if (e < end) {
            slot[h] = __ldg(evals + e);
            const float4 *p = reinterpret_cast<const float4 *>(recs + slot[h]);
            x2[h] = __ldg(p + 2);
            const uint32_t cd = __float_as_uint(x2[h].w);
            keep[h] = ((cd >> 12) & 0xfu) == (uint32_t)sdep[cd & 0xfffu];
            if (keep[h]) { x0[h] = __ldg(p); x1[h] = __ldg(p + 1); }
        }
    }
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t b0 = __ballot_sync(0xffffffffu, keep[0]), b1 = __ballot_sync(0xffffffffu, keep[1]);
    if (lane == 0) { sm.wcnt[0][w] = __popc(b0); sm.wcnt[1][w] = __popc(b1); }
    __syncthreads();
    int base0 = 0, tot0 = 0, base1 = 0, tot1 = 0;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        const int c0 = sm.wcnt[0][k], c1 = sm.wcnt[1][k];
        base0 += (k < w) ? c0 : 0;
        tot0 += c0;
        base1 += (k < w) ? c1 : 0;
        tot1 += c1;
    }
    if (keep[0]) {
        const int pos = base0 + __popc(b0 & lt);
        sm.r0[pos] = x0[0]; sm.r1[pos] = x1[0]; sm.r2[pos] = x2[0]; sm.slot[pos] = slot[0];
        sm.box[pos] = unpack_box(x2[0]);
    }
    if (keep[1]) {
        const int pos = tot0 + base1 + __popc(b1 & lt);
        sm.r0[pos] = x0[1]; sm.r1[pos] = x1[1]; sm.r2[pos] = x2[1]; sm.slot[pos] = slot[1];
        sm.box[pos] = unpack_box(x2[1]);
    }
    __syncthreads();
    const int nk = tot0 + tot1;
    // warp w keeps staged entries whose box and alpha >= 1/255 ellipse reach its quadrant
    int n = 0;
    for (int j0 = 0; j0 < nk; j0 += 32) {
        const int j = j0 + lane;
        bool hit = false;
        if (j < nk) {
            const int4 bx = sm.box[j];
            hit = reaches_quad(bx, sm.r0[j], sm.r1[j], wq.c0, wq.r0);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) sm.list[w][n + __popc(bal & lt)] = (uint8_t)j;
        n += __popc(bal);
    }
    if (lane == 0) sm.cnt[w] = n;
    __syncwarp();
    return nk;
}

// One pixel's front-to-back state.
struct Pix {
    float T, c0, c1, c2;
    bool done;
};

// Composite one staged entry into one pixel, given its base-2 exponent p2;
// branch free: an entry the pixel skips (outside the box, power > 0,
// alpha < 1/255, or the pixel already stopped) gets alpha = 0, and the entry
// at which T (1 - alpha) would drop below 1e-4 stops the pixel without being
// added; both leave T and the colour bit-identical.  Returns true at the stop.
__device__ __forceinline__ bool composite(Pix &p, float p2, float o, float r, float g, float b, bool inb)
{
    const float a0 = fminf(0.99f, __fmul_rn(o, ex2(p2)));
    const float alpha = (inb && !p.done && p2 <= 0.0f && a0 >= (1.0f / 255.0f)) ? a0 : 0.0f;
    const float Tn = __fmul_rn(p.T, __fsub_rn(1.0f, alpha));
    const bool stop = Tn < 1e-4f;
    const float wgt = stop ? 0.0f : __fmul_rn(alpha, p.T);
    p.c0 = __fmaf_rn(r, wgt, p.c0);
    p.c1 = __fmaf_rn(g, wgt, p.c1);
    p.c2 = __fmaf_rn(b, wgt, p.c2);
    p.T = stop ? p.T : Tn;
    p.done = p.done || stop;
    return stop;
}

// Does the entry need the per-pixel box test?  Only where its 3-sigma box
// clips the alpha >= 1/255 box (record flag); elsewhere the box holds every
// pixel the alpha test keeps and the test is skipped.
__device__ __forceinline__ bool is_boxed(const float4 &r2) { return (__float_as_uint(r2.w) >> 31) != 0u; }

// Per-entry column terms for a thread's pixel column: u = a2 dx^2, v = b2 dx.
__device__ __forceinline__ void column_terms(const float4 &r0, float pcx, float &dx, float &u, float &v)
{
    dx = __fsub_rn(r0.x, pcx);
    u = __fmul_rn(__fmul_rn(r0.z, dx), dx);
    v = __fmul_rn(r0.w, dx);
}

__device__ __forceinline__ void load_depth_row(const uint8_t *depth, int s, int C, uint8_t *sdep)
{
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdep[c] = depth[(size_t)s * C + c];
}

// Stage entries [start, min(start + BATCH, end)) of the tile run, keeping the
// variants that at least one of the group's states renders (variant depth ==
// that state's delivered depth of the cluster), compacted in order.  A view
// group's run holds every depth variant its states need; dropping the ones no
// state of this group renders keeps them out of shared memory and out of
// every warp's list scan.  Returns the kept count.
template <int G>
__device__ __forceinline__ int stage_kept(const Rec *__restrict__ recs, const uint32_t *__restrict__ evals,
                                          const uint8_t (*sdep)[MAX_CLUSTERS], const int (&sid)[G], uint32_t start,
                                          uint32_t end, Staged &sm)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    bool keep[2];
    uint32_t slot[2];
    // the keep decision needs only the record's cluster / depth word; the kept
    // records are read whole after the compaction (the same lines, from L1)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t e = start + (uint32_t)(h * RT + t);
        keep[h] = false;
        slot[h] = 0;
        if (e < end) {
            slot[h] = __ldg(evals + e);
            const uint32_t cd = __ldg(reinterpret_cast<const uint32_t *>(recs + slot[h]) + 11);
            const uint32_t d = (cd >> 12) & 0xfu, c = cd & 0xfffu;
#pragma unroll
            for (int g = 0; g < G; ++g) keep[h] |= sid[g] >= 0 && d == (uint32_t)sdep[g][c];
        }
    }
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t b0 = __ballot_sync(0xffffffffu, keep[0]), b1 = __ballot_sync(0xffffffffu, keep[1]);
    if (lane == 0) { sm.wcnt[0][w] = __popc(b0); sm.wcnt[1][w] = __popc(b1); }
    __syncthreads();
    int base0 = 0, tot0 = 0, base1 = 0, tot1 = 0;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        const int c0 = sm.wcnt[0][k], c1 = sm.wcnt[1][k];
        base0 += (k < w) ? c0 : 0;
        tot0 += c0;
        base1 += (k < w) ? c1 : 0;
        tot1 += c1;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!keep[h]) continue;
        const int pos = h ? tot0 + base1 + __popc(b1 & lt) : base0 + __popc(b0 & lt);
        const float4 *p = reinterpret_cast<const float4 *>(recs + slot[h]);
        const float4 r2 = __ldg(p + 2);
        sm.r0[pos] = __ldg(p);
        sm.r1[pos] = __ldg(p + 1);
        sm.r2[pos] = r2;
        sm.box[pos] = unpack_box(r2);
    }
    __syncthreads();
    return tot0 + tot1;
}

// Warp w's list of staged entries that state row `dep` renders (variant depth
// == the state's delivered depth of the entry's cluster) and whose box meets
// the warp's rows.  Returns the list length (same in all lanes).
__device__ __forceinline__ int warp_list(const Staged &sm, uint8_t *list, int nk, const uint8_t *dep,
                                         const Quad &wq)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int n = 0;
    for (int j0 = 0; j0 < nk; j0 += 32) {
        const int j = j0 + lane;
        bool hit = false;
        if (j < nk) {
            const uint32_t cd = __float_as_uint(sm.r2[j].w);
            const int4 bx = sm.box[j];
            hit = ((cd >> 12) & 0xfu) == (uint32_t)dep[cd & 0xfffu] && reaches_quad(bx, sm.r0[j], sm.r1[j], wq.c0, wq.r0);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) list[n + __popc(bal & lt)] = (uint8_t)j;
        n += __popc(bal);
    }
    __syncwarp();
    return n;
}

// Persistent forward raster.  Each block repeatedly takes a work item (one
// tile of one view group and a group of up to G states of that view group),
// stages the tile's Gaussians once per batch (the variants some state of the
// group renders) and composites them for every state of the group; items come
// costliest tile first from an atomic counter.
// Per pixel and state the arithmetic is composite(), exactly as for a single
// state, so grouping never changes a bit of the result.
template <int G, bool WRITE, bool MSE, bool LIST>
__global__ void __launch_bounds__(RT, G <= 2 ? 8 : 1) k_raster_fwd(RasterArgs a, WorkQueue q)
{
    __shared__ Staged sm;
    __shared__ uint8_t sdep[G][MAX_CLUSTERS];
    __shared__ double wsum[G][RW];
    __shared__ uint32_t s_item;
    __shared__ uint32_t s_stop[G];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t n_items = LIST ? *q.n_items_dev : q.n_items;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(q.counter, 1u);
        if (LIST && threadIdx.x < G) s_stop[threadIdx.x] = 0u;
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) break;
        uint32_t vt;
        int sid[G];
        if (LIST) {
            const uint32_t first = q.item_first[item], cnt = q.item_count[item];
            vt = q.list_vt[first];
#pragma unroll
            for (int g = 0; g < G; ++g) sid[g] = (uint32_t)g < cnt ? (int)q.list_state[first + g] : -1;
        } else {
            // largest j with item_offsets[j] <= item
            uint32_t lo = 0, hi = q.n_vt - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (q.item_offsets[mid] <= item) lo = mid; else hi = mid - 1;
            }
            vt = q.tile_order[lo];
            const int grp = q.vg_group_base[vt / a.tiles] + (int)(item - q.item_offsets[lo]);
            const int first = q.group_first[grp], cnt = q.group_count[grp];
#pragma unroll
            for (int g = 0; g < G; ++g) sid[g] = g < cnt ? q.state_order[first + g] : -1;
        }
        const int tile = (int)(vt % a.tiles);
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (sid[g] >= 0)
                for (int c = threadIdx.x; c < a.C; c += RT) sdep[g][c] = a.depth[(size_t)sid[g] * a.C + c];
        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        const Quad wq = quad_of(tx, ty, w, lane);
        const int px = wq.px, py0 = wq.py0, py1 = py0 + 1;
        const bool in0 = px < a.W && py0 < a.H, in1 = px < a.W && py1 < a.H;
        const float pcx = (float)px + 0.5f, pcy0 = (float)py0 + 0.5f, pcy1 = (float)py1 + 0.5f;
        const uint2 rg = a.ranges[vt];
        Pix p[G][2];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            p[g][0] = {1.0f, 0.0f, 0.0f, 0.0f, !in0 || sid[g] < 0};
            p[g][1] = {1.0f, 0.0f, 0.0f, 0.0f, !in1 || sid[g] < 0};
        }
        for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
            bool alive = false;
#pragma unroll
            for (int g = 0; g < G; ++g) alive |= !(p[g][0].done && p[g][1].done);
            if (__syncthreads_count(alive) == 0) break;
            const int nk = stage_kept<G>(a.recs, a.evals, sdep, sid, start, rg.y, sm);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (!__any_sync(0xffffffffu, !(p[g][0].done && p[g][1].done))) continue;
                // the state still has a live pixel: this batch's clusters decide its result
                if (LIST && lane == 0) atomicMax(&s_stop[g], min(start + (uint32_t)BATCH, rg.y) - rg.x);
                const int n = warp_list(sm, sm.list[w], nk, sdep[g], wq);
                for (int i = 0; i < n; ++i) {
                    if (p[g][0].done && p[g][1].done) break;
                    const int k = sm.list[w][i];
                    const float4 r0 = sm.r0[k], r1 = sm.r1[k], r2 = sm.r2[k];
                    float dx, u, v;
                    column_terms(r0, pcx, dx, u, v);
                    const float q0 = log2_power(u, v, r1.x, __fsub_rn(r0.y, pcy0));
                    const float q1 = log2_power(u, v, r1.x, __fsub_rn(r0.y, pcy1));
                    if (is_boxed(r2)) {           // same entry in every lane: uniform branch
                        const int4 bx = sm.box[k];
                        const bool xin = in_range(px, bx.x, bx.y);
                        composite(p[g][0], q0, r1.y, r1.z, r1.w, r2.x, xin && in_range(py0, bx.z, bx.w));
                        composite(p[g][1], q1, r1.y, r1.z, r1.w, r2.x, xin && in_range(py1, bx.z, bx.w));
                    } else {
                        composite(p[g][0], q0, r1.y, r1.z, r1.w, r2.x, true);
                        composite(p[g][1], q1, r1.y, r1.z, r1.w, r2.x, true);
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (sid[g] < 0) continue;
            const int s = sid[g];
            float o[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                o[h][0] = __fmaf_rn(p[g][h].T, a.bg0, p[g][h].c0);
                o[h][1] = __fmaf_rn(p[g][h].T, a.bg1, p[g][h].c1);
                o[h][2] = __fmaf_rn(p[g][h].T, a.bg2, p[g][h].c2);
            }
            if (WRITE) {
                const size_t si = (size_t)(s - a.img_s0);
                if (in0) {
                    float *dst = a.images + ((si * a.H + py0) * a.W + px) * 3;
                    dst[0] = o[0][0]; dst[1] = o[0][1]; dst[2] = o[0][2];
                }
                if (in1) {
                    float *dst = a.images + ((si * a.H + py1) * a.W + px) * 3;
                    dst[0] = o[1][0]; dst[1] = o[1][1]; dst[2] = o[1][2];
                }
            }
            if (MSE) {
                double se = 0.0;
                const float *rbase = a.refs + (size_t)a.ref_of_state[s] * a.H * a.W * 3;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int py = h ? py1 : py0;
                    if (h ? in1 : in0) {
                        const float *rp = rbase + ((size_t)py * a.W + px) * 3;
                        se += (double)pixel_sq_err(o[h][0], o[h][1], o[h][2], rp[0], rp[1], rp[2]);
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) se += __shfl_xor_sync(0xffffffffu, se, off);
                if (lane == 0) wsum[g][w] = se;
            }
        }
        if (MSE) {
            __syncthreads();
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (threadIdx.x == g && sid[g] >= 0) {
                    double tot = 0.0;
#pragma unroll
                    for (int k = 0; k < RW; ++k) tot += wsum[g][k];
                    a.partial[(size_t)sid[g] * a.tiles + tile] = tot;
                    if (LIST) a.stop[(size_t)sid[g] * a.tiles + tile] = s_stop[g];
                }
            }
        }
        __syncthreads();
    }
}

// Cost key of each (view group, tile), 16 bits: ascending key = descending
// entry count (counts above 65535 tie; the order only schedules work).
__global__ void k_tile_costs(const uint2 *__restrict__ ranges, uint32_t n, uint32_t *__restrict__ keys,
                             uint32_t *__restrict__ vals)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint2 r = ranges[i];
        keys[i] = 0xffffu - min(r.y - r.x, 0xffffu);
        vals[i] = i;
    }
}

__global__ void k_item_counts(const uint32_t *__restrict__ tile_order, uint32_t n, uint32_t tiles,
                              const int32_t *__restrict__ vg_ngroups, uint32_t *__restrict__ counts)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        counts[j] = (uint32_t)vg_ngroups[tile_order[j] / tiles];
}

// Per-pixel state of the adjoint walk.
struct PixB {
    float T;                  // transmittance before the current entry
    float gc;                 // dL/dC . (colour accumulated so far)
    float GK;                 // dL/dC . (C_final + T_final bg): the forward's pixel
    float g0, g1, g2;         // dL/dC
    bool active;              // in the image, dL/dC != 0 and not stopped yet
};

// Adjoint of one pixel at one staged entry (inb: in the box and the pixel
// still active).  The entry at which T (1 - alpha) would drop below 1e-4 stops
// the pixel without contributing, exactly as in composite(), so the walk ends
// where the forward ended.  With gr = dL/dC . rgb_k and the running
// gc = dL/dC . C_prefix (including k):
//   dL/dalpha_k = T_k gr - (GK - gc) / (1 - alpha_k).
// Writes (FIRST) or adds to g[9] = (S gpw dx, S gpw dy, S gpw dx^2,
// S gpw dx dy, S gpw dy^2, S gpw, dL/drgb) with gpw = dL/dpower; the conic
// and mean gradients are linear in these sums (A, B, C are per Gaussian) and
// dL/do = S gpw / o (alpha = o e^power), all formed once per Gaussian after
// the reduction.  Branch free: a skipped entry adds zeros.
template <bool FIRST>
__device__ __forceinline__ bool adjoint(PixB &p, const float4 &r0, const float4 &r1, float b, bool inb, float dx,
                                        float u, float v, float pcy, float *g)
{
    const float dy = __fsub_rn(r0.y, pcy);
    const float p2 = log2_power(u, v, r1.x, dy);
    const float araw = __fmul_rn(r1.y, ex2(p2));
    const float a0 = fminf(0.99f, araw);
    const bool hit = inb && p2 <= 0.0f && a0 >= (1.0f / 255.0f);
    const float om = __fsub_rn(1.0f, a0);                // >= 0.01
    const float Tn = __fmul_rn(p.T, om);
    const bool stop = hit && Tn < 1e-4f;
    const bool ok = hit && !stop;
    p.active = p.active && !stop;
    const float wgt = ok ? __fmul_rn(a0, p.T) : 0.0f;
    const float gr = fmaf(p.g2, b, fmaf(p.g1, r1.w, p.g0 * r1.z));
    p.gc = fmaf(wgt, gr, p.gc);
    // unused unless ok; finite either way (om >= 0.01)
    const float da = fmaf(p.T, gr, -(p.GK - p.gc) * __fdividef(1.0f, om));
    // d alpha / d power = alpha on the linear range; 0 when skipped or at the 0.99 clamp
    const float gpw = da * ((ok && araw < 0.99f) ? a0 : 0.0f);
    const float t1 = gpw * dx, t2 = gpw * dy;
    if (FIRST) {
        g[0] = t1; g[1] = t2;
        g[2] = t1 * dx; g[3] = t1 * dy; g[4] = t2 * dy;
        g[5] = gpw;
        g[6] = p.g0 * wgt; g[7] = p.g1 * wgt; g[8] = p.g2 * wgt;
    } else {
        g[0] += t1; g[1] += t2;
        g[2] = fmaf(t1, dx, g[2]); g[3] = fmaf(t1, dy, g[3]); g[4] = fmaf(t2, dy, g[4]);
        g[5] += gpw;
        g[6] = fmaf(p.g0, wgt, g[6]); g[7] = fmaf(p.g1, wgt, g[7]); g[8] = fmaf(p.g2, wgt, g[8]);
    }
    p.T = ok ? Tn : p.T;
    return ok;
}

// Sum of v[0..7] over the warp: after three exchange-and-keep-half steps and
// two plain steps, lane 4j holds the warp total of v[j].
__device__ __forceinline__ float reduce8_transpose(const float *v, int lane)
{
    float u[4], w2[2];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[i + 4];
        const float keep = b4 ? v[i + 4] : v[i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? u[i] : u[i + 2];
        const float keep = b3 ? u[i + 2] : u[i];
        w2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const float send = b2 ? w2[0] : w2[1];
    float x = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    return x;
}

// Adjoint compositing, one block per (tile, state).  The walk needs each
// pixel's final value C_final + T_final bg: with IMG it is read from the
// forward's image (the forward and this walk composite with the same
// arithmetic, so that value is the one this walk would reach), otherwise a
// first pass re-runs the forward walk.  Transmittance is never stored: the
// gradient pass walks front to back recomputing it and, for each included k,
//   dC/drgb_k   = alpha_k T_k
//   dC/dalpha_k = rgb_k T_k - (C_after_k + T_final bg) / (1 - alpha_k)
// with C_after_k = C_final - (colour accumulated up to and including k).
// Per-Gaussian sums: two pixels per thread, warp transpose reduction, block
// sum in shared memory, then float4 atomics into the record's gradient.
template <bool IMG>
__global__ void __launch_bounds__(RT, 7) k_raster_bwd(RasterBwdArgs b)
{
    const RasterArgs &a = b.f;
    __shared__ Staged sm;
    __shared__ uint8_t sdep[MAX_CLUSTERS];
    __shared__ float gacc[BATCH][9];
    const int tile = (int)(blockIdx.x / (unsigned)a.S), s = (int)(blockIdx.x % (unsigned)a.S);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = a.vg_of_state[s];
    load_depth_row(a.depth, s, a.C, sdep);
    for (int j = threadIdx.x; j < BATCH * 9; j += RT) (&gacc[0][0])[j] = 0.0f;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const Quad wq = quad_of(tx, ty, w, lane);
    const int px = wq.px, py0 = wq.py0, py1 = py0 + 1;
    const bool in0 = px < a.W && py0 < a.H, in1 = px < a.W && py1 < a.H;
    const float pcx = (float)px + 0.5f, pcy0 = (float)py0 + 0.5f, pcy1 = (float)py1 + 0.5f;
    const uint2 rg = a.ranges[(size_t)v * a.tiles + tile];

    // ---- final pixel values
    float fin[2][3];
    if (IMG) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            fin[h][0] = fin[h][1] = fin[h][2] = 0.0f;
            if (h ? in1 : in0) {
                const float *ip = b.img_fwd + (((size_t)s * a.H + (h ? py1 : py0)) * a.W + px) * 3;
                fin[h][0] = ip[0]; fin[h][1] = ip[1]; fin[h][2] = ip[2];
            }
        }
    } else {
        Pix f[2] = {{1.0f, 0.0f, 0.0f, 0.0f, !in0}, {1.0f, 0.0f, 0.0f, 0.0f, !in1}};
        for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
            if (__syncthreads_count(!(f[0].done && f[1].done)) == 0) break;
            stage_batch(a.recs, a.evals, sdep, start, rg.y, wq, sm);
            const int n = sm.cnt[w];
            for (int i = 0; i < n; ++i) {
                if (f[0].done && f[1].done) break;
                const int k = sm.list[w][i];
                const float4 r0 = sm.r0[k], r1 = sm.r1[k], r2 = sm.r2[k];
                float dx, u, v;
                column_terms(r0, pcx, dx, u, v);
                const float q0 = log2_power(u, v, r1.x, __fsub_rn(r0.y, pcy0));
                const float q1 = log2_power(u, v, r1.x, __fsub_rn(r0.y, pcy1));
                bool b0 = true, b1 = true;
                if (is_boxed(r2)) {
                    const int4 bx = sm.box[k];
                    const bool xin = in_range(px, bx.x, bx.y);
                    b0 = xin && in_range(py0, bx.z, bx.w);
                    b1 = xin && in_range(py1, bx.z, bx.w);
                }
                composite(f[0], q0, r1.y, r1.z, r1.w, r2.x, b0);
                composite(f[1], q1, r1.y, r1.z, r1.w, r2.x, b1);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            fin[h][0] = __fmaf_rn(f[h].T, a.bg0, f[h].c0);
            fin[h][1] = __fmaf_rn(f[h].T, a.bg1, f[h].c1);
            fin[h][2] = __fmaf_rn(f[h].T, a.bg2, f[h].c2);
        }
    }
    PixB q[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const bool in = h ? in1 : in0;
        const int py = h ? py1 : py0;
        PixB &p = q[h];
        p.T = 1.0f; p.gc = 0.0f;
        p.g0 = p.g1 = p.g2 = 0.0f;
        if (in) {
            const float *gp = b.dL_dimg + (((size_t)s * a.H + py) * a.W + px) * 3;
            p.g0 = gp[0]; p.g1 = gp[1]; p.g2 = gp[2];
        }
        p.GK = p.g0 * fin[h][0] + p.g1 * fin[h][1] + p.g2 * fin[h][2];
        p.active = in && (p.g0 != 0.0f || p.g1 != 0.0f || p.g2 != 0.0f);
    }

    // ---- gradient pass
    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(q[0].active || q[1].active) == 0) break;
        const int nk = stage_batch(a.recs, a.evals, sdep, start, rg.y, wq, sm);
        const int n = sm.cnt[w];
        if (__any_sync(0xffffffffu, q[0].active || q[1].active)) {
            for (int i = 0; i < n; ++i) {
                if ((i & 7) == 0 && !__any_sync(0xffffffffu, q[0].active || q[1].active)) break;
                const int k = sm.list[w][i];
                float g[9];
                bool contrib;
                const float4 r0 = sm.r0[k], r1 = sm.r1[k], r2 = sm.r2[k];
                float dx, u, v;
                column_terms(r0, pcx, dx, u, v);
                if (is_boxed(r2)) {           // same entry in every lane: uniform branch
                    const int4 bx = sm.box[k];
                    const bool xin = in_range(px, bx.x, bx.y);
                    contrib = adjoint<true>(q[0], r0, r1, r2.x, q[0].active && xin && in_range(py0, bx.z, bx.w),
                                            dx, u, v, pcy0, g);
                    contrib |= adjoint<false>(q[1], r0, r1, r2.x, q[1].active && xin && in_range(py1, bx.z, bx.w),
                                              dx, u, v, pcy1, g);
                } else {
                    contrib = adjoint<true>(q[0], r0, r1, r2.x, q[0].active, dx, u, v, pcy0, g);
                    contrib |= adjoint<false>(q[1], r0, r1, r2.x, q[1].active, dx, u, v, pcy1, g);
                }
                if (__ballot_sync(0xffffffffu, contrib)) {
                    const float x = reduce8_transpose(g, lane);
                    float g8 = g[8];
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) g8 += __shfl_xor_sync(0xffffffffu, g8, off);
                    if ((lane & 3) == 0) atomicAdd(&gacc[k][lane >> 2], x);
                    if (lane == 1) atomicAdd(&gacc[k][8], g8);
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nk; k += RT) {
            float x[9];
            bool any = false;
#pragma unroll
            for (int j = 0; j < 9; ++j) { x[j] = gacc[k][j]; gacc[k][j] = 0.0f; any |= (x[j] != 0.0f); }
            if (any) {
                // conic and mean gradients from the per-Gaussian sums (records hold the scaled conic)
                const float A = sm.r0[k].z * INV_K_AC, B = sm.r0[k].w * INV_K_B, C = sm.r1[k].x * INV_K_AC;
                const float gmx = -(A * x[0] + B * x[1]), gmy = -(C * x[1] + B * x[0]);
                float4 *dst = b.rec_grad + (size_t)sm.slot[k] * 3;
                atomicAdd(dst, make_float4(gmx, gmy, -0.5f * x[2], -x[3]));
                atomicAdd(dst + 1, make_float4(-0.5f * x[4], __fdividef(x[5], sm.r1[k].y), x[6], x[7]));
                atomicAdd(dst + 2, make_float4(x[8], 0.0f, 0.0f, 0.0f));
            }
        }
    }
}

// mse[s] = sum_t partial[s][t] / (3 H W) in a fixed order; psnr = 10 log10(1/mse)
__global__ void k_mse_reduce(const double *__restrict__ partial, int S, int parts, double inv_count,
                             double *__restrict__ mse, double *__restrict__ psnr)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= S) return;
    double acc = 0.0;
    for (int t = lane; t < parts; t += 32) acc += partial[(size_t)warp * parts + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const double m = acc * inv_count;
        mse[warp] = m;
        if (psnr) psnr[warp] = m > 0.0 ? 10.0 * log10(1.0 / m) : __longlong_as_double(0x7ff0000000000000LL);
    }
}

// Squared-error partial sum of image s vs refs[ref_index[s]] over one chunk
// of MSE_CHUNK_PIX pixels (four per thread), and optionally
// dL/dimage = weight * 2 (image - ref) / (3 H W).
__global__ void __launch_bounds__(256) k_image_mse(const float *__restrict__ images, const float *__restrict__ refs,
                                                   const int32_t *__restrict__ ref_index, size_t npix,
                                                   float gscale, double *__restrict__ partial, int parts,
                                                   float *__restrict__ dL)
{
    __shared__ double wsum[8];
    const int s = blockIdx.y;
    const float *im = images + (size_t)s * npix * 3;
    const float *rf = refs + (size_t)ref_index[s] * npix * 3;
    float x[4][3], y[4][3];
    const size_t base = (size_t)blockIdx.x * MSE_CHUNK_PIX + threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t p = base + (size_t)k * 256;
#pragma unroll
        for (int c = 0; c < 3; ++c) { x[k][c] = 0.0f; y[k][c] = 0.0f; }
        if (p < npix) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { x[k][c] = __ldg(im + 3 * p + c); y[k][c] = __ldg(rf + 3 * p + c); }
        }
    }
    double se = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t p = base + (size_t)k * 256;
        if (p < npix) {
            se += (double)pixel_sq_err(x[k][0], x[k][1], x[k][2], y[k][0], y[k][1], y[k][2]);
            if (dL) {
                float *d = dL + ((size_t)s * npix + p) * 3;
#pragma unroll
                for (int c = 0; c < 3; ++c) d[c] = gscale * (x[k][c] - y[k][c]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += wsum[w];
        partial[(size_t)s * parts + blockIdx.x] = tot;
    }
}

}  // namespace

template <int G, bool WRITE, bool MSE, bool LIST>
static void launch_fwd_t(const RasterArgs &a, const WorkQueue &q, int blocks, cudaStream_t st)
{
    k_raster_fwd<G, WRITE, MSE, LIST><<<blocks, RT, 0, st>>>(a, q);
}

// The explicit work list (tile reuse) renders squared-error partials only.
template <int G>
static void launch_fwd_g(const RasterArgs &a, const WorkQueue &q, int blocks, cudaStream_t st)
{
    if (q.item_first) launch_fwd_t<G, false, true, true>(a, q, blocks, st);
    else if (a.images && a.refs) launch_fwd_t<G, true, true, false>(a, q, blocks, st);
    else if (a.images) launch_fwd_t<G, true, false, false>(a, q, blocks, st);
    else launch_fwd_t<G, false, true, false>(a, q, blocks, st);
}

void launch_raster_fwd(const RasterArgs &a, const WorkQueue &q, int G, int blocks, cudaStream_t st)
{
    if ((!q.item_first && q.n_items == 0) || (!a.images && !a.refs)) return;
    static const char *names[2][4] = {{"raster_fwd_g1", "raster_fwd_g2", "raster_fwd_g4", "raster_fwd_g8"},
                                      {"raster_fwd_mse_g1", "raster_fwd_mse_g2", "raster_fwd_mse_g4",
                                       "raster_fwd_mse_g8"}};
    const int gi = G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : 3;
    ProfScope ps_(names[a.refs ? 1 : 0][gi], st);
    switch (G) {
    case 1: launch_fwd_g<1>(a, q, blocks, st); break;
    case 2: launch_fwd_g<2>(a, q, blocks, st); break;
    case 4: launch_fwd_g<4>(a, q, blocks, st); break;
    default: launch_fwd_g<8>(a, q, blocks, st); break;
    }
    count_launch();
}

template <int G, bool WRITE, bool MSE, bool LIST>
static int occ_t()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_raster_fwd<G, WRITE, MSE, LIST>, RT, 0);
    return n > 0 ? n : 1;
}

template <int G>
static int occ_g(bool write, bool mse, bool list)
{
    if (list) return occ_t<G, false, true, true>();
    if (write && mse) return occ_t<G, true, true, false>();
    if (write) return occ_t<G, true, false, false>();
    return occ_t<G, false, true, false>();
}

// Resident blocks per SM of each instantiation (queried once, then cached, so
// launches made during stream capture issue no runtime queries).
int raster_fwd_blocks_per_sm(int G, bool write, bool mse, bool list)
{
    static int cache[4][4] = {};
    const int gi = G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : 3;
    const int mi = list ? 3 : (write && mse) ? 0 : write ? 1 : 2;
    if (!cache[gi][mi]) {
        switch (G) {
        case 1: cache[gi][mi] = occ_g<1>(write, mse, list); break;
        case 2: cache[gi][mi] = occ_g<2>(write, mse, list); break;
        case 4: cache[gi][mi] = occ_g<4>(write, mse, list); break;
        default: cache[gi][mi] = occ_g<8>(write, mse, list); break;
        }
    }
    return cache[gi][mi];
}

void launch_tile_costs(const uint2 *ranges, uint32_t n, uint32_t *keys, uint32_t *vals, int sms, cudaStream_t st)
{
    if (n == 0) return;
    unsigned b = (n + 255) / 256;
    if (b > (unsigned)sms * 8) b = sms * 8;
    ProfScope ps_("tile_costs", st);
    k_tile_costs<<<b, 256, 0, st>>>(ranges, n, keys, vals);
    count_launch();
}

void launch_item_counts(const uint32_t *tile_order, uint32_t n, uint32_t tiles, const int32_t *vg_ngroups,
                        uint32_t *counts, int sms, cudaStream_t st)
{
    if (n == 0) return;
    unsigned b = (n + 255) / 256;
    if (b > (unsigned)sms * 8) b = sms * 8;
    ProfScope ps_("item_counts", st);
    k_item_counts<<<b, 256, 0, st>>>(tile_order, n, tiles, vg_ngroups, counts);
    count_launch();
}

void launch_raster_bwd(const RasterBwdArgs &b, cudaStream_t st)
{
    if (b.f.S == 0 || b.f.tiles == 0) return;
    const unsigned grid = b.f.tiles * (unsigned)b.f.S;
    ProfScope ps_(b.img_fwd ? "raster_bwd" : "raster_bwd_2pass", st);
    if (b.img_fwd) k_raster_bwd<true><<<grid, RT, 0, st>>>(b);
    else k_raster_bwd<false><<<grid, RT, 0, st>>>(b);
    count_launch();
}

void launch_mse_reduce(const double *partial, int S, int parts, double inv_count, double *mse, double *psnr,
                       cudaStream_t st)
{
    if (S == 0) return;
    const int threads = 256, blocks = (S * 32 + threads - 1) / threads;
    ProfScope ps_("mse_reduce", st);
    k_mse_reduce<<<blocks, threads, 0, st>>>(partial, S, parts, inv_count, mse, psnr);
    count_launch();
}

void launch_image_mse(const float *images, const float *refs, const int32_t *ref_index, int S, int H, int W,
                      float weight, double *partial, int parts, float *dL, cudaStream_t st)
{
    if (S == 0) return;
    const size_t npix = (size_t)H * W;
    const float gscale = (float)(2.0 * (double)weight / (double)(npix * 3));
    dim3 grid((unsigned)parts, (unsigned)S);
    ProfScope ps_("image_mse", st);
    k_image_mse<<<grid, 256, 0, st>>>(images, refs, ref_index, npix, gscale, partial, parts, dL);
    count_launch();
}

}  // namespace dgs
