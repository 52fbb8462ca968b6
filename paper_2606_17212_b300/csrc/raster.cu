// Tile rasterization of delivery states: forward compositing with an optional
// fused FP64 squared-error epilogue, and the adjoint compositing kernel.
//
// One warp renders one 16x16 region of a sort tile for one state: lane l owns
// column l & 15 of the region and its rows 8 (l >> 4) .. 8 (l >> 4) + 7, held
// as four vertical pixel pairs in packed FP32x2 registers, so every per-pixel
// FP32 operation of a pair issues once; the forward and the adjoint use the
// same regions.  A warp walks the tile's run of the batch-wide
// sorted entry list, which holds every depth variant any state of the view
// group needs, in chunks of 32 entries: it keeps the variants this state
// renders (variant depth == the state's delivered depth of the Gaussian's
// cluster) whose alpha >= 1/255 ellipse reaches the tile, appends them in run
// order to its own shared-memory queue, and composites them; warps never wait
// on each other.  Filtering a sorted run keeps it sorted, so every pixel sees
// exactly the (depth, Gaussian) order it would see alone: batched ==
// per-state, bit for bit.
//
// Per pixel and Gaussian the work is a handful of FP32 operations and one MUFU
// exp (two MUFU operations in the adjoint): these kernels are bound by the
// FP32 pipe and instruction issue, not by HBM.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr int WARPS = 4;              // warps per block; each takes its own (tile, state) items
constexpr int RT = 32 * WARPS;        // threads per block
constexpr int QCAP = 64;              // per-warp queue of staged entries (ring, power of two)
constexpr int CHUNK = 32;             // run entries examined per staging step (one per lane)
constexpr int NPAIR = 4;              // vertical pixel pairs per lane in the forward (8 rows: a warp per tile)
// Resident blocks per SM.  Measured on the training workload (250k Gaussians,
// 64 states, 512x512, 32 px tiles): the forward at 4 (117-124 registers) beats
// 5 (96 registers); the adjoint's 16 x 16 regions (4 pixel pairs per lane) at
// 4 blocks (128 registers, no spills) beat 16 x 8 regions (2 pairs) at 6
// blocks (80 registers; 3.97 vs 4.08 ms), which beat 5, 7 or 8 blocks: the
// per-entry warp reduction is shared by twice as many pixels.  A call with
// too few (region, state) items to fill the GPU twice (a single state) takes
// the 16 x 8 regions, which give twice the warps.
constexpr int FWD_MIN_BLOCKS = 4;
// BATCH: the adjoint batches the per-lane sums of several entries before
// one warp reduction (else each entry is reduced at once: 6 blocks of 16 x 8
// regions leave no shared memory for a batch).
template <int NP> struct BwdShape;    // pixel pairs per lane in the adjoint (a warp per 16 x 4 NP region)
template <> struct BwdShape<4> { static constexpr int MIN_BLOCKS = 4; static constexpr bool BATCH = true; };
template <> struct BwdShape<2> { static constexpr int MIN_BLOCKS = 6; static constexpr bool BATCH = false; };
constexpr int BWD_NP_BATCH = 4, BWD_NP_FEW = 2;
constexpr uint32_t FULL = 0xffffffffu;
constexpr float T_STOP = 1e-4f;       // a pixel stops before the entry that would bring T below this
constexpr float A_MAX = 0.99f;        // opacity clamp

// ------------------------------------------------------------ packed FP32x2
// Two FP32 values in one 64-bit register pair; each lane of an operation is
// rounded exactly as the scalar IEEE operation (round to nearest, no flush).
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
// Halves of a pair.  Both are written as one unpacking move, which ptxas
// resolves to a register reference; measured, extracting them with 64-bit
// shifts in C made both raster kernels 4-7% slower.
#pragma nv_diag_suppress 550
__device__ __forceinline__ float lo(f2 x)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
    return a;
}
__device__ __forceinline__ float hi(f2 x)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
    return b;
}
#pragma nv_diag_default 550
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// 2^x on the MUFU unit (ex2.approx.ftz: relative error ~2^-22, tiny results flush to 0)
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1/x on the MUFU unit (rcp.approx.ftz: ~1 ulp)
__device__ __forceinline__ float rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1.0f when x >= y, else 0.0f (one compare-and-set)
__device__ __forceinline__ float ge1(float x, float y)
{
    float r;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
    return r;
}
// 1.0f when x < y, else 0.0f
__device__ __forceinline__ float lt1(float x, float y)
{
    float r;
    asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
    return r;
}

// alpha = o 2^p2 = 2^(p2 + log2 o): each staged entry carries log2 o, which
// a lane adds to its column's constant exponent term, so alpha is one ex2
// and alpha >= 1/255 is e = p2 + log2 o >= TAU0 = -log2 255 for every entry
// (the test does not wait for the ex2).  In exact arithmetic e <= 0; an e
// that FP32 rounding leaves at or above +0 (Gaussian centre on the pixel
// centre, o near 1) passes, as the exact arithmetic does.  The forward takes
// the test as a compare and a select, the adjoint as a compare-and-set (1 or
// 0) and one packed multiply per pixel pair: the same decision.  lg2.approx
// and ex2.approx err by ~2^-22 relative, so the decision can differ from the
// exact alpha >= 1/255 only for alpha within ~1e-6 relative of 1/255.
constexpr float TAU0 = -7.99435343685886f;   // float nearest -log2 255

__device__ __forceinline__ float lg2(float x)
{
    float l;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    return l;
}

// ------------------------------------------------------------ staging
// A warp's queue of staged entries, read by all lanes at once (broadcast).
// Fields are duplicated where the packed arithmetic wants a pair.
struct Queue {
    float4 s0[QCAP];                  // my, my, c2, c2          (records hold the scaled conic)
    float4 s1[QCAP];                  // log2 o, log2 o, r, r
    float4 s2[QCAP];                  // g, g, b, b
    float4 s3[QCAP];                  // mx, a2, b2, -
    uint4 s4[QCAP];                   // box x, box y, kind (bit 0: boxed, bit 1: clamp), record slot
};

struct WarpSmem {
    Queue q;
    float4 pre[3][32];                // records of the next chunk, copied asynchronously (lane: its entry)
    uint8_t dep[MAX_CLUSTERS];        // the state's delivered depth per cluster
};

// The adjoint's batch of per-lane entry sums awaiting their warp reduction:
// entry e of the batch, lane l: (S1, S4) at float2 index e RB_STRIDE / 2 + l,
// (S5, Sr) at + 32 + l, (Sg, Sb) at + 64 + l.  RB_STRIDE = 200 words (= 8
// mod 32) lets the reduction's lanes (4 per entry, source lanes q + 4 i)
// read 64-bit words without bank conflicts.
constexpr int RB = 8;                 // entries per batch
constexpr int RB_STRIDE = 200;        // words per batch entry (3 x 64 used)
struct RedBuf {
    float2 v[RB * RB_STRIDE / 2];
    uint32_t slot[RB];                // record slot of each batch entry
    float mx[RB];                     // its mean x (the moments' dx = mx - pixel centre)
};

// Can Gaussian (mx, my, conic A B C, opacity o) reach alpha >= 1/255 at some
// pixel centre of the rectangle [x0, x1] x [y0, y1]?  alpha >= 1/255 needs
// q(d) = A dx^2 + 2 B dx dy + C dy^2 <= rho = 2 ln(255 o) with d = p - m.  The
// minimum of the convex q over the rectangle is 0 when it holds the mean, else
// it lies on an edge (1-D quadratic, clamped vertex).  rho is inflated by
// 1e-3 relative + 1e-3 so FP32 rounding never drops a pixel that composites
// (the 1e-3 also covers undoing the records' scaling of the conic);
// skipping a Gaussian that stays below 1/255 on the whole rectangle changes nothing.
__device__ __forceinline__ bool ellipse_meets_rect(const float4 &r0, const float4 &r1, float x0, float x1,
                                                   float y0, float y1)
{
    const float A = r0.z * INV_K_AC, B = r0.w * INV_K_B, C = r1.x * INV_K_AC, o = r1.y;   // records: scaled
    const float rho = fmaf(2.0f * __logf(255.0f * o), 1.001f, 1e-3f);
    const float X0 = x0 - r0.x, X1 = x1 - r0.x, Y0 = y0 - r0.y, Y1 = y1 - r0.y;
    if (X0 <= 0.0f && X1 >= 0.0f && Y0 <= 0.0f && Y1 >= 0.0f) return true;
    float best = 3.4e38f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {     // vertical edges dx = X: minimise over dy in [Y0, Y1]
        const float X = e ? X1 : X0;
        const float dy = fminf(fmaxf(__fdividef(-B * X, C), Y0), Y1);
        best = fminf(best, A * X * X + 2.0f * B * X * dy + C * dy * dy);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {     // horizontal edges dy = Y: minimise over dx in [X0, X1]
        const float Y = e ? Y1 : Y0;
        const float dx = fminf(fmaxf(__fdividef(-B * Y, A), X0), X1);
        best = fminf(best, A * dx * dx + 2.0f * B * dx * Y + C * Y * Y);
    }
    return best <= rho;
}

// A warp's region: 16 columns x 4 NP rows of a sort tile, at pixel offset
// (ox, oy) inside it.  Lane l owns column l & 15 and rows 2 NP (l >> 4) ..
// + 2 NP - 1 of the region, as NP vertical pairs.
template <int NP>
struct Lane {
    int lane, px, py0;
    int rx0, ry0;                     // the region's first pixel
    float pcx;                        // pixel-centre x
    f2 pcy[NP];                       // pixel-centre y of each pair (rows 2j, 2j + 1)
    uint32_t inimg;                   // bit r: row r of the column lies in the image
};

template <int NP>
__device__ __forceinline__ Lane<NP> lane_of(int tile, int ox, int oy, const RasterArgs &a)
{
    Lane<NP> L;
    L.lane = threadIdx.x & 31;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    L.rx0 = (tx << a.tile_shift) + ox;
    L.ry0 = (ty << a.tile_shift) + oy;
    L.px = L.rx0 + (L.lane & 15);
    L.py0 = L.ry0 + 2 * NP * (L.lane >> 4);
    L.pcx = (float)L.px + 0.5f;
#pragma unroll
    for (int j = 0; j < NP; ++j)
        L.pcy[j] = pk((float)(L.py0 + 2 * j) + 0.5f, (float)(L.py0 + 2 * j + 1) + 0.5f);
    L.inimg = 0;
    if (L.px < a.W) {
        const int rows = min(2 * NP, a.H - L.py0);
        L.inimg = rows <= 0 ? 0u : ((1u << rows) - 1u);
    }
    return L;
}

// Start copying each lane's record (the lane's run entry of the next chunk,
// record slot `slot`) into the warp's prefetch area; the copies land while
// the warp composites the entries it has already staged.
template <bool L1>
__device__ __forceinline__ void prefetch_records(const Rec *__restrict__ recs, uint32_t slot, bool valid,
                                                 WarpSmem &sm)
{
    const int lane = threadIdx.x & 31;
    if (valid) {
        const char *src = reinterpret_cast<const char *>(recs + slot);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sm.pre[k][lane]);
            if (L1)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + 16 * k) : "memory");
            else
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + 16 * k) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void prefetch_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
}

// Examine the prefetched chunk (run entries e .. e + 31, one per lane; lanes
// past the run's end hold nothing): keep the entries this state renders whose
// pixel box meets the region and whose alpha ellipse reaches its pixel
// centres [x0, x0 + 15] x [y0, y0 + h], and append them in run order at
// `tail`.  Returns the new tail.
__device__ __forceinline__ uint32_t stage_chunk(const uint8_t *dep, uint32_t slot, bool valid, int rx0, int ry0,
                                                int h, WarpSmem &sm, uint32_t tail)
{
    const int lane = threadIdx.x & 31;
    bool keep = false;
    float4 r0 = make_float4(0, 0, 0, 0), r1 = r0, r2 = r0;
    if (valid) {
        r2 = sm.pre[2][lane];
        const uint32_t cd = __float_as_uint(r2.w), bx = __float_as_uint(r2.y), by = __float_as_uint(r2.z);
        // the state's variant, whose pixel box meets the region, whose alpha ellipse reaches it
        if (((cd >> 12) & 0xfu) == (uint32_t)dep[cd & REC_CLUSTER] && (int)(bx & 0xffffu) <= rx0 + 15 &&
            (int)(bx >> 16) >= rx0 && (int)(by & 0xffffu) <= ry0 + h && (int)(by >> 16) >= ry0) {
            r0 = sm.pre[0][lane];
            r1 = sm.pre[1][lane];
            const float x0 = (float)rx0 + 0.5f, y0 = (float)ry0 + 0.5f;
            keep = ellipse_meets_rect(r0, r1, x0, x0 + 15.0f, y0, y0 + (float)h);
        }
    }
    const uint32_t bal = __ballot_sync(FULL, keep);
    if (keep) {
        const uint32_t k = (tail + __popc(bal & ((1u << lane) - 1u))) & (QCAP - 1);
        Queue &q = sm.q;
        q.s0[k] = make_float4(r0.y, r0.y, r1.x, r1.x);
        const float lo2o = lg2(r1.y);
        q.s1[k] = make_float4(lo2o, lo2o, r1.z, r1.z);
        q.s2[k] = make_float4(r1.w, r1.w, r2.x, r2.x);
        q.s3[k] = make_float4(r0.x, r0.z, r0.w, 0.0f);
        const uint32_t cd = __float_as_uint(r2.w);
        q.s4[k] = make_uint4(__float_as_uint(r2.y), __float_as_uint(r2.z),
                             (cd >> 31) | ((cd & REC_CLAMP) ? 2u : 0u), slot);
    }
    __syncwarp();
    return tail + (uint32_t)__popc(bal);
}

// Per-entry, per-lane terms of one staged entry: the column's exponent terms
// u = a2 dx^2 + log2 o, v = b2 dx (shared by the lane's pixels), the
// broadcast pairs, and the rows of the lane that lie in the entry's pixel box
// (only where the record's 3-sigma box clips its alpha box; else all rows).
struct Ent {
    f2 my, c2, r, g, b, uu, vv;
    uint32_t rows;                    // bit r: row r passes the box test
    float dx;
};

// s4: the entry's box and slot word as loaded by the dispatch (PRE), else read here.
template <int NP, bool BOXED, bool PRE>
__device__ __forceinline__ Ent load_entry(const Queue &q, int k, const uint4 &s4_, const Lane<NP> &L)
{
    Ent E;
    const float4 s0 = q.s0[k], s1 = q.s1[k], s2 = q.s2[k], s3 = q.s3[k];
    E.my = pk(s0.x, s0.y);
    E.c2 = pk(s0.z, s0.w);
    E.r = pk(s1.z, s1.w);
    E.g = pk(s2.x, s2.y);
    E.b = pk(s2.z, s2.w);
    E.dx = __fsub_rn(s3.x, L.pcx);
    const float u = __fadd_rn(__fmul_rn(__fmul_rn(s3.y, E.dx), E.dx), s1.x), v = __fmul_rn(s3.z, E.dx);
    E.uu = pk(u, u);
    E.vv = pk(v, v);
    E.rows = 0xffu;
    if (BOXED) {
        const uint4 s4 = PRE ? s4_ : q.s4[k];
        const int xlo = (int)(s4.x & 0xffffu), xhi = (int)(s4.x >> 16);
        const int ylo = (int)(s4.y & 0xffffu), yhi = (int)(s4.y >> 16);
        const int rlo = max(ylo - L.py0, 0), rhi = min(yhi - L.py0, 2 * NP - 1);
        const bool xin = (unsigned)(L.px - xlo) <= (unsigned)(xhi - xlo);
        E.rows = (xin && rlo <= rhi) ? ((2u << rhi) - (1u << rlo)) : 0u;
    }
    return E;
}

// Base-2 exponent e = a2 dx^2 + b2 dx dy + c2 dy^2 + log2 o of a pixel pair
// and the clamped opacity alpha of each pixel (0 where the entry is skipped:
// outside the box or alpha < 1/255).  Returns the pair (alpha0, alpha1); `ar`
// gets the unclamped o 2^p2 = 2^e (for the clamp's derivative in the adjoint).
__device__ __forceinline__ f2 pair_alpha_clamped(const Ent &E, f2 pcy, int j, f2 &dy, f2 &ar)
{
    dy = sub2(E.my, pcy);
    const f2 p2 = fma2(fma2(E.c2, dy, E.vv), dy, E.uu);
    ar = pk(ex2(lo(p2)), ex2(hi(p2)));
    const bool h0 = lo(p2) >= TAU0 && ((E.rows >> (2 * j)) & 1u);
    const bool h1 = hi(p2) >= TAU0 && ((E.rows >> (2 * j + 1)) & 1u);
    return pk(h0 ? fminf(A_MAX, lo(ar)) : 0.0f, h1 ? fminf(A_MAX, hi(ar)) : 0.0f);
}

// The same with the kind of the entry known at compile time: without CLAMP
// the record cannot reach the 0.99 clamp (o <= 0.98 and a well-conditioned
// conic: p2 <= 0, see the projection), so min(0.99, o 2^p2) is o 2^p2 and
// the clamp is left out; the result is the same.
template <bool BOXED, bool CLAMP>
__device__ __forceinline__ f2 pair_alpha(const Ent &E, f2 pcy, int j, f2 &dy, f2 &ar)
{
    dy = sub2(E.my, pcy);
    const f2 p2 = fma2(fma2(E.c2, dy, E.vv), dy, E.uu);
    ar = pk(ex2(lo(p2)), ex2(hi(p2)));
    const f2 keep = pk(ge1(lo(p2), TAU0), ge1(hi(p2), TAU0));
    const f2 a = mul2(CLAMP ? pk(fminf(A_MAX, lo(ar)), fminf(A_MAX, hi(ar))) : ar, keep);
    if (!BOXED) return a;
    return pk(((E.rows >> (2 * j)) & 1u) ? lo(a) : 0.0f, ((E.rows >> (2 * j + 1)) & 1u) ? hi(a) : 0.0f);
}

// ------------------------------------------------------------ forward
// Front-to-back state of a pixel pair.  A pixel that stops (T (1 - alpha)
// would fall below 1e-4: the entry is not added) keeps T = 0 from then on, so
// every later entry adds exactly zero, and its transmittance at the stop is
// kept in Tk; the final transmittance is T + Tk (one of them is zero).
// (Tracking T + Tk directly, as U - alpha T, is one operation less per pair
// but measured 4% slower.)
struct FwdPair {
    f2 T, Tk, cr, cg, cb;
};

__device__ __forceinline__ void fwd_pair(FwdPair &P, const Ent &E, f2 al)
{
    const f2 w = mul2(al, P.T);                  // alpha T
    const f2 Tn = sub2(P.T, w);                  // T (1 - alpha)
    const f2 s = pk(ge1(lo(Tn), T_STOP), ge1(hi(Tn), T_STOP));   // 1: composite, 0: stop (or stopped)
    const f2 wp = mul2(w, s);
    P.cr = fma2(E.r, wp, P.cr);
    P.cg = fma2(E.g, wp, P.cg);
    P.cb = fma2(E.b, wp, P.cb);
    P.Tk = fma2(P.T, sub2(pk(1.0f, 1.0f), s), P.Tk);
    P.T = mul2(Tn, s);
}

// The forward treats every entry as one that may reach the clamp (one min
// per pixel): measured, separate code for the records that cannot made the
// forward slower, not faster.
template <int NP>
struct FwdLane {
    static constexpr bool CLAMP_KINDS = false;
    static constexpr bool RECS_L1 = true;     // record prefetch cached in L1 (cp.async.ca)
    FwdPair p[NP];
    __device__ __forceinline__ void init(const Lane<NP> &L)
    {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            p[j].T = pk((L.inimg >> (2 * j)) & 1u ? 1.0f : 0.0f, (L.inimg >> (2 * j + 1)) & 1u ? 1.0f : 0.0f);
            p[j].Tk = p[j].cr = p[j].cg = p[j].cb = 0ull;
        }
    }
    template <bool BOXED, bool CLAMP>
    __device__ __forceinline__ void entry(const Queue &q, int k, const uint4 &s4, const Lane<NP> &L)
    {
        const Ent E = load_entry<NP, BOXED, false>(q, k, s4, L);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            f2 dy, ar;
            const f2 al = pair_alpha_clamped(E, L.pcy[j], j, dy, ar);
            fwd_pair(p[j], E, al);
        }
    }
    __device__ __forceinline__ bool live() const
    {
        f2 any = 0ull;
#pragma unroll
        for (int j = 0; j < NP; ++j) any |= p[j].T;
        return __any_sync(FULL, any != 0ull);
    }
    __device__ __forceinline__ void finish(const Lane<NP> &) {}
    // final colour of pair j: C + (T + Tk) bg
    __device__ __forceinline__ void out(int j, float bg0, float bg1, float bg2, f2 &o0, f2 &o1, f2 &o2) const
    {
        const f2 Tf = add2(p[j].T, p[j].Tk);
        o0 = fma2(Tf, pk(bg0, bg0), p[j].cr);
        o1 = fma2(Tf, pk(bg1, bg1), p[j].cg);
        o2 = fma2(Tf, pk(bg2, bg2), p[j].cb);
    }
};

// Hand staged entry k to `pix` with the arithmetic its kind needs (the same
// entry in every lane: a uniform branch).  Kind bit 0: boxed; bit 1: the
// record may reach the alpha clamp (told apart only where PIX::CLAMP_KINDS).
template <class PIX, int NP>
__device__ __forceinline__ void dispatch_entry(PIX &pix, const Queue &q, int k, const Lane<NP> &L)
{
    // the adjoint wants the whole word (its slot); the forward only the kind
    const uint4 s4 = PIX::CLAMP_KINDS ? q.s4[k] : make_uint4(0u, 0u, q.s4[k].z, 0u);
    const uint32_t kind = s4.z;
    if (!PIX::CLAMP_KINDS) {
        if (kind & 1u) pix.template entry<true, true>(q, k, s4, L);
        else pix.template entry<false, true>(q, k, s4, L);
        return;
    }
    switch (kind) {
    case 1: pix.template entry<true, false>(q, k, s4, L); break;
    case 0: pix.template entry<false, false>(q, k, s4, L); break;
    case 3: pix.template entry<true, true>(q, k, s4, L); break;
    default: pix.template entry<false, true>(q, k, s4, L); break;
    }
}

// Walk the tile run [start, end) for one state: stage chunks into the queue
// and hand every staged entry, in run order, to `pix` until no pixel of the
// tile is live.  Returns the run position past the last examined entry.
template <int NP, class PIX>
__device__ __forceinline__ uint32_t walk(const RasterArgs &a, const Lane<NP> &L, WarpSmem &sm, uint32_t start,
                                         uint32_t end, PIX &pix)
{
    const int h = 4 * NP - 1;
    uint32_t e = start, head = 0, tail = 0;
    if (!pix.live()) return e;
    // pipeline: the records of chunk e are in flight, the slots of chunk e + 32 loaded
    uint32_t slot = e + L.lane < end ? __ldg(a.evals + e + L.lane) : 0u;
    prefetch_records<PIX::RECS_L1>(a.recs, slot, e + L.lane < end, sm);
    uint32_t slot_next = e + CHUNK + L.lane < end ? __ldg(a.evals + e + CHUNK + L.lane) : 0u;
    for (;;) {
        while (tail - head < (uint32_t)CHUNK && e < end) {
            prefetch_wait();
            tail = stage_chunk(sm.dep, slot, e + L.lane < end, L.rx0, L.ry0, h, sm, tail);
            e += CHUNK;
            slot = slot_next;
            if (e < end) prefetch_records<PIX::RECS_L1>(a.recs, slot, e + L.lane < end, sm);
            slot_next = e + CHUNK + L.lane < end ? __ldg(a.evals + e + CHUNK + L.lane) : 0u;
        }
        if (head == tail) break;
        const uint32_t n = min(tail - head, (uint32_t)CHUNK);
        bool live = true;
        for (uint32_t i = 0; i < n; ++i) {
            const int k = (int)((head + i) & (QCAP - 1));
            dispatch_entry(pix, sm.q, k, L);
            if ((i & 3u) == 3u && !pix.live()) { live = false; break; }
        }
        head += n;
        if (!live || !pix.live()) break;
    }
    prefetch_wait();                  // no copy may land in the prefetch area after the walk
    pix.finish(L);
    return min(e, end);
}

__device__ __forceinline__ void load_depth(const RasterArgs &a, int s, WarpSmem &sm)
{
    const uint8_t *row = a.depth + (size_t)s * a.C;
    for (int c = threadIdx.x & 31; c < a.C; c += 32) sm.dep[c] = row[c];
    __syncwarp();
}

// Persistent forward raster.  Each warp repeatedly takes a work item (one
// tile of one view group and one of its states), walks the tile's run and
// writes the state's pixels and/or its FP64 squared-error partial; items come
// costliest tile first from an atomic counter (or from an explicit work list).
// Per pixel the arithmetic is fwd_pair(), exactly as for a single state.
// One work item of the forward raster: (view-group tile, state) number `item`
// of queue q.  Every lane of the warp calls it with the same item.
template <bool WRITE, bool MSE, bool LIST, int SHIFT>
__device__ __forceinline__ void fwd_item(const RasterArgs &a, const WorkQueue &q, uint32_t item, WarpSmem &sm,
                                         int lane)
{
    uint32_t vt;
    int s;
    if (LIST) {
        const uint32_t first = q.item_first[item];
        vt = q.list_vt[first];
        s = (int)q.list_state[first];
    } else {
        // largest j with item_offsets[j] <= item: a 32-way search, one
        // probe per lane per step (item_offsets is non-decreasing)
        uint32_t lo_ = 0, span = q.n_vt;
        while (span > 1) {
            const uint32_t stride = (span + 31) / 32;
            const uint32_t j = lo_ + (uint32_t)lane * stride;
            const bool le = j < lo_ + span && q.item_offsets[j] <= item;
            const uint32_t bal = __ballot_sync(FULL, le);     // lanes 0 .. k-1 (lane 0 always)
            const uint32_t k = 31 - __clz(bal);
            lo_ += k * stride;
            span = min(stride, span - k * stride);
        }
        vt = q.tile_order[lo_];
        const int grp = q.vg_group_base[vt / a.tiles] + (int)(item - q.item_offsets[lo_]);
        s = q.state_order[q.group_first[grp]];
    }
    const int tile = (int)(vt % a.tiles);
    load_depth(a, s, sm);
    const uint2 rg = a.ranges[vt];
    const float *rbase = MSE ? a.refs + (size_t)a.ref_of_state[s] * a.H * a.W * 3 : nullptr;
    // the tile's 16 x 16 regions in row-major order, each walked on its own
    constexpr int rpx = 1 << (SHIFT - 4);
    uint32_t stop = 0;
    for (int reg = 0; reg < rpx * rpx; ++reg) {
        const Lane<NPAIR> L = lane_of<NPAIR>(tile, (reg % rpx) * BLOCK, (reg / rpx) * BLOCK, a);
        // a region of a 32 px tile can lie past the image edge (warp-uniform); 16 px tiles never do
        if (SHIFT > 4 && (L.rx0 >= a.W || L.ry0 >= a.H)) continue;
        FwdLane<NPAIR> f;
        f.init(L);
        const uint32_t e = walk(a, L, sm, rg.x, rg.y, f);
        stop = max(stop, e - rg.x);
        double se = 0.0;
#pragma unroll
        for (int j = 0; j < NPAIR; ++j) {
            f2 o0, o1, o2;
            f.out(j, a.bg0, a.bg1, a.bg2, o0, o1, o2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 2 * j + h;
                if (!((L.inimg >> r) & 1u)) continue;
                const float c0 = h ? hi(o0) : lo(o0), c1 = h ? hi(o1) : lo(o1), c2 = h ? hi(o2) : lo(o2);
                const size_t pix = (size_t)(L.py0 + r) * a.W + L.px;
                if (WRITE) {
                    float *dst = a.images + ((size_t)(s - a.img_s0) * a.H * a.W + pix) * 3;
                    dst[0] = c0; dst[1] = c1; dst[2] = c2;
                }
                if (MSE) {
                    const float *rp = rbase + pix * 3;
                    se += (double)pixel_sq_err(c0, c1, c2, rp[0], rp[1], rp[2]);
                    if (a.dL) {   // the loss gradient, as the separate image-MSE pass forms it
                        float *dst = a.dL + ((size_t)(s - a.img_s0) * a.H * a.W + pix) * 3;
                        dst[0] = a.gscale * (c0 - rp[0]);
                        dst[1] = a.gscale * (c1 - rp[1]);
                        dst[2] = a.gscale * (c2 - rp[2]);
                    }
                }
            }
        }
        if (MSE) {
            // one partial per 16 x 16 pixel block: the same sum whatever the tile size
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) se += __shfl_xor_sync(FULL, se, off);
            if (lane == 0)
                a.partial[(size_t)s * a.blocks + (size_t)(L.ry0 / BLOCK) * a.blocks_x + L.rx0 / BLOCK] = se;
        }
    }
    if (LIST && lane == 0) a.stop[(size_t)s * a.tiles + tile] = stop;
}

template <bool WRITE, bool MSE, bool LIST, int SHIFT>
__global__ void __launch_bounds__(RT, FWD_MIN_BLOCKS) k_raster_fwd(RasterArgs a, WorkQueue q)
{
    __shared__ WarpSmem smem[WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem &sm = smem[w];
    const uint32_t n_items = LIST ? *q.n_items_dev : q.n_items;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(q.counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) break;
        fwd_item<WRITE, MSE, LIST, SHIFT>(a, q, item, sm, lane);
        __syncwarp();
    }
}

static_assert(sizeof(RasterArgs) % 4 == 0 && sizeof(WorkQueue) % 4 == 0 && sizeof(RasterBwdArgs) % 4 == 0,
              "argument structs are copied word by word");
// Copy a struct of `bytes` (a multiple of 4) word by word across the warp.
__device__ __forceinline__ void copy_words(void *dst, const void *src, size_t bytes, int lane)
{
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    for (int i = lane; i < (int)(bytes / 4); i += 32) d[i] = s[i];
}

// The forward raster of several scenes in one persistent launch: job k has
// its own arguments and queue, its items are [item_off[k], item_off[k + 1])
// of one shared counter, so warps move on to any scene's work as they finish.
template <int SHIFT>
__global__ void __launch_bounds__(RT, FWD_MIN_BLOCKS) k_raster_fwd_multi(const RasterArgs *__restrict__ args,
                                                                          const WorkQueue *__restrict__ queues,
                                                                          const uint32_t *__restrict__ item_off,
                                                                          int n_jobs, uint32_t *counter)
{
    __shared__ WarpSmem smem[WARPS];
    __shared__ RasterArgs jargs[WARPS];        // the warp's current job, copied from global memory
    __shared__ __align__(16) unsigned char jqueue_raw[WARPS][sizeof(WorkQueue)];   // (WorkQueue has initialisers)
    WorkQueue *jqueue = reinterpret_cast<WorkQueue *>(&jqueue_raw[0][0]);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem &sm = smem[w];
    const uint32_t n_items = item_off[n_jobs];
    int job = -1;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) break;
        int lo = 0, hi = n_jobs - 1;           // the last job whose first item is <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= item) lo = mid; else hi = mid - 1;
        }
        if (lo != job) {
            copy_words(&jargs[w], &args[lo], sizeof(RasterArgs), lane);
            copy_words(&jqueue[w], &queues[lo], sizeof(WorkQueue), lane);
            __syncwarp();
            job = lo;
        }
        fwd_item<true, false, false, SHIFT>(jargs[w], jqueue[w], item - item_off[lo], sm, lane);
        __syncwarp();
    }
}

// ------------------------------------------------------------ adjoint
// Per-pixel state of the adjoint walk, for a pixel pair.  With gr = dL/dC .
// rgb_k and Qn = dL/dC . (colour accumulated up to and including k) -
// dL/dC . (C_final + T_final bg):
//   dL/dalpha_k = T_k gr + Qn / (1 - alpha_k)
// (the forward's final pixel is read from its image, or recomputed by a first
// walk).  T follows the forward exactly (same operations), so the walk stops
// where the forward stopped.
struct BwdPair {
    f2 T, Qn, g0, g1, g2;
};

// Sums of one entry over a lane's pixels, packed by pair row parity:
// S5 = sum dL/dpower, S1 = sum dL/dpower dy, S4 = sum dL/dpower dy^2 (dx is
// the lane's column: its moments follow from these), and the colour sums
// sum dL/dC (alpha T).  dy = my - pixel centre (the sign of the offsets does
// not matter to the moments the projection adjoint uses).
struct BwdSums {
    f2 S1, S4, S5, Sr, Sg, Sb;
};

template <bool FIRST, bool CLAMP>
__device__ __forceinline__ void bwd_pair(BwdPair &P, BwdSums &S, const Ent &E, f2 al, f2 ar, f2 dy)
{
    const f2 w = mul2(al, P.T);
    const f2 Tn = sub2(P.T, w);
    const f2 s = pk(ge1(lo(Tn), T_STOP), ge1(hi(Tn), T_STOP));   // 1: composite, 0: stop (or stopped)
    const f2 wp = mul2(w, s);
    const f2 gr = fma2(P.g2, E.b, fma2(P.g1, E.g, mul2(P.g0, E.r)));
    P.Qn = fma2(wp, gr, P.Qn);
    const f2 om = sub2(pk(1.0f, 1.0f), al);                        // >= 0.01
    const f2 da = fma2(P.Qn, pk(rcp(lo(om)), rcp(hi(om))), mul2(P.T, gr));
    // d alpha / d power = alpha on the linear range; 0 when skipped, stopped or clamped
    f2 alin = mul2(al, s);
    if (CLAMP) alin = mul2(alin, pk(lt1(lo(ar), A_MAX), lt1(hi(ar), A_MAX)));
    const f2 gpw = mul2(da, alin);
    const f2 t2 = mul2(gpw, dy);
    if (FIRST) {
        S.S1 = t2; S.S4 = mul2(t2, dy); S.S5 = gpw;
        S.Sr = mul2(P.g0, wp); S.Sg = mul2(P.g1, wp); S.Sb = mul2(P.g2, wp);
    } else {
        S.S1 = add2(S.S1, t2); S.S4 = fma2(t2, dy, S.S4); S.S5 = add2(S.S5, gpw);
        S.Sr = fma2(P.g0, wp, S.Sr); S.Sg = fma2(P.g1, wp, S.Sg); S.Sb = fma2(P.g2, wp, S.Sb);
    }
    P.T = mul2(Tn, s);
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
        u[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? u[i] : u[i + 2];
        const float keep = b3 ? u[i + 2] : u[i];
        w2[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    const float send = b2 ? w2[0] : w2[1];
    float x = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(FULL, send, 4);
    x += __shfl_xor_sync(FULL, x, 2);
    x += __shfl_xor_sync(FULL, x, 1);
    return x;
}

template <int NP>
struct BwdLane {
    static constexpr bool CLAMP_KINDS = true;
    // the batch leaves little L1 beside shared memory: the record prefetch
    // bypasses it (cp.async.cg; measured 0.5% faster than .ca here, 0.5%
    // slower in the forward)
    static constexpr bool RECS_L1 = false;
    BwdPair p[NP];
    float4 *rec_grad;
    RedBuf *rb;                       // the warp's batch of entry sums
    uint32_t nb;                      // entries in the batch
    __device__ __forceinline__ bool live() const
    {
        f2 any = 0ull;
#pragma unroll
        for (int j = 0; j < NP; ++j) any |= p[j].T;
        return __any_sync(FULL, any != 0ull);
    }
    template <bool BOXED, bool CLAMP>
    __device__ __forceinline__ void entry(const Queue &q, int k, const uint4 &s4, const Lane<NP> &L)
    {
        const Ent E = load_entry<NP, BOXED, true>(q, k, s4, L);
        BwdSums S;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            f2 dy, ar;
            const f2 al = pair_alpha<BOXED, CLAMP>(E, L.pcy[j], j, dy, ar);
            if (j == 0) bwd_pair<true, CLAMP>(p[j], S, E, al, ar, dy);
            else bwd_pair<false, CLAMP>(p[j], S, E, al, ar, dy);
        }
        const float s1 = lo(S.S1) + hi(S.S1), s4v = lo(S.S4) + hi(S.S4), s5 = lo(S.S5) + hi(S.S5);
        const float sr = lo(S.Sr) + hi(S.Sr), sg = lo(S.Sg) + hi(S.Sg), sb = lo(S.Sb) + hi(S.Sb);
        if (!BwdShape<NP>::BATCH) {
            // entries that changed no lane's sums are skipped with one vote
            const uint32_t nz = (__float_as_uint(s1) | __float_as_uint(s4v) | __float_as_uint(s5) |
                                 __float_as_uint(sr) | __float_as_uint(sg) | __float_as_uint(sb)) << 1;
            if (__any_sync(FULL, nz != 0u)) reduce_now(s4.w, L, E.dx, s1, s4v, s5, sr, sg, sb);
            return;
        }
        // every entry joins the batch (zero sums add nothing; a vote to skip
        // them cost more than the batch work it saved)
        // the lane's sums join the batch; the warp reduces a full batch at once
        float2 *row = rb->v + nb * (RB_STRIDE / 2);
        row[L.lane] = make_float2(s1, s4v);
        row[32 + L.lane] = make_float2(s5, sr);
        row[64 + L.lane] = make_float2(sg, sb);
        if (L.lane == 0) {
            rb->slot[nb] = s4.w;
            rb->mx[nb] = q.s3[k].x;
        }
        if (++nb == (uint32_t)RB) flush(L);
    }
    // One entry's warp reduction at once (no batch).
    __device__ __forceinline__ void reduce_now(uint32_t slot, const Lane<NP> &L, float dx, float s1, float s4,
                                               float s5, float sr, float sg, float sb)
    {
        // the entry's pixel moments over the lane's pixels (dx is the lane's column
        // offset, the same for all its pixels); the projection adjoint turns their
        // sums into the conic, mean and opacity gradients
        const float m0 = dx * s5;
        float v[8];
        v[0] = m0;                 // sum dL/dpower dx
        v[1] = s1;                 // sum dL/dpower dy
        v[2] = dx * m0;            // sum dL/dpower dx^2
        v[3] = dx * s1;            // sum dL/dpower dx dy
        v[4] = s4;                 // sum dL/dpower dy^2
        v[5] = s5;                 // sum dL/dpower
        v[6] = sr;                 // sum dL/dC alpha T (per channel)
        v[7] = sg;
        float x = reduce8_transpose(v, L.lane);
        float xb = sb;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) xb += __shfl_xor_sync(FULL, xb, off);
        // lane 4 j holds the total of v[j], lane 1 the blue sum
        if ((L.lane & 3) == 0 || L.lane == 1) {
            const int idx = L.lane == 1 ? 8 : (L.lane >> 2);
            float *dst = reinterpret_cast<float *>(rec_grad + (size_t)slot * 3);
            atomicAdd(dst + idx, L.lane == 1 ? xb : x);
        }
    }
    // Reduce the batch: four lanes per entry, lane 4 e + q summing source
    // lanes q, q + 4, ..., q + 28 of entry e, then a transpose over the four.
    // The moments over the source lane's pixels (dx is its column offset,
    // computed exactly as the entry's lanes compute it):
    //   v0 = S dL/dpower dx, v1 = S dL/dpower dy, v2 = S dL/dpower dx^2,
    //   v3 = S dL/dpower dx dy, v4 = S dL/dpower dy^2, v5 = S dL/dpower,
    //   v6, v7, blue = S dL/dC alpha T per channel;
    // the projection adjoint turns them into the conic, mean and opacity
    // gradients.  One atomic add per moment goes to the record.
    __device__ __forceinline__ void flush(const Lane<NP> &L)
    {
        __syncwarp();
        const int e = L.lane >> 2, qd = L.lane & 3;
        // the plain sums packed as (S1, S4), (S5, Sr), (Sg, Sb); the dx moments
        // per column (source lanes c and c + 16 share it)
        f2 a14 = 0ull, a5r = 0ull, agb = 0ull;
        float v0 = 0.0f, v2 = 0.0f, v3 = 0.0f;
        if (e < (int)nb) {
            const f2 *row = reinterpret_cast<const f2 *>(rb->v + e * (RB_STRIDE / 2));
            const float mx = rb->mx[e];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int l = qd + 4 * c;
                const f2 x0 = row[l], y0 = row[32 + l], z0 = row[64 + l];
                const f2 x1 = row[l + 16], y1 = row[48 + l], z1 = row[80 + l];
                a14 = add2(a14, add2(x0, x1));
                a5r = add2(a5r, add2(y0, y1));
                agb = add2(agb, add2(z0, z1));
                const float dx = __fsub_rn(mx, (float)(L.rx0 + l) + 0.5f);
                const float s5 = lo(y0) + lo(y1), s1 = lo(x0) + lo(x1);
                const float m0 = dx * s5;
                v0 += m0;
                v2 = fmaf(dx, m0, v2);
                v3 = fmaf(dx, s1, v3);
            }
        }
        float v[8] = {v0, lo(a14), v2, v3, hi(a14), lo(a5r), hi(a5r), lo(agb)};
        float blue = hi(agb);
        // fold the entry's four lanes: lane 4 e + q ends with v[2 q], v[2 q + 1]
        float u[4];
        const bool b1 = qd & 2, b0 = qd & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float send = b1 ? v[i] : v[i + 4], keep = b1 ? v[i + 4] : v[i];
            u[i] = keep + __shfl_xor_sync(FULL, send, 2);
        }
        float w[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = b0 ? u[i] : u[i + 2], keep = b0 ? u[i + 2] : u[i];
            w[i] = keep + __shfl_xor_sync(FULL, send, 1);
        }
        blue += __shfl_xor_sync(FULL, blue, 1);
        blue += __shfl_xor_sync(FULL, blue, 2);
        if (e < (int)nb) {
            float *dst = reinterpret_cast<float *>(rec_grad + (size_t)rb->slot[e] * 3);
            atomicAdd(dst + 2 * qd, w[0]);
            atomicAdd(dst + 2 * qd + 1, w[1]);
            if (qd == 0) atomicAdd(dst + 8, blue);
        }
        __syncwarp();
        nb = 0;
    }
    __device__ __forceinline__ void finish(const Lane<NP> &L)
    {
        if (BwdShape<NP>::BATCH && nb) flush(L);
    }
};

// Adjoint compositing, one warp per (16x16 region, state).  Transmittance is never
// stored: the walk goes front to back recomputing it, and for each included k
//   dC/drgb_k   = alpha_k T_k
//   dC/dalpha_k = rgb_k T_k - (C_after_k + T_final bg) / (1 - alpha_k)
// with C_after_k = C_final - (colour accumulated up to and including k).  The
// final pixel value is read from the forward's image (IMG) or recomputed by a
// first forward walk.  Per-Gaussian pixel moments: the lane's sums over its
// pixels, reduced over the warp eight entries at a time (16 x 16 regions) or
// entry by entry (16 x 8), one atomic add per moment.
// Work items of the adjoint raster of one call: (tile, 16x16 region, state).
__host__ __device__ __forceinline__ size_t bwd_items(const RasterArgs &a, int np)
{
    const int RH = 4 * np;
    const int regs = (1 << (a.tile_shift - 4)) * ((1 << a.tile_shift) / RH);
    return (size_t)a.tiles * regs * a.S;
}

// One adjoint work item (every lane of the warp calls it with the same item < bwd_items).
template <bool IMG, int NP>
__device__ __forceinline__ void bwd_item(const RasterBwdArgs &b, size_t item, WarpSmem &sm, RedBuf *rb)
{
    constexpr int RH = 4 * NP;     // region height (NP pixel pairs per lane)
    const RasterArgs &a = b.f;
    const int rpx = 1 << (a.tile_shift - 4), rpy = (1 << a.tile_shift) / RH, regs = rpx * rpy;
    const int s = (int)(item % (unsigned)a.S);
    const int tr = (int)(item / (unsigned)a.S), tile = tr / regs, reg = tr % regs;
    const Lane<NP> L = lane_of<NP>(tile, (reg % rpx) * BLOCK, (reg / rpx) * RH, a);
    if (L.rx0 >= a.W || L.ry0 >= a.H) return;        // region outside the image
    const int v = a.vg_of_state[s];
    load_depth(a, s, sm);
    const uint2 rg = a.ranges[(size_t)v * a.tiles + tile];

    // final pixel values
    float fin[NP][2][3];
    if (IMG) {
#pragma unroll
        for (int r = 0; r < 2 * NP; ++r) {
            float *f = fin[r >> 1][r & 1];
            f[0] = f[1] = f[2] = 0.0f;
            if ((L.inimg >> r) & 1u) {
                const float *ip = b.img_fwd + (((size_t)s * a.H + (L.py0 + r)) * a.W + L.px) * 3;
                f[0] = ip[0]; f[1] = ip[1]; f[2] = ip[2];
            }
        }
    } else {
        FwdLane<NP> f;
        f.init(L);
        walk(a, L, sm, rg.x, rg.y, f);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            f2 o0, o1, o2;
            f.out(j, a.bg0, a.bg1, a.bg2, o0, o1, o2);
            fin[j][0][0] = lo(o0); fin[j][0][1] = lo(o1); fin[j][0][2] = lo(o2);
            fin[j][1][0] = hi(o0); fin[j][1][1] = hi(o1); fin[j][1][2] = hi(o2);
        }
    }
    BwdLane<NP> B;
    B.rec_grad = b.rec_grad;
    B.rb = rb;
    B.nb = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        float g[2][3], T[2], Q[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = 2 * j + h;
            g[h][0] = g[h][1] = g[h][2] = 0.0f;
            if ((L.inimg >> r) & 1u) {
                const float *gp = b.dL_dimg + (((size_t)s * a.H + (L.py0 + r)) * a.W + L.px) * 3;
                g[h][0] = gp[0]; g[h][1] = gp[1]; g[h][2] = gp[2];
            }
            Q[h] = -(g[h][0] * fin[j][h][0] + g[h][1] * fin[j][h][1] + g[h][2] * fin[j][h][2]);
            T[h] = (g[h][0] != 0.0f || g[h][1] != 0.0f || g[h][2] != 0.0f) ? 1.0f : 0.0f;
        }
        B.p[j].T = pk(T[0], T[1]);
        B.p[j].Qn = pk(Q[0], Q[1]);
        B.p[j].g0 = pk(g[0][0], g[1][0]);
        B.p[j].g1 = pk(g[0][1], g[1][1]);
        B.p[j].g2 = pk(g[0][2], g[1][2]);
    }
    walk(a, L, sm, rg.x, rg.y, B);
}

// Dynamic shared memory of the adjoint kernels: WARPS WarpSmem, then (when
// batching) WARPS RedBuf.
template <int NP>
constexpr size_t bwd_smem()
{
    return WARPS * (sizeof(WarpSmem) + (BwdShape<NP>::BATCH ? sizeof(RedBuf) : 0));
}

template <int NP>
__device__ __forceinline__ RedBuf *red_buf(unsigned char *dsm, int w)
{
    return BwdShape<NP>::BATCH ? reinterpret_cast<RedBuf *>(dsm + WARPS * sizeof(WarpSmem)) + w : nullptr;
}

template <bool IMG, int NP>
__global__ void __launch_bounds__(RT, BwdShape<NP>::MIN_BLOCKS) k_raster_bwd(RasterBwdArgs b)
{
    extern __shared__ __align__(16) unsigned char bwd_dsm[];
    WarpSmem *smem = reinterpret_cast<WarpSmem *>(bwd_dsm);
    const int w = threadIdx.x >> 5;
    const size_t item = (size_t)blockIdx.x * WARPS + w;
    if (item >= bwd_items(b.f, NP)) return;
    bwd_item<IMG, NP>(b, item, smem[w], red_buf<NP>(bwd_dsm, w));
}

// The adjoint raster of several scenes in one launch: warp g takes item
// g - item_off[k] of job k, the last job with item_off[k] <= g.
__global__ void __launch_bounds__(RT, BwdShape<BWD_NP_BATCH>::MIN_BLOCKS) k_raster_bwd_multi(const RasterBwdArgs *__restrict__ jobs,
                                                                         const size_t *__restrict__ item_off,
                                                                         int n_jobs)
{
    extern __shared__ __align__(16) unsigned char bwd_dsm[];
    WarpSmem *smem = reinterpret_cast<WarpSmem *>(bwd_dsm);
    __shared__ RasterBwdArgs jargs[WARPS];     // the warp's job, copied from global memory
    const int w = threadIdx.x >> 5;
    const size_t g = (size_t)blockIdx.x * WARPS + w;
    if (g >= item_off[n_jobs]) return;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    copy_words(&jargs[w], &jobs[lo], sizeof(RasterBwdArgs), threadIdx.x & 31);
    __syncwarp();
    bwd_item<true, BWD_NP_BATCH>(jargs[w], g - item_off[lo], smem[w], red_buf<BWD_NP_BATCH>(bwd_dsm, w));
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
// of MSE_CHUNK_PIX pixels (four consecutive pixels per thread, read as three
// 16-byte vectors where aligned), and optionally
// dL/dimage = weight * 2 (image - ref) / (3 H W).
__global__ void __launch_bounds__(256) k_image_mse(const float *__restrict__ images, const float *__restrict__ refs,
                                                   const int32_t *__restrict__ ref_index, size_t npix,
                                                   float gscale, double *__restrict__ partial, int parts,
                                                   float *__restrict__ dL)
{
    static_assert(MSE_CHUNK_PIX == 4 * 256, "four pixels per thread");
    __shared__ double wsum[8];
    const int s = blockIdx.y;
    const float *im = images + (size_t)s * npix * 3;
    const float *rf = refs + (size_t)ref_index[s] * npix * 3;
    float *dl = dL ? dL + (size_t)s * npix * 3 : nullptr;
    const size_t p0 = (size_t)blockIdx.x * MSE_CHUNK_PIX + 4 * (size_t)threadIdx.x;
    float x[12], y[12];
    const bool vec = p0 + 4 <= npix && ((reinterpret_cast<uintptr_t>(im + 3 * p0) | reinterpret_cast<uintptr_t>(rf + 3 * p0) |
                                         (dl ? reinterpret_cast<uintptr_t>(dl + 3 * p0) : 0)) & 15) == 0;
    const int np = p0 >= npix ? 0 : (int)min((size_t)4, npix - p0);
    if (vec) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(im + 3 * p0) + q);
            const float4 b = __ldg(reinterpret_cast<const float4 *>(rf + 3 * p0) + q);
            x[4 * q] = a.x; x[4 * q + 1] = a.y; x[4 * q + 2] = a.z; x[4 * q + 3] = a.w;
            y[4 * q] = b.x; y[4 * q + 1] = b.y; y[4 * q + 2] = b.z; y[4 * q + 3] = b.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const bool in = k / 3 < np;
            x[k] = in ? __ldg(im + 3 * p0 + k) : 0.0f;
            y[k] = in ? __ldg(rf + 3 * p0 + k) : 0.0f;
        }
    }
    double se = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < np) se += (double)pixel_sq_err(x[3 * k], x[3 * k + 1], x[3 * k + 2], y[3 * k], y[3 * k + 1], y[3 * k + 2]);
    if (dl) {
        float d[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) d[k] = gscale * (x[k] - y[k]);
        if (vec) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                reinterpret_cast<float4 *>(dl + 3 * p0)[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k)
                if (k / 3 < np) dl[3 * p0 + k] = d[k];
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

// Resident blocks per SM of each forward instantiation (its register and
// shared-memory use), queried once and cached so that launches made during
// stream capture issue no runtime queries; the persistent grid is that many
// blocks per SM.
template <bool WRITE, bool MSE, bool LIST, int SHIFT>
static int fwd_occupancy()
{
    static int n = 0;
    if (!n) {
        int m = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_raster_fwd<WRITE, MSE, LIST, SHIFT>, RT, 0);
        n = m > 0 ? m : 1;
    }
    return n;
}

template <bool WRITE, bool MSE, bool LIST>
static void launch_fwd_t(const RasterArgs &a, const WorkQueue &q, int sms, cudaStream_t st)
{
    if (a.tile_shift == 5)
        k_raster_fwd<WRITE, MSE, LIST, 5><<<sms * fwd_occupancy<WRITE, MSE, LIST, 5>(), RT, 0, st>>>(a, q);
    else
        k_raster_fwd<WRITE, MSE, LIST, 4><<<sms * fwd_occupancy<WRITE, MSE, LIST, 4>(), RT, 0, st>>>(a, q);
}

template <int SHIFT>
static int fwd_multi_occupancy()
{
    static int n = 0;
    if (!n) {
        int m = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_raster_fwd_multi<SHIFT>, RT, 0);
        n = m > 0 ? m : 1;
    }
    return n;
}

void launch_raster_fwd_multi(const RasterArgs *args, const WorkQueue *queues, const uint32_t *item_off, int n_jobs,
                             uint32_t *counter, int tile_shift, int sms, cudaStream_t st)
{
    if (n_jobs <= 0) return;
    ProfScope ps_("raster_fwd", st);
    if (tile_shift == 5)
        k_raster_fwd_multi<5><<<sms * fwd_multi_occupancy<5>(), RT, 0, st>>>(args, queues, item_off, n_jobs, counter);
    else
        k_raster_fwd_multi<4><<<sms * fwd_multi_occupancy<4>(), RT, 0, st>>>(args, queues, item_off, n_jobs, counter);
    count_launch();
}

size_t raster_bwd_items(const RasterArgs &a)
{
    const int RH = 4 * BWD_NP_BATCH;
    const size_t regs = (size_t)(1 << (a.tile_shift - 4)) * (size_t)((1 << a.tile_shift) / RH);
    return (size_t)a.tiles * regs * (size_t)a.S;
}

void launch_raster_bwd_multi(const RasterBwdArgs *jobs, const size_t *item_off, int n_jobs, size_t total_items,
                             cudaStream_t st)
{
    if (n_jobs <= 0 || total_items == 0) return;
    ProfScope ps_("raster_bwd", st);
    k_raster_bwd_multi<<<(unsigned)((total_items + WARPS - 1) / WARPS), RT, bwd_smem<BWD_NP_BATCH>(), st>>>(jobs, item_off, n_jobs);
    count_launch();
}

template <bool WRITE, bool MSE, bool LIST>
static void query_t()
{
    fwd_occupancy<WRITE, MSE, LIST, 4>();
    fwd_occupancy<WRITE, MSE, LIST, 5>();
}

// Every work item is one (view-group tile, state); the explicit work list
// (tile reuse) renders squared-error partials only.  G (states per item) is 1.
void launch_raster_fwd(const RasterArgs &a, const WorkQueue &q, int G, int sms, cudaStream_t st)
{
    (void)G;
    if ((!q.item_first && q.n_items == 0) || (!a.images && !a.refs)) return;
    ProfScope ps_(a.refs ? "raster_fwd_mse" : "raster_fwd", st);
    if (q.item_first) launch_fwd_t<false, true, true>(a, q, sms, st);
    else if (a.images && a.refs) launch_fwd_t<true, true, false>(a, q, sms, st);
    else if (a.images) launch_fwd_t<true, false, false>(a, q, sms, st);
    else launch_fwd_t<false, true, false>(a, q, sms, st);
    count_launch();
}

template <class K>
static void bwd_attributes(K *kernel, size_t smem)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

// Occupancy queries (once per process) and kernel attributes (once per
// device), before any stream capture: a context's creation calls it.
void raster_fwd_query_occupancy()
{
    static uint64_t attr_done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !((attr_done >> dev) & 1u)) {
        bwd_attributes(k_raster_bwd<true, BWD_NP_BATCH>, bwd_smem<BWD_NP_BATCH>());
        bwd_attributes(k_raster_bwd<false, BWD_NP_BATCH>, bwd_smem<BWD_NP_BATCH>());
        bwd_attributes(k_raster_bwd<true, BWD_NP_FEW>, bwd_smem<BWD_NP_FEW>());
        bwd_attributes(k_raster_bwd<false, BWD_NP_FEW>, bwd_smem<BWD_NP_FEW>());
        bwd_attributes(k_raster_bwd_multi, bwd_smem<BWD_NP_BATCH>());
        attr_done |= 1ull << dev;
    }
    static bool done = false;
    if (done) return;
    query_t<true, true, false>();
    query_t<true, false, false>();
    query_t<false, true, false>();
    query_t<false, true, true>();
    fwd_multi_occupancy<4>();
    fwd_multi_occupancy<5>();
    done = true;
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

// One warp per (region, state), WARPS warps per block; the region height by
// the item count (see BwdShape).
void launch_raster_bwd(const RasterBwdArgs &b, int sms, cudaStream_t st)
{
    if (b.f.S == 0 || b.f.tiles == 0) return;
    const size_t big = bwd_items(b.f, BWD_NP_BATCH);
    const bool batch = big >= (size_t)2 * sms * BwdShape<BWD_NP_BATCH>::MIN_BLOCKS * WARPS;
    const size_t items = batch ? big : bwd_items(b.f, BWD_NP_FEW);
    const unsigned grid = (unsigned)((items + WARPS - 1) / WARPS);
    ProfScope ps_(b.img_fwd ? "raster_bwd" : "raster_bwd_2pass", st);
    if (batch) {
        if (b.img_fwd) k_raster_bwd<true, BWD_NP_BATCH><<<grid, RT, bwd_smem<BWD_NP_BATCH>(), st>>>(b);
        else k_raster_bwd<false, BWD_NP_BATCH><<<grid, RT, bwd_smem<BWD_NP_BATCH>(), st>>>(b);
    } else {
        if (b.img_fwd) k_raster_bwd<true, BWD_NP_FEW><<<grid, RT, bwd_smem<BWD_NP_FEW>(), st>>>(b);
        else k_raster_bwd<false, BWD_NP_FEW><<<grid, RT, bwd_smem<BWD_NP_FEW>(), st>>>(b);
    }
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
