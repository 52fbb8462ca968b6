// Tile rasterization of delivery states: forward compositing with an optional
// fused FP64 squared-error epilogue, and the adjoint compositing kernel.
//
// One 256-thread block renders one 16x16 tile of one state.  The tile's run of
// the batch-wide sorted entry list holds every depth variant any state of the
// view group needs; each batch of 256 entries is staged in shared memory
// keeping only the variants this state renders (variant depth == the state's
// delivered depth of the Gaussian's cluster), compacted in order.  Filtering
// a sorted run keeps it sorted, so every state sees exactly the (depth,
// Gaussian) order it would see alone: batched == per-state, bit for bit.
//
// Per pixel and staged Gaussian the work is a handful of FP32 ops and one
// MUFU exp: these kernels are ALU/issue bound, not HBM bound.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr int NW = TILE_PIX / 32;   // warps per block

struct Staged {
    float4 r0[TILE_PIX];   // mx, my, A, B
    float4 r1[TILE_PIX];   // C, o, r, g
    float4 r2[TILE_PIX];   // b, box x, box y, cd
    uint32_t slot[TILE_PIX];
    int wcnt[NW];
};

// Stage entries [start, min(start + 256, end)) of the tile run, keeping the
// variants this state renders.  Returns the kept count (same in every thread).
__device__ __forceinline__ int stage_batch(const Rec *__restrict__ recs, const uint32_t *__restrict__ evals,
                                           const uint8_t *sdep, uint32_t start, uint32_t end, Staged &sm)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t e = start + (uint32_t)t;
    bool keep = false;
    float4 x0 = make_float4(0, 0, 0, 0), x1 = x0, x2 = x0;
    uint32_t slot = 0;
    if (e < end) {
        slot = __ldg(evals + e);
        const float4 *p = reinterpret_cast<const float4 *>(recs + slot);
        x2 = __ldg(p + 2);
        const uint32_t cd = __float_as_uint(x2.w);
        keep = ((cd >> 12) & 0xfu) == (uint32_t)sdep[cd & 0xfffu];
        if (keep) { x0 = __ldg(p); x1 = __ldg(p + 1); }
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) sm.wcnt[w] = __popc(bal);
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const int c = sm.wcnt[k];
        base += (k < w) ? c : 0;
        total += c;
    }
    if (keep) {
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        sm.r0[pos] = x0; sm.r1[pos] = x1; sm.r2[pos] = x2; sm.slot[pos] = slot;
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ bool in_box(const float4 &r2, int px, int py)
{
    const uint32_t bx = __float_as_uint(r2.y), by = __float_as_uint(r2.z);
    return px >= (int)(bx & 0xffffu) && px <= (int)(bx >> 16) && py >= (int)(by & 0xffffu) && py <= (int)(by >> 16);
}

// power = -1/2 (A dx^2 + C dy^2) - B dx dy, with explicit rounding so every
// kernel that evaluates it gets the same bits.
__device__ __forceinline__ float power_of(float A, float B, float C, float dx, float dy)
{
    const float q = __fmaf_rn(A, __fmul_rn(dx, dx), __fmul_rn(C, __fmul_rn(dy, dy)));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(B, __fmul_rn(dx, dy)));
}

__device__ __forceinline__ void load_depth_row(const uint8_t *depth, int s, int C, uint8_t *sdep)
{
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdep[c] = depth[(size_t)s * C + c];
}

template <bool WRITE, bool MSE>
__global__ void __launch_bounds__(TILE_PIX) k_raster_fwd(RasterArgs a)
{
    __shared__ Staged sm;
    __shared__ uint8_t sdep[MAX_CLUSTERS];
    __shared__ double wsum[NW];
    const int tile = (int)(blockIdx.x / (unsigned)a.S), s = (int)(blockIdx.x % (unsigned)a.S);
    const int v = a.vg_of_state[s];
    load_depth_row(a.depth, s, a.C, sdep);
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int px = tx * TILE + (threadIdx.x & (TILE - 1)), py = ty * TILE + (threadIdx.x / TILE);
    const bool inside = px < a.W && py < a.H;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const uint2 rg = a.ranges[(size_t)v * a.tiles + tile];
    float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    bool done = !inside;
    for (uint32_t start = rg.x; start < rg.y; start += TILE_PIX) {
        if (__syncthreads_count(!done) == 0) break;
        const int nk = stage_batch(a.recs, a.evals, sdep, start, rg.y, sm);
        if (done) continue;
        for (int k = 0; k < nk; ++k) {
            const float4 r2 = sm.r2[k];
            if (!in_box(r2, px, py)) continue;
            const float4 r0 = sm.r0[k], r1 = sm.r1[k];
            const float dx = __fsub_rn(r0.x, pcx), dy = __fsub_rn(r0.y, pcy);
            const float pw = power_of(r0.z, r0.w, r1.x, dx, dy);
            if (pw > 0.0f) continue;
            const float alpha = fminf(0.99f, __fmul_rn(r1.y, __expf(pw)));
            if (alpha < (1.0f / 255.0f)) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
            if (Tn < 1e-4f) { done = true; break; }
            const float wgt = __fmul_rn(alpha, T);
            c0 = __fmaf_rn(r1.z, wgt, c0);
            c1 = __fmaf_rn(r1.w, wgt, c1);
            c2 = __fmaf_rn(r2.x, wgt, c2);
            T = Tn;
        }
    }
    const float o0 = __fmaf_rn(T, a.bg0, c0), o1 = __fmaf_rn(T, a.bg1, c1), o2 = __fmaf_rn(T, a.bg2, c2);
    if (WRITE && inside) {
        float *dst = a.images + (((size_t)s * a.H + py) * a.W + px) * 3;
        dst[0] = o0; dst[1] = o1; dst[2] = o2;
    }
    if (MSE) {
        double se = 0.0;
        if (inside) {
            const float *rp = a.refs + (((size_t)a.ref_of_state[s] * a.H + py) * a.W + px) * 3;
            const double d0 = (double)o0 - (double)rp[0], d1 = (double)o1 - (double)rp[1];
            const double d2 = (double)o2 - (double)rp[2];
            se = d0 * d0 + d1 * d1 + d2 * d2;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = se;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) tot += wsum[w];
            a.partial[(size_t)s * a.tiles + tile] = tot;
        }
    }
}

// Adjoint compositing.  Pass 1 re-runs the forward walk to get each pixel's
// final colour, final transmittance and stop position; pass 2 walks front to
// back again and, for each included Gaussian k,
//   dC/drgb_k   = alpha_k T_k
//   dC/dalpha_k = rgb_k T_k - (C_after_k + T_final bg) / (1 - alpha_k)
// where C_after_k = C_final - (colour accumulated up to and including k).
// Per-Gaussian sums are reduced per warp, then per block in shared memory,
// then added to the record's gradient with one float4 atomic per 4 values.
__global__ void __launch_bounds__(TILE_PIX) k_raster_bwd(RasterBwdArgs b)
{
    const RasterArgs &a = b.f;
    __shared__ Staged sm;
    __shared__ uint8_t sdep[MAX_CLUSTERS];
    __shared__ float gacc[TILE_PIX][9];
    const int tile = (int)(blockIdx.x / (unsigned)a.S), s = (int)(blockIdx.x % (unsigned)a.S);
    const int lane = threadIdx.x & 31;
    const int v = a.vg_of_state[s];
    load_depth_row(a.depth, s, a.C, sdep);
    for (int j = threadIdx.x; j < TILE_PIX * 9; j += TILE_PIX) (&gacc[0][0])[j] = 0.0f;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int px = tx * TILE + (threadIdx.x & (TILE - 1)), py = ty * TILE + (threadIdx.x / TILE);
    const bool inside = px < a.W && py < a.H;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const uint2 rg = a.ranges[(size_t)v * a.tiles + tile];

    // ---- pass 1: forward walk
    float T = 1.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    bool done = !inside;
    uint32_t stop = 0xffffffffu, kept = 0;
    for (uint32_t start = rg.x; start < rg.y; start += TILE_PIX) {
        if (__syncthreads_count(!done) == 0) break;
        const int nk = stage_batch(a.recs, a.evals, sdep, start, rg.y, sm);
        if (!done) {
            for (int k = 0; k < nk; ++k) {
                const float4 r2 = sm.r2[k];
                if (!in_box(r2, px, py)) continue;
                const float4 r0 = sm.r0[k], r1 = sm.r1[k];
                const float dx = __fsub_rn(r0.x, pcx), dy = __fsub_rn(r0.y, pcy);
                const float pw = power_of(r0.z, r0.w, r1.x, dx, dy);
                if (pw > 0.0f) continue;
                const float alpha = fminf(0.99f, __fmul_rn(r1.y, __expf(pw)));
                if (alpha < (1.0f / 255.0f)) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                if (Tn < 1e-4f) { done = true; stop = kept + (uint32_t)k; break; }
                const float wgt = __fmul_rn(alpha, T);
                c0 = __fmaf_rn(r1.z, wgt, c0);
                c1 = __fmaf_rn(r1.w, wgt, c1);
                c2 = __fmaf_rn(r2.x, wgt, c2);
                T = Tn;
            }
        }
        kept += (uint32_t)nk;
    }
    const float Tf = T, Cf0 = c0, Cf1 = c1, Cf2 = c2;
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    if (inside) {
        const float *gp = b.dL_dimg + (((size_t)s * a.H + py) * a.W + px) * 3;
        g0 = gp[0]; g1 = gp[1]; g2 = gp[2];
    }
    const float sb0 = Tf * a.bg0, sb1 = Tf * a.bg1, sb2 = Tf * a.bg2;

    // ---- pass 2: gradients
    T = 1.0f; c0 = 0.0f; c1 = 0.0f; c2 = 0.0f;
    bool active = inside && stop > 0 && (g0 != 0.0f || g1 != 0.0f || g2 != 0.0f);
    kept = 0;
    for (uint32_t start = rg.x; start < rg.y; start += TILE_PIX) {
        if (__syncthreads_count(active) == 0) break;
        const int nk = stage_batch(a.recs, a.evals, sdep, start, rg.y, sm);
        for (int k = 0; k < nk; ++k) {
            float gv[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) gv[j] = 0.0f;
            bool contrib = false;
            if (active && kept + (uint32_t)k >= stop) active = false;
            if (active) {
                const float4 r2 = sm.r2[k];
                if (in_box(r2, px, py)) {
                    const float4 r0 = sm.r0[k], r1 = sm.r1[k];
                    const float dx = __fsub_rn(r0.x, pcx), dy = __fsub_rn(r0.y, pcy);
                    const float pw = power_of(r0.z, r0.w, r1.x, dx, dy);
                    if (pw <= 0.0f) {
                        const float ex = __expf(pw);
                        const float araw = __fmul_rn(r1.y, ex);
                        const float alpha = fminf(0.99f, araw);
                        if (alpha >= (1.0f / 255.0f)) {
                            const float one_m = __fsub_rn(1.0f, alpha);
                            const float wgt = __fmul_rn(alpha, T);
                            c0 = __fmaf_rn(r1.z, wgt, c0);
                            c1 = __fmaf_rn(r1.w, wgt, c1);
                            c2 = __fmaf_rn(r2.x, wgt, c2);
                            const float inv = 1.0f / one_m;
                            const float da = g0 * (r1.z * T - ((Cf0 - c0) + sb0) * inv) +
                                             g1 * (r1.w * T - ((Cf1 - c1) + sb1) * inv) +
                                             g2 * (r2.x * T - ((Cf2 - c2) + sb2) * inv);
                            gv[6] = g0 * wgt; gv[7] = g1 * wgt; gv[8] = g2 * wgt;
                            if (araw < 0.99f) {
                                const float gpw = da * alpha;
                                gv[5] = da * ex;
                                gv[0] = -gpw * (r0.z * dx + r0.w * dy);
                                gv[1] = -gpw * (r1.x * dy + r0.w * dx);
                                gv[2] = -0.5f * gpw * dx * dx;
                                gv[3] = -gpw * dx * dy;
                                gv[4] = -0.5f * gpw * dy * dy;
                            }
                            T = __fmul_rn(T, one_m);
                            contrib = true;
                        }
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    float x = gv[j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    gv[j] = x;
                }
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < 9; ++j) atomicAdd(&gacc[k][j], gv[j]);
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nk; k += TILE_PIX) {
            float x[9];
            bool any = false;
#pragma unroll
            for (int j = 0; j < 9; ++j) { x[j] = gacc[k][j]; gacc[k][j] = 0.0f; any |= (x[j] != 0.0f); }
            if (any) {
                float4 *dst = b.rec_grad + (size_t)sm.slot[k] * 3;
                atomicAdd(dst, make_float4(x[0], x[1], x[2], x[3]));
                atomicAdd(dst + 1, make_float4(x[4], x[5], x[6], x[7]));
                atomicAdd(dst + 2, make_float4(x[8], 0.0f, 0.0f, 0.0f));
            }
        }
        kept += (uint32_t)nk;
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

// Squared-error partial sums of image s vs refs[ref_index[s]] over one chunk of
// 256 * 16 values, and optionally dL/dimage = weight * 2 (image - ref) / count.
__global__ void __launch_bounds__(256) k_image_mse(const float *__restrict__ images, const float *__restrict__ refs,
                                                   const int32_t *__restrict__ ref_index, size_t per_image,
                                                   float gscale, double *__restrict__ partial, int parts,
                                                   float *__restrict__ dL)
{
    __shared__ double wsum[8];
    const int s = blockIdx.y;
    const float *im = images + (size_t)s * per_image;
    const float *rf = refs + (size_t)ref_index[s] * per_image;
    double se = 0.0;
    const size_t base = (size_t)blockIdx.x * 4096;
    for (int k = 0; k < 16; ++k) {
        const size_t j = base + (size_t)k * 256 + threadIdx.x;
        if (j < per_image) {
            const float x = im[j], y = rf[j];
            const double d = (double)x - (double)y;
            se += d * d;
            if (dL) dL[(size_t)s * per_image + j] = gscale * (x - y);
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

void launch_raster_fwd(const RasterArgs &a, cudaStream_t st)
{
    if (a.S == 0 || a.tiles == 0 || (!a.images && !a.refs)) return;
    // one block per (tile, state), tile-major so states sharing a tile list run together
    const unsigned grid = a.tiles * (unsigned)a.S;
    ProfScope ps_(a.refs ? "raster_fwd_mse" : "raster_fwd", st);
    if (a.images && a.refs) k_raster_fwd<true, true><<<grid, TILE_PIX, 0, st>>>(a);
    else if (a.images) k_raster_fwd<true, false><<<grid, TILE_PIX, 0, st>>>(a);
    else k_raster_fwd<false, true><<<grid, TILE_PIX, 0, st>>>(a);
    count_launch();
}

void launch_raster_bwd(const RasterBwdArgs &b, cudaStream_t st)
{
    if (b.f.S == 0 || b.f.tiles == 0) return;
    const unsigned grid = b.f.tiles * (unsigned)b.f.S;
    ProfScope ps_("raster_bwd", st);
    k_raster_bwd<<<grid, TILE_PIX, 0, st>>>(b);
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
    const size_t per = (size_t)H * W * 3;
    const float gscale = (float)(2.0 * (double)weight / (double)per);
    dim3 grid((unsigned)parts, (unsigned)S);
    ProfScope ps_("image_mse", st);
    k_image_mse<<<grid, 256, 0, st>>>(images, refs, ref_index, per, gscale, partial, parts, dL);
    count_launch();
}

}  // namespace dgs
