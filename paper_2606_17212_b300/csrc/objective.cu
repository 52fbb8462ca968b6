// The packet-conditioned training objective (Section 4, Eq. 2) over a batch of
// rendered states, forward and gradient:
//   D_s = MSE(I_s, ref_s) + w_ssim (1 - SSIM(I_s, ref_s))
//   L   = mean_s D_s + lambda_c CVaR_q(D) + lambda_t F + lambda_m M + a mean_{s in anchors} D_s
// (the rate term has weight 0 in the paper's locked setting and is absent).
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5), zero-padded same-size
// filtering, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels.  Its
// local statistics are separable blurs done in shared memory per 32x16 tile
// (5-pixel halo); the forward writes, per pixel and channel, the derivatives of
// the SSIM value with respect to the three blurred moments it depends on
// (mean of x, of x^2, of x y), and the gradient kernel blurs those back:
//   dSSIM/dx = (G * d_mx + 2 x (G * d_exx) + y (G * d_exy)) / (3 H W).
// Everything is FP32 except the sums over pixels, states and pairs (FP64;
// the SSIM forward adds each thread's six values in FP32 first).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr int OT_W = 32, OT_H = 16;          // output tile
constexpr int HR = 5;                        // window radius (11 taps)
constexpr int RG_W = OT_W + 2 * HR, RG_H = OT_H + 2 * HR;   // 42 x 26 region
constexpr int OT_THREADS = 256;
constexpr float SSIM_C1 = 0.01f * 0.01f, SSIM_C2 = 0.03f * 0.03f;
// The blurs keep each thread's inputs in registers: a horizontal-pass thread
// makes HX consecutive outputs of one region row from 2 HR + HX inputs, a
// vertical-pass thread VY consecutive output rows of one column.  Every
// output is still the sum over the 11 taps in tap order (the same fmaf
// chain), so the maps are the plain per-output filter's, bit for bit.
constexpr int HX = 4, VY = 2;
constexpr int HS = OT_W + 1;                 // padded row stride of the horizontal results

// Two FP32 values in one 64-bit register pair, each lane rounded as the
// scalar IEEE operation.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpk(f2 x, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
#pragma nv_diag_suppress 550
__device__ __forceinline__ float lo(f2 x)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
    return a;
}
#pragma nv_diag_default 550
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The normalised 11-tap Gaussian window (sigma 1.5), computed by every thread.
__device__ __forceinline__ void window(float *g)
{
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 2 * HR + 1; ++k) {
        const float d = (float)(k - HR);
        g[k] = expf(-d * d / (2.0f * 1.5f * 1.5f));
        s += g[k];
    }
#pragma unroll
    for (int k = 0; k < 2 * HR + 1; ++k) g[k] /= s;
}

__device__ double block_sum_d(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < OT_THREADS / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Forward: one block per (32x16 tile, state).  Writes the three per-pixel
// derivative maps (channel-planar [S][3][H][W] each) and the tile's FP64 sums
// of the SSIM values and of the squared errors (part[s][tile][0..1]).
__global__ void __launch_bounds__(OT_THREADS, 5) k_ssim_fwd(const float *__restrict__ images,
                                                         const float *__restrict__ refs,
                                                         const int32_t *__restrict__ ref_index, int H, int W,
                                                         int tiles_x, int n_tiles, float *__restrict__ d_mx,
                                                         float *__restrict__ d_exx, float *__restrict__ d_exy,
                                                         double *__restrict__ part)
{
    static_assert(RG_H * (OT_W / HX) <= OT_THREADS && OT_W * OT_H == OT_THREADS * VY, "blur thread layout");
    __shared__ float xs[RG_H][RG_W * 3], ys[RG_H][RG_W * 3];       // region, channel-interleaved rows
    __shared__ f2 hm[RG_H][HS], hq[RG_H][HS];     // row blurs of (x, y) and (x^2, y^2)
    __shared__ float hc[RG_H][HS];                 // row blur of x y
    __shared__ double red[OT_THREADS / 32];
    const int tile = blockIdx.x % n_tiles, s = blockIdx.x / n_tiles;
    const int x0 = (tile % tiles_x) * OT_W, y0 = (tile / tiles_x) * OT_H;
    const size_t npix = (size_t)H * W;
    const float *img = images + (size_t)s * npix * 3;
    const float *ref = refs + (size_t)ref_index[s] * npix * 3;
    float g[2 * HR + 1];
    window(g);
    f2 G[2 * HR + 1];
#pragma unroll
    for (int k = 0; k < 2 * HR + 1; ++k) G[k] = pk(g[k], g[k]);
    // the region, warp by row and lane by float of the channel-interleaved row
    // (float f of a row lies in the image iff 0 <= (x0 - HR) 3 + f < 3 W)
    for (int r = threadIdx.x >> 5; r < RG_H; r += OT_THREADS / 32) {
        const int gy = y0 - HR + r;
        const long long f0 = (long long)(x0 - HR) * 3;
        const bool row_in = gy >= 0 && gy < H;
        for (int q = threadIdx.x & 31; q < RG_W * 3; q += 32) {
            const long long f = f0 + q;
            const bool in = row_in && f >= 0 && f < 3LL * W;
            const size_t o = (size_t)gy * W * 3 + (size_t)f;
            xs[r][q] = in ? img[o] : 0.0f;
            ys[r][q] = in ? ref[o] : 0.0f;
        }
    }
    __syncthreads();
    // each thread's six values (two rows, three channels) summed in FP32, then
    // FP64 over the block: the FP64 pipe is slow, and six FP32 additions err
    // by ~1e-7 relative
    float fsum32 = 0.0f, esum32 = 0.0f;
    for (int c = 0; c < 3; ++c) {
        // horizontal pass over the region rows, the tile's columns: thread
        // (row r, columns c0 .. c0 + HX - 1)
        if (threadIdx.x < RG_H * (OT_W / HX)) {
            const int r = threadIdx.x / (OT_W / HX), c0 = (threadIdx.x % (OT_W / HX)) * HX;
            f2 m[HX], q[HX];
            float xy[HX];
#pragma unroll
            for (int j = 0; j < HX; ++j) { m[j] = q[j] = 0ull; xy[j] = 0.0f; }
#pragma unroll
            for (int i = 0; i < HX + 2 * HR; ++i) {
                const float xv = xs[r][(c0 + i) * 3 + c], yv = ys[r][(c0 + i) * 3 + c];
                const f2 v = pk(xv, yv), v2 = mul2(v, v);
                const float vxy = xv * yv;
#pragma unroll
                for (int j = 0; j < HX; ++j) {
                    const int k = i - j;
                    if (k < 0 || k > 2 * HR) continue;
                    m[j] = fma2(G[k], v, m[j]);
                    q[j] = fma2(G[k], v2, q[j]);
                    xy[j] = fmaf(lo(G[k]), vxy, xy[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < HX; ++j) { hm[r][c0 + j] = m[j]; hq[r][c0 + j] = q[j]; hc[r][c0 + j] = xy[j]; }
        }
        __syncthreads();
        // vertical pass and the per-pixel value and derivatives: thread
        // (column col, rows r0 .. r0 + VY - 1)
        const int col = threadIdx.x % OT_W, r0 = (threadIdx.x / OT_W) * VY;
        f2 mm[VY], qq[VY];
        float cc[VY];
#pragma unroll
        for (int j = 0; j < VY; ++j) { mm[j] = qq[j] = 0ull; cc[j] = 0.0f; }
#pragma unroll
        for (int i = 0; i < VY + 2 * HR; ++i) {
            const f2 a = hm[r0 + i][col], b = hq[r0 + i][col];
            const float e = hc[r0 + i][col];
#pragma unroll
            for (int j = 0; j < VY; ++j) {
                const int k = i - j;
                if (k < 0 || k > 2 * HR) continue;
                mm[j] = fma2(G[k], a, mm[j]);
                qq[j] = fma2(G[k], b, qq[j]);
                cc[j] = fmaf(lo(G[k]), e, cc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < VY; ++j) {
            const int r = r0 + j;
            const int gy = y0 + r, gx = x0 + col;
            float mx, my, exx, eyy;
            unpk(mm[j], mx, my);
            unpk(qq[j], exx, eyy);
            const float exy = cc[j];
            if (gy < H && gx < W) {
                const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                const float a1 = 2.f * mx * my + SSIM_C1, a2 = 2.f * sxy + SSIM_C2;
                const float b1 = mx * mx + my * my + SSIM_C1, b2 = sxx + syy + SSIM_C2;
                // four fast reciprocals (relative error ~1e-7) instead of IEEE divisions
                const float ra1 = __fdividef(1.f, a1), ra2 = __fdividef(1.f, a2);
                const float rb1 = __fdividef(1.f, b1), rb2 = __fdividef(1.f, b2);
                const float f = a1 * a2 * rb1 * rb2;
                const size_t o = ((size_t)s * 3 + c) * npix + (size_t)gy * W + gx;
                d_mx[o] = 2.f * f * (my * (ra1 - ra2) + mx * (rb2 - rb1));
                d_exx[o] = -f * rb2;
                d_exy[o] = 2.f * f * ra2;
                fsum32 += f;
                const float d = xs[r + HR][(col + HR) * 3 + c] - ys[r + HR][(col + HR) * 3 + c];
                esum32 += d * d;
            }
        }
        __syncthreads();
    }
    const double fsum = block_sum_d((double)fsum32, red);
    const double esum = block_sum_d((double)esum32, red);
    if (threadIdx.x == 0) {
        part[((size_t)s * n_tiles + tile) * 2 + 0] = fsum;
        part[((size_t)s * n_tiles + tile) * 2 + 1] = esum;
    }
}

// Temporal pairs: FP64 partial sums over chunks of 1024 pixels of
// || (I_j - I_i) - (R_j - R_i) ||^2; tpart[pair][chunk].
__global__ void __launch_bounds__(256) k_temporal(const float *__restrict__ images, const float *__restrict__ refs,
                                                  const int32_t *__restrict__ ref_index,
                                                  const int2 *__restrict__ pairs, size_t npix, int chunks,
                                                  double *__restrict__ tpart)
{
    __shared__ double red[8];
    const int pr = blockIdx.y;
    const int2 pq = pairs[pr];
    const float *ii = images + (size_t)pq.x * npix * 3, *ij = images + (size_t)pq.y * npix * 3;
    const float *ri = refs + (size_t)ref_index[pq.x] * npix * 3, *rj = refs + (size_t)ref_index[pq.y] * npix * 3;
    double acc = 0.0;
    const size_t base = (size_t)blockIdx.x * 1024 * 3;
    for (int k = threadIdx.x; k < 1024 * 3; k += 256) {
        const size_t o = base + k;
        if (o < npix * 3) {
            const float e = (ij[o] - ii[o]) - (rj[o] - ri[o]);
            acc += (double)(e * e);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        tpart[(size_t)pr * chunks + blockIdx.x] = t;
    }
}

// One block: per-state D, the CVaR tail (the ceil(q S) largest D, ties to the
// lower state index), the prefix hinge M, the anchor term, F and L; the
// per-state weights dL/dD_s.  Sorts (D, index) pairs in dynamic shared memory.
__global__ void __launch_bounds__(1024) k_objective(const double *__restrict__ part, int n_tiles,
                                                    const double *__restrict__ tpart, int chunks, int n_t,
                                                    const int2 *__restrict__ pm, int n_m,
                                                    const int32_t *__restrict__ anchors, int n_a, int S,
                                                    double inv_vals, ObjectiveParams prm, double *__restrict__ D,
                                                    double *__restrict__ weight, double *__restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ double red[32];
    int P = 1;
    while (P < S) P <<= 1;
    double *key = reinterpret_cast<double *>(dyn);           // [P] -D (ascending = largest D first)
    int *idx2 = reinterpret_cast<int *>(key + P);            // [P] state index
    double dsum = 0.0;
    for (int s = threadIdx.x; s < P; s += blockDim.x) {
        if (s < S) {
            double f = 0.0, e = 0.0;
            for (int t = 0; t < n_tiles; ++t) {
                f += part[((size_t)s * n_tiles + t) * 2 + 0];
                e += part[((size_t)s * n_tiles + t) * 2 + 1];
            }
            const double d = e * inv_vals + prm.ssim_weight * (1.0 - f * inv_vals);
            D[s] = d;
            weight[s] = 1.0 / (double)S;
            dsum += d;
            key[s] = -d;
            idx2[s] = s;
        } else {
            key[s] = __longlong_as_double(0x7ff0000000000000LL);   // +inf sorts last
            idx2[s] = 0x7fffffff;
        }
    }
    // block sum of D
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dsum;
    __syncthreads();
    // bitonic sort of (key, index), ascending by key then index
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const double ka = key[i], kb = key[ixj];
                    const int ia = idx2[i], ib = idx2[ixj];
                    const bool gt = ka > kb || (ka == kb && ia > ib);
                    const bool up = (i & k) == 0;
                    if (gt == up) { key[i] = kb; key[ixj] = ka; idx2[i] = ib; idx2[ixj] = ia; }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += red[w];
        const double meanD = tot / (double)S;
        const int kc = (int)ceil(prm.cvar_q * (double)S);
        double cvar = 0.0;
        for (int t = 0; t < kc; ++t) {
            cvar -= key[t];
            weight[idx2[t]] += prm.lambda_c / (double)kc;
        }
        cvar = kc > 0 ? cvar / (double)kc : 0.0;
        double M = 0.0;
        for (int p = 0; p < n_m; ++p) {
            const int i = pm[p].x, j = pm[p].y;
            if (D[j] > D[i]) {
                M += (D[j] - D[i]) / (double)n_m;
                weight[j] += prm.lambda_m / (double)n_m;
                weight[i] -= prm.lambda_m / (double)n_m;
            }
        }
        double A = 0.0;
        for (int a = 0; a < n_a; ++a) {
            A += D[anchors[a]] / (double)n_a;
            weight[anchors[a]] += prm.anchor_weight / (double)n_a;
        }
        double F = 0.0;
        for (int p = 0; p < n_t; ++p) {
            double e = 0.0;
            for (int c = 0; c < chunks; ++c) e += tpart[(size_t)p * chunks + c];
            F += e * inv_vals / (double)n_t;
        }
        *loss = meanD + prm.lambda_c * cvar + prm.lambda_t * F + prm.lambda_m * M + prm.anchor_weight * A;
    }
}

// Gradient: one block per (32x16 tile, state).  Blurs the three derivative
// maps back per channel and writes
//   dL/dI_s = weight_s (2 (x - y) / N - w_ssim dSSIM/dx) + temporal terms,
// with the temporal terms +-lambda_t 2 e / (N n_t) of every pair holding s
// (tlist: CSR over states of (partner, +1 for the later state / -1 for the
// earlier one)).
__global__ void __launch_bounds__(OT_THREADS) k_objective_grad(
    const float *__restrict__ images, const float *__restrict__ refs, const int32_t *__restrict__ ref_index,
    int H, int W, int tiles_x, int n_tiles, const float *__restrict__ d_mx, const float *__restrict__ d_exx,
    const float *__restrict__ d_exy, const double *__restrict__ weight, float ssim_weight, float tscale,
    const int32_t *__restrict__ toff, const int2 *__restrict__ tlist, float *__restrict__ dL)
{
    __shared__ float pm_[RG_H][RG_W], pxx[RG_H][RG_W], pxy[RG_H][RG_W];
    __shared__ f2 hmx[RG_H][HS];                   // row blurs of (d_mx, d_exx)
    __shared__ float hxy[RG_H][HS];                // row blur of d_exy
    const int tile = blockIdx.x % n_tiles, s = blockIdx.x / n_tiles;
    const int x0 = (tile % tiles_x) * OT_W, y0 = (tile / tiles_x) * OT_H;
    const size_t npix = (size_t)H * W;
    const float inv_n = 1.0f / (float)(npix * 3);
    const float ws = (float)weight[s];
    const float *img = images + (size_t)s * npix * 3;
    const float *ref = refs + (size_t)ref_index[s] * npix * 3;
    float g[2 * HR + 1];
    window(g);
    f2 G[2 * HR + 1];
#pragma unroll
    for (int k = 0; k < 2 * HR + 1; ++k) G[k] = pk(g[k], g[k]);
    const int t0 = toff[s], t1 = toff[s + 1];
    for (int c = 0; c < 3; ++c) {
        const size_t plane = ((size_t)s * 3 + c) * npix;
        for (int i = threadIdx.x; i < RG_H * RG_W; i += OT_THREADS) {
            const int r = i / RG_W, q = i % RG_W;
            const int gy = y0 - HR + r, gx = x0 - HR + q;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const size_t o = plane + (size_t)gy * W + gx;
            pm_[r][q] = in ? d_mx[o] : 0.0f;
            pxx[r][q] = in ? d_exx[o] : 0.0f;
            pxy[r][q] = in ? d_exy[o] : 0.0f;
        }
        __syncthreads();
        // horizontal pass: thread (row r, columns c0 .. c0 + HX - 1)
        if (threadIdx.x < RG_H * (OT_W / HX)) {
            const int r = threadIdx.x / (OT_W / HX), c0 = (threadIdx.x % (OT_W / HX)) * HX;
            f2 ab[HX];
            float e[HX];
#pragma unroll
            for (int j = 0; j < HX; ++j) { ab[j] = 0ull; e[j] = 0.0f; }
#pragma unroll
            for (int i = 0; i < HX + 2 * HR; ++i) {
                const f2 v = pk(pm_[r][c0 + i], pxx[r][c0 + i]);
                const float w = pxy[r][c0 + i];
#pragma unroll
                for (int j = 0; j < HX; ++j) {
                    const int k = i - j;
                    if (k < 0 || k > 2 * HR) continue;
                    ab[j] = fma2(G[k], v, ab[j]);
                    e[j] = fmaf(g[k], w, e[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < HX; ++j) { hmx[r][c0 + j] = ab[j]; hxy[r][c0 + j] = e[j]; }
        }
        __syncthreads();
        // vertical pass: thread (column col, rows r0 .. r0 + VY - 1)
        const int col = threadIdx.x % OT_W, r0 = (threadIdx.x / OT_W) * VY;
        f2 vb[VY];
        float vc[VY];
#pragma unroll
        for (int j = 0; j < VY; ++j) { vb[j] = 0ull; vc[j] = 0.0f; }
#pragma unroll
        for (int i = 0; i < VY + 2 * HR; ++i) {
            const f2 a = hmx[r0 + i][col];
            const float w = hxy[r0 + i][col];
#pragma unroll
            for (int j = 0; j < VY; ++j) {
                const int k = i - j;
                if (k < 0 || k > 2 * HR) continue;
                vb[j] = fma2(G[k], a, vb[j]);
                vc[j] = fmaf(g[k], w, vc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < VY; ++j) {
            const int r = r0 + j;
            const int gy = y0 + r, gx = x0 + col;
            if (gy < H && gx < W) {
                float bm, bxx;
                unpk(vb[j], bm, bxx);
                const float bxy = vc[j];
                const size_t o = ((size_t)gy * W + gx) * 3 + c;
                const float xv = img[o], yv = ref[o];
                const float dssim = (bm + 2.f * xv * bxx + yv * bxy) * inv_n;
                float gval = ws * (2.f * (xv - yv) * inv_n - ssim_weight * dssim);
                for (int t = t0; t < t1; ++t) {
                    const int2 e = tlist[t];               // partner, sign
                    const int sp = e.x;
                    const float xj = images[(size_t)sp * npix * 3 + o];
                    const float yj = refs[(size_t)ref_index[sp] * npix * 3 + o];
                    // e = (later - earlier) - (ref later - ref earlier); sign +1 when s is the later state
                    const float ev = (float)e.y * ((xv - xj) - (yv - yj));
                    gval += (float)e.y * tscale * 2.f * ev * inv_n;
                }
                dL[(size_t)s * npix * 3 + o] = gval;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int objective_tiles(int H, int W, int *tiles_x)
{
    *tiles_x = (W + OT_W - 1) / OT_W;
    return *tiles_x * ((H + OT_H - 1) / OT_H);
}

void launch_ssim_fwd(const float *images, const float *refs, const int32_t *ref_index, int S, int H, int W,
                     float *d_mx, float *d_exx, float *d_exy, double *part, cudaStream_t st)
{
    if (S == 0) return;
    int tx;
    const int nt = objective_tiles(H, W, &tx);
    ProfScope ps_("ssim_fwd", st);
    k_ssim_fwd<<<(unsigned)(nt * S), OT_THREADS, 0, st>>>(images, refs, ref_index, H, W, tx, nt, d_mx, d_exx,
                                                           d_exy, part);
    count_launch();
}

void launch_temporal(const float *images, const float *refs, const int32_t *ref_index, const int2 *pairs,
                     int n_pairs, int H, int W, double *tpart, int chunks, cudaStream_t st)
{
    if (n_pairs == 0) return;
    ProfScope ps_("temporal", st);
    k_temporal<<<dim3((unsigned)chunks, (unsigned)n_pairs), 256, 0, st>>>(images, refs, ref_index, pairs,
                                                                          (size_t)H * W, chunks, tpart);
    count_launch();
}

size_t objective_smem(int S)
{
    int P = 1;
    while (P < S) P <<= 1;
    return (size_t)P * (sizeof(double) + sizeof(int));
}

// The objective kernel's dynamic shared-memory limit, set once (before any
// stream capture that launches it).
int objective_prepare()
{
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_objective, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
            return -1;
        attr = true;
    }
    return 0;
}

int launch_objective(const double *part, int n_tiles, const double *tpart, int chunks, int n_t, const int2 *pm,
                     int n_m, const int32_t *anchors, int n_a, int S, double inv_vals, const ObjectiveParams &prm,
                     double *D, double *weight, double *loss, cudaStream_t st)
{
    const size_t smem = objective_smem(S);
    if (objective_prepare() != 0) return -1;
    ProfScope ps_("objective", st);
    k_objective<<<1, 1024, smem, st>>>(part, n_tiles, tpart, chunks, n_t, pm, n_m, anchors, n_a, S, inv_vals, prm,
                                        D, weight, loss);
    count_launch();
    return 0;
}

void launch_objective_grad(const float *images, const float *refs, const int32_t *ref_index, int S, int H, int W,
                           const float *d_mx, const float *d_exx, const float *d_exy, const double *weight,
                           float ssim_weight, float tscale, const int32_t *toff, const int2 *tlist, float *dL,
                           cudaStream_t st)
{
    if (S == 0) return;
    int tx;
    const int nt = objective_tiles(H, W, &tx);
    ProfScope ps_("objective_grad", st);
    k_objective_grad<<<(unsigned)(nt * S), OT_THREADS, 0, st>>>(images, refs, ref_index, H, W, tx, nt, d_mx, d_exx,
                                                                 d_exy, weight, ssim_weight, tscale, toff, tlist,
                                                                 dL);
    count_launch();
}

}  // namespace dgs
