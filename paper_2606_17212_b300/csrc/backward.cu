// Adjoint of decode + deformation + projection.
//
// One thread per Gaussian gathers the screen-space gradients of every record
// (view group, depth variant) of that Gaussian, runs the chain rule through
// projection, Eq. 1 deformation and decode, and adds the result once to the
// caller's gradient arrays: no atomics, deterministic.  Refinement layer l
// receives the sum over variants d > l (layer l is part of every variant of
// depth >= l + 1); the base receives the sum over all variants; layers no
// state delivered receive nothing.  Temporal coefficients u_k receive
// b_k(t) times the mean gradient of each record.  With a cluster affine
// (Eq. 1), the base mean receives A_{c,t}^T times each record's mean
// gradient, and each record's mean gradient is kept for k_affine_grad, which
// forms the keyframe gradients per (view group, cluster).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "gauss_math.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr int MAX_RANK = 8;

__device__ __forceinline__ int cluster_of_b(const int32_t *offs, int C, int i)
{
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Read a record's pixel moments (issued one record ahead of their use).
__device__ __forceinline__ void load_record(const float4 *p, float4 &a, float4 &b, float4 &c)
{
    a = p[0]; b = p[1]; c = p[2];
}

// Clear a record whose moments were read and are not all zero, so the buffer
// is zero for the next backward (each record is read by exactly one thread,
// once).  Called when its values are in use, so the prefetch of the next
// record does not wait for this test.
__device__ __forceinline__ void clear_record(float4 *p)
{
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    p[0] = z; p[1] = z; p[2] = z;
}

// RK > 0: exactly RK temporal coefficients (the accumulators stay in registers);
// RK = 0: any rank up to MAX_RANK.
template <int SH, int RK>
__global__ void __launch_bounds__(128, SH == 0 ? 4 : 1) k_project_bwd(SceneDev s, const ViewGroup *__restrict__ vgs, int V,
                                                     const uint32_t *__restrict__ need,
                                                     const uint32_t *__restrict__ recBase,
                                                     float4 *__restrict__ rec_grad, GradDev g)
{
    constexpr int NC = NCol<SH>::value;
    constexpr int K = 11 + NC;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const int c = cluster_of_b(s.offs, s.C, i);
        if (i < s.offs[c] || i >= s.offs[c + 1]) continue;   // offsets validated on the host; never taken
        const int li = i - s.offs[c];
        Attr<SH> acc;
#pragma unroll
        for (int k = 0; k < 3; ++k) { acc.mu[k] = 0.0f; acc.ls[k] = 0.0f; }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.q[k] = 0.0f;
        acc.logit = 0.0f;
#pragma unroll
        for (int k = 0; k < NC; ++k) acc.col[k] = 0.0f;
        constexpr int NR = RK > 0 ? RK : MAX_RANK;
        const int nr = RK > 0 ? RK : min(s.R, MAX_RANK);
        float gu[NR][3];
#pragma unroll
        for (int r = 0; r < NR; ++r) gu[r][0] = gu[r][1] = gu[r][2] = 0.0f;
        float gm0[3] = {0.0f, 0.0f, 0.0f};    // base-mean gradient through the affine
        bool any = false;
        for (int d = s.L; d >= 1; --d) {
            bool decoded = false;
            Attr<SH> a;
            // view groups holding a record of (this Gaussian, depth d), in order; the
            // next record's gradient is loaded while the current one is processed
            // with at most 64 view groups, the view groups holding depth d are read
            // into a mask first (independent loads), then walked bit by bit
            uint64_t vmask = 0;
            if (V <= 64) {
#pragma unroll 8
                for (int v = 0; v < V; ++v)
                    vmask |= (uint64_t)((__ldg(need + (size_t)v * s.C + c) >> d) & 1u) << v;
            }
            auto next_vg = [&](int v) {
                if (V <= 64) {
                    const uint64_t rest = v >= 64 ? 0ull : vmask >> v;
                    return rest ? v + __ffsll((long long)rest) - 1 : V;
                }
                while (v < V && !(((need[(size_t)v * s.C + c] & ~1u) >> d) & 1u)) ++v;
                return v;
            };
            auto slot_of = [&](int v) {
                const uint32_t nd = need[(size_t)v * s.C + c] & ~1u;
                return recBase[(size_t)v * s.C + c] + (uint32_t)li * __popc(nd) + __popc(nd & ((1u << d) - 1u));
            };
            int vn = next_vg(0);
            uint32_t slot_n = 0;
            float4 n0 = make_float4(0, 0, 0, 0), n1 = n0, n2 = n0;
            if (vn < V) {
                slot_n = slot_of(vn);
                load_record(rec_grad + (size_t)slot_n * 3, n0, n1, n2);
            }
            while (vn < V) {
                const int v = vn;
                const uint32_t slot = slot_n;
                const float4 q0 = n0, q1 = n1, q2 = n2;
                vn = next_vg(v + 1);
                if (vn < V) {
                    slot_n = slot_of(vn);
                    load_record(rec_grad + (size_t)slot_n * 3, n0, n1, n2);
                }
                if (q0.x == 0.f && q0.y == 0.f && q0.z == 0.f && q0.w == 0.f && q1.x == 0.f && q1.y == 0.f &&
                    q1.z == 0.f && q1.w == 0.f && q2.x == 0.f)
                    continue;
                clear_record(rec_grad + (size_t)slot * 3);
                if (!decoded) {
                    load_base<SH>(s, i, a);
                    for (int l = 1; l < d; ++l) add_layer<SH>(s, i, l, a);
                    decoded = true;
                }
                const ViewGroup vg = vgs[v];
                Proj P; Fwd F;
                project_fwd<SH>(s, i, c, a, vg, P, F);
                if (!P.live) continue;
                // screen-space gradients from the raster's pixel moments of dL/dpower
                // (power = -(A dx^2 + 2 B dx dy + C dy^2) / 2, alpha = o e^power)
                const float gg[9] = {-(P.A * q0.x + P.B * q0.y), -(P.B * q0.x + P.C * q0.y), -0.5f * q0.z, -q0.w,
                                     -0.5f * q1.x, __fdividef(q1.y, P.o), q1.z, q1.w, q2.x};
                float gmu[3];
                project_bwd<SH>(a, vg, P, F, gg, acc, gmu);
                if (s.affine) {
                    float A[12], w;
                    int k0, k1;
                    affine_at(s, c, vg.time, A, k0, k1, w);
#pragma unroll
                    for (int k = 0; k < 3; ++k) gm0[k] += A[k] * gmu[0] + A[4 + k] * gmu[1] + A[8 + k] * gmu[2];
#pragma unroll
                    for (int k = 0; k < 3; ++k) g.rec_gmu[(size_t)slot * 3 + k] = gmu[k];
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r >= nr) break;
                    const float bk = temporal_basis(r, vg.time);
#pragma unroll
                    for (int k = 0; k < 3; ++k) gu[r][k] = fmaf(bk, gmu[k], gu[r][k]);
                }
                any = true;
            }
            if (!any) continue;
            // acc now sums the variants of depth >= d
            float *dst;
            if (d >= 2 && s.res_mode == 1) {
                // decoded symbols: no refinement gradient
            } else if (d >= 2) {
                // res_mode 2: the decoded-refinement gradient goes to the workspace for k_quant_grad
                dst = (s.res_mode == 2 ? g.gq : g.res) + ((size_t)(d - 2) * s.n + i) * K;
#pragma unroll
                for (int k = 0; k < 3; ++k) { dst[k] += acc.mu[k]; dst[3 + k] += acc.ls[k]; }
#pragma unroll
                for (int k = 0; k < 4; ++k) dst[6 + k] += acc.q[k];
                dst[10] += acc.logit;
#pragma unroll
                for (int k = 0; k < NC; ++k) dst[11 + k] += acc.col[k];
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    g.mu0[3 * i + k] += s.affine ? gm0[k] : acc.mu[k];
                    g.ls[3 * i + k] += acc.ls[k];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) g.quat[4 * i + k] += acc.q[k];
                g.logit[i] += acc.logit;
#pragma unroll
                for (int k = 0; k < NC; ++k) g.colour[(size_t)NC * i + k] += acc.col[k];
            }
        }
        if (any) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (r >= nr) break;
#pragma unroll
                for (int k = 0; k < 3; ++k) g.u[((size_t)r * s.n + i) * 3 + k] += gu[r][k];
            }
        }
    }
}

// Quantized refinements (res_mode 2): straight-through gradient to the float
// refinements (zero where the symbol clips) and the learned-step gradient
// sum_i g (v - x / step) (g v where clipped), block-reduced per component.
// One block per (layer, 256 Gaussians); component sums via shared memory.
__global__ void __launch_bounds__(256) k_quant_grad(SceneDev s, const float *__restrict__ gq, float *__restrict__ g_res,
                                                    float *__restrict__ g_step)
{
    __shared__ float part[64];
    const int blocks_per_layer = (s.n + 255) / 256;
    const int l = blockIdx.x / blocks_per_layer;             // 0-based refinement layer
    const int i = (blockIdx.x % blocks_per_layer) * 256 + threadIdx.x;
    for (int k = threadIdx.x; k < s.K; k += blockDim.x) part[k] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < s.K; ++k) {
        float c = 0.0f;
        if (i < s.n) {
            const size_t o = ((size_t)l * s.n + i) * s.K + k;
            const float gv = gq[o];
            if (gv != 0.0f) {
                const float x = s.res[o], st = s.res_step[(size_t)l * s.K + k];
                bool cl;
                const float v = quant_symbol(x, st, cl);
                if (!cl) g_res[o] += gv;
                c = gv * (cl ? v : v - __fdiv_rn(x, st));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (lane == 0 && c != 0.0f) atomicAdd(&part[k], c);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < s.K; k += blockDim.x)
        if (part[k] != 0.0f) atomicAdd(g_step + (size_t)l * s.K + k, part[k]);
}

// Keyframe gradients of the cluster affine: one block per (view group v,
// cluster c) sums dL/dmu (x) (mubar, 1) over the records of (v, c) and adds the
// sum to the two keyframes of v's time with their interpolation weights.
__global__ void __launch_bounds__(256) k_affine_grad(SceneDev s, const ViewGroup *__restrict__ vgs,
                                                     const uint32_t *__restrict__ need,
                                                     const uint32_t *__restrict__ recBase,
                                                     const float *__restrict__ rec_gmu, float *__restrict__ g_aff)
{
    __shared__ float red[8][12];
    const int v = blockIdx.x / s.C, c = blockIdx.x % s.C;
    const uint32_t nd = need[(size_t)v * s.C + c] & ~1u;
    if (!nd) return;
    const uint32_t nvar = (uint32_t)__popc(nd);
    const uint32_t r0 = recBase[(size_t)v * s.C + c], r1 = recBase[(size_t)v * s.C + c + 1];
    const int i0 = s.offs[c];
    float acc[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) acc[e] = 0.0f;
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const int i = i0 + (int)((r - r0) / nvar);
        const float g0 = rec_gmu[(size_t)r * 3], g1 = rec_gmu[(size_t)r * 3 + 1], g2 = rec_gmu[(size_t)r * 3 + 2];
        const float m[4] = {__ldg(s.mu0 + 3 * i), __ldg(s.mu0 + 3 * i + 1), __ldg(s.mu0 + 3 * i + 2), 1.0f};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[k] = fmaf(g0, m[k], acc[k]);
            acc[4 + k] = fmaf(g1, m[k], acc[4 + k]);
            acc[8 + k] = fmaf(g2, m[k], acc[8 + k]);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < 12; ++e) {
        float x = acc[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[w][e] = x;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        float tot = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += red[k][threadIdx.x];
        float A[12], wt;
        int k0, k1;
        affine_at(s, c, vgs[v].time, A, k0, k1, wt);
        atomicAdd(g_aff + ((size_t)c * s.aT + k0) * 12 + threadIdx.x, (1.0f - wt) * tot);
        atomicAdd(g_aff + ((size_t)c * s.aT + k1) * 12 + threadIdx.x, wt * tot);
    }
}

}  // namespace

void launch_project_bwd(const SceneDev &s, const ViewGroup *vgs, int V, const uint32_t *need,
                        const uint32_t *recBase, float4 *rec_grad, const GradDev &g, size_t rec_cap,
                        int sms, cudaStream_t st)
{
    if (s.n == 0) return;
    if (s.affine && rec_cap) cudaMemsetAsync(g.rec_gmu, 0, sizeof(float) * 3 * rec_cap, st);
    if (s.res_mode == 2 && s.L > 1) cudaMemsetAsync(g.gq, 0, sizeof(float) * (size_t)(s.L - 1) * s.n * s.K, st);
    long long b = (s.n + 127) / 128;
    if (b > (long long)sms * 32) b = (long long)sms * 32;
    {
        ProfScope ps_("project_bwd", st);
        // the workloads' rank-2 temporal bases take the specialised kernels
        if (s.sh == 0 && s.R == 2) k_project_bwd<0, 2><<<(unsigned)b, 128, 0, st>>>(s, vgs, V, need, recBase, rec_grad, g);
        else if (s.sh == 0) k_project_bwd<0, 0><<<(unsigned)b, 128, 0, st>>>(s, vgs, V, need, recBase, rec_grad, g);
        else if (s.R == 2) k_project_bwd<3, 2><<<(unsigned)b, 128, 0, st>>>(s, vgs, V, need, recBase, rec_grad, g);
        else k_project_bwd<3, 0><<<(unsigned)b, 128, 0, st>>>(s, vgs, V, need, recBase, rec_grad, g);
        count_launch();
    }
    if (s.res_mode == 2 && s.L > 1) {
        ProfScope ps_("quant_grad", st);
        k_quant_grad<<<(unsigned)((s.L - 1) * ((s.n + 255) / 256)), 256, 0, st>>>(s, g.gq, g.res, g.res_step);
        count_launch();
    }
    if (s.affine && V > 0) {
        ProfScope ps_("affine_grad", st);
        k_affine_grad<<<(unsigned)(V * s.C), 256, 0, st>>>(s, vgs, need, recBase, g.rec_gmu, g.affine);
        count_launch();
    }
}

}  // namespace dgs
