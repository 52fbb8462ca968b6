// Adjoint of decode + deformation + projection.
//
// One thread per Gaussian gathers the screen-space gradients of every record
// (view group, depth variant) of that Gaussian, runs the chain rule through
// projection, Eq. 1 deformation and decode, and adds the result once to the
// caller's gradient arrays: no atomics, deterministic.  Refinement layer l
// receives the sum over variants d > l (layer l is part of every variant of
// depth >= l + 1); the base receives the sum over all variants; layers no
// state delivered receive nothing.  Temporal coefficients u_k receive
// b_k(t) times the mean gradient of each record.
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

template <int SH>
__global__ void __launch_bounds__(128) k_project_bwd(SceneDev s, const ViewGroup *__restrict__ vgs, int V,
                                                     const uint32_t *__restrict__ need,
                                                     const uint32_t *__restrict__ recBase,
                                                     const float4 *__restrict__ rec_grad, GradDev g)
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
        float gu[MAX_RANK][3];
#pragma unroll
        for (int r = 0; r < MAX_RANK; ++r) gu[r][0] = gu[r][1] = gu[r][2] = 0.0f;
        bool any = false;
        for (int d = s.L; d >= 1; --d) {
            bool decoded = false;
            Attr<SH> a;
            for (int v = 0; v < V; ++v) {
                const uint32_t nd = need[(size_t)v * s.C + c] & ~1u;
                if (!((nd >> d) & 1u)) continue;
                const uint32_t slot = recBase[(size_t)v * s.C + c] + (uint32_t)li * __popc(nd) +
                                      __popc(nd & ((1u << d) - 1u));
                const float4 q0 = rec_grad[(size_t)slot * 3], q1 = rec_grad[(size_t)slot * 3 + 1];
                const float4 q2 = rec_grad[(size_t)slot * 3 + 2];
                if (q0.x == 0.f && q0.y == 0.f && q0.z == 0.f && q0.w == 0.f && q1.x == 0.f && q1.y == 0.f &&
                    q1.z == 0.f && q1.w == 0.f && q2.x == 0.f)
                    continue;
                if (!decoded) {
                    load_base<SH>(s, i, a);
                    for (int l = 1; l < d; ++l) add_layer<SH>(s, i, l, a);
                    decoded = true;
                }
                const ViewGroup vg = vgs[v];
                Proj P; Fwd F;
                project_fwd<SH>(s, i, a, vg, P, F);
                if (!P.live) continue;
                const float gg[9] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x};
                float gmu[3];
                project_bwd<SH>(a, vg, P, F, gg, acc, gmu);
                for (int r = 0; r < s.R && r < MAX_RANK; ++r) {
                    const float bk = temporal_basis(r, vg.time);
#pragma unroll
                    for (int k = 0; k < 3; ++k) gu[r][k] = fmaf(bk, gmu[k], gu[r][k]);
                }
                any = true;
            }
            if (!any) continue;
            // acc now sums the variants of depth >= d
            float *dst;
            if (d >= 2) {
                dst = g.res + ((size_t)(d - 2) * s.n + i) * K;
#pragma unroll
                for (int k = 0; k < 3; ++k) { dst[k] += acc.mu[k]; dst[3 + k] += acc.ls[k]; }
#pragma unroll
                for (int k = 0; k < 4; ++k) dst[6 + k] += acc.q[k];
                dst[10] += acc.logit;
#pragma unroll
                for (int k = 0; k < NC; ++k) dst[11 + k] += acc.col[k];
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) { g.mu0[3 * i + k] += acc.mu[k]; g.ls[3 * i + k] += acc.ls[k]; }
#pragma unroll
                for (int k = 0; k < 4; ++k) g.quat[4 * i + k] += acc.q[k];
                g.logit[i] += acc.logit;
#pragma unroll
                for (int k = 0; k < NC; ++k) g.colour[(size_t)NC * i + k] += acc.col[k];
            }
        }
        if (any) {
            for (int r = 0; r < s.R && r < MAX_RANK; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) g.u[((size_t)r * s.n + i) * 3 + k] += gu[r][k];
        }
    }
}

}  // namespace

void launch_project_bwd(const SceneDev &s, const ViewGroup *vgs, int V, const uint32_t *need,
                        const uint32_t *recBase, const float4 *rec_grad, const GradDev &g, int sms,
                        cudaStream_t st)
{
    if (s.n == 0) return;
    long long b = (s.n + 127) / 128;
    if (b > (long long)sms * 32) b = (long long)sms * 32;
    ProfScope ps_("project_bwd", st);
    if (s.sh == 0) k_project_bwd<0><<<(unsigned)b, 128, 0, st>>>(s, vgs, V, need, recBase, rec_grad, g);
    else k_project_bwd<3><<<(unsigned)b, 128, 0, st>>>(s, vgs, V, need, recBase, rec_grad, g);
    count_launch();
}

}  // namespace dgs
