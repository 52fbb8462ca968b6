// Counterfactual render utility of completion groups (Section 5, Eq. 3 and
// Eq. 4): paired masks m and m u g for every sampled context, and the per-group
// statistics of Delta_g(m) = D(I, R(m)) - D(I, R(m u g)) over its contexts.
// The distortions themselves come from the batched utility pass (all 2 G M
// states in one batch), so these kernels only move masks and reduce doubles.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr int ST_THREADS = 256;

// out rows [0, G M) = the contexts; rows [G M, 2 G M) = the same contexts with
// the group's packet bit (cluster c, layer l) = c * L + l set.
__global__ void k_pair_masks(const uint32_t *__restrict__ ctx_masks, const int2 *__restrict__ groups, int G, int M,
                             int words, int L, uint32_t *__restrict__ out)
{
    const size_t n = (size_t)G * M * words;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / words;
        const int w = (int)(i % words);
        const int2 g = groups[row / M];
        const int bit = g.x * L + g.y;
        const uint32_t m = ctx_masks[i];
        out[i] = m;
        out[n + i] = (w == bit / 32) ? (m | (1u << (bit % 32))) : m;
    }
}

__device__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < ST_THREADS / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// One block per group: Delta for each of its M contexts, then (Eq. 4) the mean
// over contexts, the population standard deviation, the q-quantile by linear
// interpolation between order statistics (position q (M - 1)) and the
// risk-adjusted utility ((1 - alpha) mean + alpha Q) / (1 + beta std).
// stats[g] = (mean, Q, std, utility).
__global__ void __launch_bounds__(ST_THREADS) k_group_stats(const double *__restrict__ mse, int G, int M, double alpha,
                                                            double beta, double q, double *__restrict__ delta,
                                                            double *__restrict__ stats)
{
    __shared__ double x[DGS_UTILITY_MAX_CONTEXTS];
    __shared__ double red[ST_THREADS / 32];
    const int g = blockIdx.x;
    const size_t GM = (size_t)G * M;
    int P = 1;
    while (P < M) P <<= 1;
    double s = 0.0;
    for (int j = threadIdx.x; j < P; j += ST_THREADS) {
        if (j < M) {
            const size_t k = (size_t)g * M + j;
            const double d = mse[k] - mse[GM + k];
            if (delta) delta[k] = d;
            x[j] = d;
            s += d;
        } else {
            x[j] = __longlong_as_double(0x7ff0000000000000LL);   // +inf sorts last
        }
    }
    const double mean = block_sum(s, red) / (double)M;
    double v = 0.0;
    for (int j = threadIdx.x; j < M; j += ST_THREADS) v += (x[j] - mean) * (x[j] - mean);
    const double sd = sqrt(block_sum(v, red) / (double)M);
    // bitonic sort of the P padded values (ascending)
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += ST_THREADS) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const double a = x[i], b = x[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { x[i] = b; x[ixj] = a; }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        const double h = q * (double)(M - 1);
        const int lo = (int)floor(h);
        const int hi = lo + 1 < M ? lo + 1 : M - 1;
        const double Q = x[lo] + (h - (double)lo) * (x[hi] - x[lo]);
        stats[(size_t)g * 4 + 0] = mean;
        stats[(size_t)g * 4 + 1] = Q;
        stats[(size_t)g * 4 + 2] = sd;
        stats[(size_t)g * 4 + 3] = ((1.0 - alpha) * mean + alpha * Q) / (1.0 + beta * sd);
    }
}

}  // namespace

void launch_pair_masks(const uint32_t *ctx_masks, const int2 *groups, int G, int M, int words, int L,
                       uint32_t *out, int sms, cudaStream_t st)
{
    const size_t n = (size_t)G * M * words;
    if (n == 0) return;
    size_t b = (n + 255) / 256;
    if (b > (size_t)sms * 16) b = (size_t)sms * 16;
    ProfScope ps_("pair_masks", st);
    k_pair_masks<<<(unsigned)b, 256, 0, st>>>(ctx_masks, groups, G, M, words, L, out);
    count_launch();
}

void launch_group_stats(const double *mse, int G, int M, double alpha, double beta, double q, double *delta,
                        double *stats, cudaStream_t st)
{
    if (G == 0) return;
    ProfScope ps_("group_stats", st);
    k_group_stats<<<G, ST_THREADS, 0, st>>>(mse, G, M, alpha, beta, q, delta, stats);
    count_launch();
}

}  // namespace dgs
