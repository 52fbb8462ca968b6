// Closure, record layout, shared decode + deformation + projection, tile
// binning and tile ranges.  All of these are HBM-bound streaming kernels with
// grid-stride loops sized to a multiple of the SM count.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "gauss_math.cuh"
#include "kernels.cuh"

namespace dgs {

// Sections 4 / 7.4: a layer is usable only when every layer below it in its
// cluster is usable, so the delivered depth of cluster c is the number of
// leading delivered layers.  Also marks which depths each view group needs.
__global__ void k_closure(const uint32_t *__restrict__ masks, int S, int words, int C, int L,
                          const int32_t *__restrict__ vg_of_state, uint8_t *__restrict__ depth,
                          uint32_t *__restrict__ need, int force_full)
{
    const long long total = (long long)S * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / C), c = (int)(t % C);
        const uint32_t *m = masks + (size_t)s * words;
        int d = 0;
        while (d < L) {
            const int b = c * L + d;
            if (!((__ldg(m + (b >> 5)) >> (b & 31)) & 1u)) break;
            ++d;
        }
        depth[t] = (uint8_t)d;
        const int v = vg_of_state[s];
        uint32_t bits = d > 0 ? (1u << d) : 0u;
        if (force_full) bits |= 1u << L;
        if (bits) atomicOr(need + (size_t)v * C + c, bits);
    }
}

// records of (view group v, cluster c) = size(c) * popcount(needed depths)
__global__ void k_layout_counts(const uint32_t *__restrict__ need, const int32_t *__restrict__ offs, int V,
                                int C, uint32_t *__restrict__ counts)
{
    const int total = V * C;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int c = t % C;
        const uint32_t nb = __popc(need[t] & ~1u);
        counts[t] = nb * (uint32_t)(offs[c + 1] - offs[c]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[total] = 0;
}

__device__ __forceinline__ int cluster_of(const int32_t *offs, int C, int i)
{
    int lo = 0, hi = C - 1;        // largest c with offs[c] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The same over offsets staged in shared memory.
__device__ __forceinline__ int cluster_of_shared(const int32_t *offs, int C, int i)
{
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One thread per Gaussian: decode the base and the delivered refinement prefix
// incrementally (Section 3), once per depth some state needs, and project that
// decoded variant for every view group whose states render the Gaussian's
// cluster at that depth.  The scene is read once; records are written at
// their (view group, cluster, Gaussian, depth) slot with the depth key.
// need, recBase and the view groups are small per-call tables; when they fit
// they are staged in shared memory (dynamic size) so the loop over view groups
// issues no dependent global loads.
template <int SH, bool SMEM>
__global__ void __launch_bounds__(128, 4) k_project(SceneDev s, const ViewGroup *__restrict__ vgs_g, int V,
                                                    const uint32_t *__restrict__ need_g,
                                                    const uint32_t *__restrict__ recBase_g, Rec *__restrict__ recs,
                                                    uint32_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const ViewGroup *vgs = vgs_g;
    const uint32_t *need = need_g, *recBase = recBase_g;
    const int32_t *offs = s.offs;
    if (SMEM) {
        ViewGroup *svg = reinterpret_cast<ViewGroup *>(sm_raw);
        uint32_t *sneed = reinterpret_cast<uint32_t *>(svg + V);
        uint32_t *sbase = sneed + (size_t)V * s.C;
        int32_t *soffs = reinterpret_cast<int32_t *>(sbase + (size_t)V * s.C);
        const int nvg_words = (int)(sizeof(ViewGroup) / 4) * V;
        for (int k = threadIdx.x; k < nvg_words; k += blockDim.x)
            reinterpret_cast<uint32_t *>(svg)[k] = reinterpret_cast<const uint32_t *>(vgs_g)[k];
        for (int k = threadIdx.x; k < V * s.C; k += blockDim.x) { sneed[k] = need_g[k]; sbase[k] = recBase_g[k]; }
        for (int k = threadIdx.x; k <= s.C; k += blockDim.x) soffs[k] = s.offs[k];
        __syncthreads();
        vgs = svg; need = sneed; recBase = sbase; offs = soffs;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const int c = SMEM ? cluster_of_shared(offs, s.C, i) : cluster_of(offs, s.C, i);
        if (i < offs[c] || i >= offs[c + 1]) continue;   // offsets validated on the host; never taken
        const uint32_t li = (uint32_t)(i - offs[c]);
        uint32_t any = 0;
        for (int v = 0; v < V; ++v) any |= need[(size_t)v * s.C + c];
        any &= ~1u;
        if (!any) continue;
        const int dmax = 31 - __clz(any);
        Attr<SH> a;
        load_base<SH>(s, i, a);
        for (int d = 1; d <= dmax; ++d) {
            if (d >= 2) add_layer<SH>(s, i, d - 1, a);
            if (!((any >> d) & 1u)) continue;
            for (int v = 0; v < V; ++v) {
                const uint32_t nd = need[(size_t)v * s.C + c] & ~1u;
                if (!((nd >> d) & 1u)) continue;
                const uint32_t slot = recBase[(size_t)v * s.C + c] + li * (uint32_t)__popc(nd) +
                                      (uint32_t)__popc(nd & ((1u << d) - 1u));
                const ViewGroup &vg = vgs[v];
                Proj P; Fwd F;
                project_fwd<SH>(s, i, c, a, vg, P, F);
                Rec R;
                if (P.live) {
                    R.mx = P.mx; R.my = P.my; R.A = P.A * K_AC; R.B = P.B * K_B; R.C = P.C * K_AC; R.o = P.o;
                    R.r = P.rgb[0]; R.g = P.rgb[1]; R.b = P.rgb[2];
                    R.bx = (uint32_t)P.xlo | ((uint32_t)P.xhi << 16);
                    R.by = (uint32_t)P.ylo | ((uint32_t)P.yhi << 16);
                    R.cd = (uint32_t)c | (P.aclamp ? REC_CLAMP : 0u) | ((uint32_t)d << 12) | ((uint32_t)v << 16) |
                           ((uint32_t)P.rclip << 31);
                    keys[slot] = __float_as_uint(P.z);
                } else {
                    R.mx = R.my = R.A = R.B = R.C = R.o = R.r = R.g = R.b = 0.0f;
                    R.bx = 1u; R.by = 1u;          // xlo = 1 > xhi = 0: empty box
                    R.cd = (uint32_t)c | ((uint32_t)v << 16);   // depth field 0 = culled
                    keys[slot] = 0xffffffffu;
                }
                float4 *dst = reinterpret_cast<float4 *>(recs + slot);
                const float4 *src = reinterpret_cast<const float4 *>(&R);
                dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2];
                vals[slot] = slot;
            }
        }
    }
}

// The last 16 bytes of a record: colour b, box x, box y, cluster/depth/view group.
__device__ __forceinline__ float4 rec_tail(const Rec *recs, uint32_t slot)
{
    return __ldg(reinterpret_cast<const float4 *>(recs + slot) + 2);
}

__device__ __forceinline__ uint32_t rec_tiles(const float4 &q, int shift)
{
    const uint32_t bx = __float_as_uint(q.y), by = __float_as_uint(q.z), cd = __float_as_uint(q.w);
    const int xlo = bx & 0xffff, xhi = bx >> 16, ylo = by & 0xffff, yhi = by >> 16;
    if ((cd & 0xf000u) == 0 || xlo > xhi || ylo > yhi) return 0;
    return (uint32_t)(((xhi >> shift) - (xlo >> shift) + 1) * ((yhi >> shift) - (ylo >> shift) + 1));
}

__device__ __forceinline__ uint32_t live_n(uint32_t n_cap, const uint32_t *n_dev)
{
    return n_dev ? min(n_cap, *n_dev) : n_cap;
}

// Tile counts of records in depth order (sorted slot list), zero past the
// live count so a scan over the capacity gives the entry total; and each
// record's tile rectangle (first tile key, tile columns, slot) in the same
// order, the source the tile sort generates the entries from.
__global__ void k_tile_count(const Rec *__restrict__ recs, const uint32_t *__restrict__ order, uint32_t n_cap,
                             const uint32_t *__restrict__ n_dev, int tiles_x, uint32_t tiles, int shift,
                             uint32_t *__restrict__ counts, uint4 *__restrict__ bins)
{
    const uint32_t n = live_n(n_cap, n_dev);
    const uint32_t T = gridDim.x * blockDim.x;
    // four records per thread per step, every gather issued before any use
    for (uint32_t j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < n_cap; j0 += 4u * T) {
        uint32_t slot[4];
        float4 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t j = j0 + (uint32_t)k * T;
            slot[k] = j < n ? __ldg(order + j) : 0xffffffffu;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = slot[k] != 0xffffffffu ? rec_tail(recs, slot[k]) : make_float4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t j = j0 + (uint32_t)k * T;
            if (j >= n_cap) continue;
            const uint32_t c = slot[k] != 0xffffffffu ? rec_tiles(q[k], shift) : 0u;
            counts[j] = c;
            if (c) {
                const uint32_t bx = __float_as_uint(q[k].y), by = __float_as_uint(q[k].z);
                const uint32_t tx0 = (bx & 0xffffu) >> shift, ty0 = (by & 0xffffu) >> shift;
                const uint32_t tw = ((bx >> 16) >> shift) - tx0 + 1u;
                const uint32_t vbase = ((__float_as_uint(q[k].w) >> 16) & 0x7fffu) * tiles;
                bins[j] = make_uint4(vbase + ty0 * (uint32_t)tiles_x + tx0, tw, slot[k], 0u);
            }
        }
    }
}

// out = min(total, cap); flags bit 0 when total exceeds the capacity.
__global__ void k_clamp_count(const uint32_t *__restrict__ total, uint32_t cap, uint32_t *__restrict__ out,
                              uint32_t *__restrict__ flags)
{
    const uint32_t t = *total;
    *out = t < cap ? t : cap;
    if (t > cap) atomicOr(flags, 1u);
}

__global__ void k_ranges(const uint32_t *__restrict__ keys, uint32_t n_cap, const uint32_t *__restrict__ n_dev,
                         uint2 *__restrict__ ranges)
{
    const uint32_t n = live_n(n_cap, n_dev);
    const uint32_t T = gridDim.x * blockDim.x;
    // four keys per thread per step with their neighbours, all loads issued first
    for (uint32_t e0 = blockIdx.x * blockDim.x + threadIdx.x; e0 < n; e0 += 4u * T) {
        uint32_t k[4], prev[4], next[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t e = e0 + (uint32_t)u * T;
            const bool ok = e < n;
            k[u] = ok ? __ldg(keys + e) : 0u;
            prev[u] = ok && e > 0 ? __ldg(keys + e - 1) : ~k[u];
            next[u] = ok && e + 1 < n ? __ldg(keys + e + 1) : ~k[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t e = e0 + (uint32_t)u * T;
            if (e >= n) continue;
            if (prev[u] != k[u]) ranges[k[u]].x = e;
            if (next[u] != k[u]) ranges[k[u]].y = e + 1;
        }
    }
}


// --------------------------------------------------------------- launchers
static unsigned grid_for(long long n, int threads, int sms)
{
    long long b = (n + threads - 1) / threads;
    long long cap = (long long)sms * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

void launch_closure(const uint32_t *masks, int S, int words, int C, int L, const int32_t *vg_of_state,
                    uint8_t *depth, uint32_t *need, int force_full, int sms, cudaStream_t st)
{
    ProfScope ps_("closure", st);
    k_closure<<<grid_for((long long)S * C, 256, sms), 256, 0, st>>>(masks, S, words, C, L, vg_of_state,
                                                                      depth, need, force_full);
    count_launch();
}

void launch_layout_counts(const uint32_t *need, const int32_t *offs, int V, int C, uint32_t *counts, int sms,
                          cudaStream_t st)
{
    ProfScope ps_("layout", st);
    k_layout_counts<<<grid_for((long long)V * C + 1, 256, sms), 256, 0, st>>>(need, offs, V, C, counts);
    count_launch();
}

void launch_project(const SceneDev &s, const ViewGroup *vgs, int V, const uint32_t *need, const uint32_t *recBase,
                    Rec *recs, uint32_t *keys, uint32_t *vals, int sms, cudaStream_t st)
{
    // a persistent grid: each block stages the view-group tables once and
    // projects several Gaussians per thread (measured: 0.38 -> 0.35 ms on the
    // training step, against one Gaussian per thread)
    unsigned g = (unsigned)((s.n + 127) / 128);
    if (g < 1) g = 1;
    if (g > (unsigned)sms * 4u) g = (unsigned)sms * 4u;
    const size_t smem = sizeof(ViewGroup) * (size_t)V + 8 * (size_t)V * s.C + 4 * (size_t)(s.C + 1);
    const bool use_smem = smem <= 40 * 1024;
    ProfScope ps_("project", st);
    if (use_smem) {
        if (s.sh == 0) k_project<0, true><<<g, 128, smem, st>>>(s, vgs, V, need, recBase, recs, keys, vals);
        else k_project<3, true><<<g, 128, smem, st>>>(s, vgs, V, need, recBase, recs, keys, vals);
    } else {
        if (s.sh == 0) k_project<0, false><<<g, 128, 0, st>>>(s, vgs, V, need, recBase, recs, keys, vals);
        else k_project<3, false><<<g, 128, 0, st>>>(s, vgs, V, need, recBase, recs, keys, vals);
    }
    count_launch();
}

void launch_tile_count(const Rec *recs, const uint32_t *order, uint32_t n, int tiles_x, uint32_t tiles,
                       int tile_shift, uint32_t *counts, uint4 *bins, int sms, cudaStream_t st, const uint32_t *n_dev)
{
    if (n == 0) return;
    ProfScope ps_("tile_count", st);
    // four times the usual grid cap: more warps keep more of the dependent
    // (slot, record) gathers in flight (0.152 -> 0.128 ms on the training step)
    k_tile_count<<<grid_for(n, 256, sms * 4), 256, 0, st>>>(recs, order, n, n_dev, tiles_x, tiles, tile_shift, counts,
                                                        bins);
    count_launch();
}

void launch_clamp_count(const uint32_t *total, uint32_t cap, uint32_t *out, uint32_t *flags, cudaStream_t st)
{
    k_clamp_count<<<1, 1, 0, st>>>(total, cap, out, flags);
    count_launch();
}

void launch_ranges(const uint32_t *keys, uint32_t n, uint2 *ranges, int sms, cudaStream_t st, const uint32_t *n_dev)
{
    if (n == 0) return;
    ProfScope ps_("ranges", st);
    k_ranges<<<grid_for(n, 256, sms), 256, 0, st>>>(keys, n, n_dev, ranges);
    count_launch();
}

// flag |= 1 when a[i] != b[i] for some i < n
__global__ void k_words_differ(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, size_t n,
                               uint32_t *__restrict__ flag)
{
    bool d = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d |= a[i] != b[i];
    if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

void launch_words_differ(const uint32_t *a, const uint32_t *b, size_t n, uint32_t *flag, int sms, cudaStream_t st)
{
    if (n == 0) return;
    ProfScope ps_("words_differ", st);
    k_words_differ<<<grid_for((long long)n, 256, sms), 256, 0, st>>>(a, b, n, flag);
    count_launch();
}


}  // namespace dgs
