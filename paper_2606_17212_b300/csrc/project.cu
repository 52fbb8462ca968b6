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

// One thread per (view group, Gaussian): decode the base and the delivered
// refinement prefix incrementally (Section 3) and project every depth some
// state of the view group needs.  Writes Rec, its depth key and its slot.
template <int SH>
__global__ void __launch_bounds__(256) k_project(SceneDev s, const ViewGroup *__restrict__ vgs, int V,
                                                 const uint32_t *__restrict__ need,
                                                 const uint32_t *__restrict__ recBase, Rec *__restrict__ recs,
                                                 uint32_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const long long total = (long long)V * s.n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / s.n), i = (int)(t % s.n);
        const int c = cluster_of(s.offs, s.C, i);
        if (i < s.offs[c] || i >= s.offs[c + 1]) continue;   // offsets validated on the host; never taken
        const uint32_t nd = need[(size_t)v * s.C + c] & ~1u;
        if (!nd) continue;
        const ViewGroup vg = vgs[v];
        const int cnt = __popc(nd);
        uint32_t slot = recBase[(size_t)v * s.C + c] + (uint32_t)(i - s.offs[c]) * cnt;
        const int dmax = 31 - __clz(nd);
        Attr<SH> a;
        load_base<SH>(s, i, a);
        for (int d = 1; d <= dmax; ++d) {
            if (d >= 2) add_layer<SH>(s, i, d - 1, a);
            if (!((nd >> d) & 1u)) continue;
            Proj P; Fwd F;
            project_fwd<SH>(s, i, a, vg, P, F);
            Rec R;
            if (P.live) {
                R.mx = P.mx; R.my = P.my; R.A = P.A; R.B = P.B; R.C = P.C; R.o = P.o;
                R.r = P.rgb[0]; R.g = P.rgb[1]; R.b = P.rgb[2];
                R.bx = (uint32_t)P.xlo | ((uint32_t)P.xhi << 16);
                R.by = (uint32_t)P.ylo | ((uint32_t)P.yhi << 16);
                R.cd = (uint32_t)c | ((uint32_t)d << 12) | ((uint32_t)v << 16);
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
            ++slot;
        }
    }
}

// The last 16 bytes of a record: colour b, box x, box y, cluster/depth/view group.
__device__ __forceinline__ float4 rec_tail(const Rec *recs, uint32_t slot)
{
    return __ldg(reinterpret_cast<const float4 *>(recs + slot) + 2);
}

__device__ __forceinline__ uint32_t rec_tiles(const float4 &q)
{
    const uint32_t bx = __float_as_uint(q.y), by = __float_as_uint(q.z), cd = __float_as_uint(q.w);
    const int xlo = bx & 0xffff, xhi = bx >> 16, ylo = by & 0xffff, yhi = by >> 16;
    if ((cd & 0xf000u) == 0 || xlo > xhi || ylo > yhi) return 0;
    return (uint32_t)((xhi / TILE - xlo / TILE + 1) * (yhi / TILE - ylo / TILE + 1));
}

// Tile counts of records in depth order (sorted slot list).
__global__ void k_tile_count(const Rec *__restrict__ recs, const uint32_t *__restrict__ order, uint32_t n,
                             uint32_t *__restrict__ counts)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        counts[j] = rec_tiles(rec_tail(recs, order[j]));
    }
}

// Emit one (view group * tiles + tile, slot) entry per overlapped tile, in
// depth order, so a stable sort on the tile key leaves every tile's run
// ordered by (depth, Gaussian, depth variant).
__global__ void k_emit(const Rec *__restrict__ recs, const uint32_t *__restrict__ order,
                       const uint32_t *__restrict__ offsets, uint32_t n, int tiles_x, uint32_t tiles,
                       uint32_t *__restrict__ ekeys, uint32_t *__restrict__ evals)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const uint32_t slot = order[j];
        const float4 q = rec_tail(recs, slot);
        if (rec_tiles(q) == 0) continue;
        const uint32_t bx = __float_as_uint(q.y), by = __float_as_uint(q.z);
        const int xlo = bx & 0xffff, xhi = bx >> 16, ylo = by & 0xffff, yhi = by >> 16;
        const uint32_t v = __float_as_uint(q.w) >> 16;
        uint32_t o = offsets[j];
        for (int ty = ylo / TILE; ty <= yhi / TILE; ++ty)
            for (int tx = xlo / TILE; tx <= xhi / TILE; ++tx) {
                ekeys[o] = v * tiles + (uint32_t)(ty * tiles_x + tx);
                evals[o] = slot;
                ++o;
            }
    }
}

__global__ void k_ranges(const uint32_t *__restrict__ keys, uint32_t n, uint2 *__restrict__ ranges)
{
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t k = keys[e];
        if (e == 0 || keys[e - 1] != k) ranges[k].x = e;
        if (e == n - 1 || keys[e + 1] != k) ranges[k].y = e + 1;
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
    const unsigned g = grid_for((long long)V * s.n, 256, sms);
    ProfScope ps_("project", st);
    if (s.sh == 0) k_project<0><<<g, 256, 0, st>>>(s, vgs, V, need, recBase, recs, keys, vals);
    else k_project<3><<<g, 256, 0, st>>>(s, vgs, V, need, recBase, recs, keys, vals);
    count_launch();
}

void launch_tile_count(const Rec *recs, const uint32_t *order, uint32_t n, uint32_t *counts, int sms,
                       cudaStream_t st)
{
    ProfScope ps_("tile_count", st);
    k_tile_count<<<grid_for(n, 256, sms), 256, 0, st>>>(recs, order, n, counts);
    count_launch();
}

void launch_emit(const Rec *recs, const uint32_t *order, const uint32_t *offsets, uint32_t n, int tiles_x,
                 uint32_t tiles, uint32_t *ekeys, uint32_t *evals, int sms, cudaStream_t st)
{
    ProfScope ps_("emit", st);
    k_emit<<<grid_for(n, 256, sms), 256, 0, st>>>(recs, order, offsets, n, tiles_x, tiles, ekeys, evals);
    count_launch();
}

void launch_ranges(const uint32_t *keys, uint32_t n, uint2 *ranges, int sms, cudaStream_t st)
{
    if (n == 0) return;
    ProfScope ps_("ranges", st);
    k_ranges<<<grid_for(n, 256, sms), 256, 0, st>>>(keys, n, ranges);
    count_launch();
}

}  // namespace dgs
