// Exact reuse of rendered tiles across delivery states (utility passes).
//
// A state's walk over a tile's sorted run is decided only by the delivered
// depths of the clusters whose entries it examines: an entry is composited iff
// its depth variant equals the state's delivered depth of its cluster
// (Sections 3-4), and every other step of the walk is the same for all states
// of the view group.  The forward raster records, for each rendered (state,
// tile), the run prefix P its blocks staged before every pixel of the state
// stopped (T (1 - alpha) < 1e-4, or the run's end).  Every entry in that
// prefix belongs to one of the clusters whose first entry in the run lies
// before P -- the first m(P) clusters in order of first appearance.  Any
// other state of the view group with the same delivered depths on those m
// clusters therefore walks the same entries with the same inclusions, stops
// at the same place and produces the same pixels bit for bit, so its FP64
// squared-error partial of the tile is the rendered state's.
//
// The states of each (view group, tile) are grouped by their depths on the
// first K clusters of the run (K = 0 first: one group per tile), one member of
// each group is rendered, and every member that agrees with it on its first
// m(P) clusters takes its partial; each other member is regrouped with K one
// past the first cluster where it differs from the rendered one, so K grows
// every round and groups split no finer than the walks require.  Keys hold up to SHARE_MAX_K = 15 clusters (4 bits
// each); a state that would need more is rendered on its own.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {

namespace {

constexpr uint32_t NO_POS = 0xffffffffu;
constexpr unsigned long long EMPTY_KEY = ~0ull;
constexpr int SHARE_PROBES = 32;

// First SHARE_ORDER distinct clusters of each run in order of first
// appearance: ord_c[vt][j] (0xffffffff past the run's distinct count) and the
// run-relative position of each one's first entry, ord_fp[vt][j] (ascending;
// NO_POS past the count).  The run is scanned in order, so the first
// SHARE_ORDER distinct clusters met are the ones with the smallest first
// positions and the scan stops once it has met them.
__global__ void __launch_bounds__(256) k_first_clusters(const Rec *__restrict__ recs,
                                                        const uint32_t *__restrict__ evals,
                                                        const uint2 *__restrict__ ranges, uint32_t n_vt, int C,
                                                        uint32_t *__restrict__ ord_c, uint32_t *__restrict__ ord_fp)
{
    __shared__ uint32_t fp[MAX_CLUSTERS];
    __shared__ uint32_t ndist;
    for (uint32_t vt = blockIdx.x; vt < n_vt; vt += gridDim.x) {
        for (int c = threadIdx.x; c < C; c += blockDim.x) fp[c] = NO_POS;
        if (threadIdx.x == 0) ndist = 0;
        if (threadIdx.x < SHARE_ORDER) {
            ord_c[(size_t)vt * SHARE_ORDER + threadIdx.x] = NO_POS;
            ord_fp[(size_t)vt * SHARE_ORDER + threadIdx.x] = NO_POS;
        }
        __syncthreads();
        const uint2 rg = ranges[vt];
        for (uint32_t base = rg.x; base < rg.y; base += blockDim.x) {
            const uint32_t e = base + threadIdx.x;
            if (e < rg.y) {
                const uint32_t slot = __ldg(evals + e);
                const uint32_t c = __ldg(reinterpret_cast<const uint32_t *>(recs + slot) + 11) & REC_CLUSTER;
                if (atomicMin(&fp[c], e - rg.x) == NO_POS) atomicAdd(&ndist, 1u);
            }
            __syncthreads();
            const bool enough = ndist >= (uint32_t)SHARE_ORDER;
            __syncthreads();
            if (enough) break;
        }
        // rank of each met cluster by first position (positions are distinct)
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            const uint32_t f = fp[c];
            if (f == NO_POS) continue;
            int r = 0;
            for (int c2 = 0; c2 < C; ++c2) r += fp[c2] < f ? 1 : 0;
            if (r < SHARE_ORDER) {
                ord_c[(size_t)vt * SHARE_ORDER + r] = (uint32_t)c;
                ord_fp[(size_t)vt * SHARE_ORDER + r] = f;
            }
        }
        __syncthreads();
    }
}

// Round-one pairs: every (view group tile, state of that view group), tile
// major.  vt_off[vt] = first pair of vt (exclusive scan of the view group's
// state count); vg_first[v] = first entry of view group v in state_order.
__global__ void k_pairs_init(const uint32_t *__restrict__ vt_off, uint32_t n_vt, uint32_t n_pairs, uint32_t tiles,
                             const int32_t *__restrict__ vg_first, const int32_t *__restrict__ state_order,
                             uint32_t *__restrict__ pvt, uint32_t *__restrict__ pst, uint8_t *__restrict__ pk)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pairs; i += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = n_vt - 1;       // largest vt with vt_off[vt] <= i
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (vt_off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const uint32_t v = lo / tiles;
        pvt[i] = lo;
        pst[i] = (uint32_t)state_order[vg_first[v] + (int)(i - vt_off[lo])];
        pk[i] = 0;
    }
}

// [first, end) of every run of equal keys in a sorted array (seg zeroed before).
__global__ void k_segments(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ n_dev,
                           uint2 *__restrict__ seg)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) seg[k].x = i;
        if (i + 1 == n || keys[i + 1] != k) seg[k].y = i + 1;
    }
}

// Group key of pair i: K in the top 4 bits, then the state's delivered depth
// of the run's j-th cluster in bits 4j..4j+3 (j < K); K > SHARE_MAX_K: no key.
// One thread per pair over the whole pair array (the depth loads of all pairs
// in flight together), read back coalesced by the grouping kernel.
__global__ void k_pair_keys(const uint32_t *__restrict__ pvt, const uint32_t *__restrict__ pst,
                            const uint8_t *__restrict__ pk, const uint32_t *__restrict__ n_dev,
                            const uint32_t *__restrict__ ord_c, const uint8_t *__restrict__ depth, int C,
                            unsigned long long *__restrict__ keys)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int K = pk[i];
        if (K > SHARE_MAX_K) { keys[i] = EMPTY_KEY; continue; }
        const uint32_t *oc = ord_c + (size_t)pvt[i] * SHARE_ORDER;
        const uint8_t *row = depth + (size_t)pst[i] * C;
        unsigned long long key = (unsigned long long)K << 60;
#pragma unroll
        for (int j = 0; j < SHARE_MAX_K; ++j)
            if (j < K) key |= (unsigned long long)__ldg(row + __ldg(oc + j)) << (4 * j);
        keys[i] = key;
    }
}

__device__ __forceinline__ uint32_t key_hash(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// Open-addressing insert / lookup in the block's table, at most SHARE_PROBES
// slots from the key's home slot; -1 when not placed / absent (the pair then
// renders on its own).  Many pairs of a tile share a key, so a slot is read
// before any atomic: only the first arrival of a key pays for the
// compare-and-swap.
__device__ __forceinline__ int table_insert(unsigned long long *keys, unsigned long long key)
{
    uint32_t h = key_hash(key) & (SHARE_TABLE - 1);
    for (int p = 0; p < SHARE_PROBES; ++p) {
        const unsigned long long k = *(volatile unsigned long long *)&keys[h];
        if (k == key) return (int)h;
        if (k == EMPTY_KEY) {
            const unsigned long long old = atomicCAS(&keys[h], EMPTY_KEY, key);
            if (old == EMPTY_KEY || old == key) return (int)h;
        }
        h = (h + 1) & (SHARE_TABLE - 1);
    }
    return -1;
}
__device__ __forceinline__ int table_find(const unsigned long long *keys, unsigned long long key)
{
    uint32_t h = key_hash(key) & (SHARE_TABLE - 1);
    for (int p = 0; p < SHARE_PROBES; ++p) {
        const unsigned long long k = keys[h];
        if (k == key) return (int)h;
        if (k == EMPTY_KEY) return -1;
        h = (h + 1) & (SHARE_TABLE - 1);
    }
    return -1;
}

// One block per view-group tile: group its pending pairs by their key (K and
// the depths of the run's first K clusters); each pair's representative is
// the lowest state of its group (itself when it has no key or the table is
// full).
__global__ void __launch_bounds__(256) k_share_group(const uint2 *__restrict__ seg, uint32_t n_vt,
                                                     const uint32_t *__restrict__ pst,
                                                     const unsigned long long *__restrict__ pkey,
                                                     uint32_t *__restrict__ prep)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sm_raw);
    uint32_t *reps = reinterpret_cast<uint32_t *>(keys + SHARE_TABLE);
    for (uint32_t vt = blockIdx.x; vt < n_vt; vt += gridDim.x) {
        const uint2 sg = seg[vt];
        if (sg.x >= sg.y) continue;                       // block-uniform
        for (int h = threadIdx.x; h < SHARE_TABLE; h += blockDim.x) { keys[h] = EMPTY_KEY; reps[h] = NO_POS; }
        __syncthreads();
        for (uint32_t i = sg.x + threadIdx.x; i < sg.y; i += blockDim.x) {
            const unsigned long long key = pkey[i];
            if (key == EMPTY_KEY) continue;
            const int h = table_insert(keys, key);
            // pairs come in state order, so the group's minimum is usually in place early
            const uint32_t st_i = pst[i];
            if (h >= 0 && *(volatile uint32_t *)&reps[h] > st_i) atomicMin(&reps[h], st_i);
        }
        __syncthreads();
        for (uint32_t i = sg.x + threadIdx.x; i < sg.y; i += blockDim.x) {
            const unsigned long long key = pkey[i];
            uint32_t r = pst[i];
            if (key != EMPTY_KEY) {
                const int h = table_find(keys, key);
                if (h >= 0) r = reps[h];
            }
            prep[i] = r;
        }
        __syncthreads();
    }
}

// flag[i] = 1 for the pairs rendered this round (their own representative).
__global__ void k_rep_flags(const uint32_t *__restrict__ pst, const uint32_t *__restrict__ prep,
                            const uint32_t *__restrict__ n_dev, uint32_t *__restrict__ flag)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = prep[i] == pst[i] ? 1u : 0u;
}

// Scatter the flagged pairs to pos[i] (exclusive scan of the flags).
__global__ void k_compact_pairs(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                                const uint32_t *__restrict__ n_dev, const uint32_t *__restrict__ pvt,
                                const uint32_t *__restrict__ pst, const uint8_t *__restrict__ pk,
                                uint32_t *__restrict__ ovt, uint32_t *__restrict__ ost, uint8_t *__restrict__ ok)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const uint32_t o = pos[i];
        ovt[o] = pvt[i];
        ost[o] = pst[i];
        if (ok) ok[o] = pk[i];
    }
}

// Work items of the render list: a new item every G list entries of the same
// tile (flag), then (first, count) of each item.
__global__ void k_item_flags(const uint32_t *__restrict__ lvt, const uint2 *__restrict__ seg,
                             const uint32_t *__restrict__ n_dev, int G, uint32_t *__restrict__ flag)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = ((i - seg[lvt[i]].x) % (uint32_t)G) == 0 ? 1u : 0u;
}
__global__ void k_items(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                        const uint32_t *__restrict__ lvt, const uint2 *__restrict__ seg,
                        const uint32_t *__restrict__ n_dev, int G, uint32_t *__restrict__ item_first,
                        uint32_t *__restrict__ item_count)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const uint32_t end = seg[lvt[i]].y;
        item_first[pos[i]] = i;
        item_count[pos[i]] = min((uint32_t)G, end - i);
    }
}

// After the representatives rendered: each other pair agreeing with its
// representative on the first m(P) clusters takes the representative's
// partial; the rest stay pending with K = (first cluster where they differ) + 1,
// which exceeds the group's K (m(P) > 15: rendered alone).
__global__ void k_share_resolve(const uint32_t *__restrict__ pvt, const uint32_t *__restrict__ pst,
                                uint8_t *__restrict__ pk, const uint32_t *__restrict__ prep,
                                const uint32_t *__restrict__ n_dev, TileGeom geo,
                                const uint32_t *__restrict__ ord_c, const uint32_t *__restrict__ ord_fp,
                                const uint8_t *__restrict__ depth, int C, const uint32_t *__restrict__ stop,
                                double *__restrict__ partial, uint32_t *__restrict__ pending)
{
    const uint32_t n = *n_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t s = pst[i], q = prep[i];
        if (q == s) { pending[i] = 0; continue; }
        const uint32_t tiles = geo.tiles;
        const uint32_t vt = pvt[i], tile = vt % tiles;
        const uint32_t P = stop[(size_t)q * tiles + tile];
        const uint32_t *oc = ord_c + (size_t)vt * SHARE_ORDER;
        const uint32_t *of = ord_fp + (size_t)vt * SHARE_ORDER;
        int m = 0;
        while (m < SHARE_ORDER && of[m] < P) ++m;
        if (m > SHARE_MAX_K) {                       // too many clusters reached: render alone
            pk[i] = (uint8_t)(SHARE_MAX_K + 1);
            pending[i] = 1;
            continue;
        }
        int j = 0;                                   // first of the m clusters where the depths differ
        while (j < m && depth[(size_t)s * C + oc[j]] == depth[(size_t)q * C + oc[j]]) ++j;
        if (j == m) {
            int bx0, bx1, by0, by1;
            tile_blocks(geo, tile, bx0, bx1, by0, by1);
            for (int by = by0; by < by1; ++by)
                for (int bx = bx0; bx < bx1; ++bx) {
                    const size_t b = (size_t)by * geo.blocks_x + bx;
                    partial[(size_t)s * geo.blocks + b] = partial[(size_t)q * geo.blocks + b];
                }
            pending[i] = 0;
        } else {
            // the group agreed on its first K clusters, so j >= K: regroup one cluster past
            // the disagreement (the fewest clusters that separate s from q)
            pk[i] = (uint8_t)(j + 1);
            pending[i] = 1;
        }
    }
}

unsigned grid_of(size_t n, int sms)
{
    size_t b = (n + 255) / 256;
    const size_t cap = (size_t)sms * 16;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

}  // namespace

void launch_first_clusters(const Rec *recs, const uint32_t *evals, const uint2 *ranges, uint32_t n_vt, int C,
                           uint32_t *ord_c, uint32_t *ord_fp, int sms, cudaStream_t st)
{
    if (n_vt == 0) return;
    ProfScope ps_("share_order", st);
    const unsigned g = n_vt < (uint32_t)sms * 8 ? n_vt : (unsigned)sms * 8;
    k_first_clusters<<<g, 256, 0, st>>>(recs, evals, ranges, n_vt, C, ord_c, ord_fp);
    count_launch();
}

void launch_pairs_init(const uint32_t *vt_off, uint32_t n_vt, uint32_t n_pairs, uint32_t tiles,
                       const int32_t *vg_first, const int32_t *state_order, uint32_t *pvt, uint32_t *pst,
                       uint8_t *pk, int sms, cudaStream_t st)
{
    if (n_pairs == 0) return;
    ProfScope ps_("share_pairs", st);
    k_pairs_init<<<grid_of(n_pairs, sms), 256, 0, st>>>(vt_off, n_vt, n_pairs, tiles, vg_first, state_order, pvt,
                                                         pst, pk);
    count_launch();
}

void launch_segments(const uint32_t *keys, const uint32_t *n_dev, size_t n_cap, uint2 *seg, int sms,
                     cudaStream_t st)
{
    if (n_cap == 0) return;
    k_segments<<<grid_of(n_cap, sms), 256, 0, st>>>(keys, n_dev, seg);
    count_launch();
}

void launch_share_group(const uint2 *seg, uint32_t n_vt, const uint32_t *pvt, const uint32_t *pst,
                        const uint8_t *pk, const uint32_t *n_dev, size_t n_cap, const uint32_t *ord_c,
                        const uint8_t *depth, int C, unsigned long long *keys, uint32_t *prep, int sms,
                        cudaStream_t st)
{
    if (n_vt == 0 || n_cap == 0) return;
    ProfScope ps_("share_group", st);
    k_pair_keys<<<grid_of(n_cap, sms), 256, 0, st>>>(pvt, pst, pk, n_dev, ord_c, depth, C, keys);
    count_launch();
    const size_t smem = SHARE_TABLE * (sizeof(unsigned long long) + sizeof(uint32_t));
    // per device, so set on every call (the pass is never captured: it synchronizes)
    cudaFuncSetAttribute(k_share_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned g = n_vt < (uint32_t)sms * 4 ? n_vt : (unsigned)sms * 4;
    k_share_group<<<g, 256, smem, st>>>(seg, n_vt, pst, keys, prep);
    count_launch();
}

void launch_rep_flags(const uint32_t *pst, const uint32_t *prep, const uint32_t *n_dev, size_t n_cap, uint32_t *flag,
                      int sms, cudaStream_t st)
{
    if (n_cap == 0) return;
    k_rep_flags<<<grid_of(n_cap, sms), 256, 0, st>>>(pst, prep, n_dev, flag);
    count_launch();
}

void launch_compact_pairs(const uint32_t *flag, const uint32_t *pos, const uint32_t *n_dev, size_t n_cap,
                          const uint32_t *pvt, const uint32_t *pst, const uint8_t *pk, uint32_t *ovt, uint32_t *ost,
                          uint8_t *ok, int sms, cudaStream_t st)
{
    if (n_cap == 0) return;
    k_compact_pairs<<<grid_of(n_cap, sms), 256, 0, st>>>(flag, pos, n_dev, pvt, pst, pk, ovt, ost, ok);
    count_launch();
}

void launch_item_lists(const uint32_t *lvt, const uint2 *seg, const uint32_t *n_dev, size_t n_cap, int G,
                       uint32_t *flag, uint32_t *pos, uint32_t *n_items_dev, void *scan_ws, uint32_t *item_first,
                       uint32_t *item_count, int sms, cudaStream_t st)
{
    if (n_cap == 0) return;
    k_item_flags<<<grid_of(n_cap, sms), 256, 0, st>>>(lvt, seg, n_dev, G, flag);
    count_launch();
    exclusive_scan_u32(flag, pos, n_cap, n_items_dev, scan_ws, st);
    k_items<<<grid_of(n_cap, sms), 256, 0, st>>>(flag, pos, lvt, seg, n_dev, G, item_first, item_count);
    count_launch();
}

void launch_share_resolve(const uint32_t *pvt, const uint32_t *pst, uint8_t *pk, const uint32_t *prep,
                          const uint32_t *n_dev, size_t n_cap, const TileGeom &geo, const uint32_t *ord_c,
                          const uint32_t *ord_fp, const uint8_t *depth, int C, const uint32_t *stop, double *partial,
                          uint32_t *pending, int sms, cudaStream_t st)
{
    if (n_cap == 0) return;
    ProfScope ps_("share_resolve", st);
    k_share_resolve<<<grid_of(n_cap, sms), 256, 0, st>>>(pvt, pst, pk, prep, n_dev, geo, ord_c, ord_fp, depth, C,
                                                          stop, partial, pending);
    count_launch();
}

}  // namespace dgs
