// Device-wide exclusive scan and stable LSD radix sort (u32 key, u32 value).
//
// Both are HBM-bound streaming passes.  The radix sort is the classic
// three-step LSD pass per 8-bit digit: per-block digit histogram, exclusive
// scan of the digit-major histogram table, stable scatter.  Stability inside
// a block comes from giving every warp a contiguous run of RS_ITEMS * 32 items
// that it ranks in index order (peers by eight ballots), then offsetting warps by
// the digit counts of the warps before them.  The scatter first reorders the
// block's RS_CHUNK items by digit in shared memory, then writes each digit run
// with consecutive threads on consecutive slots (coalesced stores).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dgs_internal.cuh"

namespace dgs {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;   // 4096

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_CHUNK = RS_THREADS * RS_ITEMS;         // 2048
constexpr int RS_RADIX = 256;

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

// Block-wide exclusive scan of SCAN_CHUNK values held in shared memory (padded).
__device__ uint32_t block_scan_chunk(uint32_t *sh, uint32_t *warp_tot)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t v[SCAN_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) { v[k] = sh[pad(t * SCAN_ITEMS + k)]; sum += v[k]; }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0, xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = xi - x;   // exclusive warp offsets
        if (lane == SCAN_THREADS / 32 - 1) warp_tot[SCAN_THREADS / 32] = xi;
    }
    __syncthreads();
    uint32_t run = warp_tot[w] + inc - sum;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) { sh[pad(t * SCAN_ITEMS + k)] = run; run += v[k]; }
    __syncthreads();
    return warp_tot[SCAN_THREADS / 32];
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t *in, size_t n, uint32_t *sums)
{
    const size_t base = (size_t)blockIdx.x * SCAN_CHUNK;
    uint32_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        size_t i = base + (size_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    __shared__ uint32_t wt[SCAN_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += wt[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t *in, uint32_t *out, size_t n,
                                                            const uint32_t *offsets, uint32_t *total)
{
    __shared__ uint32_t sh[SCAN_CHUNK + SCAN_CHUNK / 32];
    __shared__ uint32_t wt[SCAN_THREADS / 32 + 1];
    const size_t base = (size_t)blockIdx.x * SCAN_CHUNK;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int j = k * SCAN_THREADS + threadIdx.x;
        size_t i = base + j;
        sh[pad(j)] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t tot = block_scan_chunk(sh, wt);
    uint32_t off = offsets ? offsets[blockIdx.x] : 0u;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int j = k * SCAN_THREADS + threadIdx.x;
        size_t i = base + j;
        if (i < n) out[i] = sh[pad(j)] + off;
    }
    if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total = off + tot;
}

size_t blocks_for(size_t n, size_t chunk) { return (n + chunk - 1) / chunk; }

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Recursive scan; ws holds the block sums of every level.
cudaError_t scan_rec(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total, uint32_t *ws,
                     cudaStream_t st)
{
    if (n == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    size_t nb = blocks_for(n, SCAN_CHUNK);
    if (nb == 1) {
        k_scan_down<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr, total);
        count_launch();
        return cudaGetLastError();
    }
    uint32_t *sums = ws;
    uint32_t *next = ws + align_up(nb * sizeof(uint32_t)) / sizeof(uint32_t);
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums);
    count_launch();
    cudaError_t e = scan_rec(sums, sums, nb, nullptr, next, st);
    if (e != cudaSuccess) return e;
    k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, sums, total);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
// n_dev (optional) holds the live item count on the device (<= n, the capacity)
__device__ __forceinline__ size_t live_count(size_t n, const uint32_t *n_dev)
{
    return n_dev ? min(n, (size_t)*n_dev) : n;
}

// Per-block digit histogram.  All of a thread's keys are loaded before any
// counting (RS_ITEMS loads in flight per thread); each warp counts into its
// own row of shared counters so warps never contend, then thread d sums the
// rows for digit d.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *__restrict__ keys, size_t n_cap,
                                                        const uint32_t *n_dev, int shift, uint32_t mask,
                                                        uint32_t *__restrict__ hist, uint32_t nblocks)
{
    const size_t n = live_count(n_cap, n_dev);
    __shared__ uint32_t h[RS_WARPS][RS_RADIX];
    const int w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&h[0][0])[d] = 0;
    const size_t base = (size_t)blockIdx.x * RS_CHUNK;
    uint32_t key[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const size_t i = base + (size_t)k * RS_THREADS + threadIdx.x;
        key[k] = i < n ? __ldg(keys + i) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const size_t i = base + (size_t)k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[w][(key[k] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) tot += h[ww][threadIdx.x];
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = tot;
}

// Lanes of the warp whose digit equals this lane's (8-bit digits): one ballot
// per digit bit, restricted to the lanes holding a valid item.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, uint32_t valid)
{
    uint32_t peers = valid;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

struct ScatterSmem {
    uint32_t wh[RS_WARPS][RS_RADIX];     // per-warp digit counts, then offsets
    uint32_t dstart[RS_RADIX];           // first block-local slot of each digit
    uint32_t gbase[RS_RADIX];            // global slot of the block's first item of each digit
    uint32_t sk[RS_CHUNK], sv[RS_CHUNK]; // the block's items in (digit, index) order
    uint32_t wsum[RS_WARPS];
};

// Stable scatter of one block's RS_CHUNK items (item k of this thread has
// block-local index w * RS_ITEMS * 32 + k * 32 + lane; the first nvalid are
// live).  sm.wh must be zero on entry.  Ranks every item among the block's
// items of its digit in index order, reorders the items by digit in shared
// memory, then writes each digit run with consecutive threads on consecutive
// slots (coalesced stores).
__device__ __forceinline__ void rank_and_scatter(const uint32_t (&key)[RS_ITEMS], const uint32_t (&val)[RS_ITEMS],
                                                 uint32_t nvalid, int shift, uint32_t mask,
                                                 const uint32_t *__restrict__ offsets, uint32_t nblocks,
                                                 uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                 ScatterSmem &sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t wbase = (uint32_t)w * (RS_ITEMS * 32);
    uint32_t rank[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const bool ok = wbase + (uint32_t)(k * 32 + lane) < nvalid;
        uint32_t d = ok ? ((key[k] >> shift) & mask) : 0u;
        uint32_t peers = digit_peers(d, __ballot_sync(0xffffffffu, ok));
        uint32_t before = ok ? sm.wh[w][d] : 0u;
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (ok && lane == leader) sm.wh[w][d] = before + __popc(peers);
        __syncwarp();
        rank[k] = ok ? before + __popc(peers & lt) : 0xffffffffu;
    }
    __syncthreads();
    // thread = digit: exclusive prefix across warps, digit total, then a
    // block-wide exclusive scan of the totals gives each digit's local start
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) { uint32_t c = sm.wh[ww][d]; sm.wh[ww][d] = run; run += c; }
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm.wsum[w] = inc;
    __syncthreads();
    uint32_t woff = 0;
    for (int ww = 0; ww < w; ++ww) woff += sm.wsum[ww];
    sm.dstart[d] = woff + inc - run;
    sm.gbase[d] = offsets[(size_t)d * nblocks + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        if (rank[k] == 0xffffffffu) continue;
        const uint32_t dk = (key[k] >> shift) & mask;
        const uint32_t pos = sm.dstart[dk] + sm.wh[w][dk] + rank[k];
        sm.sk[pos] = key[k];
        sm.sv[pos] = val[k];
    }
    __syncthreads();
    // consecutive threads write consecutive slots of each digit run: coalesced
    for (uint32_t i = threadIdx.x; i < nvalid; i += RS_THREADS) {
        const uint32_t kk = sm.sk[i];
        const uint32_t dk = (kk >> shift) & mask;
        const uint32_t g = sm.gbase[dk] + (i - sm.dstart[dk]);
        kout[g] = kk;
        vout[g] = sm.sv[i];
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *kin, const uint32_t *vin,
                                                           uint32_t *kout, uint32_t *vout, size_t n_cap,
                                                           const uint32_t *n_dev, int shift, uint32_t mask,
                                                           const uint32_t *offsets, uint32_t nblocks)
{
    const size_t n = live_count(n_cap, n_dev);
    __shared__ ScatterSmem sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&sm.wh[0][0])[d] = 0;
    __syncthreads();
    const size_t blk0 = (size_t)blockIdx.x * RS_CHUNK;
    const size_t base = blk0 + (size_t)w * (RS_ITEMS * 32);
    uint32_t key[RS_ITEMS], val[RS_ITEMS];
    // every load of the tile is issued before the ranking chain starts
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const size_t i = base + (size_t)k * 32 + lane;
        key[k] = i < n ? __ldg(kin + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const size_t i = base + (size_t)k * 32 + lane;
        val[k] = i < n ? __ldg(vin + i) : 0u;
    }
    const uint32_t nvalid = n <= blk0 ? 0u : (n - blk0 < (size_t)RS_CHUNK ? (uint32_t)(n - blk0) : (uint32_t)RS_CHUNK);
    rank_and_scatter(key, val, nvalid, shift, mask, offsets, nblocks, kout, vout, sm);
}

// ------------------------------------------------ first pass of the tile sort
// The tile entries of the depth-ordered records are never written unsorted:
// the first radix pass generates them from the records' tile rectangles.
// Record j (depth order) owns entries [toffs[j], toffs[j] + counts[j]); entry
// k of it is tile (ty0 + k / tw, tx0 + k % tw), key bins[j].x + (k / tw) *
// tiles_x + k % tw, value bins[j].z (the record slot).  Radix block b owns
// entries [b RS_CHUNK, (b + 1) RS_CHUNK) as in every other pass, and
// first[b] is the record holding entry b RS_CHUNK.

__device__ __forceinline__ uint32_t entries_live(uint32_t e_cap, const uint32_t *ne_dev)
{
    return ne_dev ? min(e_cap, *ne_dev) : e_cap;
}

__global__ void k_chunk_first(const uint32_t *__restrict__ toffs, const uint32_t *__restrict__ counts, uint32_t nr_cap,
                              const uint32_t *nr_dev, uint32_t e_cap, const uint32_t *ne_dev,
                              uint32_t *__restrict__ first)
{
    const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
    const uint32_t ne = entries_live(e_cap, ne_dev);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
        const uint32_t c = counts[j];
        if (c == 0) continue;
        const uint32_t s = toffs[j];
        const uint32_t e = min(s + c, ne);
        for (uint32_t b = (s + RS_CHUNK - 1) / RS_CHUNK; (size_t)b * RS_CHUNK < e; ++b) first[b] = j;
    }
}

// Walk the records overlapping entries [E0, E1) of the block, RS_THREADS at a
// time in depth order; f(e, key, slot) is called for every entry e in the
// range (e the entry's index, key its tile key, slot the record slot).
// Every thread returns after the same number of barriers.
template <typename F>
__device__ __forceinline__ void for_chunk_entries(const uint4 *__restrict__ bins, const uint32_t *__restrict__ toffs,
                                                  const uint32_t *__restrict__ counts, uint32_t nr, uint32_t r0,
                                                  uint32_t E0, uint32_t E1, int tiles_x, F f)
{
    for (uint32_t base = r0;; base += RS_THREADS) {
        const uint32_t r = base + threadIdx.x;
        bool more = false;
        if (r < nr) {
            const uint32_t s = toffs[r];
            if (s < E1) {
                more = true;
                const uint32_t c = counts[r];
                const uint32_t lo = max(s, E0), hi = min(s + c, E1);
                if (lo < hi) {
                    const uint4 bn = bins[r];
                    const uint32_t tw = bn.y;
                    uint32_t k = lo - s;
                    uint32_t col = k % tw;
                    uint32_t key = bn.x + (k / tw) * (uint32_t)tiles_x + col;
                    for (uint32_t e = lo; e < hi; ++e) {
                        f(e, key, bn.z);
                        if (++col == tw) { col = 0; key += (uint32_t)tiles_x - tw + 1u; } else { ++key; }
                    }
                }
            }
        }
        // toffs is non-decreasing: once some record starts at or past E1, all later ones do
        if (!__syncthreads_and(more)) break;
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist_bins(const uint4 *__restrict__ bins,
                                                             const uint32_t *__restrict__ toffs,
                                                             const uint32_t *__restrict__ counts, uint32_t nr_cap,
                                                             const uint32_t *nr_dev, uint32_t e_cap,
                                                             const uint32_t *ne_dev, const uint32_t *__restrict__ first,
                                                             int tiles_x, uint32_t mask, uint32_t *__restrict__ hist,
                                                             uint32_t nblocks)
{
    __shared__ uint32_t h[RS_WARPS][RS_RADIX];
    const int w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&h[0][0])[d] = 0;
    __syncthreads();
    const uint32_t ne = entries_live(e_cap, ne_dev);
    const uint32_t E0 = blockIdx.x * (uint32_t)RS_CHUNK;
    if (E0 < ne) {
        const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
        const uint32_t E1 = min(E0 + (uint32_t)RS_CHUNK, ne);
        for_chunk_entries(bins, toffs, counts, nr, first[blockIdx.x], E0, E1, tiles_x,
                          [&](uint32_t, uint32_t key, uint32_t) { atomicAdd(&h[w][key & mask], 1u); });
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) tot += h[ww][threadIdx.x];
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter_bins(const uint4 *__restrict__ bins,
                                                                const uint32_t *__restrict__ toffs,
                                                                const uint32_t *__restrict__ counts, uint32_t nr_cap,
                                                                const uint32_t *nr_dev, uint32_t e_cap,
                                                                const uint32_t *ne_dev,
                                                                const uint32_t *__restrict__ first, int tiles_x,
                                                                uint32_t mask, const uint32_t *offsets,
                                                                uint32_t nblocks, uint32_t *kout, uint32_t *vout)
{
    __shared__ ScatterSmem sm;
    const uint32_t ne = entries_live(e_cap, ne_dev);
    const uint32_t E0 = blockIdx.x * (uint32_t)RS_CHUNK;
    if (E0 >= ne) return;                    // block-uniform
    const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
    const uint32_t E1 = min(E0 + (uint32_t)RS_CHUNK, ne);
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&sm.wh[0][0])[d] = 0;
    // the block's entries, in entry order, into shared memory
    for_chunk_entries(bins, toffs, counts, nr, first[blockIdx.x], E0, E1, tiles_x,
                      [&](uint32_t e, uint32_t key, uint32_t slot) {
                          sm.sk[e - E0] = key;
                          sm.sv[e - E0] = slot;
                      });
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nvalid = E1 - E0;
    uint32_t key[RS_ITEMS], val[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t i = (uint32_t)w * (RS_ITEMS * 32) + (uint32_t)(k * 32 + lane);
        key[k] = i < nvalid ? sm.sk[i] : 0u;
        val[k] = i < nvalid ? sm.sv[i] : 0u;
    }
    __syncthreads();                         // sk / sv are reused for the reordered items
    rank_and_scatter(key, val, nvalid, 0, mask, offsets, nblocks, kout, vout, sm);
}

}  // namespace

size_t scan_workspace_bytes(size_t n)
{
    size_t tot = 0;
    while (n > (size_t)SCAN_CHUNK) {
        n = blocks_for(n, SCAN_CHUNK);
        tot += align_up(n * sizeof(uint32_t));
    }
    return tot + 256;
}

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total_out,
                               void *ws, cudaStream_t st)
{
    return scan_rec(in, out, n, total_out, (uint32_t *)ws, st);
}

size_t radix_workspace_bytes(size_t n)
{
    size_t nb = blocks_for(n > 0 ? n : 1, RS_CHUNK);
    size_t hist = (size_t)RS_RADIX * nb;
    // histogram table, its scan workspace, and the first-record table of the tile sort
    return align_up(hist * sizeof(uint32_t)) + align_up(scan_workspace_bytes(hist)) +
           align_up((nb + 1) * sizeof(uint32_t));
}

// Plain passes over digits [shift0, bits) of (k0, v0); the result is in (k1,
// v1) when *result_in_alt.
cudaError_t radix_passes(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, size_t n, int shift0, int bits,
                         void *ws, cudaStream_t st, bool *result_in_alt, const uint32_t *n_dev, const char *prof)
{
    *result_in_alt = false;
    static bool carveout_set = false;   // the scatter's shared memory allows 8 blocks per SM at full carveout
    if (!carveout_set) {
        cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_rs_scatter_bins, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        carveout_set = true;
    }
    size_t nb = blocks_for(n, RS_CHUNK);
    uint32_t *hist = (uint32_t *)ws;
    void *scan_ws = (char *)ws + align_up((size_t)RS_RADIX * nb * sizeof(uint32_t));
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int shift = shift0; shift < bits; shift += 8) {
        int w = bits - shift < 8 ? bits - shift : 8;
        uint32_t mask = (1u << w) - 1u;
        ProfScope ps_(prof, st);
        k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, st>>>(ki, n, n_dev, shift, mask, hist, (uint32_t)nb);
        count_launch();
        cudaError_t e = exclusive_scan_u32(hist, hist, (size_t)RS_RADIX * nb, nullptr, scan_ws, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, st>>>(ki, vi, ko, vo, n, n_dev, shift, mask, hist,
                                                          (uint32_t)nb);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t *tk = ki, *tv = vi;
        ki = ko; vi = vo; ko = tk; vo = tv;
        *result_in_alt = !*result_in_alt;
    }
    return cudaSuccess;
}

cudaError_t radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, size_t n,
                             int bits, void *ws, cudaStream_t st, bool *result_in_alt, const uint32_t *n_dev,
                             const char *prof)
{
    *result_in_alt = false;
    if (n == 0 || (n <= 1 && !n_dev) || bits <= 0) return cudaSuccess;
    return radix_passes(k0, v0, k1, v1, n, 0, bits, ws, st, result_in_alt, n_dev, prof);
}

cudaError_t radix_sort_entries(const uint4 *bins, const uint32_t *toffs, const uint32_t *counts, uint32_t n_rec,
                               const uint32_t *nrec_dev, int tiles_x, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                               uint32_t *v1, size_t e_cap, const uint32_t *nent_dev, int bits, void *ws,
                               cudaStream_t st, bool *result_in_alt, int sms)
{
    *result_in_alt = false;
    if (e_cap == 0 || n_rec == 0) return cudaSuccess;
    if (bits < 1) bits = 1;                  // the first pass also materialises the entries
    size_t nb = blocks_for(e_cap, RS_CHUNK);
    uint32_t *hist = (uint32_t *)ws;
    const size_t hist_bytes = align_up((size_t)RS_RADIX * nb * sizeof(uint32_t));
    void *scan_ws = (char *)ws + hist_bytes;
    uint32_t *first = (uint32_t *)((char *)ws + hist_bytes + align_up(scan_workspace_bytes((size_t)RS_RADIX * nb)));
    {
        const int w = bits < 8 ? bits : 8;
        const uint32_t mask = (1u << w) - 1u;
        ProfScope ps_("radix_tile", st);
        unsigned g = (unsigned)((n_rec + 255) / 256);
        if (g > (unsigned)sms * 16u) g = (unsigned)sms * 16u;
        k_chunk_first<<<g, 256, 0, st>>>(toffs, counts, n_rec, nrec_dev, (uint32_t)e_cap, nent_dev, first);
        count_launch();
        k_rs_hist_bins<<<(unsigned)nb, RS_THREADS, 0, st>>>(bins, toffs, counts, n_rec, nrec_dev, (uint32_t)e_cap,
                                                            nent_dev, first, tiles_x, mask, hist, (uint32_t)nb);
        count_launch();
        cudaError_t e = exclusive_scan_u32(hist, hist, (size_t)RS_RADIX * nb, nullptr, scan_ws, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter_bins<<<(unsigned)nb, RS_THREADS, 0, st>>>(bins, toffs, counts, n_rec, nrec_dev,
                                                               (uint32_t)e_cap, nent_dev, first, tiles_x, mask,
                                                               hist, (uint32_t)nb, k1, v1);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (bits <= 8) {
        *result_in_alt = true;
        return cudaSuccess;
    }
    // the remaining digits: plain passes from (k1, v1), ending in (k0, v0) after an odd count
    bool alt2 = false;
    cudaError_t e = radix_passes(k1, v1, k0, v0, e_cap, 8, bits, ws, st, &alt2, nent_dev, "radix_tile");
    *result_in_alt = !alt2;
    return e;
}

}  // namespace dgs
