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
constexpr uint32_t DROP_KEY = 0xffffffffu;              // culled records' depth key

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
    uint32_t kept;                       // items the block writes
};

// Stable scatter of one block's RS_CHUNK items (item k of this thread has
// block-local index w * RS_ITEMS * 32 + k * 32 + lane; the first nvalid are
// live; with drop, items whose key is DROP_KEY are left out as if absent).
// The digit of key k is ((k - sub) >> shift) & mask; the scanned
// table gives the block's first output slot of digit d at toff[d * tstride].
// sm.wh must be zero on entry.  Ranks every item among the block's items of
// its digit in index order, reorders the items by digit in shared memory,
// then writes each digit run with consecutive threads on consecutive slots
// (coalesced stores).
__device__ __forceinline__ void rank_and_scatter(const uint32_t (&key)[RS_ITEMS], const uint32_t (&val)[RS_ITEMS],
                                                 uint32_t nvalid, int shift, uint32_t mask, uint32_t sub,
                                                 const uint32_t *__restrict__ toff, uint32_t tstride,
                                                 uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                 ScatterSmem &sm, bool drop = false)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t wbase = (uint32_t)w * (RS_ITEMS * 32);
    uint32_t rank[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const bool ok = wbase + (uint32_t)(k * 32 + lane) < nvalid && !(drop && key[k] == DROP_KEY);
        uint32_t d = ok ? (((key[k] - sub) >> shift) & mask) : 0u;
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
    if (d == RS_RADIX - 1) sm.kept = woff + inc;
    sm.gbase[d] = toff[(size_t)d * tstride];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        if (rank[k] == 0xffffffffu) continue;
        const uint32_t dk = ((key[k] - sub) >> shift) & mask;
        const uint32_t pos = sm.dstart[dk] + sm.wh[w][dk] + rank[k];
        sm.sk[pos] = key[k];
        sm.sv[pos] = val[k];
    }
    __syncthreads();
    // consecutive threads write consecutive slots of each digit run: coalesced
    const uint32_t kept = sm.kept;
    for (uint32_t i = threadIdx.x; i < kept; i += RS_THREADS) {
        const uint32_t kk = sm.sk[i];
        const uint32_t dk = ((kk - sub) >> shift) & mask;
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
    rank_and_scatter(key, val, nvalid, shift, mask, 0u, offsets + blockIdx.x, nblocks, kout, vout, sm);
}

// ------------------------------------------------ segmented passes
// Items [start(v), start(v + 1)) form segment v = 0 .. V-1, with start(v) =
// start[v * stride] non-decreasing (start(V) is the end).  Each segment is cut
// into blocks of RS_CHUNK items (the last one partial); bbase[v] is the first
// block of segment v and bbase[V] the number of blocks.  A stable pass over
// the digit ((key - v * sub) >> shift) & mask keeps every item inside its
// segment: block bl of segment v puts its count of digit d at
// hist[RS_RADIX * bbase[v] + d * nb_v + bl] (nb_v = the segment's blocks), so
// one exclusive scan of the table in index order gives every (segment, digit,
// block) its first output slot: segments one after another, the digits of a
// segment in order, the blocks of a digit in order.  Sorting records so, with
// the view groups as segments, leaves the tile sort only the tile digits.
struct Segs {
    const uint32_t *start;
    uint32_t stride;
    const uint32_t *bbase;
    int V;
    uint32_t sub;
};

__device__ __forceinline__ uint32_t seg_start(const Segs &g, int v) { return __ldg(g.start + (size_t)v * g.stride); }

// The segment of block b < bbase[V]: the last v with bbase[v] <= b (a segment
// without items has its successor's base, so the last one is the segment that
// holds the block).
__device__ __forceinline__ int seg_of_block(const Segs &g, uint32_t b)
{
    int lo = 0, hi = g.V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(g.bbase + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Block bl of segment v and its item range [s0, s1).
struct SegBlock {
    int v;
    uint32_t bl, nb, s0, s1;
};

__device__ __forceinline__ SegBlock seg_block(const Segs &g, uint32_t b)
{
    SegBlock r;
    r.v = seg_of_block(g, b);
    const uint32_t b0 = __ldg(g.bbase + r.v);
    r.bl = b - b0;
    r.nb = __ldg(g.bbase + r.v + 1) - b0;
    r.s0 = seg_start(g, r.v) + r.bl * (uint32_t)RS_CHUNK;
    r.s1 = min(r.s0 + (uint32_t)RS_CHUNK, seg_start(g, r.v + 1));
    return r;
}

// nb[v] = blocks of segment v (v < V), nb[V] = 0: the exclusive scan of nb is bbase.
__global__ void k_seg_blocks(const uint32_t *__restrict__ start, uint32_t stride, int V, uint32_t *__restrict__ nb)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= V; v += gridDim.x * blockDim.x) {
        if (v == V) { nb[v] = 0; continue; }
        const uint32_t n = start[(size_t)(v + 1) * stride] - start[(size_t)v * stride];
        nb[v] = (n + RS_CHUNK - 1) / RS_CHUNK;
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist_seg(const uint32_t *__restrict__ keys, Segs g, int shift,
                                                            uint32_t mask, uint32_t *__restrict__ hist, bool drop)
{
    const uint32_t b = blockIdx.x;
    if (b >= __ldg(g.bbase + g.V)) {          // no items: zero this block's share of the table tail
        hist[(size_t)RS_RADIX * b + threadIdx.x] = 0u;
        return;
    }
    __shared__ uint32_t h[RS_WARPS][RS_RADIX];
    const int w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&h[0][0])[d] = 0;
    const SegBlock sb = seg_block(g, b);
    const uint32_t sub = (uint32_t)sb.v * g.sub;
    uint32_t key[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t i = sb.s0 + (uint32_t)(k * RS_THREADS) + threadIdx.x;
        key[k] = i < sb.s1 ? __ldg(keys + i) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t i = sb.s0 + (uint32_t)(k * RS_THREADS) + threadIdx.x;
        if (i < sb.s1 && !(drop && key[k] == DROP_KEY)) atomicAdd(&h[w][((key[k] - sub) >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) tot += h[ww][threadIdx.x];
    hist[(size_t)RS_RADIX * __ldg(g.bbase + sb.v) + (size_t)threadIdx.x * sb.nb + sb.bl] = tot;
}

// 5 resident blocks (48 registers, no spills) beat 4 (63 registers) and 6
__global__ void __launch_bounds__(RS_THREADS, 5) k_rs_scatter_seg(const uint32_t *kin, const uint32_t *vin,
                                                               uint32_t *kout, uint32_t *vout, Segs g, int shift,
                                                               uint32_t mask, const uint32_t *offsets, bool drop)
{
    const uint32_t b = blockIdx.x;
    if (b >= __ldg(g.bbase + g.V)) return;   // block-uniform
    __shared__ ScatterSmem sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&sm.wh[0][0])[d] = 0;
    __syncthreads();
    const SegBlock sb = seg_block(g, b);
    const uint32_t base = sb.s0 + (uint32_t)w * (RS_ITEMS * 32);
    uint32_t key[RS_ITEMS], val[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t i = base + (uint32_t)(k * 32 + lane);
        key[k] = i < sb.s1 ? __ldg(kin + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t i = base + (uint32_t)(k * 32 + lane);
        val[k] = i < sb.s1 ? __ldg(vin + i) : 0u;
    }
    rank_and_scatter(key, val, sb.s1 - sb.s0, shift, mask, (uint32_t)sb.v * g.sub,
                     offsets + (size_t)RS_RADIX * __ldg(g.bbase + sb.v) + sb.bl, sb.nb, kout, vout, sm, drop);
}

// ------------------------------------------------ first pass of the tile sort
// The tile entries of the sorted records are never written unsorted: the
// first radix pass generates them from the records' tile rectangles.  Record
// j (sorted order) owns entries [toffs[j], toffs[j] + counts[j]); entry k of
// it is tile (ty0 + k / tw, tx0 + k % tw), key bins[j].x + (k / tw) * tiles_x
// + k % tw, value bins[j].z (the record slot).  The records of view group v
// are segment v of the record order, so its entries are segment v of the
// entry order, [eseg[v], eseg[v + 1]); first[b] is the record holding the
// first entry of entry block b.

__device__ __forceinline__ uint32_t entries_live(uint32_t e_cap, const uint32_t *ne_dev)
{
    return ne_dev ? min(e_cap, *ne_dev) : e_cap;
}

// eseg[v] = first entry of the records of segment v (capped at the live entry count).
__global__ void k_entry_segs(Segs rseg, const uint32_t *__restrict__ toffs, uint32_t nr_cap,
                             const uint32_t *nr_dev, uint32_t e_cap, const uint32_t *ne_dev,
                             uint32_t *__restrict__ eseg)
{
    const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
    const uint32_t ne = entries_live(e_cap, ne_dev);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= rseg.V; v += gridDim.x * blockDim.x) {
        const uint32_t r = v < rseg.V ? seg_start(rseg, v) : nr;
        eseg[v] = r < nr ? min(toffs[r], ne) : ne;
    }
}

__global__ void k_chunk_first_seg(const uint32_t *__restrict__ toffs, const uint32_t *__restrict__ counts,
                                  uint32_t nr_cap, const uint32_t *nr_dev, Segs rseg, Segs eseg,
                                  uint32_t *__restrict__ first)
{
    const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
        const uint32_t c = counts[j];
        if (c == 0) continue;
        // the segment of record j: the last v with start(v) <= j
        int lo = 0, hi = rseg.V - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_start(rseg, mid) <= j) lo = mid; else hi = mid - 1;
        }
        const uint32_t e0 = seg_start(eseg, lo), e1 = seg_start(eseg, lo + 1);
        const uint32_t s = toffs[j], e = min(s + c, e1);
        if (s >= e) continue;
        const uint32_t bb = __ldg(eseg.bbase + lo);
        for (uint32_t k = (s - e0 + RS_CHUNK - 1) / RS_CHUNK; e0 + k * RS_CHUNK < e; ++k) first[bb + k] = j;
    }
}

// Walk the records overlapping entries [E0, E1) of the block, RS_THREADS at a
// time in order; f(e, key, slot) is called for every entry e in the range (e
// the entry's index, key its tile key, slot the record slot).  Every thread
// returns after the same number of barriers.
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
                                                             const uint32_t *nr_dev, const uint32_t *__restrict__ first,
                                                             int tiles_x, Segs g, uint32_t mask,
                                                             uint32_t *__restrict__ hist)
{
    const uint32_t b = blockIdx.x;
    if (b >= __ldg(g.bbase + g.V)) {
        hist[(size_t)RS_RADIX * b + threadIdx.x] = 0u;
        return;
    }
    __shared__ uint32_t h[RS_WARPS][RS_RADIX];
    const int w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&h[0][0])[d] = 0;
    __syncthreads();
    const SegBlock sb = seg_block(g, b);
    const uint32_t sub = (uint32_t)sb.v * g.sub;
    const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
    for_chunk_entries(bins, toffs, counts, nr, first[b], sb.s0, sb.s1, tiles_x,
                      [&](uint32_t, uint32_t key, uint32_t) { atomicAdd(&h[w][(key - sub) & mask], 1u); });
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) tot += h[ww][threadIdx.x];
    hist[(size_t)RS_RADIX * __ldg(g.bbase + sb.v) + (size_t)threadIdx.x * sb.nb + sb.bl] = tot;
}

// 6 resident blocks (40 registers, a few spilled words) beat 4 (57 registers) and 5:
// more warps hide the record walks' dependent loads (tile sort 0.63 -> 0.57 ms)
__global__ void __launch_bounds__(RS_THREADS, 6) k_rs_scatter_bins(const uint4 *__restrict__ bins,
                                                                const uint32_t *__restrict__ toffs,
                                                                const uint32_t *__restrict__ counts, uint32_t nr_cap,
                                                                const uint32_t *nr_dev,
                                                                const uint32_t *__restrict__ first, int tiles_x,
                                                                Segs g, uint32_t mask, const uint32_t *offsets,
                                                                uint32_t *kout, uint32_t *vout)
{
    const uint32_t b = blockIdx.x;
    if (b >= __ldg(g.bbase + g.V)) return;   // block-uniform
    __shared__ ScatterSmem sm;
    const SegBlock sb = seg_block(g, b);
    const uint32_t nr = nr_dev ? min(nr_cap, *nr_dev) : nr_cap;
    for (int d = threadIdx.x; d < RS_WARPS * RS_RADIX; d += RS_THREADS) (&sm.wh[0][0])[d] = 0;
    // the block's entries, in entry order, into shared memory
    for_chunk_entries(bins, toffs, counts, nr, first[b], sb.s0, sb.s1, tiles_x,
                      [&](uint32_t e, uint32_t key, uint32_t slot) {
                          sm.sk[e - sb.s0] = key;
                          sm.sv[e - sb.s0] = slot;
                      });
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nvalid = sb.s1 - sb.s0;
    uint32_t key[RS_ITEMS], val[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const uint32_t i = (uint32_t)w * (RS_ITEMS * 32) + (uint32_t)(k * 32 + lane);
        key[k] = i < nvalid ? sm.sk[i] : 0u;
        val[k] = i < nvalid ? sm.sv[i] : 0u;
    }
    __syncthreads();                         // sk / sv are reused for the reordered items
    rank_and_scatter(key, val, nvalid, 0, mask, (uint32_t)sb.v * g.sub,
                     offsets + (size_t)RS_RADIX * __ldg(g.bbase + sb.v) + sb.bl, sb.nb, kout, vout, sm);
}

// Segment starts after a pass that dropped items: segment v now starts at the
// scanned table's slot for (v, digit 0, block 0); the end (*total, the kept
// count) is start[V], which the table scan wrote.
__global__ void k_kept_starts(const uint32_t *__restrict__ table, const uint32_t *__restrict__ bbase, int V,
                              size_t bound, uint32_t *__restrict__ start)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        const uint32_t b = bbase[v];
        start[v] = (size_t)b < bound ? table[(size_t)RS_RADIX * b] : start[V];
    }
}

// Tile ranges of a single-pass tile sort, read off its scanned digit table:
// (view group v, tile t) starts at the table's slot for digit t of segment v
// and ends where digit t + 1 starts (the segment's end after the last tile).
__global__ void k_ranges_from_table(const uint32_t *__restrict__ table, Segs g, uint32_t tiles,
                                    uint2 *__restrict__ ranges)
{
    const size_t n = (size_t)g.V * tiles;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(k / tiles);
        const uint32_t t = (uint32_t)(k % tiles);
        const uint32_t b0 = __ldg(g.bbase + v), nb = __ldg(g.bbase + v + 1) - b0;
        uint32_t s0, s1;
        if (nb == 0) {
            s0 = s1 = seg_start(g, v);
        } else {
            s0 = table[(size_t)RS_RADIX * b0 + (size_t)t * nb];
            s1 = t + 1 < tiles ? table[(size_t)RS_RADIX * b0 + (size_t)(t + 1) * nb] : seg_start(g, v + 1);
        }
        ranges[k] = make_uint2(s0, s1);
    }
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

// The scatters' shared memory allows 8 blocks per SM at the full carveout.
static void sort_carveouts()
{
    static bool set = false;
    if (set) return;
    cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_rs_scatter_bins, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(k_rs_scatter_seg, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    set = true;
}

// Layout of a sort workspace for n items in V segments (V = 0: a plain sort).
struct SortWs {
    uint32_t *hist;       // digit table: RS_RADIX x (blocks of n + V)
    void *scan;           // its scan workspace
    uint32_t *first;      // entry blocks: the record holding each block's first entry
    uint32_t *rbase;      // [V + 1] first block of each record segment
    uint32_t *ebase;      // [V + 1] first block of each entry segment
    uint32_t *eseg;       // [V + 1] first entry of each segment
    void *vscan;          // scan workspace of the [V + 1] arrays
    size_t bytes;
};

static SortWs sort_ws(void *ws, size_t n, int V)
{
    const size_t bound = blocks_for(n > 0 ? n : 1, RS_CHUNK) + (size_t)V;
    char *base = (char *)ws, *p = base;
    SortWs w;
    w.hist = (uint32_t *)p; p += align_up((size_t)RS_RADIX * bound * sizeof(uint32_t));
    w.scan = p; p += align_up(scan_workspace_bytes((size_t)RS_RADIX * bound));
    w.first = (uint32_t *)p; p += align_up((bound + 1) * sizeof(uint32_t));
    w.rbase = (uint32_t *)p; p += align_up(((size_t)V + 1) * sizeof(uint32_t));
    w.ebase = (uint32_t *)p; p += align_up(((size_t)V + 1) * sizeof(uint32_t));
    w.eseg = (uint32_t *)p; p += align_up(((size_t)V + 1) * sizeof(uint32_t));
    w.vscan = p; p += align_up(scan_workspace_bytes((size_t)V + 1));
    w.bytes = (size_t)(p - base);
    return w;
}

size_t radix_workspace_bytes(size_t n, int V)
{
    return sort_ws(nullptr, n, V).bytes;
}

// bbase of the segments [start(v), start(v + 1)): block counts, then their exclusive scan.
static cudaError_t seg_bases(const uint32_t *start, uint32_t stride, int V, uint32_t *bbase, void *vscan, cudaStream_t st)
{
    k_seg_blocks<<<(unsigned)((V + 256) / 256), 256, 0, st>>>(start, stride, V, bbase);
    count_launch();
    return exclusive_scan_u32(bbase, bbase, (size_t)V + 1, nullptr, vscan, st);
}

// Segmented passes over digits [shift0, bits) of (k0, v0), ping-ponging with
// (k1, v1); *result_in_alt flips once per pass.
// With kept (device, [V + 1]), the first pass drops the items whose key is
// DROP_KEY, kept receives the compacted segment starts (kept[V] = the items
// left) and the later passes sort the compacted segments.
static cudaError_t seg_passes(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, Segs g, size_t bound,
                              int shift0, int bits, const SortWs &w, cudaStream_t st, bool *result_in_alt,
                              const char *prof, uint32_t *kept = nullptr)
{
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int shift = shift0; shift < bits; shift += 8) {
        const int wd = bits - shift < 8 ? bits - shift : 8;
        const uint32_t mask = (1u << wd) - 1u;
        const bool drop = kept && shift == shift0;
        ProfScope ps_(prof, st);
        k_rs_hist_seg<<<(unsigned)bound, RS_THREADS, 0, st>>>(ki, g, shift, mask, w.hist, drop);
        count_launch();
        cudaError_t e = exclusive_scan_u32(w.hist, w.hist, (size_t)RS_RADIX * bound, drop ? kept + g.V : nullptr,
                                           w.scan, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter_seg<<<(unsigned)bound, RS_THREADS, 0, st>>>(ki, vi, ko, vo, g, shift, mask, w.hist, drop);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (drop) {   // the compacted segments, and their blocks, for the later passes
            k_kept_starts<<<(unsigned)((g.V + 255) / 256), 256, 0, st>>>(w.hist, g.bbase, g.V, bound, kept);
            count_launch();
            e = seg_bases(kept, 1u, g.V, w.rbase, w.vscan, st);
            if (e != cudaSuccess) return e;
            g.start = kept;
            g.stride = 1u;
            g.bbase = w.rbase;
        }
        uint32_t *tk = ki, *tv = vi;
        ki = ko; vi = vo; ko = tk; vo = tv;
        *result_in_alt = !*result_in_alt;
    }
    return cudaSuccess;
}

// Plain passes over digits [shift0, bits) of (k0, v0); the result is in (k1,
// v1) when *result_in_alt.
cudaError_t radix_passes(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, size_t n, int shift0, int bits,
                         void *ws, cudaStream_t st, bool *result_in_alt, const uint32_t *n_dev, const char *prof)
{
    *result_in_alt = false;
    sort_carveouts();
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

cudaError_t radix_sort_pairs_seg(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, size_t n_cap,
                                 const uint32_t *seg_start, uint32_t stride, int V, int bits, void *ws,
                                 cudaStream_t st, bool *result_in_alt, const char *prof, uint32_t *kept)
{
    *result_in_alt = false;
    if (n_cap == 0 || V <= 0 || bits <= 0) return cudaSuccess;
    sort_carveouts();
    const SortWs w = sort_ws(ws, n_cap, V);
    const size_t bound = blocks_for(n_cap, RS_CHUNK) + (size_t)V;
    {
        ProfScope ps_(prof, st);
        cudaError_t e = seg_bases(seg_start, stride, V, w.rbase, w.vscan, st);
        if (e != cudaSuccess) return e;
    }
    const Segs g{seg_start, stride, w.rbase, V, 0u};
    return seg_passes(k0, v0, k1, v1, g, bound, 0, bits, w, st, result_in_alt, prof, kept);
}

cudaError_t radix_sort_entries(const uint4 *bins, const uint32_t *toffs, const uint32_t *counts, uint32_t n_rec,
                               const uint32_t *nrec_dev, const uint32_t *rec_start, uint32_t rec_stride, int V,
                               int tiles_x, uint32_t tiles, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                               size_t e_cap, const uint32_t *nent_dev, int bits, void *ws, cudaStream_t st,
                               bool *result_in_alt, int sms, uint2 *ranges, bool *ranges_done)
{
    *result_in_alt = false;
    if (ranges_done) *ranges_done = false;
    if (e_cap == 0 || n_rec == 0 || V <= 0) return cudaSuccess;
    if (bits < 1) bits = 1;                  // the first pass also materialises the entries
    sort_carveouts();
    const SortWs w = sort_ws(ws, e_cap, V);
    const size_t bound = blocks_for(e_cap, RS_CHUNK) + (size_t)V;
    const Segs rseg{rec_start, rec_stride, nullptr, V, 0u};
    const Segs eg{w.eseg, 1u, w.ebase, V, tiles};
    {
        const int wd = bits < 8 ? bits : 8;
        const uint32_t mask = (1u << wd) - 1u;
        ProfScope ps_("radix_tile", st);
        k_entry_segs<<<(unsigned)((V + 256) / 256), 256, 0, st>>>(rseg, toffs, n_rec, nrec_dev, (uint32_t)e_cap,
                                                                   nent_dev, w.eseg);
        count_launch();
        cudaError_t e = seg_bases(w.eseg, 1u, V, w.ebase, w.vscan, st);
        if (e != cudaSuccess) return e;
        unsigned g = (unsigned)((n_rec + 255) / 256);
        if (g > (unsigned)sms * 16u) g = (unsigned)sms * 16u;
        k_chunk_first_seg<<<g, 256, 0, st>>>(toffs, counts, n_rec, nrec_dev, rseg, eg, w.first);
        count_launch();
        k_rs_hist_bins<<<(unsigned)bound, RS_THREADS, 0, st>>>(bins, toffs, counts, n_rec, nrec_dev, w.first, tiles_x,
                                                               eg, mask, w.hist);
        count_launch();
        e = exclusive_scan_u32(w.hist, w.hist, (size_t)RS_RADIX * bound, nullptr, w.scan, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter_bins<<<(unsigned)bound, RS_THREADS, 0, st>>>(bins, toffs, counts, n_rec, nrec_dev, w.first,
                                                                  tiles_x, eg, mask, w.hist, k1, v1);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (bits <= 8) {
        *result_in_alt = true;
        if (ranges && ranges_done) {
            ProfScope ps_("ranges", st);
            const size_t n = (size_t)V * tiles;
            unsigned g = (unsigned)((n + 255) / 256);
            if (g > (unsigned)sms * 16u) g = (unsigned)sms * 16u;
            k_ranges_from_table<<<g, 256, 0, st>>>(w.hist, eg, tiles, ranges);
            count_launch();
            *ranges_done = true;
        }
        return cudaGetLastError();
    }
    // the remaining tile digits: segmented passes from (k1, v1), ending in (k0, v0) after an odd count
    bool alt2 = false;
    cudaError_t e = seg_passes(k1, v1, k0, v0, eg, bound, 8, bits, w, st, &alt2, "radix_tile");
    *result_in_alt = !alt2;
    return e;
}

}  // namespace dgs
