// C ABI entry points, the per-call planner (view groups of a state batch) and
// the context's device workspace.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <initializer_list>
#include <utility>
#include <vector>

#include "dgs_internal.cuh"
#include "kernels.cuh"

namespace dgs {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Library-wide launch profiler: CUDA events recorded on the launching stream
// around each named launch while enabled; read (and cleared) by dgs_profile_read.
namespace {
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
bool g_prof = false;
std::vector<ProfRec> g_prof_recs;
std::vector<size_t> g_prof_stack;
std::vector<cudaEvent_t> g_event_pool;
size_t g_event_next = 0;

cudaEvent_t next_event()
{
    if (g_event_next == g_event_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_event_pool.push_back(e);
    }
    return g_event_pool[g_event_next++];
}
}  // namespace

void prof_begin(const char *name, cudaStream_t st)
{
    if (!g_prof) return;
    ProfRec r{name, next_event(), next_event()};
    if (r.a) cudaEventRecord(r.a, st);
    g_prof_stack.push_back(g_prof_recs.size());
    g_prof_recs.push_back(r);
}

void prof_end(cudaStream_t st)
{
    if (!g_prof || g_prof_stack.empty()) return;
    const size_t k = g_prof_stack.back();
    g_prof_stack.pop_back();
    if (g_prof_recs[k].b) cudaEventRecord(g_prof_recs[k].b, st);
}
}  // namespace dgs

using namespace dgs;

namespace {

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    bool zeroed = false;   // (record gradients) every byte is zero between uses
};

struct Plan {
    int S = 0;           // states rendered (including appended reference states)
    int S_user = 0;      // caller's states
    int V = 0;
    int W = 0, H = 0, tiles_x = 0, tiles_y = 0;
    uint32_t tiles = 0;
    int tile_shift = 4;                  // sort tiles of 2^tile_shift pixels
    int blocks_x = 0, blocks_y = 0;      // 16 x 16 pixel blocks (squared-error partials)
    uint32_t blocks = 0;
    TileGeom geom() const
    {
        TileGeom g;
        g.tiles_x = tiles_x; g.tiles_y = tiles_y; g.tile_shift = tile_shift;
        g.blocks_x = blocks_x; g.blocks_y = blocks_y; g.tiles = tiles; g.blocks = blocks;
        return g;
    }
    std::vector<int32_t> vg_of_state;
    std::vector<ViewGroup> vgs;
};

// Outputs of the shared preparation of a batch (pointers into the workspace).
struct Lists {
    uint32_t nRec = 0, nEnt = 0;
    uint32_t nLive = 0;                                       // records left by the depth sort (context calls)
    uint32_t *depth_keys = nullptr, *depth_slots = nullptr;   // records sorted by depth
    uint32_t *ekeys = nullptr, *evals = nullptr;              // entries sorted by (view group, tile)
    uint32_t *tile_order = nullptr;                           // (view group, tile), costliest first
};

struct Tape {
    bool valid = false;
    dgs_scene scene{};
    const uint32_t *masks = nullptr;
    std::vector<float> t;
    std::vector<int32_t> cam;
    std::vector<dgs_camera> cams;
    Plan plan;
    Lists lists;
};

}  // namespace

struct dgs_ctx {
    int device = 0;
    int sms = 148;
    std::string err;
    Buf vgs, vgos, depth, need, counts, recBase, total, recs, k0, v0, k1, v1, tcount, toffs, bins, ek0, ev0, ek1, ev1,
        ranges, sortws, scanws, partial, refs, recgrad, refidx, tck0, tcv0, tck1, tcv1, icnt, ioff, qint, counter,
        pairm, grp, gmse, omaps, opart, otpart, oD, oweight, oints, recgmu, gqws,
        shord, shpair, shpair2, shrep, shflag, shpos, shlist, shitem, shkey, shstop, shseg, shcnt, shtab,
        tapemask,                  // the masks the last forward rendered (checked by the backward)
        live,                      // [V + 1] view-group starts of the depth-sorted live records; [V] = their count
        jobargs;                   // multi-scene calls: per-scene raster arguments, queues and item offsets
    bool tile_reuse = true;        // utility passes reuse rendered tiles across states (share.cu)
    int tile_size = 0;             // sort tile side in pixels: 16 or 32, or 0 (chosen per batch shape)
    size_t mem_budget = 0;         // cap on the workspace bytes (0: the device's free memory only)
    size_t ws_bytes = 0;           // workspace bytes held now
    long long chunk_splits = 0;    // batches split because their workspace did not fit
    int active_shift = 4;          // tile shift of the call in progress when tile_size is 0
    int last_shift = 0;            // tile shift of the last prepared batch (0: none yet)
    std::map<std::vector<long long>, int> tuned_tile;   // autotuner: call shape -> tile shift
    long long reuse_pairs = 0, reuse_rendered = 0;   // last distortion pass: (state, tile) pairs, rendered
    int reuse_rounds = 0;
    std::map<std::vector<long long>, int> tuned_G;   // autotuner: call shape -> states per block
    std::vector<dgs_ctx *> kids;   // multi-scene calls: one workspace per scene of the batch
    void *h_stage = nullptr;
    size_t h_stage_cap = 0;
    uint32_t *h_small = nullptr;   // pinned readback of counts
    cudaEvent_t stage_done = nullptr;   // last copy out of h_stage
    long long launch_base = 0;
    Tape tape;
};

namespace {

int fail(dgs_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

#define CK(x)                                                                                       \
    do {                                                                                            \
        cudaError_t e_ = (x);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, DGS_E_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

#define TRY(x)                     \
    do {                           \
        int r_ = (x);              \
        if (r_ != DGS_OK) return r_; \
    } while (0)

int ensure(dgs_ctx *ctx, Buf &b, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) bytes = 256;
    if (b.cap >= bytes) return DGS_OK;
    size_t want = bytes + bytes / 8;
    if (ctx->mem_budget && ctx->ws_bytes - b.cap + want > ctx->mem_budget) {
        want = bytes;
        if (ctx->ws_bytes - b.cap + want > ctx->mem_budget)
            return fail(ctx, DGS_E_OOM, "workspace of %zu bytes would exceed the budget of %zu", ctx->ws_bytes -
                        b.cap + want, ctx->mem_budget);
    }
    if (b.p) {
        CK(cudaStreamSynchronize(st));
        CK(cudaFree(b.p));
        ctx->ws_bytes -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DGS_E_OOM, "device allocation of %zu bytes failed", want);
    }
    b.cap = want;
    b.zeroed = false;
    ctx->ws_bytes += want;
    return DGS_OK;
}

// The per-record gradient buffer stays zero between backward calls: it is
// cleared once when allocated, the adjoint raster accumulates into it, and the
// projection adjoint clears every record it reads.  `zeroed` is false while a
// backward is between those two kernels (or after a failure there).
int ensure_zeroed(dgs_ctx *ctx, Buf &b, size_t bytes, cudaStream_t st)
{
    TRY(ensure(ctx, b, bytes, st));
    if (!b.zeroed) {
        CK(cudaMemsetAsync(b.p, 0, b.cap, st));
        b.zeroed = true;
    }
    return DGS_OK;
}

// A view of states [s0, s0 + n) of a batch.
dgs_states sub_states(const dgs_states *st, int s0, int n, int words)
{
    dgs_states r;
    r.masks = st->masks + (size_t)s0 * words;
    r.t = st->t + s0;
    r.cam = st->cam + s0;
    r.n_states = n;
    return r;
}

// Memory-budget batching: run call(sub-batch, first state) on the whole batch
// and, when the workspace would not fit (DGS_E_OOM), on its two halves,
// recursively.  Every state renders the same bits in any batch, so the
// outputs do not depend on the split; calls fail before writing any output
// when a workspace allocation fails.
void release_workspace(dgs_ctx *ctx, cudaStream_t st, std::initializer_list<Buf *> keep);

// keep: workspace buffers the call reads or writes across parts (never released)
template <class F>
int chunked(dgs_ctx *ctx, const dgs_states *st, int words, int s0, cudaStream_t stream, F call,
            std::initializer_list<Buf *> keep = {})
{
    const int r = call(st, s0);
    if (r != DGS_E_OOM || st->n_states <= 1) return r;
    ++ctx->chunk_splits;
    release_workspace(ctx, stream, keep);   // buffers the failed attempt grew would crowd out the parts
    const int h = st->n_states / 2;
    const dgs_states a = sub_states(st, 0, h, words), b = sub_states(st, h, st->n_states - h, words);
    TRY(chunked(ctx, &a, words, s0, stream, call, keep));
    return chunked(ctx, &b, words, s0 + h, stream, call, keep);
}

int ensure_stage(dgs_ctx *ctx, size_t bytes, cudaStream_t st)
{
    if (ctx->h_stage_cap >= bytes) return DGS_OK;
    if (ctx->h_stage) {
        CK(cudaEventSynchronize(ctx->stage_done));
        CK(cudaFreeHost(ctx->h_stage));
        ctx->h_stage = nullptr;
    }
    size_t want = bytes + bytes / 4 + 4096;
    CK(cudaMallocHost(&ctx->h_stage, want));
    ctx->h_stage_cap = want;
    return DGS_OK;
}

int check_scene(dgs_ctx *ctx, const dgs_scene *s)
{
    if (!s) return fail(ctx, DGS_E_INVALID_ARG, "scene is null");
    if (s->n < 0 || s->n_clusters < 1 || s->n_layers < 1)
        return fail(ctx, DGS_E_INVALID_ARG, "bad scene sizes n=%d C=%d L=%d", s->n, s->n_clusters, s->n_layers);
    if (s->n_clusters > MAX_CLUSTERS) return fail(ctx, DGS_E_UNSUPPORTED, "more than %d clusters", MAX_CLUSTERS);
    if (s->n_layers > MAX_LAYERS) return fail(ctx, DGS_E_UNSUPPORTED, "more than %d layers", MAX_LAYERS);
    if (s->sh_degree != 0 && s->sh_degree != 3) return fail(ctx, DGS_E_UNSUPPORTED, "sh_degree must be 0 or 3");
    if (s->temporal_rank < 0 || s->temporal_rank > 8)
        return fail(ctx, DGS_E_UNSUPPORTED, "temporal_rank must be in [0, 8]");
    if (s->n > 0) {
        if (!s->cluster_offsets || !s->mu0 || !s->log_scale || !s->quat || !s->opacity_logit || !s->colour)
            return fail(ctx, DGS_E_INVALID_ARG, "scene array is null");
        if (s->temporal_rank > 0 && !s->u) return fail(ctx, DGS_E_INVALID_ARG, "u is null");
        if (s->n_layers > 1 && s->res_mode != 1 && !s->res) return fail(ctx, DGS_E_INVALID_ARG, "res is null");
        if (s->n_layers > 1 && s->res_mode == 1 && !s->res_q) return fail(ctx, DGS_E_INVALID_ARG, "res_q is null");
        if (s->n_layers > 1 && s->res_mode != 0 && !s->res_step)
            return fail(ctx, DGS_E_INVALID_ARG, "res_step is null");
        if (((uintptr_t)s->quat & 15u) != 0) return fail(ctx, DGS_E_INVALID_ARG, "quat must be 16-byte aligned");
    }
    if (s->affine && s->affine_T < 1) return fail(ctx, DGS_E_INVALID_ARG, "affine_T must be >= 1");
    if (s->res_mode < 0 || s->res_mode > 2) return fail(ctx, DGS_E_INVALID_ARG, "res_mode must be 0, 1 or 2");
    return DGS_OK;
}

SceneDev scene_dev(const dgs_scene *s)
{
    SceneDev d;
    d.n = s->n; d.C = s->n_clusters; d.L = s->n_layers; d.sh = s->sh_degree; d.R = s->temporal_rank;
    d.nc = 3 * (s->sh_degree + 1) * (s->sh_degree + 1);
    d.K = 11 + d.nc;
    d.offs = s->cluster_offsets; d.mu0 = s->mu0; d.u = s->u; d.ls = s->log_scale; d.quat = s->quat;
    d.logit = s->opacity_logit; d.colour = s->colour; d.res = s->res;
    d.affine = s->affine; d.aT = s->affine ? s->affine_T : 0;
    d.res_q = s->res_q; d.res_step = s->res_step; d.res_mode = s->res_mode;
    return d;
}

int build_plan(dgs_ctx *ctx, const dgs_states *st, const dgs_camera *cams, int n_cams, bool add_refs, Plan &p)
{
    if (!st) return fail(ctx, DGS_E_INVALID_ARG, "states is null");
    if (st->n_states < 0) return fail(ctx, DGS_E_INVALID_ARG, "n_states < 0");
    if (!cams || n_cams < 1) return fail(ctx, DGS_E_INVALID_ARG, "need at least one camera");
    if (st->n_states > 0 && (!st->masks || !st->t || !st->cam))
        return fail(ctx, DGS_E_INVALID_ARG, "states arrays are null");
    const int W = cams[0].width, H = cams[0].height;
    if (W < 1 || H < 1 || W > 32768 || H > 32768) return fail(ctx, DGS_E_INVALID_ARG, "bad image size %dx%d", W, H);
    for (int k = 0; k < n_cams; ++k) {
        if (cams[k].width != W || cams[k].height != H)
            return fail(ctx, DGS_E_INVALID_ARG, "all cameras of a batch must share one image size");
        if (!(cams[k].fx > 0.0f) || !(cams[k].fy > 0.0f)) return fail(ctx, DGS_E_INVALID_ARG, "focal must be > 0");
    }
    p = Plan();
    p.S_user = st->n_states;
    p.W = W; p.H = H;
    p.tile_shift = ctx->tile_size == 32 ? 5 : ctx->tile_size == 16 ? 4 : ctx->active_shift;
    ctx->last_shift = p.tile_shift;
    const int T = 1 << p.tile_shift;
    p.tiles_x = (W + T - 1) / T;
    p.tiles_y = (H + T - 1) / T;
    p.tiles = (uint32_t)p.tiles_x * (uint32_t)p.tiles_y;
    p.blocks_x = (W + BLOCK - 1) / BLOCK;
    p.blocks_y = (H + BLOCK - 1) / BLOCK;
    p.blocks = (uint32_t)p.blocks_x * (uint32_t)p.blocks_y;
    std::map<std::pair<int, uint32_t>, int> groups;
    p.vg_of_state.resize(st->n_states);
    for (int s = 0; s < st->n_states; ++s) {
        const int c = st->cam[s];
        if (c < 0 || c >= n_cams) return fail(ctx, DGS_E_INVALID_ARG, "state %d: camera index %d out of range", s, c);
        uint32_t tb;
        std::memcpy(&tb, &st->t[s], 4);
        auto key = std::make_pair(c, tb);
        auto it = groups.find(key);
        int v;
        if (it == groups.end()) {
            v = (int)p.vgs.size();
            groups.emplace(key, v);
            ViewGroup g;
            const dgs_camera &cm = cams[c];
            for (int k = 0; k < 9; ++k) g.R[k] = cm.R_wc[k];
            for (int k = 0; k < 3; ++k) g.t[k] = cm.t_wc[k];
            g.fx = cm.fx; g.fy = cm.fy; g.cx = cm.cx; g.cy = cm.cy;
            g.time = st->t[s];
            for (int k = 0; k < 3; ++k)   // camera centre = -R^T t
                g.campos[k] = -(cm.R_wc[k] * cm.t_wc[0] + cm.R_wc[3 + k] * cm.t_wc[1] + cm.R_wc[6 + k] * cm.t_wc[2]);
            g.width = W; g.height = H; g.cam = c; g.pad = 0;
            p.vgs.push_back(g);
        } else {
            v = it->second;
        }
        p.vg_of_state[s] = v;
    }
    p.V = (int)p.vgs.size();
    if (p.V > 32767) return fail(ctx, DGS_E_UNSUPPORTED, "more than 32767 distinct (camera, time) pairs");
    if ((unsigned long long)(st->n_states + (add_refs ? p.V : 0)) * p.blocks * 8ull >= 0x7fffffffull)
        return fail(ctx, DGS_E_CAPACITY, "states x tiles exceeds the launch grid");
    if ((unsigned long long)p.V * p.tiles >= 0xffffffffull)
        return fail(ctx, DGS_E_CAPACITY, "view groups x tiles exceeds 32 bits");
    p.S = p.S_user;
    if (add_refs) {
        for (int v = 0; v < p.V; ++v) p.vg_of_state.push_back(v);
        p.S += p.V;
    }
    return DGS_OK;
}

int bits_for(unsigned long long maxval)
{
    int b = 1;
    while (b < 32 && (maxval >> b) != 0) ++b;
    return b;
}

// Closure, layout, projection, depth sort, binning, tile sort, ranges.
int prepare(dgs_ctx *ctx, const dgs_scene *scene, const uint32_t *masks, const Plan &p, bool force_full,
            cudaStream_t st, Lists &out)
{
    uint32_t nRec = 0, nEnt = 0;
    const int C = scene->n_clusters, L = scene->n_layers;
    const int words = (C * L + 31) / 32;
    const size_t nvc = (size_t)p.V * C;
    TRY(ensure(ctx, ctx->vgs, sizeof(ViewGroup) * (size_t)(p.V > 0 ? p.V : 1), st));
    TRY(ensure(ctx, ctx->vgos, sizeof(int32_t) * (size_t)(p.S > 0 ? p.S : 1), st));
    TRY(ensure(ctx, ctx->depth, (size_t)p.S * C, st));
    TRY(ensure(ctx, ctx->need, sizeof(uint32_t) * nvc, st));
    TRY(ensure(ctx, ctx->counts, sizeof(uint32_t) * (nvc + 1), st));
    TRY(ensure(ctx, ctx->recBase, sizeof(uint32_t) * (nvc + 1), st));
    TRY(ensure(ctx, ctx->total, 64, st));
    TRY(ensure(ctx, ctx->scanws, scan_workspace_bytes(nvc + 1), st));
    const size_t stage = sizeof(ViewGroup) * p.vgs.size() + sizeof(int32_t) * p.vg_of_state.size() + 64;
    TRY(ensure_stage(ctx, stage, st));
    CK(cudaEventSynchronize(ctx->stage_done));   // an earlier copy may still read h_stage
    char *hs = (char *)ctx->h_stage;
    std::memcpy(hs, p.vgs.data(), sizeof(ViewGroup) * p.vgs.size());
    std::memcpy(hs + sizeof(ViewGroup) * p.vgs.size(), p.vg_of_state.data(), sizeof(int32_t) * p.vg_of_state.size());
    CK(cudaMemcpyAsync(ctx->vgs.p, hs, sizeof(ViewGroup) * p.vgs.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->vgos.p, hs + sizeof(ViewGroup) * p.vgs.size(), sizeof(int32_t) * p.vg_of_state.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->stage_done, st));
    CK(cudaMemsetAsync(ctx->need.p, 0, sizeof(uint32_t) * nvc, st));
    uint8_t *depth = (uint8_t *)ctx->depth.p;
    if (p.S_user > 0)
        launch_closure(masks, p.S_user, words, C, L, (const int32_t *)ctx->vgos.p, depth, (uint32_t *)ctx->need.p,
                       force_full ? 1 : 0, ctx->sms, st);
    if (p.S > p.S_user) CK(cudaMemsetAsync(depth + (size_t)p.S_user * C, L, (size_t)(p.S - p.S_user) * C, st));
    launch_layout_counts((const uint32_t *)ctx->need.p, scene->cluster_offsets, p.V, C, (uint32_t *)ctx->counts.p,
                         ctx->sms, st);
    CK(exclusive_scan_u32((const uint32_t *)ctx->counts.p, (uint32_t *)ctx->recBase.p, nvc + 1,
                          (uint32_t *)ctx->total.p, ctx->scanws.p, st));
    CK(cudaMemcpyAsync(ctx->h_small, ctx->total.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    int32_t *hoffs = (int32_t *)(ctx->h_small + 16);
    CK(cudaMemcpyAsync(hoffs, scene->cluster_offsets, sizeof(int32_t) * (size_t)(C + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hoffs[0] != 0 || hoffs[C] != scene->n)
        return fail(ctx, DGS_E_INVALID_ARG, "cluster_offsets must start at 0 and end at n");
    for (int c = 0; c < C; ++c)
        if (hoffs[c + 1] < hoffs[c]) return fail(ctx, DGS_E_INVALID_ARG, "cluster_offsets must be non-decreasing");
    nRec = ctx->h_small[0];
    if (nRec >= 0x7fffffffu) return fail(ctx, DGS_E_CAPACITY, "too many projected records");
    TRY(ensure(ctx, ctx->recs, sizeof(Rec) * (size_t)nRec, st));
    TRY(ensure(ctx, ctx->k0, 4 * (size_t)nRec, st));
    TRY(ensure(ctx, ctx->v0, 4 * (size_t)nRec, st));
    TRY(ensure(ctx, ctx->k1, 4 * (size_t)nRec, st));
    TRY(ensure(ctx, ctx->v1, 4 * (size_t)nRec, st));
    TRY(ensure(ctx, ctx->tcount, 4 * ((size_t)nRec + 1), st));
    TRY(ensure(ctx, ctx->bins, sizeof(uint4) * ((size_t)nRec + 1), st));
    TRY(ensure(ctx, ctx->toffs, 4 * ((size_t)nRec + 1), st));
    TRY(ensure(ctx, ctx->sortws, radix_workspace_bytes(nRec, p.V), st));
    TRY(ensure(ctx, ctx->scanws, scan_workspace_bytes((size_t)nRec + 1), st));
    SceneDev sd = scene_dev(scene);
    if (nRec > 0)
        launch_project(sd, (const ViewGroup *)ctx->vgs.p, p.V, (const uint32_t *)ctx->need.p,
                       (const uint32_t *)ctx->recBase.p, (Rec *)ctx->recs.p, (uint32_t *)ctx->k0.p,
                       (uint32_t *)ctx->v0.p, ctx->sms, st);
    bool alt = false;
    // live records in (view group, depth) order: each view group's records are one
    // segment; culled records (key 0xFFFFFFFF) are dropped by the first pass
    TRY(ensure(ctx, ctx->live, 4 * ((size_t)p.V + 1), st));
    uint32_t *live = (uint32_t *)ctx->live.p;
    CK(radix_sort_pairs_seg((uint32_t *)ctx->k0.p, (uint32_t *)ctx->v0.p, (uint32_t *)ctx->k1.p,
                            (uint32_t *)ctx->v1.p, nRec, (const uint32_t *)ctx->recBase.p, (uint32_t)C, p.V, 32,
                            ctx->sortws.p, st, &alt, "radix_depth", live));
    const uint32_t *order = alt ? (const uint32_t *)ctx->v1.p : (const uint32_t *)ctx->v0.p;
    out.depth_keys = alt ? (uint32_t *)ctx->k1.p : (uint32_t *)ctx->k0.p;
    out.depth_slots = (uint32_t *)order;
    if (nRec > 0)
        launch_tile_count((const Rec *)ctx->recs.p, order, nRec, p.tiles_x, p.tiles, p.tile_shift,
                          (uint32_t *)ctx->tcount.p, (uint4 *)ctx->bins.p, ctx->sms, st, live + p.V);
    CK(exclusive_scan_u32((const uint32_t *)ctx->tcount.p, (uint32_t *)ctx->toffs.p, nRec,
                          (uint32_t *)ctx->total.p + 1, ctx->scanws.p, st));
    CK(cudaMemcpyAsync(ctx->h_small + 1, (uint32_t *)ctx->total.p + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    if (nRec > 0 && p.V > 0)
        CK(cudaMemcpyAsync(ctx->h_small + 2, live + p.V, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    nEnt = nRec > 0 ? ctx->h_small[1] : 0;
    out.nLive = nRec > 0 && p.V > 0 ? ctx->h_small[2] : 0;
    if (nEnt >= 0x7fffffffu) return fail(ctx, DGS_E_CAPACITY, "too many tile entries");
    TRY(ensure(ctx, ctx->ek0, 4 * (size_t)nEnt, st));
    TRY(ensure(ctx, ctx->ev0, 4 * (size_t)nEnt, st));
    TRY(ensure(ctx, ctx->ek1, 4 * (size_t)nEnt, st));
    TRY(ensure(ctx, ctx->ev1, 4 * (size_t)nEnt, st));
    TRY(ensure(ctx, ctx->sortws, radix_workspace_bytes(nEnt, p.V), st));
    TRY(ensure(ctx, ctx->ranges, sizeof(uint2) * (size_t)p.V * p.tiles, st));
    const int tbits = bits_for((unsigned long long)p.tiles - 1ull);
    bool ranges_done = false;
    CK(radix_sort_entries((const uint4 *)ctx->bins.p, (const uint32_t *)ctx->toffs.p, (const uint32_t *)ctx->tcount.p,
                          nRec, live + p.V, live, 1u, p.V, p.tiles_x, p.tiles,
                          (uint32_t *)ctx->ek0.p, (uint32_t *)ctx->ev0.p, (uint32_t *)ctx->ek1.p,
                          (uint32_t *)ctx->ev1.p, nEnt, nullptr, tbits, ctx->sortws.p, st, &alt, ctx->sms,
                          (uint2 *)ctx->ranges.p, &ranges_done));
    uint32_t *ekeys = alt ? (uint32_t *)ctx->ek1.p : (uint32_t *)ctx->ek0.p;
    out.ekeys = ekeys;
    out.evals = alt ? (uint32_t *)ctx->ev1.p : (uint32_t *)ctx->ev0.p;
    out.nRec = nRec;
    out.nEnt = nEnt;
    if (!ranges_done) {
        CK(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * (size_t)p.V * p.tiles, st));
        launch_ranges(ekeys, nEnt, (uint2 *)ctx->ranges.p, ctx->sms, st);
    }
    // (view group, tile) pairs in descending entry count: the raster work order
    const size_t vt = (size_t)p.V * p.tiles;
    TRY(ensure(ctx, ctx->tck0, 4 * vt, st));
    TRY(ensure(ctx, ctx->tcv0, 4 * vt, st));
    TRY(ensure(ctx, ctx->tck1, 4 * vt, st));
    TRY(ensure(ctx, ctx->tcv1, 4 * vt, st));
    TRY(ensure(ctx, ctx->sortws, radix_workspace_bytes(vt), st));
    launch_tile_costs((const uint2 *)ctx->ranges.p, (uint32_t)vt, (uint32_t *)ctx->tck0.p, (uint32_t *)ctx->tcv0.p,
                      ctx->sms, st);
    CK(radix_sort_pairs((uint32_t *)ctx->tck0.p, (uint32_t *)ctx->tcv0.p, (uint32_t *)ctx->tck1.p,
                        (uint32_t *)ctx->tcv1.p, vt, 16, ctx->sortws.p, st, &alt, nullptr, "radix_cost"));
    out.tile_order = alt ? (uint32_t *)ctx->tcv1.p : (uint32_t *)ctx->tcv0.p;
    CK(cudaGetLastError());
    return DGS_OK;
}

RasterArgs raster_args(dgs_ctx *ctx, const Plan &p, int C, const float *bg, uint32_t *sorted_evals)
{
    RasterArgs a;
    a.recs = (const Rec *)ctx->recs.p;
    a.evals = sorted_evals;
    a.ranges = (const uint2 *)ctx->ranges.p;
    a.depth = (const uint8_t *)ctx->depth.p;
    a.vg_of_state = (const int32_t *)ctx->vgos.p;
    a.S = p.S_user; a.C = C; a.W = p.W; a.H = p.H; a.tiles_x = p.tiles_x; a.tiles = p.tiles;
    a.tile_shift = p.tile_shift; a.blocks_x = p.blocks_x; a.blocks = p.blocks;
    a.bg0 = bg[0]; a.bg1 = bg[1]; a.bg2 = bg[2];
    a.images = nullptr; a.refs = nullptr; a.ref_of_state = nullptr; a.partial = nullptr;
    a.img_s0 = 0;
    a.stop = nullptr;
    a.dL = nullptr; a.gscale = 0.0f;
    return a;
}

bool same_call(const Tape &tp, const dgs_scene *sc, const dgs_states *st, const dgs_camera *cams, int n_cams)
{
    if (!tp.valid) return false;
    const dgs_scene &a = tp.scene;
    if (a.n != sc->n || a.n_clusters != sc->n_clusters || a.n_layers != sc->n_layers ||
        a.sh_degree != sc->sh_degree || a.temporal_rank != sc->temporal_rank ||
        a.cluster_offsets != sc->cluster_offsets || a.mu0 != sc->mu0 || a.u != sc->u ||
        a.log_scale != sc->log_scale || a.quat != sc->quat || a.opacity_logit != sc->opacity_logit ||
        a.colour != sc->colour || a.res != sc->res)
        return false;
    if (tp.masks != st->masks || (int)tp.t.size() != st->n_states || (int)tp.cams.size() != n_cams) return false;
    if (st->n_states > 0 && (std::memcmp(tp.t.data(), st->t, 4 * (size_t)st->n_states) != 0 ||
                             std::memcmp(tp.cam.data(), st->cam, 4 * (size_t)st->n_states) != 0))
        return false;
    return std::memcmp(tp.cams.data(), cams, sizeof(dgs_camera) * (size_t)n_cams) == 0;
}

void record_tape(Tape &tp, const dgs_scene *sc, const dgs_states *st, const dgs_camera *cams, int n_cams,
                 const Plan &p, const Lists &L)
{
    tp.valid = true;
    tp.scene = *sc;
    tp.masks = st->masks;
    tp.t.assign(st->t, st->t + st->n_states);
    tp.cam.assign(st->cam, st->cam + st->n_states);
    tp.cams.assign(cams, cams + n_cams);
    tp.plan = p;
    tp.lists = L;
}

// Device-resident state-group tables of one forward pass (states grouped by
// view group in groups of at most G).
struct QueueTabs {
    const int32_t *order = nullptr, *gfirst = nullptr, *gcount = nullptr, *gbase = nullptr, *ngroups = nullptr;
    size_t ng = 0;
    int G = 1;
};

void build_groups(const Plan &p, int s0, int s1, int G, std::vector<int32_t> &buf, size_t off[5], size_t &ng)
{
    std::vector<std::vector<int32_t>> per_vg(p.V);
    for (int s = s0; s < s1; ++s) per_vg[p.vg_of_state[s]].push_back(s);
    std::vector<int32_t> order, gfirst, gcount, gbase(p.V), ngroups(p.V);
    for (int v = 0; v < p.V; ++v) {
        gbase[v] = (int32_t)gfirst.size();
        for (size_t k = 0; k < per_vg[v].size(); k += G) {
            gfirst.push_back((int32_t)order.size() + (int32_t)k);
            gcount.push_back((int32_t)std::min<size_t>(G, per_vg[v].size() - k));
        }
        ngroups[v] = (int32_t)gfirst.size() - gbase[v];
        order.insert(order.end(), per_vg[v].begin(), per_vg[v].end());
    }
    ng = gfirst.size();
    buf.clear();
    off[0] = buf.size(); buf.insert(buf.end(), order.begin(), order.end());
    off[1] = buf.size(); buf.insert(buf.end(), gfirst.begin(), gfirst.end());
    off[2] = buf.size(); buf.insert(buf.end(), gcount.begin(), gcount.end());
    off[3] = buf.size(); buf.insert(buf.end(), gbase.begin(), gbase.end());
    off[4] = buf.size(); buf.insert(buf.end(), ngroups.begin(), ngroups.end());
}

QueueTabs tabs_at(const int32_t *dev, const size_t off[5], size_t ng, int G)
{
    QueueTabs q;
    q.order = dev + off[0]; q.gfirst = dev + off[1]; q.gcount = dev + off[2]; q.gbase = dev + off[3];
    q.ngroups = dev + off[4]; q.ng = ng; q.G = G;
    return q;
}

// Launch the persistent forward raster for uploaded group tables: per-call
// item offsets from the cost-ordered tile list, counter reset, kernel.
int make_queue(dgs_ctx *ctx, const Plan &p, const Lists &L, const QueueTabs &qt, cudaStream_t st, WorkQueue &q)
{
    const size_t vt = (size_t)p.V * p.tiles;
    TRY(ensure(ctx, ctx->icnt, 4 * (vt + 1), st));
    TRY(ensure(ctx, ctx->ioff, 4 * (vt + 1), st));
    TRY(ensure(ctx, ctx->counter, 16, st));
    TRY(ensure(ctx, ctx->scanws, scan_workspace_bytes(vt + 1), st));
    launch_item_counts(L.tile_order, (uint32_t)vt, p.tiles, qt.ngroups, (uint32_t *)ctx->icnt.p, ctx->sms, st);
    CK(exclusive_scan_u32((const uint32_t *)ctx->icnt.p, (uint32_t *)ctx->ioff.p, vt, nullptr, ctx->scanws.p, st));
    CK(cudaMemsetAsync(ctx->counter.p, 0, 4, st));
    q = WorkQueue();
    q.tile_order = L.tile_order;
    q.item_offsets = (const uint32_t *)ctx->ioff.p;
    q.n_vt = (uint32_t)vt;
    q.n_items = (uint32_t)(qt.ng * p.tiles);
    q.group_first = qt.gfirst;
    q.group_count = qt.gcount;
    q.vg_group_base = qt.gbase;
    q.state_order = qt.order;
    q.counter = (uint32_t *)ctx->counter.p;
    return DGS_OK;
}

int launch_queue(dgs_ctx *ctx, const Plan &p, const Lists &L, const RasterArgs &a, const QueueTabs &qt,
                 cudaStream_t st)
{
    WorkQueue q;
    TRY(make_queue(ctx, p, L, qt, st, q));
    launch_raster_fwd(a, q, qt.G, ctx->sms, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

// Forward raster of states [s0, s1) of the plan: group them by view group in
// groups of at most G, upload the tables through the pinned staging buffer and
// launch the persistent kernel.
int launch_fwd_pass(dgs_ctx *ctx, const Plan &p, const Lists &L, const RasterArgs &a, int s0, int s1, int G,
                    cudaStream_t st)
{
    if (s1 - s0 <= 0) return DGS_OK;
    std::vector<int32_t> buf;
    size_t off[5], ng = 0;
    build_groups(p, s0, s1, G, buf, off, ng);
    TRY(ensure(ctx, ctx->qint, 4 * buf.size(), st));
    TRY(ensure_stage(ctx, 4 * buf.size(), st));
    CK(cudaEventSynchronize(ctx->stage_done));
    std::memcpy(ctx->h_stage, buf.data(), 4 * buf.size());
    CK(cudaMemcpyAsync(ctx->qint.p, ctx->h_stage, 4 * buf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->stage_done, st));
    return launch_queue(ctx, p, L, a, tabs_at((const int32_t *)ctx->qint.p, off, ng, G), st);
}

// Autotuned forward pass: the first call of a given shape times every
// states-per-block choice (each produces the same bits) and keeps the fastest.
int fwd_pass(dgs_ctx *ctx, const dgs_scene *scene, const Plan &p, const Lists &L, const RasterArgs &a, int s0,
             int s1, cudaStream_t st)
{
    int maxper = 1;
    {
        std::vector<int> cnt(p.V, 0);
        for (int s = s0; s < s1; ++s) maxper = std::max(maxper, ++cnt[p.vg_of_state[s]]);
    }
    const std::vector<long long> key = {s1 - s0, p.V, p.W, p.H, scene->n, scene->n_clusters, scene->n_layers,
                                        a.images != nullptr, a.refs != nullptr, maxper};
    auto it = ctx->tuned_G.find(key);
    if (it != ctx->tuned_G.end()) return launch_fwd_pass(ctx, p, L, a, s0, s1, it->second, st);
    const int cands[1] = {1};
    int best = 1;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int G : cands) {
        if (G > 1 && G / 2 >= maxper) break;
        CK(cudaEventRecord(e0, st));
        TRY(launch_fwd_pass(ctx, p, L, a, s0, s1, G, st));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = G; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuned_G[key] = best;   // every trial wrote the same bits, so the outputs are final
    return DGS_OK;
}

// ------------------------------------------------------------ tile-size autotuner
// The sort tile size (16 or 32 px) changes no output bit, only the cost split
// between sorting (fewer, larger tiles: fewer entries) and rasterization
// (longer runs to walk per 16-pixel-wide region).  Unless the caller fixed it,
// the first call of each shape runs once untimed, then once per candidate,
// timed with events on its stream, and the faster size is kept for that
// shape in this context.
enum { TUNE_RENDER = 1, TUNE_UTILITY = 2 };

std::vector<long long> tile_key(int kind, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                                int n_cams)
{
    return {kind, cams && n_cams > 0 ? cams[0].width : 0, cams && n_cams > 0 ? cams[0].height : 0,
            states ? states->n_states : 0, n_cams, scene->n, scene->n_clusters, scene->n_layers, scene->sh_degree,
            scene->temporal_rank};
}

// Shift for a call of shape `key`: fixed by the caller, cached, or -1 (not tuned yet).
int known_shift(const dgs_ctx *ctx, const std::vector<long long> &key)
{
    if (ctx->tile_size) return ctx->tile_size == 32 ? 5 : 4;
    auto it = ctx->tuned_tile.find(key);
    return it == ctx->tuned_tile.end() ? -1 : it->second;
}

// Run call() (int(void)) with the tuned tile size of its shape, tuning it
// first if needed.  Every run writes the same outputs; the chosen size runs
// last, so the context's state (the lists a backward can reuse) is its.
template <class F>
int tuned_call(dgs_ctx *ctx, const std::vector<long long> &key, cudaStream_t st, F call)
{
    const int known = known_shift(ctx, key);
    if (known >= 0) {
        ctx->active_shift = known;
        return call();
    }
    // an untimed first run grows the workspace (and warms the caches) so the
    // timed runs compare the two sizes on equal terms
    ctx->active_shift = MIN_TILE_SHIFT;
    TRY(call());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = MIN_TILE_SHIFT, last = -1, r = DGS_OK;
    float best_ms = 1e30f;
    for (int sh = MIN_TILE_SHIFT; sh <= MAX_TILE_SHIFT && r == DGS_OK; ++sh) {
        ctx->active_shift = last = sh;
        CK(cudaEventRecord(e0, st));
        r = call();
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = sh; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != DGS_OK) return r;
    ctx->tuned_tile[key] = best;
    ctx->active_shift = best;
    return best == last ? DGS_OK : call();
}

int render_batched(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                   int n_cams, const float *bg, float *images, cudaStream_t st)
{
    TRY(check_scene(ctx, scene));
    if (!bg) return fail(ctx, DGS_E_INVALID_ARG, "bg is null");
    Plan p;
    TRY(build_plan(ctx, states, cams, n_cams, false, p));
    if (p.S_user > 0 && !images) return fail(ctx, DGS_E_INVALID_ARG, "images is null");
    ctx->tape.valid = false;
    if (p.S_user == 0) return DGS_OK;
    Lists L;
    TRY(prepare(ctx, scene, states->masks, p, false, st, L));
    RasterArgs a = raster_args(ctx, p, scene->n_clusters, bg, L.evals);
    a.images = images;
    TRY(fwd_pass(ctx, scene, p, L, a, 0, p.S_user, st));
    record_tape(ctx->tape, scene, states, cams, n_cams, p, L);
    // a copy of the masks rendered: the backward reuses these lists only while the masks still hold them
    const size_t mbytes = 4 * (size_t)p.S_user * (size_t)((scene->n_clusters * scene->n_layers + 31) / 32);
    TRY(ensure(ctx, ctx->tapemask, mbytes, st));
    CK(cudaMemcpyAsync(ctx->tapemask.p, states->masks, mbytes, cudaMemcpyDeviceToDevice, st));
    return DGS_OK;
}

}  // namespace


// ---------------------------------------------------------------- plans
// A plan fixes the scene, the states' times and cameras, the cameras and the
// background of a batch, and owns a workspace sized for them.  Its per-call
// entry points launch kernels only: counts stay on the device, every launch
// size depends only on the plan, nothing is allocated, copied from the host or
// synchronised, so a caller can capture them in a CUDA graph and replay them
// with new masks (and new scene values) of the same shapes.
// Scratch workspace shared by the plans created in it (they run one after
// another on one stream): records, keys, entries, sort and raster buffers.
struct dgs_arena {
    dgs_ctx ws;
    int plans = 0;
    const dgs_plan *last = nullptr;   // the plan whose lists the scratch holds
};

struct dgs_plan {
    dgs_ctx ws;                   // the plan's own tables (vgs, vgos, refidx), host staging, error message
    dgs_ctx *sc = nullptr;        // scratch buffers: &ws, or the arena's workspace
    dgs_arena *arena = nullptr;
    Plan p;
    dgs_scene scene{};
    float bg[3] = {0, 0, 0};
    int mode = 0;
    uint32_t R_cap = 0, E_cap = 0;
    Buf cnts;                     // [0] records, [1] entries, [2] min(entries, capacity), [3] overflow flags
    Buf qfwd, qref;               // state-group tables of the forward / reference passes
    QueueTabs tfwd, tref;
    Lists L;
    bool rendered = false;
    int n_refs = 0;
    int image_parts = 0;
    // Eq. 2 objective fixed by dgs_plan_set_objective: pair, anchor and
    // temporal-neighbour tables in ws.oints at these offsets (ints)
    bool obj = false;
    int obj_nt = 0, obj_nm = 0, obj_na = 0;
    size_t obj_pt = 0, obj_pm = 0, obj_tl = 0, obj_an = 0, obj_to = 0;
    dgs_objective_params obj_prm{};
};

namespace {

int plan_fail(dgs_plan *P, int code, const char *msg)
{
    P->ws.err = msg;
    P->sc->err = msg;
    return code;
}

// Capture-safe preparation: closure, layout, projection, sorts, binning and
// tile order with every count kept on the device.
int prepare_dev(dgs_plan *P, const uint32_t *masks, bool force_full, cudaStream_t st)
{
    dgs_ctx *ctx = P->sc;
    const Plan &p = P->p;
    const dgs_scene *scene = &P->scene;
    const int C = scene->n_clusters, L = scene->n_layers;
    const int words = (C * L + 31) / 32;
    const size_t nvc = (size_t)p.V * C, vt = (size_t)p.V * p.tiles;
    uint32_t *cnt = (uint32_t *)P->cnts.p;
    CK(cudaMemsetAsync(ctx->need.p, 0, 4 * nvc, st));
    if (p.S_user > 0)
        launch_closure(masks, p.S_user, words, C, L, (const int32_t *)P->ws.vgos.p, (uint8_t *)ctx->depth.p,
                       (uint32_t *)ctx->need.p, force_full ? 1 : 0, ctx->sms, st);
    launch_layout_counts((const uint32_t *)ctx->need.p, scene->cluster_offsets, p.V, C, (uint32_t *)ctx->counts.p,
                         ctx->sms, st);
    CK(exclusive_scan_u32((const uint32_t *)ctx->counts.p, (uint32_t *)ctx->recBase.p, nvc + 1, cnt + 0,
                          ctx->scanws.p, st));
    launch_project(scene_dev(scene), (const ViewGroup *)P->ws.vgs.p, p.V, (const uint32_t *)ctx->need.p,
                   (const uint32_t *)ctx->recBase.p, (Rec *)ctx->recs.p, (uint32_t *)ctx->k0.p, (uint32_t *)ctx->v0.p,
                   ctx->sms, st);
    bool alt = false;
    uint32_t *live = (uint32_t *)ctx->live.p;
    CK(radix_sort_pairs_seg((uint32_t *)ctx->k0.p, (uint32_t *)ctx->v0.p, (uint32_t *)ctx->k1.p,
                            (uint32_t *)ctx->v1.p, P->R_cap, (const uint32_t *)ctx->recBase.p, (uint32_t)C, p.V, 32,
                            ctx->sortws.p, st, &alt, "radix_depth", live));
    const uint32_t *order = alt ? (const uint32_t *)ctx->v1.p : (const uint32_t *)ctx->v0.p;
    Lists &out = P->L;
    out.depth_keys = alt ? (uint32_t *)ctx->k1.p : (uint32_t *)ctx->k0.p;
    out.depth_slots = (uint32_t *)order;
    launch_tile_count((const Rec *)ctx->recs.p, order, P->R_cap, p.tiles_x, p.tiles, p.tile_shift,
                      (uint32_t *)ctx->tcount.p, (uint4 *)ctx->bins.p, ctx->sms, st, live + p.V);
    CK(exclusive_scan_u32((const uint32_t *)ctx->tcount.p, (uint32_t *)ctx->toffs.p, P->R_cap, cnt + 1,
                          ctx->scanws.p, st));
    launch_clamp_count(cnt + 1, P->E_cap, cnt + 2, cnt + 3, st);
    const int tbits = bits_for((unsigned long long)p.tiles - 1ull);
    bool ranges_done = false;
    CK(radix_sort_entries((const uint4 *)ctx->bins.p, (const uint32_t *)ctx->toffs.p, (const uint32_t *)ctx->tcount.p,
                          P->R_cap, live + p.V, live, 1u, p.V, p.tiles_x, p.tiles,
                          (uint32_t *)ctx->ek0.p, (uint32_t *)ctx->ev0.p, (uint32_t *)ctx->ek1.p,
                          (uint32_t *)ctx->ev1.p, P->E_cap, cnt + 2, tbits, ctx->sortws.p, st, &alt, ctx->sms,
                          (uint2 *)ctx->ranges.p, &ranges_done));
    out.ekeys = alt ? (uint32_t *)ctx->ek1.p : (uint32_t *)ctx->ek0.p;
    out.evals = alt ? (uint32_t *)ctx->ev1.p : (uint32_t *)ctx->ev0.p;
    if (!ranges_done) {
        CK(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * vt, st));
        launch_ranges(out.ekeys, P->E_cap, (uint2 *)ctx->ranges.p, ctx->sms, st, cnt + 2);
    }
    launch_tile_costs((const uint2 *)ctx->ranges.p, (uint32_t)vt, (uint32_t *)ctx->tck0.p, (uint32_t *)ctx->tcv0.p,
                      ctx->sms, st);
    CK(radix_sort_pairs((uint32_t *)ctx->tck0.p, (uint32_t *)ctx->tcv0.p, (uint32_t *)ctx->tck1.p,
                        (uint32_t *)ctx->tcv1.p, vt, 16, ctx->sortws.p, st, &alt, nullptr, "radix_cost"));
    out.tile_order = alt ? (uint32_t *)ctx->tcv1.p : (uint32_t *)ctx->tcv0.p;
    out.nRec = P->R_cap;
    out.nEnt = P->E_cap;
    CK(cudaGetLastError());
    return DGS_OK;
}

int upload_tabs(dgs_plan *P, Buf &b, int s0, int s1, int G, QueueTabs &out)
{
    dgs_ctx *ctx = &P->ws;
    std::vector<int32_t> buf;
    size_t off[5], ng = 0;
    build_groups(P->p, s0, s1, G, buf, off, ng);
    TRY(ensure(ctx, b, 4 * buf.size() + 16, 0));
    CK(cudaMemcpy(b.p, buf.data(), 4 * buf.size(), cudaMemcpyHostToDevice));
    out = tabs_at((const int32_t *)b.p, off, ng, G);
    return DGS_OK;
}

int tuned_choice(dgs_ctx *ctx, const dgs_scene *scene, const Plan &p, int s0, int s1, bool images, bool refs)
{
    int maxper = 1;
    std::vector<int> cnt(p.V, 0);
    for (int s = s0; s < s1; ++s) maxper = std::max(maxper, ++cnt[p.vg_of_state[s]]);
    const std::vector<long long> key = {s1 - s0, p.V, p.W, p.H, scene->n, scene->n_clusters, scene->n_layers,
                                        images, refs, maxper};
    auto it = ctx->tuned_G.find(key);
    return it == ctx->tuned_G.end() ? 1 : it->second;
}

// Free every device and host buffer a workspace holds (not the workspace itself).
// Every device buffer of a context's workspace.
std::vector<Buf *> all_bufs(dgs_ctx *ctx)
{
    return {&ctx->vgs, &ctx->vgos, &ctx->depth, &ctx->need, &ctx->counts, &ctx->recBase, &ctx->total,
                   &ctx->recs, &ctx->k0, &ctx->v0, &ctx->k1, &ctx->v1, &ctx->tcount, &ctx->toffs, &ctx->bins, &ctx->ek0,
                   &ctx->ev0, &ctx->ek1, &ctx->ev1, &ctx->ranges, &ctx->sortws, &ctx->scanws, &ctx->partial,
                   &ctx->refs, &ctx->recgrad, &ctx->refidx, &ctx->tck0, &ctx->tcv0, &ctx->tck1, &ctx->tcv1,
                   &ctx->icnt, &ctx->ioff, &ctx->qint, &ctx->counter, &ctx->pairm, &ctx->grp, &ctx->gmse, &ctx->omaps, &ctx->opart, &ctx->otpart,
                   &ctx->oD, &ctx->oweight, &ctx->oints, &ctx->recgmu, &ctx->gqws, &ctx->shord, &ctx->shpair,
                   &ctx->shpair2, &ctx->shrep, &ctx->shflag, &ctx->shpos, &ctx->shlist, &ctx->shitem, &ctx->shkey, &ctx->shstop,
                   &ctx->shseg, &ctx->shcnt, &ctx->shtab, &ctx->tapemask, &ctx->live, &ctx->jobargs};
}

// Free the device workspace except the buffers in `keep` (after the stream's
// work is done); the next call grows it again.  The lists a backward could
// reuse are gone with it.
void release_workspace(dgs_ctx *ctx, cudaStream_t st, std::initializer_list<Buf *> keep)
{
    cudaStreamSynchronize(st);
    for (Buf *b : all_bufs(ctx)) {
        if (!b->p || std::find(keep.begin(), keep.end(), b) != keep.end()) continue;
        cudaFree(b->p);
        ctx->ws_bytes -= b->cap;
        b->p = nullptr;
        b->cap = 0;
    }
    ctx->tape.valid = false;
}

void free_ctx_buffers(dgs_ctx *ctx)
{
    for (Buf *b : all_bufs(ctx))
        if (b->p) { cudaFree(b->p); b->p = nullptr; b->cap = 0; }
    ctx->ws_bytes = 0;
    if (ctx->h_stage) { cudaFreeHost(ctx->h_stage); ctx->h_stage = nullptr; }
    if (ctx->h_small) { cudaFreeHost(ctx->h_small); ctx->h_small = nullptr; }
    if (ctx->stage_done) { cudaEventDestroy(ctx->stage_done); ctx->stage_done = nullptr; }
}

int utility_pass(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                 int n_cams, const float *bg, double *mse, double *psnr, cudaStream_t st);

bool grads_complete(const dgs_scene *scene, const dgs_scene_grad *g)
{
    return g->mu0 && g->log_scale && g->quat && g->opacity_logit && g->colour &&
           !(scene->temporal_rank > 0 && !g->u) && !(scene->n_layers > 1 && scene->res_mode != 1 && !g->res) &&
           !(scene->affine && !g->affine) && !(scene->n_layers > 1 && scene->res_mode == 2 && !g->res_step);
}

// The projection adjoint after the adjoint raster has accumulated the record
// moments of lists L (plan p) in ctx->recgrad: chain rule to the scene
// gradients, and the moments cleared again.
int project_backward(dgs_ctx *ctx, const dgs_scene *scene, const Plan &p, const Lists &L,
                     const dgs_scene_grad *grads, cudaStream_t st)
{
    const uint32_t nRec = L.nRec;
    GradDev g;
    g.mu0 = grads->mu0; g.u = grads->u; g.ls = grads->log_scale; g.quat = grads->quat;
    g.logit = grads->opacity_logit; g.colour = grads->colour; g.res = grads->res;
    g.affine = grads->affine; g.rec_gmu = nullptr;
    g.res_step = grads->res_step; g.gq = nullptr;
    if (scene->affine) {
        TRY(ensure(ctx, ctx->recgmu, sizeof(float) * 3 * ((size_t)nRec + 1), st));
        g.rec_gmu = (float *)ctx->recgmu.p;
    }
    if (scene->res_mode == 2 && scene->n_layers > 1) {
        const SceneDev sdv = scene_dev(scene);
        TRY(ensure(ctx, ctx->gqws, sizeof(float) * (size_t)(scene->n_layers - 1) * scene->n * sdv.K, st));
        g.gq = (float *)ctx->gqws.p;
    }
    launch_project_bwd(scene_dev(scene), (const ViewGroup *)ctx->vgs.p, p.V, (const uint32_t *)ctx->need.p,
                       (const uint32_t *)ctx->recBase.p, (float4 *)ctx->recgrad.p, g, nRec, ctx->sms, st);
    CK(cudaGetLastError());
    ctx->recgrad.zeroed = true;          // the projection adjoint cleared what the raster wrote
    return DGS_OK;
}

RasterArgs plan_raster_args(dgs_plan *P)
{
    RasterArgs a = raster_args(P->sc, P->p, P->scene.n_clusters, P->bg, P->L.evals);
    a.vg_of_state = (const int32_t *)P->ws.vgos.p;
    return a;
}

}  // namespace

extern "C" {

int dgs_version(void) { return DGS_VERSION; }

int dgs_create(dgs_ctx **out, int device)
{
    if (!out) return DGS_E_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DGS_E_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return DGS_E_CUDA;
    dgs_ctx *ctx = new dgs_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMallocHost((void **)&ctx->h_small, 64 + 4 * (MAX_CLUSTERS + 1)) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming) != cudaSuccess) {
        if (ctx->h_small) cudaFreeHost(ctx->h_small);
        delete ctx;
        return DGS_E_OOM;
    }
    raster_fwd_query_occupancy();
    ctx->launch_base = g_launches.load();
    *out = ctx;
    return DGS_OK;
}

void dgs_destroy(dgs_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (dgs_ctx *k : ctx->kids) dgs_destroy(k);
    free_ctx_buffers(ctx);
    delete ctx;
}

const char *dgs_last_error(const dgs_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t dgs_kernel_launches(const dgs_ctx *ctx) { return ctx ? (int64_t)(g_launches.load() - ctx->launch_base) : 0; }

void dgs_reset_kernel_launches(dgs_ctx *ctx)
{
    if (ctx) ctx->launch_base = g_launches.load();
}

void dgs_profile_enable(dgs_ctx *ctx, int on)
{
    (void)ctx;
    g_prof = on != 0;
    g_prof_recs.clear();
    g_prof_stack.clear();
    g_event_next = 0;
}

int dgs_profile_read(dgs_ctx *ctx, int max_names, char *names, double *total_ms, int64_t *launches)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(ctx, DGS_E_CUDA, "synchronize failed");
    std::vector<std::string> order;
    std::map<std::string, std::pair<double, long long>> agg;
    for (const ProfRec &r : g_prof_recs) {
        float ms = 0.0f;
        if (!r.a || !r.b || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            agg[r.name] = {ms, 1};
        } else {
            it->second.first += ms;
            it->second.second += 1;
        }
    }
    g_prof_recs.clear();
    g_prof_stack.clear();
    g_event_next = 0;
    const int n = (int)order.size() < max_names ? (int)order.size() : max_names;
    for (int k = 0; k < n; ++k) {
        if (names) {
            std::strncpy(names + 32 * k, order[k].c_str(), 31);
            names[32 * k + 31] = 0;
        }
        if (total_ms) total_ms[k] = agg[order[k]].first;
        if (launches) launches[k] = agg[order[k]].second;
    }
    return n;
}

int dgs_render_states_batched(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states,
                              const dgs_camera *cams, int n_cams, const float *bg, float *images, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    TRY(check_scene(ctx, scene));
    if (!states) return fail(ctx, DGS_E_INVALID_ARG, "states is null");
    const size_t img_vals = (cams && n_cams > 0) ? (size_t)cams[0].width * cams[0].height * 3 : 0;
    const int words = (scene->n_clusters * scene->n_layers + 31) / 32;
    return tuned_call(ctx, tile_key(TUNE_RENDER, scene, states, cams, n_cams), (cudaStream_t)stream, [&] {
        return chunked(ctx, states, words, 0, (cudaStream_t)stream, [&](const dgs_states *sub, int s0) {
            return render_batched(ctx, scene, sub, cams, n_cams, bg, images ? images + (size_t)s0 * img_vals : nullptr,
                                  (cudaStream_t)stream);
        });
    });
}

int dgs_render_state(dgs_ctx *ctx, const dgs_scene *scene, const uint32_t *mask, float t, const dgs_camera *cam,
                     const float *bg, float *image, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (!mask || !cam) return fail(ctx, DGS_E_INVALID_ARG, "mask or camera is null");
    CK(cudaSetDevice(ctx->device));
    const int32_t cam0 = 0;
    dgs_states s;
    s.masks = mask; s.t = &t; s.cam = &cam0; s.n_states = 1;
    TRY(check_scene(ctx, scene));
    return tuned_call(ctx, tile_key(TUNE_RENDER, scene, &s, cam, 1), (cudaStream_t)stream,
                      [&] { return render_batched(ctx, scene, &s, cam, 1, bg, image, (cudaStream_t)stream); });
}

int dgs_render_backward(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                        int n_cams, const float *bg, const float *images, const float *dL_dimages,
                        const dgs_scene_grad *grads, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    TRY(check_scene(ctx, scene));
    if (!bg || !grads) return fail(ctx, DGS_E_INVALID_ARG, "bg or grads is null");
    if (!states) return fail(ctx, DGS_E_INVALID_ARG, "states is null");
    {   // the tile size the forward of this shape used (any size gives the same gradients)
        const int known = known_shift(ctx, tile_key(TUNE_RENDER, scene, states, cams, n_cams));
        ctx->active_shift = known >= 0 ? known : (ctx->tape.valid ? ctx->tape.plan.tile_shift : MIN_TILE_SHIFT);
    }
    if (!dL_dimages && states->n_states > 0) return fail(ctx, DGS_E_INVALID_ARG, "dL_dimages is null");
    const size_t img_vals = (cams && n_cams > 0) ? (size_t)cams[0].width * cams[0].height * 3 : 0;
    // a batch whose workspace does not fit runs in halves (gradients accumulate)
    auto pass = [&](const dgs_states *sub, int s0) -> int {
        const float *img_s = images ? images + (size_t)s0 * img_vals : nullptr;
        const float *dL_s = dL_dimages ? dL_dimages + (size_t)s0 * img_vals : nullptr;
        Plan p;
        TRY(build_plan(ctx, sub, cams, n_cams, false, p));
        if (p.S_user == 0 || scene->n == 0) return DGS_OK;
        if (!dL_s) return fail(ctx, DGS_E_INVALID_ARG, "dL_dimages is null");
        if (!grads_complete(scene, grads)) return fail(ctx, DGS_E_INVALID_ARG, "gradient array is null");
        Lists L;
        bool reuse = same_call(ctx->tape, scene, sub, cams, n_cams) && ctx->tape.plan.tile_shift == p.tile_shift;
        if (reuse) {
            // same arguments as the last forward: its lists are reused only if the masks
            // still hold the bits it rendered (compared on the device; one host sync)
            const size_t words = (size_t)p.S_user * (size_t)((scene->n_clusters * scene->n_layers + 31) / 32);
            uint32_t *flag = (uint32_t *)ctx->total.p + 4;
            CK(cudaMemsetAsync(flag, 0, 4, st));
            launch_words_differ(sub->masks, (const uint32_t *)ctx->tapemask.p, words, flag, ctx->sms, st);
            CK(cudaMemcpyAsync(ctx->h_small + 12, flag, 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (ctx->h_small[12]) {
                if (img_s)
                    return fail(ctx, DGS_E_STALE, "the masks changed after the forward call whose images were passed");
                reuse = false;          // no forward images to disagree with: render lists for the current masks
            }
        }
        if (reuse) {
            L = ctx->tape.lists;
        } else {
            ctx->tape.valid = false;
            TRY(prepare(ctx, scene, sub->masks, p, false, st, L));
            record_tape(ctx->tape, scene, sub, cams, n_cams, p, L);
        }
        TRY(ensure_zeroed(ctx, ctx->recgrad, sizeof(float4) * 3 * (size_t)L.nRec, st));
        ctx->recgrad.zeroed = false;
        RasterBwdArgs b;
        b.f = raster_args(ctx, p, scene->n_clusters, bg, L.evals);
        b.dL_dimg = dL_s;
        b.img_fwd = img_s;
        b.rec_grad = (float4 *)ctx->recgrad.p;
        launch_raster_bwd(b, ctx->sms, st);
        return project_backward(ctx, scene, p, L, grads, st);
    };
    return chunked(ctx, states, (scene->n_clusters * scene->n_layers + 31) / 32, 0, st, pass);
}

// ---------------------------------------------------------------- several scenes
// dgs_render_scenes_batched / dgs_render_scenes_backward: every scene of the
// batch gets a workspace of its own (a child context, kept between calls), its
// closure, projection, sorts and lists are prepared there scene by scene, and
// one persistent forward raster launch (one adjoint raster launch) works
// through the (scene, tile, state) items of all of them from one queue.
}  // extern "C"

namespace {

dgs_ctx *make_kid(const dgs_ctx *parent)
{
    dgs_ctx *k = new dgs_ctx();
    k->device = parent->device;
    k->sms = parent->sms;
    if (cudaMallocHost((void **)&k->h_small, 64 + 4 * (MAX_CLUSTERS + 1)) != cudaSuccess ||
        cudaEventCreateWithFlags(&k->stage_done, cudaEventDisableTiming) != cudaSuccess) {
        if (k->h_small) cudaFreeHost(k->h_small);
        delete k;
        return nullptr;
    }
    k->launch_base = parent->launch_base;
    return k;
}

int scene_job_fail(dgs_ctx *ctx, const dgs_ctx *kid, int k, int code)
{
    return fail(ctx, code, "scene %d: %s", k, kid->err.c_str());
}

// Copy n bytes from host memory into ctx->jobargs at byte offset off through
// the pinned staging buffer (the buffer must already hold off + n bytes).
int upload_jobs(dgs_ctx *ctx, const void *src, size_t n, size_t off, cudaStream_t st)
{
    TRY(ensure_stage(ctx, n, st));
    CK(cudaEventSynchronize(ctx->stage_done));
    std::memcpy(ctx->h_stage, src, n);
    CK(cudaMemcpyAsync((char *)ctx->jobargs.p + off, ctx->h_stage, n, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->stage_done, st));
    return DGS_OK;
}

}  // namespace

extern "C" {

int dgs_render_scenes_batched(dgs_ctx *ctx, const dgs_scene_job *jobs, int n_jobs, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, DGS_E_INVALID_ARG, "jobs is null or n_jobs < 0");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    // one tile size for the whole launch: the caller's, else 32 px
    const int shift = ctx->tile_size == 16 ? 4 : 5;
    while ((int)ctx->kids.size() < n_jobs) {
        dgs_ctx *k = make_kid(ctx);
        if (!k) return fail(ctx, DGS_E_OOM, "pinned host memory for a scene workspace");
        ctx->kids.push_back(k);
    }
    std::vector<RasterArgs> args;
    std::vector<WorkQueue> queues;
    std::vector<uint32_t> off(1, 0u);
    for (int k = 0; k < n_jobs; ++k) {
        const dgs_scene_job &J = jobs[k];
        dgs_ctx *kid = ctx->kids[k];
        kid->tile_size = 1 << shift;
        kid->active_shift = shift;
        kid->tape.valid = false;
        if (!J.scene) return fail(ctx, DGS_E_INVALID_ARG, "scene %d: scene is null", k);
        if (check_scene(kid, J.scene) != DGS_OK) return scene_job_fail(ctx, kid, k, DGS_E_INVALID_ARG);
        Plan p;
        int r = build_plan(kid, &J.states, J.cams, J.n_cams, false, p);
        if (r != DGS_OK) return scene_job_fail(ctx, kid, k, r);
        if (p.S_user == 0) continue;
        if (!J.images) return fail(ctx, DGS_E_INVALID_ARG, "scene %d: images is null", k);
        Lists L;
        if ((r = prepare(kid, J.scene, J.states.masks, p, false, st, L)) != DGS_OK) return scene_job_fail(ctx, kid, k, r);
        RasterArgs a = raster_args(kid, p, J.scene->n_clusters, J.bg, L.evals);
        a.images = J.images;
        std::vector<int32_t> buf;
        size_t toff[5], ng = 0;
        build_groups(p, 0, p.S_user, 1, buf, toff, ng);
        if ((r = ensure(kid, kid->qint, 4 * buf.size(), st)) != DGS_OK ||
            (r = ensure_stage(kid, 4 * buf.size(), st)) != DGS_OK)
            return scene_job_fail(ctx, kid, k, r);
        CK(cudaEventSynchronize(kid->stage_done));
        std::memcpy(kid->h_stage, buf.data(), 4 * buf.size());
        CK(cudaMemcpyAsync(kid->qint.p, kid->h_stage, 4 * buf.size(), cudaMemcpyHostToDevice, st));
        CK(cudaEventRecord(kid->stage_done, st));
        WorkQueue q;
        if ((r = make_queue(kid, p, L, tabs_at((const int32_t *)kid->qint.p, toff, ng, 1), st, q)) != DGS_OK)
            return scene_job_fail(ctx, kid, k, r);
        record_tape(kid->tape, J.scene, &J.states, J.cams, J.n_cams, p, L);
        const size_t mbytes = 4 * (size_t)p.S_user * (size_t)((J.scene->n_clusters * J.scene->n_layers + 31) / 32);
        if ((r = ensure(kid, kid->tapemask, mbytes, st)) != DGS_OK) return scene_job_fail(ctx, kid, k, r);
        CK(cudaMemcpyAsync(kid->tapemask.p, J.states.masks, mbytes, cudaMemcpyDeviceToDevice, st));
        args.push_back(a);
        queues.push_back(q);
        off.push_back(off.back() + q.n_items);
    }
    const int n = (int)args.size();
    if (n == 0 || off.back() == 0) return DGS_OK;
    // device copies of the per-scene arguments, queues and item offsets, then one launch
    const size_t b_args = sizeof(RasterArgs) * n, b_q = sizeof(WorkQueue) * n, b_off = 4 * (size_t)(n + 1);
    const size_t o_q = (b_args + 255) & ~(size_t)255, o_off = (o_q + b_q + 255) & ~(size_t)255;
    const size_t o_cnt = (o_off + b_off + 255) & ~(size_t)255;
    TRY(ensure(ctx, ctx->jobargs, o_cnt + 16, st));
    std::vector<char> host(o_cnt);
    std::memcpy(host.data(), args.data(), b_args);
    std::memcpy(host.data() + o_q, queues.data(), b_q);
    std::memcpy(host.data() + o_off, off.data(), b_off);
    TRY(upload_jobs(ctx, host.data(), o_cnt, 0, st));
    uint32_t *counter = (uint32_t *)((char *)ctx->jobargs.p + o_cnt);
    CK(cudaMemsetAsync(counter, 0, 4, st));
    char *base = (char *)ctx->jobargs.p;
    launch_raster_fwd_multi((const RasterArgs *)base, (const WorkQueue *)(base + o_q), (const uint32_t *)(base + o_off),
                            n, counter, shift, ctx->sms, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

int dgs_render_scenes_backward(dgs_ctx *ctx, const dgs_scene_job *jobs, int n_jobs, const float *const *dL_dimages,
                               const dgs_scene_grad *grads, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !dL_dimages || !grads)))
        return fail(ctx, DGS_E_INVALID_ARG, "jobs, dL_dimages or grads is null");
    if ((int)ctx->kids.size() < n_jobs)
        return fail(ctx, DGS_E_INVALID_ARG, "dgs_render_scenes_backward needs dgs_render_scenes_batched of these jobs first");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    // every scene must be the one its workspace last rendered, with the masks it rendered
    std::vector<int> live;
    for (int k = 0; k < n_jobs; ++k) {
        const dgs_scene_job &J = jobs[k];
        dgs_ctx *kid = ctx->kids[k];
        if (J.states.n_states == 0) continue;
        if (!J.scene || !J.images || !dL_dimages[k]) return fail(ctx, DGS_E_INVALID_ARG, "scene %d: null argument", k);
        if (!kid->tape.valid || !same_call(kid->tape, J.scene, &J.states, J.cams, J.n_cams))
            return fail(ctx, DGS_E_INVALID_ARG, "scene %d: not the scene batch the last dgs_render_scenes_batched rendered", k);
        if (!grads_complete(J.scene, &grads[k])) return fail(ctx, DGS_E_INVALID_ARG, "scene %d: gradient array is null", k);
        const Plan &p = kid->tape.plan;
        const size_t words = (size_t)p.S_user * (size_t)((J.scene->n_clusters * J.scene->n_layers + 31) / 32);
        uint32_t *flag = (uint32_t *)kid->total.p + 4;
        CK(cudaMemsetAsync(flag, 0, 4, st));
        launch_words_differ(J.states.masks, (const uint32_t *)kid->tapemask.p, words, flag, ctx->sms, st);
        CK(cudaMemcpyAsync(kid->h_small + 12, flag, 4, cudaMemcpyDeviceToHost, st));
        live.push_back(k);
    }
    if (live.empty()) return DGS_OK;
    CK(cudaStreamSynchronize(st));
    for (int k : live)
        if (ctx->kids[k]->h_small[12])
            return fail(ctx, DGS_E_STALE, "scene %d: the masks changed after the forward call", k);
    std::vector<RasterBwdArgs> bargs;
    std::vector<size_t> off(1, 0);
    for (int k : live) {
        const dgs_scene_job &J = jobs[k];
        dgs_ctx *kid = ctx->kids[k];
        const Lists &L = kid->tape.lists;
        int r = ensure_zeroed(kid, kid->recgrad, sizeof(float4) * 3 * (size_t)L.nRec, st);
        if (r != DGS_OK) return scene_job_fail(ctx, kid, k, r);
        kid->recgrad.zeroed = false;
        RasterBwdArgs b;
        b.f = raster_args(kid, kid->tape.plan, J.scene->n_clusters, J.bg, L.evals);
        b.dL_dimg = dL_dimages[k];
        b.img_fwd = J.images;
        b.rec_grad = (float4 *)kid->recgrad.p;
        bargs.push_back(b);
        off.push_back(off.back() + raster_bwd_items(b.f));
    }
    const int n = (int)bargs.size();
    const size_t b_args = sizeof(RasterBwdArgs) * n, o_off = (b_args + 255) & ~(size_t)255;
    const size_t total = o_off + sizeof(size_t) * (n + 1);
    TRY(ensure(ctx, ctx->jobargs, total, st));
    std::vector<char> host(total);
    std::memcpy(host.data(), bargs.data(), b_args);
    std::memcpy(host.data() + o_off, off.data(), sizeof(size_t) * (n + 1));
    TRY(upload_jobs(ctx, host.data(), total, 0, st));
    launch_raster_bwd_multi((const RasterBwdArgs *)ctx->jobargs.p,
                            (const size_t *)((char *)ctx->jobargs.p + o_off), n, off.back(), st);
    CK(cudaGetLastError());
    for (int k : live) {
        dgs_ctx *kid = ctx->kids[k];
        const int r = project_backward(kid, jobs[k].scene, kid->tape.plan, kid->tape.lists, &grads[k], st);
        if (r != DGS_OK) return scene_job_fail(ctx, kid, k, r);
    }
    return DGS_OK;
}

int dgs_state_utility(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                      int n_cams, const float *bg, double *mse, double *psnr, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    TRY(check_scene(ctx, scene));
    if (!bg) return fail(ctx, DGS_E_INVALID_ARG, "bg is null");
    if (!states) return fail(ctx, DGS_E_INVALID_ARG, "states is null");
    const int words = (scene->n_clusters * scene->n_layers + 31) / 32;
    return tuned_call(ctx, tile_key(TUNE_UTILITY, scene, states, cams, n_cams), (cudaStream_t)stream, [&] {
        return chunked(ctx, states, words, 0, (cudaStream_t)stream, [&](const dgs_states *sub, int s0) {
            return utility_pass(ctx, scene, sub, cams, n_cams, bg, mse ? mse + s0 : nullptr, psnr ? psnr + s0 : nullptr,
                                (cudaStream_t)stream);
        });
    });
}

int dgs_group_utility(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *contexts, const int32_t *groups,
                      int n_groups, int n_contexts, const dgs_camera *cams, int n_cams, const float *bg,
                      double alpha, double beta, double q, double *delta, double *stats, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    TRY(check_scene(ctx, scene));
    if (!bg || !contexts) return fail(ctx, DGS_E_INVALID_ARG, "bg or contexts is null");
    if (n_groups < 0 || n_contexts < 1 || n_contexts > DGS_UTILITY_MAX_CONTEXTS)
        return fail(ctx, DGS_E_INVALID_ARG, "need n_groups >= 0 and 1 <= n_contexts <= %d", DGS_UTILITY_MAX_CONTEXTS);
    if ((long long)n_groups * n_contexts != (long long)contexts->n_states)
        return fail(ctx, DGS_E_INVALID_ARG, "contexts must hold n_groups * n_contexts states");
    if (2ll * n_groups * n_contexts > 0x7fffffffll) return fail(ctx, DGS_E_CAPACITY, "too many states");
    if (!(q >= 0.0 && q <= 1.0) || !(beta >= 0.0) || !(alpha == alpha))
        return fail(ctx, DGS_E_INVALID_ARG, "need 0 <= q <= 1, beta >= 0, alpha finite");
    if (n_groups == 0) return DGS_OK;
    if (!groups || !stats || !contexts->masks || !contexts->t || !contexts->cam)
        return fail(ctx, DGS_E_INVALID_ARG, "null argument");
    const int C = scene->n_clusters, L = scene->n_layers, G = n_groups, M = n_contexts;
    for (int g = 0; g < G; ++g)
        if (groups[2 * g] < 0 || groups[2 * g] >= C || groups[2 * g + 1] < 0 || groups[2 * g + 1] >= L)
            return fail(ctx, DGS_E_INVALID_ARG, "group %d = (%d, %d) is not a packet", g, groups[2 * g],
                        groups[2 * g + 1]);
    const int words = (C * L + 31) / 32;
    const size_t GM = (size_t)G * M;
    TRY(ensure(ctx, ctx->pairm, 4 * 2 * GM * words, st));
    TRY(ensure(ctx, ctx->grp, 8 * (size_t)G, st));
    TRY(ensure(ctx, ctx->gmse, 8 * 2 * GM, st));
    TRY(ensure_stage(ctx, 8 * (size_t)G, st));
    CK(cudaEventSynchronize(ctx->stage_done));   // an earlier copy may still read h_stage
    std::memcpy(ctx->h_stage, groups, 8 * (size_t)G);
    CK(cudaMemcpyAsync(ctx->grp.p, ctx->h_stage, 8 * (size_t)G, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->stage_done, st));
    launch_pair_masks(contexts->masks, (const int2 *)ctx->grp.p, G, M, words, L, (uint32_t *)ctx->pairm.p,
                      ctx->sms, st);
    std::vector<float> t2(2 * GM);
    std::vector<int32_t> c2(2 * GM);
    for (size_t k = 0; k < GM; ++k) {
        t2[k] = t2[GM + k] = contexts->t[k];
        c2[k] = c2[GM + k] = contexts->cam[k];
    }
    dgs_states s2;
    s2.masks = (const uint32_t *)ctx->pairm.p;
    s2.t = t2.data();
    s2.cam = c2.data();
    s2.n_states = (int)(2 * GM);
    TRY(tuned_call(ctx, tile_key(TUNE_UTILITY, scene, &s2, cams, n_cams), st, [&] {
        return chunked(ctx, &s2, words, 0, st, [&](const dgs_states *sub, int s0) {
            return utility_pass(ctx, scene, sub, cams, n_cams, bg, (double *)ctx->gmse.p + s0, nullptr, st);
        }, {&ctx->pairm, &ctx->grp, &ctx->gmse});     // the paired masks and the MSE output live there
    }));
    launch_group_stats((const double *)ctx->gmse.p, G, M, alpha, beta, q, delta, stats, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

int dgs_objective(dgs_ctx *ctx, const float *images, const float *refs, const int32_t *ref_index, int S, int n_refs,
                  int H, int W, const int32_t *pairs_t, int n_pairs_t, const int32_t *pairs_m, int n_pairs_m,
                  const int32_t *anchors, int n_anchors, const dgs_objective_params *params, double *loss, double *D,
                  float *dL_dimages, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (S < 1 || S > DGS_OBJECTIVE_MAX_STATES || n_refs < 1 || H < 1 || W < 1 || n_pairs_t < 0 || n_pairs_m < 0 ||
        n_anchors < 0)
        return fail(ctx, DGS_E_INVALID_ARG, "bad sizes (1 <= S <= %d)", DGS_OBJECTIVE_MAX_STATES);
    if (!images || !refs || !ref_index || !loss) return fail(ctx, DGS_E_INVALID_ARG, "null argument");
    if ((n_pairs_t && !pairs_t) || (n_pairs_m && !pairs_m) || (n_anchors && !anchors))
        return fail(ctx, DGS_E_INVALID_ARG, "null pair or anchor list");
    for (int s = 0; s < S; ++s)
        if (ref_index[s] < 0 || ref_index[s] >= n_refs)
            return fail(ctx, DGS_E_INVALID_ARG, "ref_index[%d] out of range", s);
    for (int p = 0; p < 2 * n_pairs_t; ++p)
        if (pairs_t[p] < 0 || pairs_t[p] >= S) return fail(ctx, DGS_E_INVALID_ARG, "temporal pair out of range");
    for (int p = 0; p < 2 * n_pairs_m; ++p)
        if (pairs_m[p] < 0 || pairs_m[p] >= S) return fail(ctx, DGS_E_INVALID_ARG, "prefix pair out of range");
    for (int a = 0; a < n_anchors; ++a)
        if (anchors[a] < 0 || anchors[a] >= S) return fail(ctx, DGS_E_INVALID_ARG, "anchor out of range");
    dgs_objective_params prm = {0.20, 0.30, 0.05, 0.10, 2.0, 0.50};
    if (params) prm = *params;
    if (!(prm.cvar_q >= 0.0 && prm.cvar_q <= 1.0)) return fail(ctx, DGS_E_INVALID_ARG, "cvar_q outside [0, 1]");
    const size_t npix = (size_t)H * W;
    int tx;
    const int nt = objective_tiles(H, W, &tx);
    const int chunks = (int)((npix + 1023) / 1024);
    // host tables: ref_index [S], pairs_t [2 n_t], pairs_m [2 n_m], anchors, toff [S + 1], tlist [2 n_t][2]
    std::vector<int32_t> toff(S + 1, 0), tl(4 * (size_t)n_pairs_t);
    for (int p = 0; p < n_pairs_t; ++p) { ++toff[pairs_t[2 * p] + 1]; ++toff[pairs_t[2 * p + 1] + 1]; }
    for (int s = 0; s < S; ++s) toff[s + 1] += toff[s];
    {
        std::vector<int32_t> fill(toff.begin(), toff.end() - 1);
        for (int p = 0; p < n_pairs_t; ++p) {
            const int i = pairs_t[2 * p], j = pairs_t[2 * p + 1];
            tl[2 * fill[i]] = j; tl[2 * fill[i] + 1] = -1; ++fill[i];      // i is the earlier state
            tl[2 * fill[j]] = i; tl[2 * fill[j] + 1] = +1; ++fill[j];      // j is the later state
        }
    }
    // the int2 lists first, at even offsets (8-byte aligned), then the int arrays
    const size_t o_pt = 0, o_pm = o_pt + 2 * (size_t)n_pairs_t, o_tl = o_pm + 2 * (size_t)n_pairs_m;
    const size_t o_ri = o_tl + tl.size(), o_an = o_ri + S, o_to = o_an + n_anchors, n_ints = o_to + S + 1;
    TRY(ensure(ctx, ctx->oints, 4 * n_ints + 16, st));
    TRY(ensure(ctx, ctx->omaps, sizeof(float) * 3 * (size_t)S * 3 * npix, st));
    TRY(ensure(ctx, ctx->opart, sizeof(double) * 2 * (size_t)S * nt, st));
    TRY(ensure(ctx, ctx->otpart, sizeof(double) * (size_t)(n_pairs_t > 0 ? n_pairs_t : 1) * chunks, st));
    TRY(ensure(ctx, ctx->oD, sizeof(double) * (size_t)S, st));
    TRY(ensure(ctx, ctx->oweight, sizeof(double) * (size_t)S, st));
    TRY(ensure_stage(ctx, 4 * n_ints, st));
    CK(cudaEventSynchronize(ctx->stage_done));   // an earlier copy may still read h_stage
    int32_t *h = (int32_t *)ctx->h_stage;
    std::memcpy(h + o_ri, ref_index, 4 * (size_t)S);
    if (n_pairs_t) std::memcpy(h + o_pt, pairs_t, 8 * (size_t)n_pairs_t);
    if (n_pairs_m) std::memcpy(h + o_pm, pairs_m, 8 * (size_t)n_pairs_m);
    if (n_anchors) std::memcpy(h + o_an, anchors, 4 * (size_t)n_anchors);
    std::memcpy(h + o_to, toff.data(), 4 * (size_t)(S + 1));
    if (!tl.empty()) std::memcpy(h + o_tl, tl.data(), 4 * tl.size());
    CK(cudaMemcpyAsync(ctx->oints.p, h, 4 * n_ints, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->stage_done, st));
    const int32_t *d = (const int32_t *)ctx->oints.p;
    float *maps = (float *)ctx->omaps.p;
    const size_t plane = (size_t)S * 3 * npix;
    launch_ssim_fwd(images, refs, d + o_ri, S, H, W, maps, maps + plane, maps + 2 * plane, (double *)ctx->opart.p,
                    st);
    launch_temporal(images, refs, d + o_ri, (const int2 *)(d + o_pt), n_pairs_t, H, W, (double *)ctx->otpart.p, chunks,
                    st);
    double *Dout = D ? D : (double *)ctx->oD.p;
    if (launch_objective((const double *)ctx->opart.p, nt, (const double *)ctx->otpart.p, chunks, n_pairs_t,
                         (const int2 *)(d + o_pm), n_pairs_m, d + o_an, n_anchors, S, 1.0 / (double)(npix * 3), prm,
                         Dout, (double *)ctx->oweight.p, loss, st) != 0)
        return fail(ctx, DGS_E_CUDA, "objective kernel attribute");
    if (dL_dimages)
        launch_objective_grad(images, refs, d + o_ri, S, H, W, maps, maps + plane, maps + 2 * plane,
                              (const double *)ctx->oweight.p, (float)prm.ssim_weight,
                              n_pairs_t ? (float)(prm.lambda_t / (double)n_pairs_t) : 0.0f, d + o_to,
                              (const int2 *)(d + o_tl), dL_dimages, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

}  // extern "C"

namespace {

// Eq. 3 distortion of every state against its view's complete render (one batch).
// View groups with at least this many states take the tile-reuse pass.
constexpr int SHARE_MIN_STATES = 8;

// Squared-error partials of states [0, S_user) with rendered tiles reused
// across states (share.cu): rounds of grouping, rendering one state per group
// on the explicit work list, and resolving the rest, until no pair of (view
// group tile, state) is pending.  Writes exactly the partials the plain pass
// writes, bit for bit.
int shared_mse_pass(dgs_ctx *ctx, const dgs_scene *scene, const Plan &p, const Lists &L, RasterArgs a,
                    cudaStream_t st)
{
    const uint32_t T = p.tiles, nvt = (uint32_t)((size_t)p.V * T);
    const int C = scene->n_clusters;
    const int G = 1;
    // states of each view group, in state order; pairs per view-group tile
    std::vector<int32_t> cnt(p.V, 0), vg_first(p.V + 1, 0), order(p.S_user);
    for (int s = 0; s < p.S_user; ++s) ++cnt[p.vg_of_state[s]];
    for (int v = 0; v < p.V; ++v) vg_first[v + 1] = vg_first[v] + cnt[v];
    {
        std::vector<int32_t> fill(vg_first.begin(), vg_first.end() - 1);
        for (int s = 0; s < p.S_user; ++s) order[fill[p.vg_of_state[s]]++] = s;
    }
    std::vector<uint32_t> vt_off(nvt + 1, 0);
    unsigned long long np = 0;
    for (uint32_t vt = 0; vt < nvt; ++vt) {
        vt_off[vt] = (uint32_t)np;
        np += (unsigned long long)cnt[vt / T];
    }
    if (np >= 0x7fffffffull) return fail(ctx, DGS_E_CAPACITY, "too many (tile, state) pairs for tile reuse");
    const size_t n0 = (size_t)np;
    vt_off[nvt] = (uint32_t)np;
    if (n0 == 0) return DGS_OK;
    // tables: vt_off | vg_first | order
    const size_t tab_words = (size_t)nvt + 1 + (size_t)p.V + 1 + (size_t)p.S_user;
    TRY(ensure(ctx, ctx->shtab, 4 * tab_words, st));
    TRY(ensure_stage(ctx, 4 * tab_words, st));
    CK(cudaEventSynchronize(ctx->stage_done));
    {
        char *h = (char *)ctx->h_stage;
        std::memcpy(h, vt_off.data(), 4 * ((size_t)nvt + 1));
        std::memcpy(h + 4 * ((size_t)nvt + 1), vg_first.data(), 4 * ((size_t)p.V + 1));
        std::memcpy(h + 4 * ((size_t)nvt + 1 + p.V + 1), order.data(), 4 * (size_t)p.S_user);
        CK(cudaMemcpyAsync(ctx->shtab.p, h, 4 * tab_words, cudaMemcpyHostToDevice, st));
        CK(cudaEventRecord(ctx->stage_done, st));
    }
    const uint32_t *d_vt_off = (const uint32_t *)ctx->shtab.p;
    const int32_t *d_vg_first = (const int32_t *)(d_vt_off + nvt + 1);
    const int32_t *d_order = d_vg_first + p.V + 1;
    // buffers
    const size_t pair_bytes = 9 * n0 + 64;                 // vt, state (u32) and K (u8)
    TRY(ensure(ctx, ctx->shord, 8 * (size_t)nvt * SHARE_ORDER, st));
    TRY(ensure(ctx, ctx->shpair, pair_bytes, st));
    TRY(ensure(ctx, ctx->shpair2, pair_bytes, st));
    TRY(ensure(ctx, ctx->shrep, 4 * n0, st));
    TRY(ensure(ctx, ctx->shflag, 4 * n0, st));
    TRY(ensure(ctx, ctx->shpos, 4 * n0, st));
    TRY(ensure(ctx, ctx->shlist, 8 * n0, st));
    TRY(ensure(ctx, ctx->shitem, 8 * n0, st));
    TRY(ensure(ctx, ctx->shkey, 8 * n0, st));
    TRY(ensure(ctx, ctx->shstop, 4 * (size_t)p.S_user * T, st));
    TRY(ensure(ctx, ctx->shseg, 2 * sizeof(uint2) * (size_t)nvt, st));
    TRY(ensure(ctx, ctx->shcnt, 64, st));
    TRY(ensure(ctx, ctx->scanws, scan_workspace_bytes(n0), st));
    TRY(ensure(ctx, ctx->counter, 16, st));
    uint32_t *ord_c = (uint32_t *)ctx->shord.p, *ord_fp = ord_c + (size_t)nvt * SHARE_ORDER;
    auto pair_arrays = [&](Buf &b, uint32_t *&vt, uint32_t *&stt, uint8_t *&k) {
        vt = (uint32_t *)b.p;
        stt = vt + n0;
        k = (uint8_t *)(stt + n0);
    };
    uint32_t *pvt, *pst, *nvt_a, *nst;
    uint8_t *pk, *nk;
    pair_arrays(ctx->shpair, pvt, pst, pk);
    pair_arrays(ctx->shpair2, nvt_a, nst, nk);
    uint32_t *prep = (uint32_t *)ctx->shrep.p, *flag = (uint32_t *)ctx->shflag.p, *pos = (uint32_t *)ctx->shpos.p;
    uint32_t *lvt = (uint32_t *)ctx->shlist.p, *lst = lvt + n0;
    uint32_t *ifirst = (uint32_t *)ctx->shitem.p, *icount = ifirst + n0;
    unsigned long long *keys = (unsigned long long *)ctx->shkey.p;
    uint2 *seg = (uint2 *)ctx->shseg.p, *seg2 = seg + nvt;
    uint32_t *dcnt = (uint32_t *)ctx->shcnt.p;   // [0] pending pairs, [1] render list, [2] items, [3] next pending
    const uint8_t *depth = (const uint8_t *)ctx->depth.p;

    launch_first_clusters((const Rec *)ctx->recs.p, L.evals, (const uint2 *)ctx->ranges.p, nvt, C, ord_c, ord_fp, ctx->sms, st);
    launch_pairs_init(d_vt_off, nvt, (uint32_t)n0, T, d_vg_first, d_order, pvt, pst, pk, ctx->sms, st);
    ctx->h_small[8] = (uint32_t)n0;
    CK(cudaMemcpyAsync(dcnt, ctx->h_small + 8, 4, cudaMemcpyHostToDevice, st));
    a.stop = (uint32_t *)ctx->shstop.p;
    size_t n = n0;
    ctx->reuse_pairs = (long long)n0;
    ctx->reuse_rendered = 0;
    ctx->reuse_rounds = 0;
    for (int round = 0; n > 0; ++round) {
        if (round > SHARE_MAX_K + 2) return fail(ctx, DGS_E_CUDA, "tile reuse did not converge");
        // group the pending pairs of every tile; representatives render
        CK(cudaMemsetAsync(seg, 0, sizeof(uint2) * nvt, st));
        launch_segments(pvt, dcnt + 0, n, seg, ctx->sms, st);
        launch_share_group(seg, nvt, pvt, pst, pk, dcnt + 0, n, ord_c, depth, C, keys, prep, ctx->sms, st);
        launch_rep_flags(pst, prep, dcnt + 0, n, flag, ctx->sms, st);
        CK(exclusive_scan_u32(flag, pos, n, dcnt + 1, ctx->scanws.p, st));
        launch_compact_pairs(flag, pos, dcnt + 0, n, pvt, pst, nullptr, lvt, lst, nullptr, ctx->sms, st);
        CK(cudaMemcpyAsync(ctx->h_small + 9, dcnt + 1, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const size_t nl = ctx->h_small[9];
        ctx->reuse_rendered += (long long)nl;
        ctx->reuse_rounds = round + 1;
        if (nl > 0) {
            CK(cudaMemsetAsync(seg2, 0, sizeof(uint2) * nvt, st));
            launch_segments(lvt, dcnt + 1, nl, seg2, ctx->sms, st);
            launch_item_lists(lvt, seg2, dcnt + 1, nl, G, flag, pos, dcnt + 2, ctx->scanws.p, ifirst, icount,
                              ctx->sms, st);
            CK(cudaMemsetAsync(ctx->counter.p, 0, 4, st));
            WorkQueue q{};
            q.counter = (uint32_t *)ctx->counter.p;
            q.item_first = ifirst;
            q.item_count = icount;
            q.list_vt = lvt;
            q.list_state = lst;
            q.n_items_dev = dcnt + 2;
            launch_raster_fwd(a, q, G, ctx->sms, st);
        }
        // everyone else: take the representative's partial, or regroup
        launch_share_resolve(pvt, pst, pk, prep, dcnt + 0, n, p.geom(), ord_c, ord_fp, depth, C, a.stop, a.partial, flag,
                             ctx->sms, st);
        CK(exclusive_scan_u32(flag, pos, n, dcnt + 3, ctx->scanws.p, st));
        launch_compact_pairs(flag, pos, dcnt + 0, n, pvt, pst, pk, nvt_a, nst, nk, ctx->sms, st);
        CK(cudaMemcpyAsync(dcnt + 0, dcnt + 3, 4, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->h_small + 9, dcnt + 3, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        n = ctx->h_small[9];
        std::swap(pvt, nvt_a);
        std::swap(pst, nst);
        std::swap(pk, nk);
    }
    CK(cudaGetLastError());
    return DGS_OK;
}

int utility_pass(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                 int n_cams, const float *bg, double *mse, double *psnr, cudaStream_t st)
{
    Plan p;
    TRY(build_plan(ctx, states, cams, n_cams, true, p));
    if (p.S_user > 0 && !mse) return fail(ctx, DGS_E_INVALID_ARG, "mse is null");
    ctx->tape.valid = false;
    if (p.S_user == 0) return DGS_OK;
    Lists L;
    TRY(prepare(ctx, scene, states->masks, p, true, st, L));
    uint32_t *sorted = L.evals;
    const size_t img = (size_t)p.W * p.H * 3;
    TRY(ensure(ctx, ctx->refs, sizeof(float) * img * (size_t)p.V, st));
    TRY(ensure(ctx, ctx->partial, sizeof(double) * (size_t)p.S_user * p.blocks, st));
    // complete renders of every view group (appended states S_user .. S-1)
    RasterArgs r = raster_args(ctx, p, scene->n_clusters, bg, sorted);
    r.images = (float *)ctx->refs.p;
    r.img_s0 = p.S_user;
    TRY(fwd_pass(ctx, scene, p, L, r, p.S_user, p.S, st));
    // every state: fused FP64 squared error against its view's complete render
    RasterArgs a = raster_args(ctx, p, scene->n_clusters, bg, sorted);
    a.refs = (const float *)ctx->refs.p;
    a.ref_of_state = (const int32_t *)ctx->vgos.p;
    a.partial = (double *)ctx->partial.p;
    int maxper = 0;
    {
        std::vector<int> cnt(p.V, 0);
        for (int s = 0; s < p.S_user; ++s) maxper = std::max(maxper, ++cnt[p.vg_of_state[s]]);
    }
    if (ctx->tile_reuse && maxper >= SHARE_MIN_STATES) {
        TRY(shared_mse_pass(ctx, scene, p, L, a, st));
    } else {
        ctx->reuse_pairs = ctx->reuse_rendered = (long long)p.S_user * p.tiles;
        ctx->reuse_rounds = 0;
        TRY(fwd_pass(ctx, scene, p, L, a, 0, p.S_user, st));
    }
    launch_mse_reduce((const double *)ctx->partial.p, p.S_user, (int)p.blocks, 1.0 / (double)img, mse, psnr, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

}  // namespace

extern "C" {

int dgs_debug_tile_lists(dgs_ctx *ctx, uint32_t *n_rec, uint32_t *n_ent, int32_t *n_view_groups,
                         uint32_t *tiles, uint32_t *recs, uint32_t *depth_keys, uint32_t *depth_slots,
                         uint32_t *entry_keys, uint32_t *entry_vals, uint32_t *ranges, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (!ctx->tape.valid) return fail(ctx, DGS_E_INVALID_ARG, "no forward call to export");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const Tape &tp = ctx->tape;
    if (n_rec) *n_rec = tp.lists.nRec;
    if (n_ent) *n_ent = tp.lists.nEnt;
    if (n_view_groups) *n_view_groups = tp.plan.V;
    if (tiles) *tiles = tp.plan.tiles;
    const size_t nr = tp.lists.nRec, ne = tp.lists.nEnt, nrg = (size_t)tp.plan.V * tp.plan.tiles;
    if (recs && nr) CK(cudaMemcpyAsync(recs, ctx->recs.p, sizeof(Rec) * nr, cudaMemcpyDeviceToDevice, st));
    const size_t nl = tp.lists.nLive;   // the sort dropped the culled records: 0xFFFFFFFF after the live ones
    if (depth_keys && nr) {
        CK(cudaMemsetAsync(depth_keys, 0xff, 4 * nr, st));
        if (nl) CK(cudaMemcpyAsync(depth_keys, tp.lists.depth_keys, 4 * nl, cudaMemcpyDeviceToDevice, st));
    }
    if (depth_slots && nr) {
        CK(cudaMemsetAsync(depth_slots, 0xff, 4 * nr, st));
        if (nl) CK(cudaMemcpyAsync(depth_slots, tp.lists.depth_slots, 4 * nl, cudaMemcpyDeviceToDevice, st));
    }
    if (entry_keys && ne) CK(cudaMemcpyAsync(entry_keys, tp.lists.ekeys, 4 * ne, cudaMemcpyDeviceToDevice, st));
    if (entry_vals && ne) CK(cudaMemcpyAsync(entry_vals, tp.lists.evals, 4 * ne, cudaMemcpyDeviceToDevice, st));
    if (ranges && nrg) CK(cudaMemcpyAsync(ranges, ctx->ranges.p, sizeof(uint2) * nrg, cudaMemcpyDeviceToDevice, st));
    return DGS_OK;
}

int dgs_set_tile_reuse(dgs_ctx *ctx, int enable)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    ctx->tile_reuse = enable != 0;
    return DGS_OK;
}

int dgs_set_tile_size(dgs_ctx *ctx, int size)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (size != 0 && size != 16 && size != 32) return fail(ctx, DGS_E_INVALID_ARG, "tile size must be 0, 16 or 32");
    ctx->tile_size = size;
    return DGS_OK;
}

int dgs_set_memory_budget(dgs_ctx *ctx, uint64_t bytes)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    ctx->mem_budget = (size_t)bytes;
    return DGS_OK;
}

int dgs_memory_stats(const dgs_ctx *ctx, uint64_t *workspace_bytes, int64_t *batch_splits)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (workspace_bytes) *workspace_bytes = ctx->ws_bytes;
    if (batch_splits) *batch_splits = ctx->chunk_splits;
    return DGS_OK;
}

int dgs_last_tile_size(const dgs_ctx *ctx, int32_t *tile_px)
{
    if (!ctx || !tile_px) return DGS_E_INVALID_ARG;
    *tile_px = ctx->last_shift ? 1 << ctx->last_shift : 0;
    return DGS_OK;
}

int dgs_tile_reuse_stats(const dgs_ctx *ctx, int64_t *pairs, int64_t *rendered, int32_t *rounds)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    if (pairs) *pairs = ctx->reuse_pairs;
    if (rendered) *rendered = ctx->reuse_rendered;
    if (rounds) *rounds = ctx->reuse_rounds;
    return DGS_OK;
}

int dgs_image_mse(dgs_ctx *ctx, const float *images, const float *refs, const int32_t *ref_index, int S, int n_refs,
                  int H, int W, float weight, double *mse, double *psnr, float *dL_dimages, dgs_stream stream)
{
    if (!ctx) return DGS_E_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (S < 0 || H < 1 || W < 1 || n_refs < 1) return fail(ctx, DGS_E_INVALID_ARG, "bad sizes");
    if (S == 0) return DGS_OK;
    if (!images || !refs || !ref_index || !mse) return fail(ctx, DGS_E_INVALID_ARG, "null argument");
    for (int s = 0; s < S; ++s)
        if (ref_index[s] < 0 || ref_index[s] >= n_refs)
            return fail(ctx, DGS_E_INVALID_ARG, "ref_index[%d] = %d out of range", s, ref_index[s]);
    const size_t per = (size_t)H * W * 3;
    const int parts = mse_parts(H, W);
    TRY(ensure(ctx, ctx->refidx, sizeof(int32_t) * (size_t)S, st));
    TRY(ensure(ctx, ctx->partial, sizeof(double) * (size_t)S * parts, st));
    TRY(ensure_stage(ctx, sizeof(int32_t) * (size_t)S, st));
    CK(cudaEventSynchronize(ctx->stage_done));   // an earlier copy may still read h_stage
    std::memcpy(ctx->h_stage, ref_index, sizeof(int32_t) * (size_t)S);
    CK(cudaMemcpyAsync(ctx->refidx.p, ctx->h_stage, sizeof(int32_t) * (size_t)S, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->stage_done, st));
    launch_image_mse(images, refs, (const int32_t *)ctx->refidx.p, S, H, W, weight, (double *)ctx->partial.p, parts,
                     dL_dimages, st);
    launch_mse_reduce((const double *)ctx->partial.p, S, parts, 1.0 / (double)per, mse, psnr, st);
    CK(cudaGetLastError());
    return DGS_OK;
}


int dgs_arena_create(dgs_ctx *ctx, dgs_arena **out)
{
    if (!ctx || !out) return DGS_E_INVALID_ARG;
    *out = nullptr;
    CK(cudaSetDevice(ctx->device));
    dgs_arena *A = new dgs_arena();
    A->ws.device = ctx->device;
    A->ws.sms = ctx->sms;
    if (cudaMallocHost((void **)&A->ws.h_small, 64 + 4 * (MAX_CLUSTERS + 1)) != cudaSuccess ||
        cudaEventCreateWithFlags(&A->ws.stage_done, cudaEventDisableTiming) != cudaSuccess) {
        if (A->ws.h_small) cudaFreeHost(A->ws.h_small);
        delete A;
        return fail(ctx, DGS_E_OOM, "arena host allocation failed");
    }
    *out = A;
    return DGS_OK;
}

int dgs_arena_destroy(dgs_arena *A)
{
    if (!A) return DGS_OK;
    if (A->plans > 0) return DGS_E_INVALID_ARG;
    free_ctx_buffers(&A->ws);
    delete A;
    return DGS_OK;
}

int dgs_plan_create(dgs_ctx *ctx, const dgs_scene *scene, const dgs_states *states, const dgs_camera *cams,
                    int n_cams, const float *bg, int mode, const int32_t *ref_index, int n_refs,
                    float entry_headroom, dgs_arena *arena, dgs_plan **out)
{
    if (!ctx || !out) return DGS_E_INVALID_ARG;
    *out = nullptr;
    CK(cudaSetDevice(ctx->device));
    TRY(check_scene(ctx, scene));
    if (!bg) return fail(ctx, DGS_E_INVALID_ARG, "bg is null");
    if (mode != DGS_PLAN_RENDER && mode != DGS_PLAN_UTILITY) return fail(ctx, DGS_E_INVALID_ARG, "bad plan mode");
    if (!states) return fail(ctx, DGS_E_INVALID_ARG, "states is null");
    {   // the tile size of this shape: fixed, tuned by earlier calls, or tuned now by the same context call
        const auto key = tile_key(mode == DGS_PLAN_RENDER ? TUNE_RENDER : TUNE_UTILITY, scene, states, cams, n_cams);
        if (known_shift(ctx, key) < 0 && states->n_states > 0 && cams && n_cams > 0) {
            const size_t img = (size_t)cams[0].width * cams[0].height * 3;
            void *tmp = nullptr;
            const size_t bytes = mode == DGS_PLAN_RENDER ? sizeof(float) * img * (size_t)states->n_states
                                                         : sizeof(double) * (size_t)states->n_states;
            if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, DGS_E_OOM, "plan tuning buffer");
            }
            const int rt = tuned_call(ctx, key, 0, [&] {
                return mode == DGS_PLAN_RENDER
                           ? render_batched(ctx, scene, states, cams, n_cams, bg, (float *)tmp, 0)
                           : utility_pass(ctx, scene, states, cams, n_cams, bg, (double *)tmp, nullptr, 0);
            });
            CK(cudaDeviceSynchronize());
            cudaFree(tmp);
            if (rt != DGS_OK) return rt;
        }
        const int sh = known_shift(ctx, key);
        ctx->active_shift = sh >= 0 ? sh : MIN_TILE_SHIFT;
    }
    Plan p;
    TRY(build_plan(ctx, states, cams, n_cams, mode == DGS_PLAN_UTILITY, p));
    if (p.S_user < 1) return fail(ctx, DGS_E_INVALID_ARG, "a plan needs at least one state");
    if (ref_index) {
        if (n_refs < 1) return fail(ctx, DGS_E_INVALID_ARG, "n_refs < 1");
        for (int s = 0; s < p.S_user; ++s)
            if (ref_index[s] < 0 || ref_index[s] >= n_refs)
                return fail(ctx, DGS_E_INVALID_ARG, "ref_index[%d] out of range", s);
    }
    if (!(entry_headroom >= 1.0f)) entry_headroom = 1.25f;
    if (arena && arena->ws.device != ctx->device) return fail(ctx, DGS_E_INVALID_ARG, "arena is on another device");
    dgs_plan *P = new dgs_plan();
    dgs_ctx *own = &P->ws;
    own->device = ctx->device;
    own->sms = ctx->sms;
    P->arena = arena;
    P->sc = arena ? &arena->ws : own;
    dgs_ctx *w = P->sc;             // scratch: sizing runs, capacities, tuning
    if (cudaMallocHost((void **)&own->h_small, 64 + 4 * (MAX_CLUSTERS + 1)) != cudaSuccess ||
        cudaEventCreateWithFlags(&own->stage_done, cudaEventDisableTiming) != cudaSuccess) {
        dgs_plan_destroy(P);
        return fail(ctx, DGS_E_OOM, "plan host allocation failed");
    }
    P->p = p;
    P->scene = *scene;
    P->bg[0] = bg[0]; P->bg[1] = bg[1]; P->bg[2] = bg[2];
    P->mode = mode;
    cudaStream_t st = 0;
    int r = DGS_OK;
    do {
        // exact record capacity: each state adds at most one depth per cluster
        std::vector<int> per(p.V, 0);
        for (int s = 0; s < p.S; ++s) ++per[p.vg_of_state[s]];
        unsigned long long rc = 0;
        for (int v = 0; v < p.V; ++v) rc += (unsigned long long)scene->n * (unsigned long long)std::min(per[v], scene->n_layers);
        if (rc >= 0x7fffffffull) { r = fail(ctx, DGS_E_CAPACITY, "record capacity exceeds 32 bits"); break; }
        P->R_cap = (uint32_t)std::max<unsigned long long>(rc, 1);
        // sizing run on the given masks (synchronous), then capacities
        Lists L0;
        if ((r = prepare(w, scene, states->masks, p, mode == DGS_PLAN_UTILITY, st, L0)) != DGS_OK) break;
        unsigned long long ec = (unsigned long long)((double)L0.nEnt * entry_headroom) + 65536ull;
        if (ec >= 0x7fffffffull) ec = 0x7ffffffeull;
        P->E_cap = (uint32_t)ec;
        const size_t vt = (size_t)p.V * p.tiles, R = P->R_cap, E = P->E_cap;
        if ((r = ensure(w, w->recs, sizeof(Rec) * R, st)) != DGS_OK) break;
        Buf *rb[] = {&w->k0, &w->v0, &w->k1, &w->v1};
        for (Buf *b : rb) if ((r = ensure(w, *b, 4 * R, st)) != DGS_OK) break;
        if (r != DGS_OK) break;
        if ((r = ensure(w, w->tcount, 4 * (R + 1), st)) != DGS_OK) break;
        if ((r = ensure(w, w->bins, sizeof(uint4) * (R + 1), st)) != DGS_OK) break;
        if ((r = ensure(w, w->toffs, 4 * (R + 1), st)) != DGS_OK) break;
        if ((r = ensure(w, w->live, 4 * ((size_t)p.V + 1), st)) != DGS_OK) break;
        Buf *eb[] = {&w->ek0, &w->ev0, &w->ek1, &w->ev1};
        for (Buf *b : eb) if ((r = ensure(w, *b, 4 * E, st)) != DGS_OK) break;
        if (r != DGS_OK) break;
        const size_t big = std::max(std::max(R, E), vt) + 1;
        if ((r = ensure(w, w->sortws, radix_workspace_bytes(big, p.V), st)) != DGS_OK) break;
        if ((r = ensure(w, w->scanws, scan_workspace_bytes(big), st)) != DGS_OK) break;
        if ((r = ensure(w, w->icnt, 4 * (vt + 1), st)) != DGS_OK) break;
        if ((r = ensure(w, w->ioff, 4 * (vt + 1), st)) != DGS_OK) break;
        if ((r = ensure(w, w->counter, 16, st)) != DGS_OK) break;
        if ((r = ensure(w, P->cnts, 16, st)) != DGS_OK) break;
        CK(cudaMemset(P->cnts.p, 0, 16));
        if (mode == DGS_PLAN_RENDER && (r = ensure(w, w->recgrad, sizeof(float4) * 3 * R, st)) != DGS_OK) break;
        if (mode == DGS_PLAN_RENDER && scene->affine &&
            (r = ensure(w, w->recgmu, sizeof(float) * 3 * (R + 1), st)) != DGS_OK) break;
        if (mode == DGS_PLAN_RENDER && scene->res_mode == 2 && scene->n_layers > 1 &&
            (r = ensure(w, w->gqws, sizeof(float) * (size_t)(scene->n_layers - 1) * scene->n * scene_dev(scene).K,
                        st)) != DGS_OK) break;
        const size_t img = (size_t)p.W * p.H * 3;
        if (mode == DGS_PLAN_UTILITY) {
            if ((r = ensure(w, w->refs, sizeof(float) * img * p.V, st)) != DGS_OK) break;
            if ((r = ensure(w, w->partial, sizeof(double) * (size_t)p.S_user * p.blocks, st)) != DGS_OK) break;
        }
        if (ref_index) {
            P->n_refs = n_refs;
            P->image_parts = mse_parts(p.H, p.W);
            if ((r = ensure(own, own->refidx, 4 * (size_t)p.S_user, st)) != DGS_OK) break;
            CK(cudaMemcpy(own->refidx.p, ref_index, 4 * (size_t)p.S_user, cudaMemcpyHostToDevice));
            if ((r = ensure(w, w->partial, sizeof(double) * (size_t)p.S_user *
                                               std::max<size_t>(P->image_parts, p.blocks), st)) != DGS_OK) break;
        }
        // Growing the workspace above reallocated buffers the sizing run's lists
        // point into: prepare again so every list lives in the final buffers,
        // then tune states-per-block on it and upload the tables.
        if ((r = prepare(w, scene, states->masks, p, mode == DGS_PLAN_UTILITY, st, L0)) != DGS_OK) break;
        CK(cudaDeviceSynchronize());
        if (arena) {   // the plan's own copies of its view-group tables (the arena's are overwritten by others)
            if ((r = ensure(own, own->vgs, sizeof(ViewGroup) * (size_t)p.V, st)) != DGS_OK) break;
            if ((r = ensure(own, own->vgos, sizeof(int32_t) * (size_t)p.S, st)) != DGS_OK) break;
            CK(cudaMemcpy(own->vgs.p, w->vgs.p, sizeof(ViewGroup) * (size_t)p.V, cudaMemcpyDeviceToDevice));
            CK(cudaMemcpy(own->vgos.p, w->vgos.p, sizeof(int32_t) * (size_t)p.S, cudaMemcpyDeviceToDevice));
        }
        RasterArgs a = raster_args(w, p, scene->n_clusters, P->bg, L0.evals);
        if (mode == DGS_PLAN_RENDER) {
            float *tmp = nullptr;
            if (cudaMalloc(&tmp, sizeof(float) * img * p.S_user) != cudaSuccess) {
                cudaGetLastError();
                r = fail(ctx, DGS_E_OOM, "plan tuning buffer");
                break;
            }
            a.images = tmp;
            r = fwd_pass(w, scene, p, L0, a, 0, p.S_user, st);
            CK(cudaDeviceSynchronize());
            cudaFree(tmp);
            if (r != DGS_OK) break;
            if ((r = upload_tabs(P, P->qfwd, 0, p.S_user,
                                 tuned_choice(w, scene, p, 0, p.S_user, true, false), P->tfwd)) != DGS_OK) break;
        } else {
            RasterArgs rr = a;
            rr.images = (float *)w->refs.p;
            rr.img_s0 = p.S_user;
            if ((r = fwd_pass(w, scene, p, L0, rr, p.S_user, p.S, st)) != DGS_OK) break;
            a.refs = (const float *)w->refs.p;
            a.ref_of_state = (const int32_t *)w->vgos.p;
            a.partial = (double *)w->partial.p;
            if ((r = fwd_pass(w, scene, p, L0, a, 0, p.S_user, st)) != DGS_OK) break;
            if ((r = upload_tabs(P, P->qref, p.S_user, p.S, 1, P->tref)) != DGS_OK) break;
            if ((r = upload_tabs(P, P->qfwd, 0, p.S_user,
                                 tuned_choice(w, scene, p, 0, p.S_user, false, true), P->tfwd)) != DGS_OK) break;
        }
        CK(cudaDeviceSynchronize());
    } while (0);
    if (r != DGS_OK) {
        if (!w->err.empty()) ctx->err = w->err;
        dgs_plan_destroy(P);
        return r;
    }
    if (arena) ++arena->plans;
    *out = P;
    return DGS_OK;
}

void dgs_plan_destroy(dgs_plan *P)
{
    if (!P) return;
    cudaSetDevice(P->ws.device);
    cudaDeviceSynchronize();
    Buf *own[] = {&P->cnts, &P->qfwd, &P->qref};
    for (Buf *b : own)
        if (b->p) cudaFree(b->p);
    free_ctx_buffers(&P->ws);          // with an arena: only the plan's tables live here
    if (P->arena) {
        --P->arena->plans;
        if (P->arena->last == P) P->arena->last = nullptr;
    }
    delete P;
}

const char *dgs_plan_last_error(const dgs_plan *P) { return P ? P->sc->err.c_str() : "null plan"; }

int dgs_plan_render(dgs_plan *P, const uint32_t *masks, float *images, dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (P->mode != DGS_PLAN_RENDER) return plan_fail(P, DGS_E_INVALID_ARG, "plan was not made for rendering");
    if (!masks || !images) return plan_fail(P, DGS_E_INVALID_ARG, "masks or images is null");
    dgs_ctx *ctx = P->sc;
    CK(cudaSetDevice(P->ws.device));
    cudaStream_t st = (cudaStream_t)stream;
    TRY(prepare_dev(P, masks, false, st));
    RasterArgs a = plan_raster_args(P);
    a.images = images;
    TRY(launch_queue(ctx, P->p, P->L, a, P->tfwd, st));
    P->rendered = true;
    if (P->arena) P->arena->last = P;
    return DGS_OK;
}

int dgs_plan_render_mse(dgs_plan *P, const uint32_t *masks, float *images, const float *refs, float weight,
                        double *mse, double *psnr, float *dL_dimages, dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (P->mode != DGS_PLAN_RENDER) return plan_fail(P, DGS_E_INVALID_ARG, "plan was not made for rendering");
    if (P->n_refs < 1) return plan_fail(P, DGS_E_INVALID_ARG, "plan was made without ref_index");
    if (!masks || !images || !refs || !mse) return plan_fail(P, DGS_E_INVALID_ARG, "null argument");
    dgs_ctx *ctx = P->sc;
    CK(cudaSetDevice(P->ws.device));
    cudaStream_t st = (cudaStream_t)stream;
    TRY(prepare_dev(P, masks, false, st));
    RasterArgs a = plan_raster_args(P);
    a.images = images;
    a.refs = refs;
    a.ref_of_state = (const int32_t *)P->ws.refidx.p;
    a.partial = (double *)ctx->partial.p;
    a.dL = dL_dimages;
    const size_t npix = (size_t)P->p.W * P->p.H;
    a.gscale = (float)(2.0 * (double)weight / (double)(npix * 3));   // as dgs_plan_image_mse
    TRY(launch_queue(ctx, P->p, P->L, a, P->tfwd, st));
    launch_mse_reduce((const double *)ctx->partial.p, P->p.S_user, (int)P->p.blocks, 1.0 / (double)(npix * 3), mse,
                      psnr, st);
    CK(cudaGetLastError());
    P->rendered = true;
    if (P->arena) P->arena->last = P;
    return DGS_OK;
}

int dgs_plan_backward(dgs_plan *P, const float *images, const float *dL_dimages, const dgs_scene_grad *grads,
                      dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (!P->rendered) return plan_fail(P, DGS_E_INVALID_ARG, "dgs_plan_backward needs a dgs_plan_render first");
    if (P->arena && P->arena->last != P)
        return plan_fail(P, DGS_E_INVALID_ARG, "another plan of the arena ran after this plan's render");
    if (!dL_dimages || !grads) return plan_fail(P, DGS_E_INVALID_ARG, "dL_dimages or grads is null");
    const dgs_scene *scene = &P->scene;
    if (!grads->mu0 || !grads->log_scale || !grads->quat || !grads->opacity_logit || !grads->colour ||
        (scene->temporal_rank > 0 && !grads->u) ||
        (scene->n_layers > 1 && scene->res_mode != 1 && !grads->res) || (scene->affine && !grads->affine) ||
        (scene->n_layers > 1 && scene->res_mode == 2 && !grads->res_step))
        return plan_fail(P, DGS_E_INVALID_ARG, "gradient array is null");
    dgs_ctx *ctx = P->sc;
    CK(cudaSetDevice(P->ws.device));
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->recgrad.zeroed) {
        CK(cudaMemsetAsync(ctx->recgrad.p, 0, ctx->recgrad.cap, st));
        ctx->recgrad.zeroed = true;
    }
    ctx->recgrad.zeroed = false;
    RasterBwdArgs b;
    b.f = plan_raster_args(P);
    b.dL_dimg = dL_dimages;
    b.img_fwd = images;
    b.rec_grad = (float4 *)ctx->recgrad.p;
    launch_raster_bwd(b, ctx->sms, st);
    GradDev g;
    g.mu0 = grads->mu0; g.u = grads->u; g.ls = grads->log_scale; g.quat = grads->quat;
    g.logit = grads->opacity_logit; g.colour = grads->colour; g.res = grads->res;
    g.affine = grads->affine; g.rec_gmu = scene->affine ? (float *)ctx->recgmu.p : nullptr;
    g.res_step = grads->res_step; g.gq = scene->res_mode == 2 ? (float *)ctx->gqws.p : nullptr;
    launch_project_bwd(scene_dev(scene), (const ViewGroup *)P->ws.vgs.p, P->p.V, (const uint32_t *)ctx->need.p,
                       (const uint32_t *)ctx->recBase.p, (float4 *)ctx->recgrad.p, g, P->R_cap, ctx->sms, st);
    CK(cudaGetLastError());
    ctx->recgrad.zeroed = true;
    return DGS_OK;
}

int dgs_plan_utility(dgs_plan *P, const uint32_t *masks, double *mse, double *psnr, dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (P->mode != DGS_PLAN_UTILITY) return plan_fail(P, DGS_E_INVALID_ARG, "plan was not made for utility");
    if (!masks || !mse) return plan_fail(P, DGS_E_INVALID_ARG, "masks or mse is null");
    dgs_ctx *ctx = P->sc;
    CK(cudaSetDevice(P->ws.device));
    cudaStream_t st = (cudaStream_t)stream;
    TRY(prepare_dev(P, masks, true, st));
    if (P->arena) P->arena->last = P;
    RasterArgs r = plan_raster_args(P);
    r.images = (float *)ctx->refs.p;
    r.img_s0 = P->p.S_user;
    TRY(launch_queue(ctx, P->p, P->L, r, P->tref, st));
    RasterArgs a = plan_raster_args(P);
    a.refs = (const float *)ctx->refs.p;
    a.ref_of_state = (const int32_t *)P->ws.vgos.p;
    a.partial = (double *)ctx->partial.p;
    TRY(launch_queue(ctx, P->p, P->L, a, P->tfwd, st));
    launch_mse_reduce((const double *)ctx->partial.p, P->p.S_user, (int)P->p.blocks,
                      1.0 / (double)((size_t)P->p.W * P->p.H * 3), mse, psnr, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

int dgs_plan_image_mse(dgs_plan *P, const float *images, const float *refs, float weight, double *mse,
                       double *psnr, float *dL_dimages, dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (P->n_refs < 1) return plan_fail(P, DGS_E_INVALID_ARG, "plan was made without ref_index");
    if (!images || !refs || !mse) return plan_fail(P, DGS_E_INVALID_ARG, "null argument");
    dgs_ctx *ctx = P->sc;
    CK(cudaSetDevice(P->ws.device));
    cudaStream_t st = (cudaStream_t)stream;
    launch_image_mse(images, refs, (const int32_t *)P->ws.refidx.p, P->p.S_user, P->p.H, P->p.W, weight,
                     (double *)ctx->partial.p, P->image_parts, dL_dimages, st);
    launch_mse_reduce((const double *)ctx->partial.p, P->p.S_user, P->image_parts,
                      1.0 / (double)((size_t)P->p.W * P->p.H * 3), mse, psnr, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

int dgs_plan_set_objective(dgs_plan *P, const int32_t *pairs_t, int n_pairs_t, const int32_t *pairs_m,
                           int n_pairs_m, const int32_t *anchors, int n_anchors, const dgs_objective_params *params)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (P->n_refs < 1) return plan_fail(P, DGS_E_INVALID_ARG, "plan was made without ref_index");
    const int S = P->p.S_user;
    if (S < 1 || S > DGS_OBJECTIVE_MAX_STATES || n_pairs_t < 0 || n_pairs_m < 0 || n_anchors < 0)
        return plan_fail(P, DGS_E_INVALID_ARG, "bad sizes");
    if ((n_pairs_t && !pairs_t) || (n_pairs_m && !pairs_m) || (n_anchors && !anchors))
        return plan_fail(P, DGS_E_INVALID_ARG, "null pair or anchor list");
    for (int q = 0; q < 2 * n_pairs_t; ++q)
        if (pairs_t[q] < 0 || pairs_t[q] >= S) return plan_fail(P, DGS_E_INVALID_ARG, "temporal pair out of range");
    for (int q = 0; q < 2 * n_pairs_m; ++q)
        if (pairs_m[q] < 0 || pairs_m[q] >= S) return plan_fail(P, DGS_E_INVALID_ARG, "prefix pair out of range");
    for (int a = 0; a < n_anchors; ++a)
        if (anchors[a] < 0 || anchors[a] >= S) return plan_fail(P, DGS_E_INVALID_ARG, "anchor out of range");
    dgs_objective_params prm = {0.20, 0.30, 0.05, 0.10, 2.0, 0.50};
    if (params) prm = *params;
    if (!(prm.cvar_q >= 0.0 && prm.cvar_q <= 1.0)) return plan_fail(P, DGS_E_INVALID_ARG, "cvar_q outside [0, 1]");
    dgs_ctx *ctx = &P->ws, *own = ctx;   // (CK reports through ctx)
    CK(cudaSetDevice(own->device));
    // temporal neighbour lists as dgs_objective builds them
    std::vector<int32_t> toff(S + 1, 0), tl(4 * (size_t)n_pairs_t);
    for (int q = 0; q < n_pairs_t; ++q) { ++toff[pairs_t[2 * q] + 1]; ++toff[pairs_t[2 * q + 1] + 1]; }
    for (int s = 0; s < S; ++s) toff[s + 1] += toff[s];
    {
        std::vector<int32_t> fill(toff.begin(), toff.end() - 1);
        for (int q = 0; q < n_pairs_t; ++q) {
            const int i = pairs_t[2 * q], j = pairs_t[2 * q + 1];
            tl[2 * fill[i]] = j; tl[2 * fill[i] + 1] = -1; ++fill[i];
            tl[2 * fill[j]] = i; tl[2 * fill[j] + 1] = +1; ++fill[j];
        }
    }
    const size_t o_pt = 0, o_pm = o_pt + 2 * (size_t)n_pairs_t, o_tl = o_pm + 2 * (size_t)n_pairs_m;
    const size_t o_an = o_tl + tl.size(), o_to = o_an + n_anchors, n_ints = o_to + S + 1;
    std::vector<int32_t> h(n_ints);
    if (n_pairs_t) std::memcpy(h.data() + o_pt, pairs_t, 8 * (size_t)n_pairs_t);
    if (n_pairs_m) std::memcpy(h.data() + o_pm, pairs_m, 8 * (size_t)n_pairs_m);
    if (!tl.empty()) std::memcpy(h.data() + o_tl, tl.data(), 4 * tl.size());
    if (n_anchors) std::memcpy(h.data() + o_an, anchors, 4 * (size_t)n_anchors);
    std::memcpy(h.data() + o_to, toff.data(), 4 * (size_t)(S + 1));
    const size_t npix = (size_t)P->p.H * P->p.W;
    int tx;
    const int nt = objective_tiles(P->p.H, P->p.W, &tx);
    const int chunks = (int)((npix + 1023) / 1024);
    int r;
    if ((r = ensure(own, own->oints, 4 * n_ints + 16, 0)) != DGS_OK ||
        (r = ensure(own, own->omaps, sizeof(float) * 3 * (size_t)S * 3 * npix, 0)) != DGS_OK ||
        (r = ensure(own, own->opart, sizeof(double) * 2 * (size_t)S * nt, 0)) != DGS_OK ||
        (r = ensure(own, own->otpart, sizeof(double) * (size_t)(n_pairs_t > 0 ? n_pairs_t : 1) * chunks, 0)) != DGS_OK ||
        (r = ensure(own, own->oD, sizeof(double) * (size_t)S, 0)) != DGS_OK ||
        (r = ensure(own, own->oweight, sizeof(double) * (size_t)S, 0)) != DGS_OK)
        return plan_fail(P, r, own->err.c_str());
    CK(cudaMemcpy(own->oints.p, h.data(), 4 * n_ints, cudaMemcpyHostToDevice));
    if (objective_prepare() != 0) return plan_fail(P, DGS_E_CUDA, "objective kernel attribute");
    P->obj = true;
    P->obj_nt = n_pairs_t; P->obj_nm = n_pairs_m; P->obj_na = n_anchors;
    P->obj_pt = o_pt; P->obj_pm = o_pm; P->obj_tl = o_tl; P->obj_an = o_an; P->obj_to = o_to;
    P->obj_prm = prm;
    return DGS_OK;
}

int dgs_plan_objective(dgs_plan *P, const float *images, const float *refs, double *loss, double *D,
                       float *dL_dimages, dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    if (!P->obj) return plan_fail(P, DGS_E_INVALID_ARG, "dgs_plan_set_objective was not called");
    if (!images || !refs || !loss) return plan_fail(P, DGS_E_INVALID_ARG, "null argument");
    dgs_ctx *ctx = &P->ws, *own = ctx;   // (CK reports through ctx)
    CK(cudaSetDevice(own->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int S = P->p.S_user, H = P->p.H, W = P->p.W;
    const size_t npix = (size_t)H * W;
    int tx;
    const int nt = objective_tiles(H, W, &tx);
    const int chunks = (int)((npix + 1023) / 1024);
    const int32_t *d = (const int32_t *)own->oints.p;
    const int32_t *ridx = (const int32_t *)own->refidx.p;
    float *maps = (float *)own->omaps.p;
    const size_t plane = (size_t)S * 3 * npix;
    launch_ssim_fwd(images, refs, ridx, S, H, W, maps, maps + plane, maps + 2 * plane, (double *)own->opart.p, st);
    launch_temporal(images, refs, ridx, (const int2 *)(d + P->obj_pt), P->obj_nt, H, W, (double *)own->otpart.p,
                    chunks, st);
    double *Dout = D ? D : (double *)own->oD.p;
    if (launch_objective((const double *)own->opart.p, nt, (const double *)own->otpart.p, chunks, P->obj_nt,
                         (const int2 *)(d + P->obj_pm), P->obj_nm, d + P->obj_an, P->obj_na, S,
                         1.0 / (double)(npix * 3), P->obj_prm, Dout, (double *)own->oweight.p, loss, st) != 0)
        return plan_fail(P, DGS_E_CUDA, "objective kernel attribute");
    if (dL_dimages)
        launch_objective_grad(images, refs, ridx, S, H, W, maps, maps + plane, maps + 2 * plane,
                              (const double *)own->oweight.p, (float)P->obj_prm.ssim_weight,
                              P->obj_nt ? (float)(P->obj_prm.lambda_t / (double)P->obj_nt) : 0.0f, d + P->obj_to,
                              (const int2 *)(d + P->obj_tl), dL_dimages, st);
    CK(cudaGetLastError());
    return DGS_OK;
}

int dgs_plan_tile_size(const dgs_plan *P, int32_t *tile_px)
{
    if (!P || !tile_px) return DGS_E_INVALID_ARG;
    *tile_px = 1 << P->p.tile_shift;
    return DGS_OK;
}

int dgs_plan_status(dgs_plan *P, int64_t *n_records, int64_t *n_entries, dgs_stream stream)
{
    if (!P) return DGS_E_INVALID_ARG;
    dgs_ctx *ctx = &P->ws;
    CK(cudaSetDevice(P->ws.device));
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->h_small, P->cnts.p, 16, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n_records) *n_records = ctx->h_small[0];
    if (n_entries) *n_entries = ctx->h_small[1];
    if (ctx->h_small[3]) {
        CK(cudaMemsetAsync((uint32_t *)P->cnts.p + 3, 0, 4, st));
        return plan_fail(P, DGS_E_CAPACITY, "tile entries exceeded the plan's capacity: results are incomplete");
    }
    return DGS_OK;
}

}  // extern "C"
