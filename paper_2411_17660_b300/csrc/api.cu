// api.cu -- the C ABI of include/gsr.h: argument checks, the workspace
// layout, and the launch sequence of the forward and backward passes.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <new>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"

struct gsr_ctx {
    int tile = 16;
    uint32_t spin = gsr::kDefaultSpin;
    int flags = 0;
    int binning = GSR_BIN_TILE;
    int batch = 32;   // list entries a blend warp stages per round (32 or 64)
    int fwd_rows = 16;   // pixel rows of a forward blend warp's block (8, or 16 at tiles 16 and 32)
    int sm_count = 0;
    std::string err;
    struct Rec {
        const void *ws;
        size_t bytes;
        int N, V, deg;
        int tile, binning;   // the configuration that rendered it (gsr_autotune changes the context's)
        std::vector<int> dims;
        bool median;   // the forward recorded the median-depth contributors
        bool surfels;  // the forward rendered surfels
    };
    std::vector<Rec> recs;  // recent forwards, for the backward's checks
    // caller-provided stage events (gsr_set_stage_events), 0..9
    bool timing = false;
    cudaEvent_t ev[GSR_STAGE_EVENTS] = {};
    void mark(int slot, cudaStream_t st) {
        if (timing && ev[slot]) cudaEventRecord(ev[slot], st);
    }
};

namespace gsr {
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// NVTX ranges around a call and each of its stages, for timeline tools and
// ncu's --nvtx filters; a stage's range ends where the next one begins, and
// all close on every return.  Without an attached tool the calls do nothing.
struct CallTrace {
    bool stage_open = false;
    explicit CallTrace(const char *call) { nvtxRangePushA(call); }
    void stage(const char *name) {
        if (stage_open) nvtxRangePop();
        nvtxRangePushA(name);
        stage_open = true;
    }
    ~CallTrace() {
        if (stage_open) nvtxRangePop();
        nvtxRangePop();
    }
};

struct Layout {
    size_t hdr, counts, offsets, scan_partials, rec, rec4, rec5, radius, aux;
    size_t keys0, keys1, vals0, vals1, hist, tile_cursor, tile_order, order_bins, lookback, ranges, T_final, last, median,
        vg_grads, pose_partials;
    size_t total;
    uint64_t VN;
    uint32_t cap, lb_tiles, scan_blocks, pose_blocks, total_pixels, total_tiles;
    int tbits;   // bits of a global tile id
};

void make_layout(int N, const gsr_view *views, int V, int tile, size_t cap, Layout &L) {
    L.VN = (uint64_t)V * (uint64_t)N;
    uint64_t px = 0, tiles = 0;
    for (int v = 0; v < V; ++v) {
        px += (uint64_t)views[v].H * views[v].W;
        tiles += (uint64_t)((views[v].W + tile - 1) / tile) * ((views[v].H + tile - 1) / tile);
    }
    L.total_pixels = (uint32_t)px;
    L.total_tiles = (uint32_t)tiles;
    int tbits = 1;
    while ((1ull << tbits) < tiles) ++tbits;
    L.tbits = tbits;
    L.cap = (uint32_t)cap;
    L.lb_tiles = (uint32_t)((cap + kSortTile - 1) / kSortTile);
    L.scan_blocks = (uint32_t)((L.VN + kScanChunk - 1) / kScanChunk);
    if (L.scan_blocks == 0) L.scan_blocks = 1;
    L.pose_blocks = (uint32_t)((N + 31) / 32);   // one pose partial per 32-Gaussian block
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.hdr = take(sizeof(WsHeader));
    L.counts = take(4 * L.VN);
    L.offsets = take(4 * L.VN);
    L.scan_partials = take(8ull * L.scan_blocks);
    L.rec = take(64 * L.VN);
    L.rec4 = take(16 * L.VN);
    L.rec5 = take(16 * L.VN);
    L.radius = take(4 * L.VN);
    L.aux = take(8ull * L.total_pixels);
    L.hist = take(4ull * kMaxPasses * kRadix);
    L.ranges = take(8ull * L.total_tiles);
    L.tile_cursor = take(4ull * L.total_tiles);
    L.tile_order = take(4ull * L.total_tiles);
    L.order_bins = take(4ull * 2 * 33);
    L.T_final = take(4ull * L.total_pixels);
    L.last = take(4ull * L.total_pixels);
    L.median = take(4ull * L.total_pixels);
    L.vg_grads = take(4ull * kVGGradsMax * L.VN);
    L.pose_partials = take(24ull * V * (L.pose_blocks ? L.pose_blocks : 1));
    L.keys0 = take(8 * cap);
    L.keys1 = take(8 * cap);
    L.vals0 = take(4 * cap);
    L.vals1 = take(4 * cap);
    L.lookback = take(2ull * L.lb_tiles * kRadix * 4);
    L.total = o;
}

// Largest key capacity (a multiple of the sort tile) whose layout fits.
uint32_t capacity_for(int N, const gsr_view *views, int V, int tile, size_t bytes) {
    Layout L0;
    make_layout(N, views, V, tile, 0, L0);
    if (bytes <= L0.total + 8 * 256) return 0;
    const double per_key = 24.0 + 2.0 * kRadix * 4 / kSortTile;
    uint64_t cap = (uint64_t)((double)(bytes - L0.total - 8 * 256) / per_key);
    cap = cap / kSortTile * kSortTile;
    const uint64_t kMaxCap = ((1ull << 30) - 1) / kSortTile * kSortTile;
    if (cap > kMaxCap) cap = kMaxCap;
    while (cap > 0) {
        Layout L;
        make_layout(N, views, V, tile, cap, L);
        if (L.total <= bytes) break;
        cap -= kSortTile;
    }
    return (uint32_t)cap;
}

// Which key buffers the sort passes through and where the sorted ids end:
// radix, 8-bit passes over (tile, depth bits); per-tile, passes over the tile
// id only (or one bucket scatter), then each tile's words are sorted in
// shared memory.  Depends on the primitive, so it is set again for surfels.
void set_sort_plan(Ws &w, int tbits) {
    if (bucket_binning(w))
        w.passes = 1;   // the scatter writes keys[1]
    else
        w.passes = w.bin_tile ? (tbits + 7) / 8 : (32 + tbits + 7) / 8;
    w.sorted = w.vals[w.bin_tile ? (w.passes + 1) & 1 : w.passes & 1];
    // The blends take their tiles most keys first, so that the heaviest do not
    // trail the last wave (uneven, 19k tiles: 5.27 -> 5.12 ms per step);
    // with many tiles per SM there is little tail to save and the spatial
    // order keeps more of the records shared in L2 (outdoor, 261k tiles:
    // 45.32 ms unordered, 45.46 ordered).  The bucket grouping lists the
    // order itself; the other groupings list it after the ranges
    // (launch_tile_order).
    w.order_tiles = !w.surfels && w.total_tiles <= kOrderMaxTiles;
}

Ws make_ws(void *base, const Layout &L, int N, int V, const gsr_ctx &ctx) {
    char *b = static_cast<char *>(base);
    Ws w;
    w.hdr = reinterpret_cast<WsHeader *>(b + L.hdr);
    w.counts = reinterpret_cast<uint32_t *>(b + L.counts);
    w.offsets = reinterpret_cast<uint32_t *>(b + L.offsets);
    w.scan_partials = reinterpret_cast<unsigned long long *>(b + L.scan_partials);
    w.rec = reinterpret_cast<float4 *>(b + L.rec);
    w.radius = reinterpret_cast<float *>(b + L.radius);
    w.rec4 = reinterpret_cast<float4 *>(b + L.rec4);
    w.rec5 = reinterpret_cast<float4 *>(b + L.rec5);
    w.aux = reinterpret_cast<float *>(b + L.aux);
    w.surfels = 0;
    w.vg_stride = kVGGrads;
    w.keys[0] = reinterpret_cast<unsigned long long *>(b + L.keys0);
    w.keys[1] = reinterpret_cast<unsigned long long *>(b + L.keys1);
    w.vals[0] = reinterpret_cast<uint32_t *>(b + L.vals0);
    w.vals[1] = reinterpret_cast<uint32_t *>(b + L.vals1);
    w.bin_tile = ctx.binning == GSR_BIN_TILE;
    w.hist = reinterpret_cast<uint32_t *>(b + L.hist);
    w.tile_cursor = reinterpret_cast<uint32_t *>(b + L.tile_cursor);
    w.tile_order = reinterpret_cast<uint32_t *>(b + L.tile_order);
    w.order_bins = reinterpret_cast<uint32_t *>(b + L.order_bins);
    w.lookback = reinterpret_cast<uint32_t *>(b + L.lookback);
    w.ranges = reinterpret_cast<uint2 *>(b + L.ranges);
    w.T_final = reinterpret_cast<float *>(b + L.T_final);
    w.last = reinterpret_cast<uint32_t *>(b + L.last);
    w.median = reinterpret_cast<uint32_t *>(b + L.median);
    w.vg_grads = reinterpret_cast<float *>(b + L.vg_grads);
    w.pose_partials = reinterpret_cast<float *>(b + L.pose_partials);
    w.N = (uint32_t)N;
    w.V = (uint32_t)V;
    w.VN = (uint32_t)L.VN;
    w.cap = L.cap;
    w.lb_tiles = L.lb_tiles;
    w.scan_blocks = L.scan_blocks;
    w.pose_blocks = L.pose_blocks;
    w.total_pixels = L.total_pixels;
    w.total_tiles = L.total_tiles;
    w.spin_limit = ctx.spin;
    w.test_flags = ctx.flags;
    set_sort_plan(w, L.tbits);
    return w;
}

// Clears the header (all but its record of clean gradient rows, which ends
// it), the radix histograms of the sort, the bucket grouping's tile counters
// (tile_counts, when it runs) and the fused loss's scalar (loss, when there
// is one).
__global__ void __launch_bounds__(1024) init_header_kernel(WsHeader *h, uint32_t cap, uint32_t tiles, uint32_t *hist,
                                                           uint32_t *tile_counts, float *loss, uint32_t *order_bins) {
    uint32_t *p = reinterpret_cast<uint32_t *>(h);
    static_assert(offsetof(WsHeader, rows_clean) == sizeof(WsHeader) - 4 * kRowsCleanWords, "record ends the header");
    for (int i = threadIdx.x; i < (int)(sizeof(WsHeader) / 4) - kRowsCleanWords; i += blockDim.x) p[i] = 0u;
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) hist[i] = 0u;
    for (int i = threadIdx.x; i < 2 * 33; i += blockDim.x) order_bins[i] = 0u;
    if (tile_counts)
        for (uint32_t i = threadIdx.x; i < tiles; i += blockDim.x) tile_counts[i] = 0u;
    if (loss && threadIdx.x == 0) *loss = 0.f;
    __syncthreads();
    if (threadIdx.x == 0) {
        h->key_capacity = cap;
        h->tiles = tiles;
    }
}

void launch_init(const Ws &w, uint32_t cap, float *loss, cudaStream_t st) {
    init_header_kernel<<<1, 1024, 0, st>>>(w.hdr, cap, w.total_tiles, w.hist,
                                           bucket_binning(w) ? w.tile_cursor : nullptr, loss, w.order_bins);
}

gsr_status fail(gsr_ctx *ctx, gsr_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
gsr_status fail(gsr_ctx *ctx, gsr_status s, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

gsr_status cuda_fail(gsr_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, GSR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

gsr_status check_views(gsr_ctx *ctx, const gsr_view *views, int V, bool need_outputs) {
    if (!views) return fail(ctx, GSR_EINVAL, "views is NULL");
    if (V < 1 || V > GSR_MAX_VIEWS) return fail(ctx, GSR_EINVAL, "V=%d outside 1..%d", V, GSR_MAX_VIEWS);
    uint64_t px = 0;
    for (int v = 0; v < V; ++v) {
        const gsr_view &w = views[v];
        if (w.H < 1 || w.W < 1 || w.H > 16384 || w.W > 16384)
            return fail(ctx, GSR_EINVAL, "view %d: size %dx%d outside 1..16384", v, w.W, w.H);
        if (!(w.fx > 0.f) || !(w.fy > 0.f) || !std::isfinite(w.fx) || !std::isfinite(w.fy) ||
            !std::isfinite(w.cx) || !std::isfinite(w.cy))
            return fail(ctx, GSR_EINVAL, "view %d: intrinsics must be finite with fx, fy > 0", v);
        if (!w.T_cw) return fail(ctx, GSR_EINVAL, "view %d: T_cw is NULL", v);
        if (need_outputs && !w.color) return fail(ctx, GSR_EINVAL, "view %d: color output is NULL", v);
        px += (uint64_t)w.H * w.W;
    }
    if (px >= (1ull << 32)) return fail(ctx, GSR_EINVAL, "more than 2^32 pixels in the batch");
    return GSR_OK;
}

gsr_status check_gaussians(gsr_ctx *ctx, const gsr_gaussians *gs, int V) {
    if (!gs) return fail(ctx, GSR_EINVAL, "gaussians is NULL");
    if (gs->N < 0) return fail(ctx, GSR_EINVAL, "N=%d is negative", gs->N);
    if (gs->sh_degree < 0 || gs->sh_degree > 3) return fail(ctx, GSR_EINVAL, "sh_degree=%d outside 0..3", gs->sh_degree);
    if ((uint64_t)gs->N * (uint64_t)V >= (1ull << 31)) return fail(ctx, GSR_EINVAL, "N*V must be below 2^31");
    if (gs->N > 0 && (!gs->means || !gs->log_scales || !gs->quats || !gs->opacity_logits || !gs->sh))
        return fail(ctx, GSR_EINVAL, "a Gaussian parameter pointer is NULL");
    return GSR_OK;
}

GaussianPtrs gaussian_ptrs(const gsr_gaussians *gs) {
    GaussianPtrs g;
    g.N = gs->N;
    g.sh_degree = gs->sh_degree;
    g.means = gs->means;
    g.log_scales = gs->log_scales;
    g.quats = gs->quats;
    g.opacity_logits = gs->opacity_logits;
    g.sh = gs->sh;
    return g;
}

bool want_median(const gsr_view *views, int V) {
    for (int v = 0; v < V; ++v)
        if (views[v].median_depth) return true;
    return false;
}

void fill_views(ViewTable &vt, const gsr_view *views, const gsr_view_grad *grads, int V, int tile, int batch = 32,
                int fwd_rows = 16) {
    memset(&vt, 0, sizeof vt);
    vt.V = V;
    vt.tile = tile;
    vt.batch = batch;
    vt.fwd_rows = tile == 8 ? 8 : fwd_rows;
    uint32_t toff = 0, poff = 0;
    for (int v = 0; v < V; ++v) {
        ViewParams &p = vt.v[v];
        const gsr_view &w = views[v];
        p.H = w.H;
        p.W = w.W;
        p.fx = w.fx;
        p.fy = w.fy;
        p.cx = w.cx;
        p.cy = w.cy;
        p.T_cw = w.T_cw;
        p.color = w.color;
        p.depth = w.depth;
        p.alpha = w.alpha;
        p.median_depth = w.median_depth;
        p.normal = p.distortion = nullptr;
        p.d_normal = p.d_distortion = nullptr;
        if (grads) {
            p.d_color = grads[v].d_color;
            p.d_depth = grads[v].d_depth;
            p.d_alpha = grads[v].d_alpha;
            p.d_median_depth = grads[v].d_median_depth;
            p.d_pose = grads[v].d_pose;
        }
        p.tiles_x = (w.W + tile - 1) / tile;
        p.tiles_y = (w.H + tile - 1) / tile;
        p.tile_offset = toff;
        p.pixel_offset = poff;
        toff += (uint32_t)(p.tiles_x * p.tiles_y);
        poff += (uint32_t)(w.H * w.W);
    }
    vt.total_tiles = toff;
    vt.total_pixels = poff;
}

// The backward checks that its workspace holds a forward of the same
// Gaussians and views (and of the same kind).
void remember_forward(gsr_ctx *ctx, const void *ws_ptr, size_t ws_bytes, const gsr_gaussians *gs,
                      const gsr_view *views, int V, bool median, bool surfels) {
    gsr_ctx::Rec r{ws_ptr, ws_bytes, gs->N, V, gs->sh_degree, ctx->tile, ctx->binning, {}, median, surfels};
    for (int v = 0; v < V; ++v) {
        r.dims.push_back(views[v].H);
        r.dims.push_back(views[v].W);
    }
    for (auto it = ctx->recs.begin(); it != ctx->recs.end(); ++it)
        if (it->ws == ws_ptr) {
            ctx->recs.erase(it);
            break;
        }
    ctx->recs.push_back(r);
    if (ctx->recs.size() > 64) ctx->recs.erase(ctx->recs.begin());
}

const gsr_ctx::Rec *find_forward(gsr_ctx *ctx, const void *ws_ptr, size_t ws_bytes, const gsr_gaussians *gs,
                                 const gsr_view *views, int V) {
    const gsr_ctx::Rec *rec = nullptr;
    for (const auto &r : ctx->recs)
        if (r.ws == ws_ptr) rec = &r;
    bool match = rec && rec->bytes == ws_bytes && rec->N == gs->N && rec->V == V && rec->deg == gs->sh_degree &&
                 rec->tile == ctx->tile && rec->binning == ctx->binning;
    for (int v = 0; match && v < V; ++v)
        match = rec->dims[2 * v] == views[v].H && rec->dims[2 * v + 1] == views[v].W;
    return match ? rec : nullptr;
}

int sm_count(gsr_ctx *ctx) {
    if (ctx->sm_count == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            ctx->sm_count = n;
        else
            ctx->sm_count = 148;
    }
    return ctx->sm_count;
}

}  // namespace

void set_ctx_error(gsr_ctx *ctx, const char *msg) {
    if (ctx) ctx->err = msg;
}

}  // namespace gsr

using namespace gsr;

extern "C" {

gsr_status gsr_create(const gsr_config *cfg, gsr_ctx **out) {
    if (!out) return GSR_EINVAL;
    *out = nullptr;
    int tile = 16, flags = 0, binning = GSR_BIN_TILE, batch = 32, fwd_rows = 0;
    uint32_t spin = kDefaultSpin;
    if (cfg) {
        if (cfg->batch != 0 && cfg->batch != 32 && cfg->batch != 64) return GSR_EINVAL;
        if (cfg->batch != 0) batch = cfg->batch;
        if (cfg->fwd_rows != 0 && cfg->fwd_rows != 8 && cfg->fwd_rows != 16) return GSR_EINVAL;
        fwd_rows = cfg->fwd_rows;
        if (cfg->tile != 0) tile = cfg->tile;
        if (cfg->spin_limit != 0) spin = cfg->spin_limit;
        if (cfg->flags & ~GSR_TEST_STALL_SORT) return GSR_EINVAL;
        flags = cfg->flags;
        if (cfg->binning != GSR_BIN_TILE && cfg->binning != GSR_BIN_RADIX) return GSR_EINVAL;
        binning = cfg->binning;
    }
    if (tile != 8 && tile != 16 && tile != 32) return GSR_EINVAL;
    if (tile == 32 && batch == 64) return GSR_EINVAL;   // the blends' staging would exceed 48 KB of shared memory
    if (tile == 8 && fwd_rows == 16) return GSR_EINVAL;  // a tile of 8 rows holds no 16-row block
    if (fwd_rows == 0) fwd_rows = tile == 8 ? 8 : 16;
    gsr_ctx *c = new (std::nothrow) gsr_ctx;
    if (!c) return GSR_EINVAL;
    c->tile = tile;
    c->spin = spin;
    c->flags = flags;
    c->binning = binning;
    c->batch = batch;
    c->fwd_rows = fwd_rows;
    *out = c;
    return GSR_OK;
}

gsr_status gsr_destroy(gsr_ctx *ctx) {
    delete ctx;
    return GSR_OK;
}

gsr_status gsr_workspace_size(gsr_ctx *ctx, int N, const gsr_view *views, int V, size_t key_capacity, size_t *bytes) {
    if (!ctx || !bytes) return fail(ctx, GSR_EINVAL, "ctx and bytes must be non-NULL");
    gsr_status s = check_views(ctx, views, V, false);
    if (s != GSR_OK) return s;
    if (N < 0) return fail(ctx, GSR_EINVAL, "N=%d is negative", N);
    if (key_capacity == 0) {
        key_capacity = (size_t)8 * V * (size_t)N;
        if (key_capacity < (1u << 20)) key_capacity = 1u << 20;
    }
    key_capacity = (key_capacity + kSortTile - 1) / kSortTile * kSortTile;
    if (key_capacity >= (1u << 30)) return fail(ctx, GSR_EINVAL, "key_capacity must be below 2^30");
    Layout L;
    make_layout(N, views, V, ctx->tile, key_capacity, L);
    *bytes = L.total + 8 * 256;
    return GSR_OK;
}

namespace {

// The L1 loss that gsr_render_l1 fuses into the forward blend.
struct FusedL1 {
    const gsr_l1_view *targets;
    float color_weight, depth_weight;
    float *loss;
};

gsr_status render_impl(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V, const FusedL1 *l1,
                       void *ws_ptr, size_t ws_bytes, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    gsr_status s = check_views(ctx, views, V, true);
    if (s != GSR_OK) return s;
    if ((s = check_gaussians(ctx, gs, V)) != GSR_OK) return s;
    if (!ws_ptr || (reinterpret_cast<uintptr_t>(ws_ptr) & 255))
        return fail(ctx, GSR_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    const uint32_t cap = capacity_for(gs->N, views, V, ctx->tile, ws_bytes);
    if (cap == 0) return fail(ctx, GSR_EINVAL, "workspace of %zu bytes holds no tile keys", ws_bytes);
    Layout L;
    make_layout(gs->N, views, V, ctx->tile, cap, L);
    ViewTable vt;
    fill_views(vt, views, nullptr, V, ctx->tile, ctx->batch, ctx->fwd_rows);
    if (l1) {
        for (int v = 0; v < V; ++v) {
            vt.v[v].l1_target_color = l1->targets[v].target_color;
            vt.v[v].l1_target_depth = l1->targets[v].target_depth;
            vt.v[v].l1_d_color = l1->targets[v].d_color;
            vt.v[v].l1_d_depth = l1->targets[v].d_depth;
        }
        vt.l1_loss = l1->loss;
        vt.l1_color_weight = l1->color_weight;
        vt.l1_depth_weight = l1->depth_weight;
    }
    const Ws w = make_ws(ws_ptr, L, gs->N, V, *ctx);
    const GaussianPtrs gp = gaussian_ptrs(gs);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    CallTrace tr(l1 ? "gsr_render_l1" : "gsr_render");
    ctx->mark(0, st);
    tr.stage("preprocess");
    launch_init(w, cap, l1 ? l1->loss : nullptr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init");
    if ((e = launch_preprocess_fwd(vt, gp, w, sm_count(ctx), st)) != cudaSuccess) return cuda_fail(ctx, e, "preprocess");
    ctx->mark(1, st);
    tr.stage("scan+duplicate");
    if ((e = launch_scan_duplicate(vt, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "scan/duplicate");
    ctx->mark(2, st);
    tr.stage("sort");
    if ((e = launch_sort(w, sm_count(ctx), st)) != cudaSuccess) return cuda_fail(ctx, e, "sort");
    ctx->mark(3, st);
    tr.stage("ranges");
    if ((e = launch_ranges(w, sm_count(ctx), st)) != cudaSuccess) return cuda_fail(ctx, e, "ranges");
    ctx->mark(4, st);
    tr.stage("blend");
    if ((e = launch_blend_fwd(vt, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "blend");
    ctx->mark(5, st);

    remember_forward(ctx, ws_ptr, ws_bytes, gs, views, V, want_median(views, V), false);
    return GSR_OK;
}

}  // namespace

gsr_status gsr_render(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V, void *ws_ptr,
                      size_t ws_bytes, gsr_stream stream) {
    return render_impl(ctx, gs, views, V, nullptr, ws_ptr, ws_bytes, stream);
}

gsr_status gsr_render_l1(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V,
                         const gsr_l1_view *targets, float color_weight, float depth_weight, float *loss,
                         void *ws_ptr, size_t ws_bytes, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    if (!targets || !loss || !views || V < 1 || V > GSR_MAX_VIEWS)
        return fail(ctx, GSR_EINVAL, "targets, loss and views must be non-NULL and 1 <= V <= %d", GSR_MAX_VIEWS);
    for (int v = 0; v < V; ++v)
        if (!targets[v].target_color || !targets[v].d_color)
            return fail(ctx, GSR_EINVAL, "view %d: target_color and d_color must be non-NULL", v);
    const FusedL1 l1{targets, color_weight, depth_weight, loss};
    return render_impl(ctx, gs, views, V, &l1, ws_ptr, ws_bytes, stream);
}

gsr_status gsr_render_backward(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views,
                               const gsr_view_grad *grads, int V, const gsr_grads *out, void *ws_ptr,
                               size_t ws_bytes, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    gsr_status s = check_views(ctx, views, V, false);
    if (s != GSR_OK) return s;
    if ((s = check_gaussians(ctx, gs, V)) != GSR_OK) return s;
    if (!grads) return fail(ctx, GSR_EINVAL, "grads is NULL");
    if (!out || (gs->N > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh)))
        return fail(ctx, GSR_EINVAL, "an output gradient pointer is NULL");
    if (!out->densify_grad != !out->densify_count || !out->densify_grad != !out->densify_radius)
        return fail(ctx, GSR_EINVAL, "densify_grad, densify_count and densify_radius must be all NULL or all set");
    const gsr_ctx::Rec *rec = find_forward(ctx, ws_ptr, ws_bytes, gs, views, V);
    if (!rec || rec->surfels)
        return fail(ctx, GSR_ENOTREADY, "no forward with these Gaussians and views on this workspace");
    for (int v = 0; v < V; ++v)
        if (grads[v].d_median_depth && !rec->median)
            return fail(ctx, GSR_ENOTREADY, "view %d: a median-depth gradient needs a forward that rendered median depth", v);
    const uint32_t cap = capacity_for(gs->N, views, V, ctx->tile, ws_bytes);
    Layout L;
    make_layout(gs->N, views, V, ctx->tile, cap, L);
    ViewTable vt;
    fill_views(vt, views, grads, V, ctx->tile, ctx->batch, ctx->fwd_rows);
    const Ws w = make_ws(ws_ptr, L, gs->N, V, *ctx);
    const GaussianPtrs gp = gaussian_ptrs(gs);
    GradPtrs gout;
    gout.means = out->means;
    gout.log_scales = out->log_scales;
    gout.quats = out->quats;
    gout.opacity_logits = out->opacity_logits;
    gout.sh = out->sh;
    gout.accumulate = out->accumulate;
    gout.densify_grad = out->densify_grad;
    gout.densify_count = out->densify_count;
    gout.densify_radius = out->densify_radius;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // the per-pair gradient rows are zero here: cleared by the last backward
    // after reading them, or by the forward when the header did not record
    // them as clean (rows_known_clean in common.cuh)
    CallTrace tr("gsr_render_backward");
    ctx->mark(6, st);
    ctx->mark(7, st);
    tr.stage("blend backward");
    cudaError_t e;
    if ((e = launch_blend_bwd(vt, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "blend backward");
    ctx->mark(8, st);
    tr.stage("preprocess backward");
    if ((e = launch_preprocess_bwd(vt, gp, w, gout, st)) != cudaSuccess) return cuda_fail(ctx, e, "preprocess backward");
    ctx->mark(9, st);
    return GSR_OK;
}

gsr_status gsr_render_surfels(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views,
                              const gsr_surfel_out *extra, int V, void *ws_ptr, size_t ws_bytes, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    gsr_status s = check_views(ctx, views, V, true);
    if (s != GSR_OK) return s;
    if ((s = check_gaussians(ctx, gs, V)) != GSR_OK) return s;
    if (want_median(views, V)) return fail(ctx, GSR_EINVAL, "surfels render no median depth");
    if (!ws_ptr || (reinterpret_cast<uintptr_t>(ws_ptr) & 255))
        return fail(ctx, GSR_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    const uint32_t cap = capacity_for(gs->N, views, V, ctx->tile, ws_bytes);
    if (cap == 0) return fail(ctx, GSR_EINVAL, "workspace of %zu bytes holds no tile keys", ws_bytes);
    Layout L;
    make_layout(gs->N, views, V, ctx->tile, cap, L);
    ViewTable vt;
    fill_views(vt, views, nullptr, V, ctx->tile, ctx->batch, ctx->fwd_rows);
    if (extra)
        for (int v = 0; v < V; ++v) {
            vt.v[v].normal = extra[v].normal;
            vt.v[v].distortion = extra[v].distortion;
        }
    Ws w = make_ws(ws_ptr, L, gs->N, V, *ctx);
    w.surfels = 1;
    w.vg_stride = kVGGradsMax;
    set_sort_plan(w, L.tbits);
    const GaussianPtrs gp = gaussian_ptrs(gs);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    CallTrace tr("gsr_render_surfels");
    ctx->mark(0, st);
    tr.stage("preprocess");
    launch_init(w, cap, nullptr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init");
    if ((e = launch_surfel_preprocess_fwd(vt, gp, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "preprocess");
    ctx->mark(1, st);
    tr.stage("scan+duplicate");
    if ((e = launch_scan_duplicate(vt, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "scan/duplicate");
    ctx->mark(2, st);
    tr.stage("sort");
    if ((e = launch_sort(w, sm_count(ctx), st)) != cudaSuccess) return cuda_fail(ctx, e, "sort");
    ctx->mark(3, st);
    tr.stage("ranges");
    if ((e = launch_ranges(w, sm_count(ctx), st)) != cudaSuccess) return cuda_fail(ctx, e, "ranges");
    ctx->mark(4, st);
    tr.stage("blend");
    if ((e = launch_surfel_blend_fwd(vt, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "blend");
    ctx->mark(5, st);
    remember_forward(ctx, ws_ptr, ws_bytes, gs, views, V, false, true);
    return GSR_OK;
}

gsr_status gsr_render_surfels_backward(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views,
                                       const gsr_view_grad *grads, const gsr_surfel_grad *extra, int V,
                                       const gsr_grads *out, void *ws_ptr, size_t ws_bytes, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    gsr_status s = check_views(ctx, views, V, false);
    if (s != GSR_OK) return s;
    if ((s = check_gaussians(ctx, gs, V)) != GSR_OK) return s;
    if (!grads) return fail(ctx, GSR_EINVAL, "grads is NULL");
    if (!out || (gs->N > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh)))
        return fail(ctx, GSR_EINVAL, "an output gradient pointer is NULL");
    if (out->densify_grad || out->densify_count || out->densify_radius)
        return fail(ctx, GSR_EINVAL, "surfels produce no densification statistics");
    for (int v = 0; v < V; ++v)
        if (grads[v].d_median_depth) return fail(ctx, GSR_EINVAL, "surfels render no median depth");
    const gsr_ctx::Rec *rec = find_forward(ctx, ws_ptr, ws_bytes, gs, views, V);
    if (!rec || !rec->surfels)
        return fail(ctx, GSR_ENOTREADY, "no surfel forward with these Gaussians and views on this workspace");
    const uint32_t cap = capacity_for(gs->N, views, V, ctx->tile, ws_bytes);
    Layout L;
    make_layout(gs->N, views, V, ctx->tile, cap, L);
    ViewTable vt;
    fill_views(vt, views, grads, V, ctx->tile, ctx->batch, ctx->fwd_rows);
    if (extra)
        for (int v = 0; v < V; ++v) {
            vt.v[v].d_normal = extra[v].d_normal;
            vt.v[v].d_distortion = extra[v].d_distortion;
        }
    Ws w = make_ws(ws_ptr, L, gs->N, V, *ctx);
    w.surfels = 1;
    w.vg_stride = kVGGradsMax;
    set_sort_plan(w, L.tbits);
    const GaussianPtrs gp = gaussian_ptrs(gs);
    GradPtrs gout;
    gout.means = out->means;
    gout.log_scales = out->log_scales;
    gout.quats = out->quats;
    gout.opacity_logits = out->opacity_logits;
    gout.sh = out->sh;
    gout.accumulate = out->accumulate;
    gout.densify_grad = gout.densify_count = gout.densify_radius = nullptr;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    CallTrace tr("gsr_render_surfels_backward");
    ctx->mark(6, st);   // gradient rows are cleared by the forward and after use
    ctx->mark(7, st);
    tr.stage("blend backward");
    cudaError_t e;
    if ((e = launch_surfel_blend_bwd(vt, w, st)) != cudaSuccess) return cuda_fail(ctx, e, "blend backward");
    ctx->mark(8, st);
    tr.stage("preprocess backward");
    if ((e = launch_surfel_preprocess_bwd(vt, gp, w, gout, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "preprocess backward");
    ctx->mark(9, st);
    return GSR_OK;
}

gsr_status gsr_read_info(gsr_ctx *ctx, const void *ws, size_t ws_bytes, gsr_info *info, gsr_stream stream) {
    if (!ctx || !ws || !info || ws_bytes < sizeof(WsHeader)) return fail(ctx, GSR_EINVAL, "bad arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
    WsHeader h;
    e = cudaMemcpy(&h, ws, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read header");
    info->status = h.status;
    info->keys = h.keys > 0xffffffffull ? 0xffffffffu : (uint32_t)h.keys;
    info->key_capacity = h.key_capacity;
    info->tiles = h.tiles;
    info->pairs_contributing = h.pairs_contrib;
    info->pairs_visible = h.pairs_visible;
    info->pairs_backward = h.pairs_bwd > 0xffffffffull ? 0xffffffffu : (uint32_t)h.pairs_bwd;
    return GSR_OK;
}

gsr_status gsr_get_status(gsr_ctx *ctx, const void *ws, size_t ws_bytes, gsr_stream stream) {
    gsr_info info;
    const gsr_status s = gsr_read_info(ctx, ws, ws_bytes, &info, stream);
    return s != GSR_OK ? s : static_cast<gsr_status>(info.status);
}

namespace {

// Forward + backward of one tuning candidate on the caller's buffers: the
// rendered colour serves as its own upstream gradient.
gsr_status tune_step(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V, const gsr_grads *grads,
                     void *ws, size_t ws_bytes, gsr_stream stream) {
    gsr_view_grad vg[GSR_MAX_VIEWS];
    for (int v = 0; v < V; ++v) vg[v] = gsr_view_grad{views[v].color, nullptr, nullptr, nullptr, nullptr};
    gsr_status s = gsr_render(ctx, gs, views, V, ws, ws_bytes, stream);
    if (s != GSR_OK) return s;
    return gsr_render_backward(ctx, gs, views, vg, V, grads, ws, ws_bytes, stream);
}

}  // namespace

gsr_status gsr_autotune(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V, const gsr_grads *grads,
                        void *ws, size_t ws_bytes, int reps, gsr_tune_entry *entries, int max_entries,
                        int *n_entries, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    if (!grads || (max_entries > 0 && !entries) || max_entries < 0 || reps < 1 || reps > 100)
        return fail(ctx, GSR_EINVAL, "gsr_autotune: grads must be non-NULL, 1 <= reps <= 100, entries for max_entries");
    gsr_status s = check_views(ctx, views, V, true);
    if (s != GSR_OK) return s;
    if ((s = check_gaussians(ctx, gs, V)) != GSR_OK) return s;
    if (ctx->flags) return fail(ctx, GSR_EINVAL, "gsr_autotune: a context with test flags cannot be tuned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int tile0 = ctx->tile, binning0 = ctx->binning, batch0 = ctx->batch, rows0 = ctx->fwd_rows;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ctx, e, "gsr_autotune: event");
    }
    static const int kTiles[] = {8, 16, 32}, kBinnings[] = {GSR_BIN_TILE, GSR_BIN_RADIX}, kBatches[] = {32, 64},
                     kRows[] = {16, 8};
    int n = 0, best = -1;
    float best_ms = 0.f;
    int best_cfg[4] = {tile0, binning0, batch0, rows0};
    gsr_status first_fail = GSR_OK, hard = GSR_OK;
    for (int tile : kTiles)
        for (int binning : kBinnings)
            for (int batch : kBatches)
                for (int rows : kRows) {
                if (hard != GSR_OK || (tile == 32 && batch == 64)) continue;   // 32/64: not supported (shared memory)
                if (tile == 8 && rows == 16) continue;                          // no 16-row block in an 8-row tile
                ctx->tile = tile;
                ctx->binning = binning;
                ctx->batch = batch;
                ctx->fwd_rows = rows;
                gsr_tune_entry r{tile, binning, batch, rows, -1.f, GSR_OK};
                // the warm-up run also tells whether the keys fit this workspace
                gsr_status cs = tune_step(ctx, gs, views, V, grads, ws, ws_bytes, stream);
                gsr_info info{};
                if (cs == GSR_OK) cs = gsr_read_info(ctx, ws, ws_bytes, &info, stream);
                if (cs == GSR_OK) cs = static_cast<gsr_status>(info.status);
                for (int k = 0; cs == GSR_OK && k < reps; ++k) {
                    float ms = 0.f;
                    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { cs = cuda_fail(ctx, e, "gsr_autotune: record"); break; }
                    cs = tune_step(ctx, gs, views, V, grads, ws, ws_bytes, stream);
                    if (cs != GSR_OK) break;
                    if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                        (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
                        cs = cuda_fail(ctx, e, "gsr_autotune: timing");
                        break;
                    }
                    r.ms = k == 0 ? ms : std::min(r.ms, ms);
                }
                r.status = cs;
                if (cs != GSR_OK) {
                    r.ms = -1.f;
                    if (first_fail == GSR_OK) first_fail = cs;
                    if (cs == GSR_ECUDA) hard = cs;
                } else if (best < 0 || r.ms < best_ms) {
                    best = n;
                    best_ms = r.ms;
                    best_cfg[0] = tile;
                    best_cfg[1] = binning;
                    best_cfg[2] = batch;
                    best_cfg[3] = rows;
                }
                if (n < max_entries) entries[n] = r;
                ++n;
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_entries) *n_entries = std::min(n, max_entries);
    ctx->tile = best_cfg[0];
    ctx->binning = best_cfg[1];
    ctx->batch = best_cfg[2];
    ctx->fwd_rows = best_cfg[3];
    if (hard != GSR_OK) return hard;
    if (best < 0) return fail(ctx, first_fail, "gsr_autotune: no candidate ran (%s); grow the workspace",
                              gsr_status_string(first_fail));
    return GSR_OK;
}

gsr_status gsr_l1_loss(gsr_ctx *ctx, const gsr_view *views, const gsr_l1_view *targets, int V, float color_weight,
                       float depth_weight, float *loss, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    gsr_status s = check_views(ctx, views, V, true);
    if (s != GSR_OK) return s;
    if (!targets || !loss) return fail(ctx, GSR_EINVAL, "targets and loss must be non-NULL");
    for (int v = 0; v < V; ++v)
        if (!targets[v].target_color || !targets[v].d_color)
            return fail(ctx, GSR_EINVAL, "view %d: target_color and d_color must be non-NULL", v);
    ViewTable vt;
    fill_views(vt, views, nullptr, V, ctx->tile, ctx->batch, ctx->fwd_rows);
    CallTrace tr("gsr_l1_loss");
    cudaError_t e = launch_l1_loss(vt, targets, color_weight, depth_weight, loss, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "l1 loss");
    return GSR_OK;
}

gsr_status gsr_rgbd_loss(gsr_ctx *ctx, const gsr_view *views, const gsr_l1_view *targets, int V, float lambda1,
                         float lambda2, float *loss, gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    gsr_status s = check_views(ctx, views, V, true);
    if (s != GSR_OK) return s;
    if (!targets || !loss) return fail(ctx, GSR_EINVAL, "targets and loss must be non-NULL");
    if (!(lambda1 >= 0.f && lambda1 <= 1.f && lambda2 >= 0.f && lambda2 <= 1.f))
        return fail(ctx, GSR_EINVAL, "lambda1 and lambda2 must lie in [0, 1]");
    for (int v = 0; v < V; ++v)
        if (!targets[v].target_color || !targets[v].d_color)
            return fail(ctx, GSR_EINVAL, "view %d: target_color and d_color must be non-NULL", v);
    ViewTable vt;
    fill_views(vt, views, nullptr, V, ctx->tile, ctx->batch, ctx->fwd_rows);
    CallTrace tr("gsr_rgbd_loss");
    cudaError_t e = launch_rgbd_loss(vt, targets, lambda1, lambda2, loss, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rgbd loss");
    return GSR_OK;
}

gsr_status gsr_set_stage_events(gsr_ctx *ctx, void *const *events) {
    if (!ctx) return GSR_EINVAL;
    ctx->timing = events != nullptr;
    for (int k = 0; k < GSR_STAGE_EVENTS; ++k) ctx->ev[k] = events ? static_cast<cudaEvent_t>(events[k]) : nullptr;
    return GSR_OK;
}

const char *gsr_last_error(const gsr_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

const char *gsr_status_string(gsr_status s) {
    switch (s) {
        case GSR_OK: return "GSR_OK";
        case GSR_EINVAL: return "GSR_EINVAL";
        case GSR_ECAPACITY: return "GSR_ECAPACITY";
        case GSR_ECUDA: return "GSR_ECUDA";
        case GSR_ETIMEOUT: return "GSR_ETIMEOUT";
        case GSR_ENOTREADY: return "GSR_ENOTREADY";
        case GSR_EINTERNAL: return "GSR_EINTERNAL";
    }
    return "unknown";
}

int gsr_abi_version(void) { return GSR_ABI_VERSION; }

gsr_status gsr_density_workspace_size(gsr_ctx *ctx, int N, size_t *bytes) {
    if (!ctx || !bytes) return fail(ctx, GSR_EINVAL, "ctx and bytes must be non-NULL");
    if (N < 0) return fail(ctx, GSR_EINVAL, "N=%d is negative", N);
    *bytes = density_workspace_bytes(N);
    return GSR_OK;
}

}  // extern "C"

namespace {

// Shared checks of the density calls: Gaussians, the output arrays and the workspace.
gsr_status check_density(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_gaussians_out *out, int min_room,
                         const void *ws, size_t ws_bytes) {
    gsr_status s = check_gaussians(ctx, gs, 1);
    if (s != GSR_OK) return s;
    if (out) {
        if (out->N < min_room) return fail(ctx, GSR_EINVAL, "out has room for %d Gaussians, needs %d", out->N, min_room);
        if (out->N > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh))
            return fail(ctx, GSR_EINVAL, "an output array is NULL");
        if (out->means == gs->means || out->log_scales == gs->log_scales || out->quats == gs->quats ||
            out->opacity_logits == gs->opacity_logits || out->sh == gs->sh)
            return fail(ctx, GSR_EINVAL, "out must not be the input arrays");
    }
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < density_workspace_bytes(gs->N))
        return fail(ctx, GSR_EINVAL, "workspace must be 256-byte aligned and hold gsr_density_workspace_size bytes");
    return GSR_OK;
}

}  // namespace

extern "C" {

gsr_status gsr_densify_adc(gsr_ctx *ctx, const gsr_gaussians *gs, const float *grad, const float *count,
                           const float *radius, const float *split_normals, const gsr_adc_params *params,
                           const gsr_gaussians_out *out, int *out_count, void *ws, size_t ws_bytes,
                           gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    if (!gs || !params || !out || !out_count) return fail(ctx, GSR_EINVAL, "gs, params, out and out_count must be non-NULL");
    gsr_status s = check_density(ctx, gs, out, 0, ws, ws_bytes);
    if (s != GSR_OK) return s;
    if (gs->N > 0 && (!grad || !count || !split_normals || (params->max_screen_radius > 0.f && !radius)))
        return fail(ctx, GSR_EINVAL, "grad, count, split_normals (and radius with max_screen_radius) must be non-NULL");
    if (!(params->min_opacity > 0.f && params->min_opacity < 1.f) || !(params->split_scale > 0.f) ||
        !(params->max_screen_radius >= 0.f) || !(params->max_world_scale >= 0.f) || !(params->grad_threshold >= 0.f))
        return fail(ctx, GSR_EINVAL, "adc thresholds out of range");
    CallTrace tr("gsr_densify_adc");
    cudaError_t e = launch_densify_adc(gaussian_ptrs(gs), grad, count, radius, split_normals, *params, *out, out_count,
                                       ws, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GSR_OK : cuda_fail(ctx, e, "densify");
}

gsr_status gsr_mcmc_relocate(gsr_ctx *ctx, const gsr_gaussians *gs, const uint32_t *draws, float min_opacity,
                             const gsr_gaussians_out *out, int *relocated, void *ws, size_t ws_bytes,
                             gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    if (!gs || !out || !relocated) return fail(ctx, GSR_EINVAL, "gs, out and relocated must be non-NULL");
    gsr_status s = check_density(ctx, gs, out, gs->N, ws, ws_bytes);
    if (s != GSR_OK) return s;
    if (gs->N > 0 && !draws) return fail(ctx, GSR_EINVAL, "draws must be non-NULL");
    if (!(min_opacity > 0.f && min_opacity < 1.f)) return fail(ctx, GSR_EINVAL, "min_opacity must lie in (0, 1)");
    CallTrace tr("gsr_mcmc_relocate");
    cudaError_t e = launch_mcmc_relocate(gaussian_ptrs(gs), draws, min_opacity, *out, relocated, ws,
                                         reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GSR_OK : cuda_fail(ctx, e, "relocate");
}

gsr_status gsr_mcmc_noise(gsr_ctx *ctx, const gsr_gaussians *gs, const float *eta, float scale, float *means_out,
                          gsr_stream stream) {
    if (!ctx) return GSR_EINVAL;
    if (!gs) return fail(ctx, GSR_EINVAL, "gs must be non-NULL");
    gsr_status s = check_gaussians(ctx, gs, 1);
    if (s != GSR_OK) return s;
    if (gs->N > 0 && (!eta || !means_out)) return fail(ctx, GSR_EINVAL, "eta and means_out must be non-NULL");
    if (!std::isfinite(scale)) return fail(ctx, GSR_EINVAL, "scale must be finite");
    CallTrace tr("gsr_mcmc_noise");
    cudaError_t e = launch_mcmc_noise(gaussian_ptrs(gs), eta, scale, means_out, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GSR_OK : cuda_fail(ctx, e, "noise");
}

size_t gsr_abi_sizeof(int which) {
    switch (which) {
        case 0: return sizeof(gsr_config);
        case 1: return sizeof(gsr_gaussians);
        case 2: return sizeof(gsr_view);
        case 3: return sizeof(gsr_view_grad);
        case 4: return sizeof(gsr_grads);
        case 5: return sizeof(gsr_info);
        case 6: return sizeof(gsr_l1_view);
        case 7: return sizeof(gsr_surfel_out);
        case 8: return sizeof(gsr_surfel_grad);
        case 9: return sizeof(gsr_adc_params);
        case 10: return sizeof(gsr_gaussians_out);
        case 11: return sizeof(gsr_tune_entry);
    }
    return 0;
}

}  // extern "C"
