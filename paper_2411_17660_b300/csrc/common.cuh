// common.cuh -- constants, launch-parameter structs and small numeric helpers
// shared by the rasteriser kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

namespace gsr {

// ---------------------------------------------------------------- rules
// Readings of the rendering rules (3DGS conventions the paper inherits,
// Sec. 3.3): near plane, low-pass dilation, 3-sigma cutoff, alpha skip and
// clamp, transmittance stop, Jacobian clamp.
constexpr float kNearZ = 0.2f;
constexpr float kDilation = 0.3f;
constexpr float kCutoffD2 = 9.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kFovClamp = 1.3f;
// The blend works with s = 0.5*log2(e)*d^2, so exp(-d^2/2) = 2^-s.
constexpr float kHalfLog2e = 0.721347520444481703680f;      // 0.5 / ln 2
constexpr float kSqrtHalfLog2e = 0.849321800288019133f;     // sqrt(0.5 / ln 2)
// Scale of the blend backward's position and conic-factor sums (gradient
// row components 0..4): -2 ln 2 sqrt(0.5 / ln 2) = -sqrt(2 ln 2)
constexpr float kRowScale = -1.17741002251547466f;
constexpr float kLn2 = 0.693147180559945309417f;
constexpr float kLog2_255 = 7.99435343685885793f;           // log2(255)

constexpr int kMaxPasses = 8;     // 8-bit radix digits of a 64-bit key
constexpr int kRadix = 256;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 12;    // keys per thread per sort tile
constexpr int kLookBatch = 32;    // predecessor flags read per wide look-back round
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr int kVGGradsMax = 16;   // surfels: a, b (6), p_z, u_c, v_c, ln sigma, rgb, normal
constexpr int kVGGrads = 10;      // per (view, Gaussian) screen-space grads
constexpr uint32_t kDefaultSpin = 1u << 24;

// ---------------------------------------------------------------- params
struct ViewParams {
    int H, W;
    float fx, fy, cx, cy;
    const float *T_cw;
    float *color, *depth, *alpha, *median_depth;
    const float *d_color, *d_depth, *d_alpha, *d_median_depth;
    float *normal, *distortion;               // surfels only
    const float *d_normal, *d_distortion;     // surfels only
    float *d_pose;
    // L1 loss fused into the forward blend (gsr_render_l1); NULL otherwise
    const float *l1_target_color, *l1_target_depth;
    float *l1_d_color, *l1_d_depth;
    int tiles_x, tiles_y;
    uint32_t tile_offset;   // first global tile id of this view
    uint32_t pixel_offset;  // first pixel in the concatenated per-pixel buffers
};

// Passed by value (__grid_constant__) so that a captured CUDA graph replays
// it without any host-side copy.
struct ViewTable {
    int V;
    int tile;
    int batch;                // list entries a blend warp stages per round: 32 or 64
    int fwd_rows;             // pixel rows of a forward blend warp's block: 8 or 16 (16 needs tile >= 16)
    uint32_t total_tiles;
    uint32_t total_pixels;
    float *l1_loss;           // fused L1 loss: the device scalar it adds to, or NULL
    float l1_color_weight, l1_depth_weight;
    ViewParams v[GSR_MAX_VIEWS];
};

struct GaussianPtrs {
    int N, sh_degree;
    const float *means, *log_scales, *quats, *opacity_logits, *sh;
};

// Device-side state at the start of the workspace.
constexpr int kRowsCleanWords = 8;

struct WsHeader {
    int32_t status;                 // first device error (gsr_status)
    uint32_t key_capacity;
    uint32_t tiles;
    uint32_t sort_final;            // key buffer holding the sorted result
    unsigned long long keys;        // tile keys of all pairs: the scan's total, or the sum of the reservations
    unsigned long long pairs_contrib;
    uint32_t sort_counter[kMaxPasses];
    uint32_t bwd_groups;            // preprocess backward: groups taken (reset by the pose reduction)
    uint32_t pre_items;             // preprocess forward: work items taken (zeroed by the init kernel)
    uint32_t pairs_visible;         // (view, Gaussian) pairs with tile keys (records written), Gaussians only
    uint32_t order_counter;         // tile-order count kernel: blocks done (zeroed by the init kernel)
    unsigned long long pairs_bwd;   // checked builds: contributor pairs the blend backward took
    uint32_t pad[64 - 14 - kMaxPasses - kRowsCleanWords];
    // The layout whose screen-gradient rows are known to be all zero (tag,
    // byte offset of the rows in the workspace, N, V, row stride); kept by the
    // init kernel, see rows_known_clean below.
    uint32_t rows_clean[kRowsCleanWords];
};
static_assert(sizeof(WsHeader) == 256, "header must stay one 256-byte block");

// Typed views of one workspace; offsets come from the host layout code.
struct Ws {
    WsHeader *hdr;
    uint32_t *counts;        // [V*N] tiles touched by (view, Gaussian)
    uint32_t *offsets;       // [V*N] exclusive scan of counts
    unsigned long long *scan_partials;  // [scan_blocks]
    // [V*N][4] one 64-byte record per pair: rec[4i] (u_hi, v_hi, u_lo, v_lo),
    // rec[4i+1] (m00, m01, m11, s_max), rec[4i+2] (r, g, b, z), rec[4i+3]
    // (log2 opacity, Sxx, Sxy, Syy); a pair's record fills whole 32-byte
    // sectors, so writing the visible pairs' records never leaves a sector
    // partly written (which L2 would complete with a read from DRAM)
    float4 *rec;
    float *radius;           // [V*N] 3 sqrt(lambda_max(Sigma')) if the pair is visible for densification, else 0
    float4 *rec4;            // [V*N] surfels: (n_x, n_y, n_z, 0) normal towards the camera
    float4 *rec5;            // [V*N] surfels: (x_lo, y_lo, x_hi, y_hi) pixel bounds of the cutoff region
    float *aux;              // surfels: [2][total_pixels] sum w z, sum w z^2 of the forward
    int surfels;             // 1: records, tile coverage and gradient rows are the surfel ones
    uint32_t vg_stride;      // floats per (Gaussian, view) gradient row: 10, or 16 for surfels
    // Binning buffers, double-buffered by pass parity.  Radix: keys =
    // (tile << 32 | depth bits), vals = Gaussian id.  Per-tile: the u32 tile
    // keys live in vals[] and the (depth bits << 32 | Gaussian id) words in
    // keys[] (tile_keys / tile_words below).
    unsigned long long *keys[2];
    uint32_t *vals[2];
    uint32_t *sorted;        // [keys] Gaussian ids in (tile, depth, id) order
    int bin_tile;
    uint32_t *hist;          // [kMaxPasses][256]
    uint32_t *tile_cursor;   // [total_tiles] bucket binning: keys per tile, then each tile's next free slot
    uint32_t *tile_order;    // [total_tiles] the blends' launch order, most keys first
    uint32_t *order_bins;    // [2][33] tile counts by key-count bit length, then each bin's next slot
    int order_tiles;         // the blends take their tiles from tile_order
    uint32_t *lookback;      // [2][lb_tiles][256] look-back flags, by pass parity
    uint2 *ranges;           // [total_tiles] [start, end) in the sorted list
    float *T_final;          // [total_pixels]
    uint32_t *last;          // [total_pixels] list position where the pixel stopped, or its tile list's end
    uint32_t *median;        // [total_pixels] median-depth contributor index + 1 (0: none)
    float *vg_grads;         // [N][V][10] screen-space gradients of each (Gaussian, view)
    float *pose_partials;    // [V][pose_blocks][6]
    uint32_t N, V, VN;
    uint32_t cap, lb_tiles, scan_blocks, pose_blocks;
    uint32_t total_pixels, total_tiles;
    int passes;
    uint32_t spin_limit;
    int test_flags;
};

// Screen-gradient rows.  The blend backward accumulates into the rows of the
// visible pairs, which must start at zero; the preprocess backward clears
// every row it reads.  So between iterations on one layout the rows stay
// zero, and the forward clears them only when the header does not record
// this layout as clean: a fresh or foreign workspace, another layout (N, V,
// image sizes or key capacity moved the rows), surfel rows, or a backward
// whose preprocess half did not run.  The Gaussian blend forward records
// the layout once the preprocess has cleared (or found clean) the rows; the
// blend backward withdraws the record and the pose reduction after the
// preprocess backward restores it; the surfel forward withdraws it.
constexpr uint32_t kRowsCleanTag0 = 0x52c3e9a1u, kRowsCleanTag1 = 0x0d7b46f5u;

__device__ __forceinline__ void rows_clean_record(const Ws &ws, uint32_t (&d)[kRowsCleanWords]) {
    const unsigned long long off =
        (unsigned long long)(reinterpret_cast<const char *>(ws.vg_grads) - reinterpret_cast<const char *>(ws.hdr));
    d[0] = kRowsCleanTag0;
    d[1] = kRowsCleanTag1;
    d[2] = (uint32_t)off;
    d[3] = (uint32_t)(off >> 32);
    d[4] = ws.N;
    d[5] = ws.V;
    d[6] = ws.vg_stride;
    d[7] = 0u;
}

__device__ __forceinline__ bool rows_known_clean(const Ws &ws) {
    uint32_t d[kRowsCleanWords];
    rows_clean_record(ws, d);
    bool same = true;
#pragma unroll
    for (int k = 0; k < kRowsCleanWords; ++k) same &= ws.hdr->rows_clean[k] == d[k];
    return same;
}

// One thread records the layout as clean (or withdraws the record).
__device__ __forceinline__ void set_rows_clean(const Ws &ws, bool clean) {
    uint32_t d[kRowsCleanWords];
    rows_clean_record(ws, d);
#pragma unroll
    for (int k = 0; k < kRowsCleanWords; ++k) ws.hdr->rows_clean[k] = clean ? d[k] : 0u;
}

// Gaussians (not surfels) binned per tile emit their tile keys in the
// preprocess: each warp reserves its pairs' keys with one atomic on the key
// count.  Every tile's words are sorted completely afterwards, so the order
// in which the unsorted keys land does not matter.  The other paths place
// the keys by an exclusive scan of the tile counts.  (The surfel preprocess
// takes one Gaussian per thread, so a warp with one large surfel would emit
// its keys with one lane for every view: 0.054 -> 0.39 ms measured.)
__host__ __device__ __forceinline__ bool keys_in_preprocess(const Ws &w) { return w.bin_tile && !w.surfels; }

// With per-tile binning and at most kBucketMaxTiles tiles (a shared-memory
// counter each) the unsorted keys -- from the preprocess, or from the
// duplication for surfels -- are grouped by tile with counting kernels
// instead of the onesweep passes over the tile bits.
constexpr uint32_t kBucketMaxTiles = 1u << 15;
// Up to this many tiles the blends take them most keys first.
constexpr uint32_t kOrderMaxTiles = 1u << 16;
__host__ __device__ __forceinline__ bool bucket_binning(const Ws &w) {
    return w.bin_tile && w.total_tiles <= kBucketMaxTiles;
}

__device__ __forceinline__ void set_status(WsHeader *h, int code) {
    atomicCAS(reinterpret_cast<int *>(&h->status), 0, code);
}

// Checked builds (-DGSR_CHECKED; `python -m paper_2411_17660_b300.build
// --checked` makes libgsr_checked.so) verify the data-dependent indices of the
// kernels: a failed check records GSR_EINTERNAL in the status word and the
// caller skips the access, instead of trapping.  Release builds compile the
// checks out (the expression is then true).
#ifdef GSR_CHECKED
#define GSR_CHECK(hdr, ok) ((ok) || (set_status((hdr), GSR_EINTERNAL), false))
#else
#define GSR_CHECK(hdr, ok) true
#endif

// A tile's [start, end) range, checked against the sorted key count (empty
// when the check fails).
__device__ __forceinline__ uint2 checked_range(const uint2 *ranges, uint32_t tile, WsHeader *hdr, uint32_t cap) {
    uint2 r = ranges[tile];
    if (!GSR_CHECK(hdr, r.x <= r.y && r.y <= min(hdr->keys, (unsigned long long)cap))) r = make_uint2(0u, 0u);
    return r;
}

// ---------------------------------------------------------------- numerics
// Error-free transformations (Knuth TwoSum, FMA-based TwoProd) written with
// round-to-nearest intrinsics so that no contraction or reassociation can
// change them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// w.x + t with a compensated dot product (Ogita-Rump-Oishi Dot2): result as
// hi + lo, accurate to about one FP32 rounding of the exact value.
__device__ __forceinline__ void dot3_plus(float w0, float w1, float w2, float t, float x0, float x1,
                                          float x2, float &hi, float &lo) {
    float p, s, h, r, q;
    two_prod(w0, x0, p, s);
    two_prod(w1, x1, h, r);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
    two_prod(w2, x2, h, r);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
    two_sum(p, t, p, q);
    s = __fadd_rn(s, q);
    hi = __fadd_rn(p, s);
    lo = __fsub_rn(s, __fsub_rn(hi, p));
}

// f*(xh+xl)/(zh+zl) + c as hi + lo (double-float), for pixel coordinates
// whose fractional part must survive |u| up to thousands of pixels.  rz is
// an approximation of 1/zh (rcp.approx: within about one unit in the last
// place): the quotient's high part q1 = xh rz is then within a few units of
// xh/zh, the FMA forms its remainder xh - q1 zh with an error of about
// 2^-46 |xh| at most, and the low part q2 = remainder rz corrects q1, so
// q1 + q2 carries the quotient to about 2^-44 -- far below the 2^-24 of the
// pixel coordinate's low part.
__device__ __forceinline__ void project_coord(float f, float c, float xh, float xl, float zh, float zl, float rz,
                                              float &hi, float &lo) {
    const float q1 = __fmul_rn(xh, rz);
    float r = __fmaf_rn(-q1, zh, xh);          // remainder xh - q1*zh
    r = __fadd_rn(r, __fsub_rn(xl, __fmul_rn(q1, zl)));
    const float q2 = __fmul_rn(r, rz);
    float p, pe;
    two_prod(f, q1, p, pe);
    pe = __fmaf_rn(f, q2, pe);
    float s, se;
    two_sum(p, c, s, se);
    se = __fadd_rn(se, pe);
    hi = __fadd_rn(s, se);
    lo = __fsub_rn(se, __fsub_rn(hi, s));
}

// a*d - b*c with the FMA trick (Kahan): accurate even under cancellation.
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    const float w = __fmul_rn(b, c);
    const float e = __fmaf_rn(-b, c, w);
    const float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Relaxed GPU-scope accesses for inter-block flags.
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int view_of_tile(const ViewTable &vt, uint32_t tile) {
    int v = 0;
    while (v + 1 < vt.V && tile >= vt.v[v + 1].tile_offset) ++v;
    return v;
}

}  // namespace gsr
