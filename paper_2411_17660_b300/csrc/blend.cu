// blend.cu -- per-pixel front-to-back compositing (Sec. 3.3, Eq.
// "rendering": C = sum_i c_i alpha_i prod_{j<i}(1 - alpha_j)) and its
// back-to-front backward.
//
// One CTA of one warp per block of pixels of a screen tile (all views
// concatenated; the blocks of a tile are consecutive CTAs): 8x16 blocks
// (four pixels per lane) where the tile is that tall, else 8x8 blocks (two
// pixels per lane; also the forward's median-depth variant).
// Each warp walks its tile's depth-sorted list in chunks of 32 entries: the
// 32 lanes load one entry each, keep only the Gaussians whose cutoff ellipse
// reaches the warp's block (an exact convex minimum of d^2 over the block),
// compact the survivors into the warp's shared-memory slots with a ballot,
// and then every lane composites them for its pixels.  A warp leaves as soon
// as all its lanes have hit the transmittance stop; warps never wait for each
// other.
//
// The backward recomputes the blend state from the stored final
// transmittance and last contributor: walking back, T_i = T_{i+1}/(1-alpha_i)
// and the colour/depth behind each entry accumulate as B <- B(1-a) + c a.
// Per-Gaussian gradients of the pixels of a warp are summed in registers
// (four pixels per lane) and with a transposing warp butterfly before one set
// of global atomics per (warp, Gaussian); when at most four lanes touch a
// Gaussian they issue their atomics directly instead.
//
// A lane's pixels share their column: rows y, y + 4 (and y + 8, y + 12) form
// row pairs whose per-pixel terms run on packed FP32 pairs (fma.rn.f32x2, the
// same rounding as two scalar operations), and both kernels form s from the
// same linear forms, so the forward and the backward take bit-identical
// decisions.  The forward stages each entry as plain scalars (its shared
// loads would otherwise bound it); the backward stages duplicated operand
// pairs, so that one 128-bit shared load yields two ready register pairs.
// Both run their row pairs without branches.
#include <type_traits>

#include "kernels.cuh"

namespace gsr {

namespace {

// A warp covers a block of 8 columns and BH rows: lane (x, y), y < 4, owns
// the pixel rows y + 4 r of column x.  The forward's blocks are 8x8 (rows y
// and y + 4); the backward's are 8x16 where the tile allows.
constexpr int kSubW = 8, kSubH = 8, kRowStep = 4;
constexpr unsigned kFull = 0xffffffffu;

// A CTA is one warp with its block of 8 columns and BH rows; the blocks of a
// tile are consecutive CTAs, each reading the whole tile list.  A CTA's slot
// on the SM is then held only while its own warp works, not until the
// slowest warp of its tile finishes (window blend backward 0.2190 -> 0.2120
// ms against a CTA per tile of 16; at tile 32 against a CTA per 16 x 16 or
// per tile, uneven blend backward 1.525 -> 1.477, 1.590 ms).
template <int TS, int BH = kSubH>
struct BlendShape {
    static_assert(TS % kSubW == 0 && TS % BH == 0, "a tile holds whole warp blocks");
    static constexpr int CX = TS / kSubW;          // CTAs (warp blocks) per tile row
    static constexpr int CTAS = CX * (TS / BH);    // CTAs per tile
    static constexpr int WARPS = 1;
    static constexpr int THREADS = 32;
};

// s = 0.5 log2(e) d^2 = p1^2 + p2^2, with the Cholesky factor m of
// 0.5 log2(e) Sigma'^-1 and the mean at offset (ur, vr) from the origin of
// the pixel offsets (x, y): p1 = m00 (x - ur) + m01 (y - vr) = m00 x + m01 y + a
// and p2 = m11 (y - vr) = m11 y + b.  The constants a, b are formed once per
// staged entry; a pixel then needs three FMAs for p1, p2.  Round-to-nearest
// intrinsics throughout, so that the forward and the backward take
// bit-identical decisions.
__device__ __forceinline__ void lin_consts(float ur, float vr, float m00, float m01, float m11, float &a, float &b) {
    a = -__fmaf_rn(m01, vr, __fmul_rn(m00, ur));
    b = -__fmul_rn(m11, vr);
}

// Forward: staged entry of a warp's slot k, three float4 (no duplicated
// pairs: the blend forward is bound by the bytes its shared-memory loads
// deliver to the warp, 128 per clock and SM, so each entry is loaded once
// as plain scalars).
//   q0 = (m00, a, m01, m11)   Cholesky factor of 0.5 log2(e) Sigma'^-1, constant a
//   q1 = (b, s_max, l, list index as bits)   l = log2(opacity)
//   q2 = (r, g, b, z)
constexpr int kFwdQuads = 3;
// Backward: staged entry of a warp's slot k, five float4 of pairs and one
// float4, so that one 128-bit shared load yields two ready register pairs
// (the backward has arithmetic enough per entry that its shared loads are
// not what bounds it).
//   e0 = (-ur, -ur, -vr, -vr)  mean relative to the offsets' origin
//   e1 = (m00, m00, m01, m01)
//   e2 = (m11, m11, l, l)
//   e3 = (r, r, g, g), e4 = (b, b, z, z)
//   x  = (s_max, list index, Gaussian index, -)
constexpr int kBwdQuads = 5;

// Below this log2(opacity), 2^(log2(opacity) - s) stays under the 0.99
// alpha clamp for every s >= 0 even with ex2.approx's error (a relative
// 2^-21 at most against the 1.5e-5 margin), so the clamp is the identity.
constexpr float kLog2ClampFree = -0.01452f;   // log2(0.99) = -0.0144996, less 2e-5

// 1.0f where a <= b, else 0.0f (also for a NaN): one instruction that gives
// both the cutoff mask that scales alpha and the composited-pair count.
__device__ __forceinline__ float le_mask(float a, float b) {
    float r;
    asm("set.le.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

template <int R>
struct RowTag {
    static constexpr int value = R;
};

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// s of a lane's two pixels, at rows ly.x and ly.y of one column: t = m00 x +
// a (the same for both pixels) comes from the caller, once per entry.
__device__ __forceinline__ float2 pair_s2(float2 t, float2 ly, float2 m01, float2 m11, float2 b, float2 &p1,
                                          float2 &p2) {
    p1 = __ffma2_rn(m01, ly, t);
    p2 = __ffma2_rn(m11, ly, b);
    return __ffma2_rn(p1, p1, __fmul2_rn(p2, p2));
}

// Backward block height: 16 rows (two packed row pairs per lane) when the
// tile is at least that tall.
template <int TS>
struct BwdBlock {
    static constexpr int H = TS >= 16 ? 16 : kSubH;
    // resident blocks per SM asked of the compiler: 24 warps, 80 registers
    // (window: 0.2227 ms against 0.2306 with 28 warps at 72 registers, which
    // spill; the uncapped 115 registers, with their lower occupancy, were
    // slower still)
    static constexpr int MIN_BLOCKS = 768 / BlendShape<TS, H>::THREADS;
};

// Forward block height: 16 rows (two packed row pairs per lane) when the
// tile is at least that tall, as in the backward: the per-entry work that
// does not depend on the pixel (shared loads, the linear forms' constant,
// the stop vote, the loop) and the staging then serve twice the pixels.
// ROWS is the configured block height (gsr_config.fwd_rows: 16 shares each
// staged entry among twice the pixels, 8 evaluates fewer entries that reach
// no pixel; which is faster depends on the scene, so the autotuner picks).
// The median-depth variant keeps one row pair per lane: its per-pixel
// median state would not fit the registers of two.
template <int TS, bool MED, int ROWS>
struct FwdBlock {
    static constexpr int H = TS >= 16 && !MED && ROWS == 16 ? 16 : kSubH;
    // resident warps: 32 (64 registers) with two row pairs per lane, 36 (56
    // registers) with one
    static constexpr int WARPS_PER_SM = H == 16 ? 32 : 36;
    static constexpr int MIN_BLOCKS = WARPS_PER_SM * 32 / BlendShape<TS, H>::THREADS < 32
                                          ? WARPS_PER_SM * 32 / BlendShape<TS, H>::THREADS
                                          : 32;
};

// Whether min over the warp's block of pixel centres of s can reach s_max.
// s(dx, dy) = (m00 dx + m01 dy)^2 + (m11 dy)^2; for fixed dy the first term's
// minimum over dx in [dx0, dx1] is max(0, m00 dx0 + m01 dy, -(m00 dx1 + m01 dy))^2,
// a convex function of dy whose minimum over [dy0, dy1] lies at an end or at
// one of three stationary points, all clamped into the interval.
template <int BH>
__device__ __forceinline__ bool touches_block(float ur, float vr, float m00, float m01, float m11, float smax) {
    const float dx0 = -ur, dx1 = (float)(kSubW - 1) - ur;
    const float dy0 = -vr, dy1 = (float)(BH - 1) - vr;
    const float a0 = m00 * dx0, a1 = m00 * dx1;
    const float inv_den = rcp_approx(m01 * m01 + m11 * m11);   // m11 > 0
    auto f = [&](float dy) {
        const float t = m01 * dy;
        const float p = fmaxf(0.f, fmaxf(a0 + t, -(a1 + t)));
        const float q = m11 * dy;
        return p * p + q * q;
    };
    auto cl = [&](float y) { return fminf(fmaxf(y, dy0), dy1); };
    float smin = fminf(f(dy0), f(dy1));
    smin = fminf(smin, f(cl(0.f)));
    smin = fminf(smin, f(cl(-m01 * a0 * inv_den)));
    smin = fminf(smin, f(cl(-m01 * a1 * inv_den)));
    // tolerance for the rounding of both this minimum and the per-pixel s:
    // a few units in the last place of the largest term of the linear forms
    const float A = fabsf(m00) * fmaxf(fabsf(dx0), fabsf(dx1)) + (fabsf(m01) + fabsf(m11)) * fmaxf(fabsf(dy0), fabsf(dy1));
    return smin <= smax + 1e-3f * (1.f + smax) + 1e-2f + 0x1p-17f * A;
}

// One level of a transposing butterfly: L values per lane become ceil(L/2)
// values, each summed over the lane pair (lane, lane ^ LEVEL).  The lower
// lane keeps the first half, the upper lane the second (zero-padded).  The
// sums run two at a time on packed FP32 pairs.
template <int L, int LEVEL>
__device__ __forceinline__ void butterfly_level(const float *in, float *out, int lane) {
    constexpr int H = (L + 1) / 2;
    const bool hi = (lane & LEVEL) != 0;
    float keep[H], recv[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float lo_keep = in[i];
        const float hi_keep = (H + i < L) ? in[H + i] : 0.f;
        const float send = hi ? lo_keep : hi_keep;
        keep[i] = hi ? hi_keep : lo_keep;
        recv[i] = __shfl_xor_sync(kFull, send, LEVEL);
    }
#pragma unroll
    for (int i = 0; i + 1 < H; i += 2) {
        const float2 r = __fadd2_rn(make_float2(keep[i], keep[i + 1]), make_float2(recv[i], recv[i + 1]));
        out[i] = r.x;
        out[i + 1] = r.y;
    }
    if constexpr (H % 2 == 1) out[H - 1] = __fadd_rn(keep[H - 1], recv[H - 1]);
}

// Sums 10 per-lane values over the warp with 12 shuffles (instead of 50):
// afterwards lane l holds the total of component sum10_slot(l) (where that
// slot is valid), and its partner lane l^1 holds the same total.
__device__ __forceinline__ float warp_sum10(const float (&v)[kVGGrads], int lane) {
    static_assert(kVGGrads == 10, "butterfly is laid out for 10 values");
    float a[5], b[3], c[2];
    butterfly_level<10, 16>(v, a, lane);
    butterfly_level<5, 8>(a, b, lane);
    butterfly_level<3, 4>(b, c, lane);
    float d;
    butterfly_level<2, 2>(c, &d, lane);
    d += __shfl_xor_sync(kFull, d, 1);
    return d;
}

// The component that warp_sum10 leaves in lane `lane`, and whether it is one
// (the halving of 10 values leaves some lanes without a component); it
// depends on the lane alone, so callers form it once.
__device__ __forceinline__ void sum10_slot(int lane, int &comp, bool &valid) {
    int base = 0, left = 10;
    const int lev[4] = {16, 8, 4, 2}, half[4] = {5, 3, 2, 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (lane & lev[k]) {
            base += half[k];
            left = max(0, left - half[k]);
        } else {
            left = min(left, half[k]);
        }
    }
    comp = base;
    valid = left == 1;
}

// Both blends form a pixel's row offset from the mean relative to the last
// row above it that is a multiple of kRowOrigin (the first row of a 16-row
// band), whatever their own warp blocks: the forward's 8-row blocks and the
// backward's 16-row ones (or 8-row ones at tile 8) then form s with the same
// FP32 operations for every pixel, so the two kernels take the same
// decisions, at every tile size.
constexpr int kRowOrigin = 16;
__device__ __forceinline__ int row_origin(int Y0) { return Y0 - Y0 % kRowOrigin; }

struct WarpTile {
    int v;
    int X0, Y0;         // pixel of lane 0 (origin of the warp's block)
    int px, py;         // this lane's first pixel; the others sit kRowStep rows below
    uint2 range;
};

template <int TS, int BH = kSubH>
__device__ __forceinline__ WarpTile warp_tile(const ViewTable &vt, const Ws &ws) {
    using S = BlendShape<TS, BH>;
    WarpTile w;
    const uint32_t slot = blockIdx.x / S::CTAS, q = blockIdx.x % S::CTAS;   // tile slot, block in the tile
    uint32_t tile = slot;
    if (ws.order_tiles) {   // tiles with the most keys first (bucket scan or launch_tile_order)
        const uint32_t t = ws.tile_order[slot];
        tile = t < vt.total_tiles ? t : slot;
    }
    w.v = view_of_tile(vt, tile);
    const ViewParams &vp = vt.v[w.v];
    const uint32_t lt = tile - vp.tile_offset;
    const int tx = (int)(lt % (uint32_t)vp.tiles_x), ty = (int)(lt / (uint32_t)vp.tiles_x);
    const int lane = threadIdx.x & 31;
    w.X0 = tx * TS + (int)(q % S::CX) * kSubW;
    w.Y0 = ty * TS + (int)(q / S::CX) * BH;
    w.px = w.X0 + (lane & (kSubW - 1));
    w.py = w.Y0 + lane / kSubW;
    w.range = checked_range(ws.ranges, tile, ws.hdr, ws.cap);
    return w;
}

// Loads entries [base, base + 32 CH) of the tile list (lane-parallel: entry
// base + 32 k + lane on each lane, k < CH), tests each against the warp's
// block of BH rows and compacts the survivors into the warp's slots in list
// order; Stage writes one survivor's slot.  Returns the number of survivors.
// CH = 2 (the 64-entry batch) halves the staging rounds (and the warp's
// done tests between them), at the price of staging up to 64 entries past a
// warp's transmittance stop.
// vr is the mean's row offset from row Yr (the origin the per-pixel offsets
// are formed from); the block test takes it relative to the block's first
// row Y0 >= Yr.
template <int BH, int CH, typename Stage>
__device__ __forceinline__ int stage_chunk(const Ws &ws, const uint32_t *vals, size_t vN, uint32_t base, uint32_t end,
                                           int X0, int Y0, int Yr, Stage &&write) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t g[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        const uint32_t idx = base + 32u * k + lane;
        g[k] = idx < end ? vals[idx] : 0xffffffffu;
        if (idx < end) (void)GSR_CHECK(ws.hdr, g[k] < ws.N);   // a listed id >= N: only after another error
    }
    int n = 0;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        bool keep = false;
        float4 r1 = make_float4(0.f, 0.f, 0.f, 0.f);
        float ur = 0.f, vr = 0.f;
        if (g[k] < ws.N) {
            const float4 *rec = ws.rec + 4 * (vN + g[k]);
            const float4 r0 = rec[0];
            r1 = rec[1];
            ur = __fadd_rn(__fsub_rn(r0.x, (float)X0), r0.z);
            vr = __fadd_rn(__fsub_rn(r0.y, (float)Yr), r0.w);
            keep = touches_block<BH>(ur, Y0 == Yr ? vr : __fsub_rn(vr, (float)(Y0 - Yr)), r1.x, r1.y, r1.z, r1.w);
        }
        const unsigned ballot = __ballot_sync(kFull, keep);
        if (keep) {
            const float4 *rec = ws.rec + 4 * (vN + g[k]);
            write(n + __popc(ballot & lanemask_lt()), ur, vr, r1, rec[2], rec[3].x, base + 32u * k + lane, g[k]);
        }
        n += __popc(ballot);
    }
    __syncwarp();
    return n;
}

// MED: also record, per pixel, the median-depth contributor (the last one
// entered with transmittance above 0.5) and its depth.
// L1: the epilogue also takes the L1 loss terms of its pixels (gsr_render_l1),
// with the expressions of the stand-alone L1 kernel, so that the gradients
// match it bit for bit.
//
// A lane's two pixels (rows y and y + 4 of its column) share the entry's
// scalars; the terms that are already pairs (s, alpha, w, T, the pair
// count) run as packed FP32 pairs, without branches: a pixel that an entry
// does not reach, or that has stopped, composites it with w = 0, which leaves
// its sums unchanged.
template <int TS, int CH, bool MED, bool L1, int ROWS>
__global__ void __launch_bounds__(BlendShape<TS, FwdBlock<TS, MED, ROWS>::H>::THREADS, FwdBlock<TS, MED, ROWS>::MIN_BLOCKS)
    blend_fwd_kernel(const __grid_constant__ ViewTable vt, const Ws ws) {
    constexpr int BH = FwdBlock<TS, MED, ROWS>::H, NR = BH / kRowStep, NP = NR / 2;
    using S = BlendShape<TS, BH>;
    __shared__ float4 sF[S::WARPS][kFwdQuads][32 * CH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the preprocess left this layout's gradient rows zero (rows_known_clean)
    if (blockIdx.x == 0 && threadIdx.x == 0) set_rows_clean(ws, true);
    const WarpTile wt = warp_tile<TS, BH>(vt, ws);
    const ViewParams &vp = vt.v[wt.v];
    const uint32_t *vals = ws.sorted;
    const size_t vN = (size_t)wt.v * ws.N;
    const float lxf = (float)(lane & (kSubW - 1)), lyf = (float)(lane / kSubW);
    const float2 neg2 = make_float2(-1.f, -1.f);

    // A row that lies outside the view, or has met the transmittance stop,
    // sits at the row offset kFar (the largest finite float): its p2 = m11
    // kFar + b overflows (m11 > 0 is a Cholesky diagonal, far above 1e-19)
    // and p1 is finite or infinite but never NaN, so s = +inf, which no
    // entry reaches and whose 2^(l - s) is 0.  T never falls below the stop,
    // so an entry that reaches no row leaves Tn = T and cannot trigger the
    // stop either.
    const int Yr = row_origin(wt.Y0);
    const float yoff = (float)(wt.Y0 - Yr);
    const float kFar = 0x1.fffffep127f;
    // per pixel (pair p: .x row 2p, .y row 2p + 1, i.e. rows y + 8p and y + 8p + 4)
    float2 ly[NP], T[NP], C0[NP], C1[NP], C2[NP], D[NP], Zm[NP], cnt[NP];
    // last: the list position of the entry the pixel stopped at, or the
    // list's end -- the backward's contributors are the entries before it
    // that reach the pixel (every one of them was composited)
    uint32_t last[NR], mi[NR];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int r0 = 2 * p * kRowStep, r1 = r0 + kRowStep;
        ly[p] = make_float2(wt.px < vp.W && wt.py + r0 < vp.H ? lyf + yoff + (float)r0 : kFar,
                            wt.px < vp.W && wt.py + r1 < vp.H ? lyf + yoff + (float)r1 : kFar);
        T[p] = make_float2(1.f, 1.f);
        C0[p] = C1[p] = C2[p] = D[p] = Zm[p] = cnt[p] = make_float2(0.f, 0.f);   // cnt: composited pairs (exact in FP32)
        last[2 * p] = last[2 * p + 1] = wt.range.y;
        mi[2 * p] = mi[2 * p + 1] = 0u;
    }
    const float4(&F)[kFwdQuads][32 * CH] = sF[warp];
    auto all_stopped = [&]() {
        bool far = true;
#pragma unroll
        for (int p = 0; p < NP; ++p) far = far && ly[p].x == kFar && ly[p].y == kFar;
        return __all_sync(kFull, far);
    };

    bool stopped_all = false;
    for (uint32_t base = wt.range.x; base < wt.range.y; base += 32 * CH) {
        if (stopped_all || all_stopped()) break;
        bool clamp_chunk = false;
        const int n = stage_chunk<BH, CH>(ws, vals, vN, base, wt.range.y, wt.X0, wt.Y0, Yr,
                                          [&](int slot, float ur, float vr, float4 r1, float4 r2, float log2o,
                                              uint32_t idx, uint32_t) {
                                              float a, b;
                                              lin_consts(ur, vr, r1.x, r1.y, r1.z, a, b);
                                              clamp_chunk |= log2o > kLog2ClampFree;
                                              sF[warp][0][slot] = make_float4(r1.x, a, r1.y, r1.z);
                                              sF[warp][1][slot] = make_float4(b, r1.w, log2o, __uint_as_float(idx));
                                              sF[warp][2][slot] = r2;
                                          });
        // the entries in list order, with the stop rule
        auto run = [&](auto clamp) {
#pragma unroll 2
            for (int j = 0; j < n; ++j) {
                const float4 q0 = F[0][j], q1 = F[1][j];
                // s with the same FP32 operations as the backward
                const float t = __fmaf_rn(q0.x, lxf, q0.y);                     // m00 x + a
                float2 w[NP], Tn[NP], m[NP];
                bool st = false;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    // packed: each half is the same fma.rn as the scalar form
                    const float2 p1 = __ffma2_rn(make_float2(q0.z, q0.z), ly[p], make_float2(t, t));
                    const float2 p2 = __ffma2_rn(make_float2(q0.w, q0.w), ly[p], make_float2(q1.x, q1.x));
                    const float2 s = __ffma2_rn(p1, p1, __fmul2_rn(p2, p2));
                    m[p] = make_float2(le_mask(s.x, q1.y), le_mask(s.y, q1.y));   // the entry reaches the pixel
                    // alpha = min(0.99, 2^(log2(sigma) - s)), times the mask;
                    // chunks whose Gaussians all lie below kLog2ClampFree skip the clamp
                    const float2 earg = __ffma2_rn(s, neg2, make_float2(q1.z, q1.z));   // 0.0877 -> 0.0855 ms
                    float2 e = make_float2(ex2_approx(earg.x), ex2_approx(earg.y));
                    if constexpr (decltype(clamp)::value) e = make_float2(fminf(kAlphaMax, e.x), fminf(kAlphaMax, e.y));
                    w[p] = __fmul2_rn(__fmul2_rn(e, m[p]), T[p]);
                    Tn[p] = __ffma2_rn(w[p], neg2, T[p]);                    // T (1 - alpha)
                    st = st || Tn[p].x < kTStop || Tn[p].y < kTStop;          // stop before this entry
                }
                if (MED) {   // a stopping entry has T < 0.01, so the reach mask is enough here
                    const uint32_t id1 = __float_as_uint(q1.w) + 1u;
                    const float z = F[2][j].w;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (m[p].x != 0.f && T[p].x > 0.5f) Zm[p].x = z, mi[2 * p] = id1;
                        if (m[p].y != 0.f && T[p].y > 0.5f) Zm[p].y = z, mi[2 * p + 1] = id1;
                    }
                }
                if (__builtin_expect(__any_sync(kFull, st), 0)) {
                    // a pixel of the warp meets the stop; it keeps its T and
                    // takes nothing more (its row moves to the far offset)
                    const uint32_t idx = __float_as_uint(q1.w);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (Tn[p].x < kTStop) w[p].x = 0.f, Tn[p].x = T[p].x, ly[p].x = kFar, last[2 * p] = idx, m[p].x = 0.f;
                        if (Tn[p].y < kTStop)
                            w[p].y = 0.f, Tn[p].y = T[p].y, ly[p].y = kFar, last[2 * p + 1] = idx, m[p].y = 0.f;
                    }
                    // every pixel of the warp has stopped: this entry adds
                    // nothing (w = 0 and Tn = T everywhere), nor does any
                    // later one, so the warp leaves the chunk (and then the
                    // list) here instead of at the chunk's end
                    if (all_stopped()) {
                        stopped_all = true;
                        break;
                    }
                }
                const float4 q2 = F[2][j];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    cnt[p] = __fadd2_rn(cnt[p], m[p]);
                    // colour and depth sums of both rows, packed (window blend forward
                    // 0.0898 -> 0.0877 ms with the linear forms above)
                    C0[p] = __ffma2_rn(w[p], make_float2(q2.x, q2.x), C0[p]);
                    C1[p] = __ffma2_rn(w[p], make_float2(q2.y, q2.y), C1[p]);
                    C2[p] = __ffma2_rn(w[p], make_float2(q2.z, q2.z), C2[p]);
                    D[p] = __ffma2_rn(w[p], make_float2(q2.w, q2.w), D[p]);
                    T[p] = Tn[p];
                }
            }
        };
        if (__any_sync(kFull, clamp_chunk))
            run(std::true_type{});
        else
            run(std::false_type{});
        __syncwarp();
    }
    uint32_t ncon = 0;
    float Ta[NR], C0a[NR], C1a[NR], C2a[NR], Da[NR], Zma[NR];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        ncon += (uint32_t)cnt[p].x + (uint32_t)cnt[p].y;
        Ta[2 * p] = T[p].x, Ta[2 * p + 1] = T[p].y;
        C0a[2 * p] = C0[p].x, C0a[2 * p + 1] = C0[p].y;
        C1a[2 * p] = C1[p].x, C1a[2 * p + 1] = C1[p].y;
        C2a[2 * p] = C2[p].x, C2a[2 * p + 1] = C2[p].y;
        Da[2 * p] = D[p].x, Da[2 * p + 1] = D[p].y;
        Zma[2 * p] = Zm[p].x, Zma[2 * p + 1] = Zm[p].y;
    }
    // L1: the targets of the lane's pixels, loaded together before any store
    // (a store to a gradient image could otherwise alias the next load)
    float tgt[L1 ? NR : 1][4];
    if constexpr (L1) {
        const size_t HW = (size_t)vp.H * vp.W;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int py = wt.py + q * kRowStep;
            const bool in = wt.px < vp.W && py < vp.H;
            const size_t pix = in ? (size_t)py * vp.W + wt.px : 0;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) tgt[q][ch] = in ? __ldg(vp.l1_target_color + ch * HW + pix) : 0.f;
            tgt[q][3] = in && vp.l1_target_depth ? __ldg(vp.l1_target_depth + pix) : 0.f;
        }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int py = wt.py + q * kRowStep;
        if (wt.px < vp.W && py < vp.H) {
            const size_t HW = (size_t)vp.H * vp.W, pix = (size_t)py * vp.W + wt.px;
            vp.color[pix] = C0a[q];
            vp.color[HW + pix] = C1a[q];
            vp.color[2 * HW + pix] = C2a[q];
            if (vp.depth) vp.depth[pix] = Da[q];
            if (vp.alpha) vp.alpha[pix] = 1.f - Ta[q];
            ws.T_final[vp.pixel_offset + pix] = Ta[q];
            ws.last[vp.pixel_offset + pix] = last[q];
            if (MED) {
                if (vp.median_depth) vp.median_depth[pix] = Zma[q];
                ws.median[vp.pixel_offset + pix] = mi[q];
            }
        }
    }
    const uint32_t tot = __reduce_add_sync(kFull, ncon);
    if (lane == 0 && tot) atomicAdd(&ws.hdr->pairs_contrib, (unsigned long long)tot);
    if constexpr (L1) {
        // mean over the view's pixels (and 3 channels) of |C - C*|, |D - D*|
        const size_t HW = (size_t)vp.H * vp.W;
        const float kc = vt.l1_color_weight / (3.f * (float)HW), kd = vt.l1_depth_weight / (float)HW;
        const bool dterm = vp.l1_target_depth != nullptr;
        auto sgn = [](float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); };
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int py = wt.py + q * kRowStep;
            if (wt.px < vp.W && py < vp.H) {
                const size_t pix = (size_t)py * vp.W + wt.px;
                const float c[3] = {C0a[q], C1a[q], C2a[q]};
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float d = c[ch] - tgt[q][ch];
                    part += fabsf(d) * kc;
                    vp.l1_d_color[ch * HW + pix] = sgn(d) * kc;
                }
                float g = 0.f;
                if (dterm) {
                    const float d = Da[q] - tgt[q][3];
                    part += fabsf(d) * kd;
                    g = sgn(d) * kd;
                }
                if (vp.l1_d_depth) vp.l1_d_depth[pix] = g;
            }
        }
        // one atomic per block: every warp of the block reaches this point
        __shared__ float s_part[S::WARPS];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
        if (lane == 0) s_part[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < S::WARPS; ++k) s += s_part[k];
            atomicAdd(vt.l1_loss, s);
        }
    }
}

// A lane's gradient sums over its pixels, kept as pairs (A[2] is not used: the
// dx term follows from A[0]).  SET starts them with pair p's terms, otherwise
// they are added.
template <bool SET>
__device__ __forceinline__ void pair_sums(float2 (&A)[kVGGrads], float2 dp1, float2 dp2, float2 glo, float2 w,
                                          float2 dy, float2 gR, float2 gG, float2 gB, float2 gZ) {
    if (SET) {
        A[0] = dp1;
        A[1] = dp2;
        A[3] = __fmul2_rn(dp1, dy);
        A[4] = __fmul2_rn(dp2, dy);
        A[5] = glo;
        A[6] = __fmul2_rn(gR, w);
        A[7] = __fmul2_rn(gG, w);
        A[8] = __fmul2_rn(gB, w);
        A[9] = __fmul2_rn(gZ, w);
    } else {
        A[0] = __fadd2_rn(A[0], dp1);
        A[1] = __fadd2_rn(A[1], dp2);
        A[3] = __ffma2_rn(dp1, dy, A[3]);
        A[4] = __ffma2_rn(dp2, dy, A[4]);
        A[5] = __fadd2_rn(A[5], glo);
        A[6] = __ffma2_rn(gR, w, A[6]);
        A[7] = __ffma2_rn(gG, w, A[7]);
        A[8] = __ffma2_rn(gB, w, A[8]);
        A[9] = __ffma2_rn(gZ, w, A[9]);
    }
}

// MED: dL/d(median depth) goes to the z of each pixel's median contributor.
// A lane owns NR = BH / 4 pixel rows of its column; rows 2p and 2p + 1 (y + 8p
// and y + 8p + 4) form pair p, whose arithmetic runs on packed FP32 pairs.
template <int TS, int CH, bool MED>
__global__ void __launch_bounds__(BlendShape<TS, BwdBlock<TS>::H>::THREADS, BwdBlock<TS>::MIN_BLOCKS)
    blend_bwd_kernel(const __grid_constant__ ViewTable vt, const Ws ws) {
    constexpr int BH = BwdBlock<TS>::H;
    constexpr int NR = BH / kRowStep, NP = NR / 2;
    using S = BlendShape<TS, BH>;
    __shared__ float4 sE[S::WARPS][kBwdQuads][32 * CH];
    __shared__ float4 sX[S::WARPS][32 * CH];  // (s_max, list index, Gaussian index, -)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the rows fill up here until the preprocess backward clears them again
    if (blockIdx.x == 0 && threadIdx.x == 0) set_rows_clean(ws, false);
    const WarpTile wt = warp_tile<TS, BH>(vt, ws);
    const ViewParams &vp = vt.v[wt.v];
    const uint32_t *vals = ws.sorted;
    const size_t vN = (size_t)wt.v * ws.N;
    const float lxf = (float)(lane & (kSubW - 1)), lyf = (float)(lane / kSubW);
    const float2 lx2 = make_float2(lxf, lxf);
    const float2 one2 = make_float2(1.f, 1.f), neg2 = make_float2(-1.f, -1.f);
    const int Yr = row_origin(wt.Y0);             // the row offsets' origin (see row_origin)
    const float yoff = (float)(wt.Y0 - Yr);

    // per pixel (pair p: .x row 2p, .y row 2p + 1): Q = gC . (colour behind)
    // + gD (depth behind), normalised by the transmittance in front of the
    // current entry
    float2 T[NP], Q[NP], gR[NP], gG[NP], gB[NP], gZ[NP], gA[NP];
    uint32_t last[NR], mi[NR], lmax = 0;
    float gM[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        float t = 1.f, g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        last[r] = mi[r] = 0;
        gM[r] = 0.f;
        const int py = wt.py + r * kRowStep;
        if (wt.px < vp.W && py < vp.H) {
            const size_t HW = (size_t)vp.H * vp.W, pix = (size_t)py * vp.W + wt.px;
            t = ws.T_final[vp.pixel_offset + pix];
            last[r] = ws.last[vp.pixel_offset + pix];
            if (vp.d_color) {
                g[0] = vp.d_color[pix];
                g[1] = vp.d_color[HW + pix];
                g[2] = vp.d_color[2 * HW + pix];
            }
            if (vp.d_depth) g[3] = vp.d_depth[pix];
            if (vp.d_alpha) g[4] = vp.d_alpha[pix] * t;
            if (MED && vp.d_median_depth) {
                gM[r] = vp.d_median_depth[pix];
                mi[r] = ws.median[vp.pixel_offset + pix];
            }
        }
        lmax = max(lmax, last[r]);
        const int p = r / 2;
        if (r & 1) {
            T[p].y = t, gR[p].y = g[0], gG[p].y = g[1], gB[p].y = g[2], gZ[p].y = g[3], gA[p].y = g[4];
        } else {
            T[p].x = t, gR[p].x = g[0], gG[p].x = g[1], gB[p].x = g[2], gZ[p].x = g[3], gA[p].x = g[4];
        }
        Q[p] = make_float2(0.f, 0.f);
    }
    const uint32_t wlast = __reduce_max_sync(kFull, lmax);
    // the lane's component of the warp sums, and whether it writes it (one
    // lane of each partner pair)
    int sum_comp;
    bool sum_writer;
    sum10_slot(lane, sum_comp, sum_writer);
    sum_writer = sum_writer && (lane & 1) == 0;
    // the lane's row offsets from the origin, per pair
    float2 lyp[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
        lyp[p] = make_float2(lyf + yoff + (float)(2 * p * kRowStep), lyf + yoff + (float)((2 * p + 1) * kRowStep));
#ifdef GSR_CHECKED
    unsigned long long nbwd = 0;   // the contributor pairs this warp takes (the same in every lane)
#endif
    float *grads = ws.vg_grads + (size_t)wt.v * kVGGrads;   // + g V 10: (Gaussian, view) rows of 10
    const size_t row = (size_t)ws.V * kVGGrads;

    for (uint32_t end = wlast; end > wt.range.x;) {
        const uint32_t begin = end - wt.range.x > 32u * CH ? end - 32u * CH : wt.range.x;
        bool clamp_chunk = false;
        const int n = stage_chunk<BH, CH>(ws, vals, vN, begin, end, wt.X0, wt.Y0, Yr,
                                      [&](int slot, float ur, float vr, float4 r1, float4 r2, float log2o,
                                          uint32_t idx, uint32_t g) {
                                          clamp_chunk |= log2o > kLog2ClampFree;
                                          float4(&e)[kBwdQuads][32 * CH] = sE[warp];
                                          e[0][slot] = make_float4(-ur, -ur, -vr, -vr);
                                          e[1][slot] = make_float4(r1.x, r1.x, r1.y, r1.y);
                                          e[2][slot] = make_float4(r1.z, r1.z, log2o, log2o);
                                          e[3][slot] = make_float4(r2.x, r2.x, r2.y, r2.y);
                                          e[4][slot] = make_float4(r2.z, r2.z, r2.w, r2.w);
                                          sX[warp][slot] = make_float4(r1.w, __uint_as_float(idx),
                                                                       __uint_as_float(g), 0.f);
                                      });
        // entry j; CLAMP: the chunk holds a Gaussian that can reach the alpha clamp
        auto entry = [&](int j, auto clamp) {
            constexpr bool CLAMP = decltype(clamp)::value;
            const float4 e0 = sE[warp][0][j], e1 = sE[warp][1][j], e2 = sE[warp][2][j];
            const float4 x = sX[warp][j];
            const uint32_t eidx = __float_as_uint(x.y);
            const float dx = __fadd_rn(lxf, e0.x);                    // the gradient's column offset
            // the constants a, b of lin_consts, and t = m00 x + a: the same
            // FP32 operations as the forward (negation is exact)
            const float2 a2 = __ffma2_rn(hi2(e1), hi2(e0), __fmul2_rn(lo2(e1), lo2(e0)));
            const float2 b2 = __fmul2_rn(lo2(e2), hi2(e0));
            const float2 t = __ffma2_rn(lo2(e1), lx2, a2);
            float2 dy[NP], s[NP], p1[NP], p2[NP];
            bool c[NR];
            unsigned m[NR], cmask = 0u;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float2 ly = lyp[p];
                dy[p] = __fadd2_rn(ly, hi2(e0));
                s[p] = pair_s2(t, ly, hi2(e1), lo2(e2), b2, p1[p], p2[p]);
                c[2 * p] = eidx < last[2 * p] && s[p].x <= x.x;
                c[2 * p + 1] = eidx < last[2 * p + 1] && s[p].y <= x.x;
                m[2 * p] = __ballot_sync(kFull, c[2 * p]);
                m[2 * p + 1] = __ballot_sync(kFull, c[2 * p + 1]);
                cmask |= m[2 * p] | m[2 * p + 1];
            }
            if (cmask == 0u) return;
#ifdef GSR_CHECKED
#pragma unroll
            for (int r = 0; r < NR; ++r) nbwd += (unsigned long long)__popc(m[r]);
#endif
            const float4 e3 = sE[warp][3][j], e4 = sE[warp][4][j];
            float2 A[kVGGrads];
            // Both rows of pair p, packed.  Branch-free: a pixel without a
            // contribution runs with alpha = 0, which leaves its T and Q
            // unchanged and makes every gradient term zero.
            auto packed = [&](int p, float2 &dp1, float2 &dp2, float2 &glo, float2 &w) {
                const float2 arg = __ffma2_rn(s[p], neg2, hi2(e2));
                const float2 raw = make_float2(c[2 * p] ? ex2_approx(arg.x) : 0.f,
                                               c[2 * p + 1] ? ex2_approx(arg.y) : 0.f);
                float2 al = raw;
                if constexpr (CLAMP) al = make_float2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y));
                const float2 om = __ffma2_rn(al, neg2, one2);
                const float2 rom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                const float2 Ti = __fmul2_rn(T[p], rom);
                w = __fmul2_rn(al, Ti);
                // dL/dalpha = T_i (g.c_i - Q) + gA T_final / (1 - alpha), and
                // Q <- Q (1 - alpha) + alpha g.c_i, with g.c = gC.rgb + gD z
                const float2 gc = __ffma2_rn(gR[p], lo2(e3),
                                             __ffma2_rn(gG[p], hi2(e3),
                                                        __ffma2_rn(gB[p], lo2(e4), __fmul2_rn(gZ[p], hi2(e4)))));
                const float2 dgq = __ffma2_rn(Q[p], neg2, gc);
                const float2 dA = __ffma2_rn(Ti, dgq, __fmul2_rn(gA[p], rom));
                Q[p] = __ffma2_rn(al, dgq, Q[p]);
                T[p] = Ti;
                // no gradient to position or opacity through the 0.99 clamp
                glo = __fmul2_rn(dA, raw);                              // dL/d ln(sigma)
                if constexpr (CLAMP) {
                    glo.x = raw.x <= kAlphaMax ? glo.x : 0.f;
                    glo.y = raw.y <= kAlphaMax ? glo.y : 0.f;
                }
                // dL/dp = 2 p dL/ds = -2 ln 2 p glo: the factor -2 ln 2 is
                // applied once per (view, Gaussian) by the preprocess backward
                dp1 = __fmul2_rn(p1[p], glo);
                dp2 = __fmul2_rn(p2[p], glo);
            };
            if constexpr (NP == 2) {
                // Both pairs in one straight run where the entry reaches rows
                // of both halves of the block in the warp, so that their
                // independent chains interleave; only the reached pair where
                // it reaches one half (a warp-uniform branch).  Rows the entry
                // does not reach within a computed pair run with alpha = 0.
                // (Scalar paths for single reached rows took more registers
                // than the 80 of 24 resident warps.)
                const bool h0 = (m[0] | m[1]) != 0u, h1 = (m[2] | m[3]) != 0u;
                if (h0 && h1) {
                    float2 dp1[NP], dp2[NP], glo[NP], w[NP];
#pragma unroll
                    for (int p = 0; p < NP; ++p) packed(p, dp1[p], dp2[p], glo[p], w[p]);
                    pair_sums<true>(A, dp1[0], dp2[0], glo[0], w[0], dy[0], gR[0], gG[0], gB[0], gZ[0]);
                    pair_sums<false>(A, dp1[1], dp2[1], glo[1], w[1], dy[1], gR[1], gG[1], gB[1], gZ[1]);
                } else if (h0) {
                    float2 dp1, dp2, glo, w;
                    packed(0, dp1, dp2, glo, w);
                    pair_sums<true>(A, dp1, dp2, glo, w, dy[0], gR[0], gG[0], gB[0], gZ[0]);
                } else {
                    float2 dp1, dp2, glo, w;
                    packed(1, dp1, dp2, glo, w);
                    pair_sums<true>(A, dp1, dp2, glo, w, dy[1], gR[1], gG[1], gB[1], gZ[1]);
                }
            } else {
                // pair 0 sets the sums (to zero when it is not reached), later pairs add
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const unsigned ma = m[2 * p], mb = m[2 * p + 1];
                    if ((ma | mb) == 0u) {
                        if (p == 0) {
#pragma unroll
                            for (int k = 0; k < kVGGrads; ++k) A[k] = make_float2(0.f, 0.f);
                        }
                        continue;
                    }
                    float2 dp1, dp2, glo, w;
                    if (ma != 0u && mb != 0u) {
                        packed(p, dp1, dp2, glo, w);
                    } else {
                        // Only one row of the pair is reached in the warp: scalar
                        // work on it, its results in its own half of the pairs.
                        auto one_row = [&](auto tag) {
                            constexpr int R = decltype(tag)::value;
                            const bool cq = c[2 * p + R];
                            const float sq = R ? s[p].y : s[p].x;
                            const float p1q = R ? p1[p].y : p1[p].x, p2q = R ? p2[p].y : p2[p].x;
                            float &Tq = R ? T[p].y : T[p].x;
                            float &Qq = R ? Q[p].y : Q[p].x;
                            const float gRq = R ? gR[p].y : gR[p].x, gGq = R ? gG[p].y : gG[p].x;
                            const float gBq = R ? gB[p].y : gB[p].x, gZq = R ? gZ[p].y : gZ[p].x;
                            const float gAq = R ? gA[p].y : gA[p].x;
                            const float raw = cq ? ex2_approx(__fmaf_rn(sq, -1.f, e2.z)) : 0.f;
                            const float al = CLAMP ? fminf(kAlphaMax, raw) : raw;
                            const float rom = rcp_approx(__fmaf_rn(al, -1.f, 1.f));
                            const float Ti = Tq * rom;
                            const float wq = al * Ti;
                            const float gc = fmaf(gRq, e3.x, fmaf(gGq, e3.z, fmaf(gBq, e4.x, gZq * e4.z)));
                            const float dgq = __fmaf_rn(Qq, -1.f, gc);
                            const float dA = fmaf(Ti, dgq, gAq * rom);
                            Qq = fmaf(al, dgq, Qq);
                            Tq = Ti;
                            const float gl = !CLAMP || raw <= kAlphaMax ? dA * raw : 0.f;
                            const float ds2 = gl;   // without -2 ln 2, as in the packed path
                            auto put = [](float v) { return R ? make_float2(0.f, v) : make_float2(v, 0.f); };
                            dp1 = put(p1q * ds2);
                            dp2 = put(p2q * ds2);
                            glo = put(gl);
                            w = put(wq);
                        };
                        if (ma == 0u)
                            one_row(RowTag<1>{});
                        else
                            one_row(RowTag<0>{});
                    }
                    if (p == 0)
                        pair_sums<true>(A, dp1, dp2, glo, w, dy[p], gR[p], gG[p], gB[p], gZ[p]);
                    else
                        pair_sums<false>(A, dp1, dp2, glo, w, dy[p], gR[p], gG[p], gB[p], gZ[p]);
                }
            }
            float gv[kVGGrads];
            gv[0] = A[0].x + A[0].y;                                    // du, dv follow from these and m
            gv[1] = A[1].x + A[1].y;
            gv[2] = dx * gv[0];
#pragma unroll
            for (int k = 3; k < kVGGrads; ++k) gv[k] = A[k].x + A[k].y;
            if (MED) {
#pragma unroll
                for (int r = 0; r < NR; ++r) gv[9] += eidx + 1u == mi[r] ? gM[r] : 0.f;
            }
            float *gp = grads + (size_t)__float_as_uint(x.z) * row;
            if (__popc(cmask) <= 4) {
                // up to four lanes: their own atomics are cheaper than a reduction
                // (measured: 0.259 ms against 0.261 with two, 0.260 with eight)
                if ((cmask >> lane) & 1u) {
#pragma unroll
                    for (int k = 0; k < kVGGrads; ++k) atomicAdd(gp + k, gv[k]);
                }
            } else {
                const float sum = warp_sum10(gv, lane);
                if (sum_writer) atomicAdd(gp + sum_comp, sum);
            }
        };
        if (__any_sync(kFull, clamp_chunk)) {
            for (int j = n - 1; j >= 0; --j) entry(j, std::true_type{});
        } else {
            for (int j = n - 1; j >= 0; --j) entry(j, std::false_type{});
        }
        __syncwarp();
        end = begin;
    }
#ifdef GSR_CHECKED
    if (lane == 0 && nbwd) atomicAdd(&ws.hdr->pairs_bwd, nbwd);
#endif
}

// The median-depth variant has 8-row blocks at either ROWS (FwdBlock), so
// it is instantiated once, with ROWS 8.
template <int TS, int CH, int ROWS>
cudaError_t launch_fwd_rows(const ViewTable &vt, const Ws &ws, cudaStream_t st, bool med, bool l1) {
    constexpr int TM = BlendShape<TS, FwdBlock<TS, true, 8>::H>::THREADS;       // with median depth
    constexpr int TP = BlendShape<TS, FwdBlock<TS, false, ROWS>::H>::THREADS;   // without
    const unsigned cm = vt.total_tiles * BlendShape<TS, FwdBlock<TS, true, 8>::H>::CTAS;
    const unsigned cp = vt.total_tiles * BlendShape<TS, FwdBlock<TS, false, ROWS>::H>::CTAS;
    if (med && l1)
        blend_fwd_kernel<TS, CH, true, true, 8><<<cm, TM, 0, st>>>(vt, ws);
    else if (med)
        blend_fwd_kernel<TS, CH, true, false, 8><<<cm, TM, 0, st>>>(vt, ws);
    else if (l1)
        blend_fwd_kernel<TS, CH, false, true, ROWS><<<cp, TP, 0, st>>>(vt, ws);
    else
        blend_fwd_kernel<TS, CH, false, false, ROWS><<<cp, TP, 0, st>>>(vt, ws);
    return cudaGetLastError();
}

template <int TS, int CH>
cudaError_t launch_fwd_t(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    bool med = false;
    for (int v = 0; v < vt.V; ++v) med |= vt.v[v].median_depth != nullptr;
    const bool l1 = vt.l1_loss != nullptr;
    if constexpr (TS >= 16) {
        if (vt.fwd_rows == 16) return launch_fwd_rows<TS, CH, 16>(vt, ws, st, med, l1);
    }
    return launch_fwd_rows<TS, CH, 8>(vt, ws, st, med, l1);
}

template <int TS, int CH>
cudaError_t launch_bwd_t(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    bool med = false;
    for (int v = 0; v < vt.V; ++v) med |= vt.v[v].d_median_depth != nullptr;
    constexpr int T = BlendShape<TS, BwdBlock<TS>::H>::THREADS;
    const unsigned ctas = vt.total_tiles * BlendShape<TS, BwdBlock<TS>::H>::CTAS;
    if (med)
        blend_bwd_kernel<TS, CH, true><<<ctas, T, 0, st>>>(vt, ws);
    else
        blend_bwd_kernel<TS, CH, false><<<ctas, T, 0, st>>>(vt, ws);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_fwd(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (vt.total_tiles == 0) return cudaSuccess;
    switch (vt.tile) {
        // the 64-entry batch at tile 32 would need more than 48 KB of static shared memory
        case 8: return vt.batch == 64 ? launch_fwd_t<8, 2>(vt, ws, st) : launch_fwd_t<8, 1>(vt, ws, st);
        case 32: return launch_fwd_t<32, 1>(vt, ws, st);
        default: return vt.batch == 64 ? launch_fwd_t<16, 2>(vt, ws, st) : launch_fwd_t<16, 1>(vt, ws, st);
    }
}

cudaError_t launch_blend_bwd(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (vt.total_tiles == 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: return vt.batch == 64 ? launch_bwd_t<8, 2>(vt, ws, st) : launch_bwd_t<8, 1>(vt, ws, st);
        case 32: return launch_bwd_t<32, 1>(vt, ws, st);
        default: return vt.batch == 64 ? launch_bwd_t<16, 2>(vt, ws, st) : launch_bwd_t<16, 1>(vt, ws, st);
    }
}

}  // namespace gsr
