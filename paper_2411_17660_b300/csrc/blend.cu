// blend.cu -- per-pixel front-to-back compositing (Sec. 3.3, Eq.
// "rendering": C = sum_i c_i alpha_i prod_{j<i}(1 - alpha_j)) and its
// back-to-front backward.
//
// One CTA per screen tile (all views concatenated), one warp per 8x4 block
// of pixels, one pixel per lane.  Each warp walks its tile's depth-sorted
// list in chunks of 32 entries: the 32 lanes load one entry each, keep only
// the Gaussians whose cutoff ellipse reaches the warp's 8x4 block (an exact
// convex minimum of d^2 over the block), compact the survivors into the
// warp's shared-memory slots with a ballot, and then every lane composites
// them for its pixel.  A warp leaves as soon as all its lanes have hit the
// transmittance stop; warps never wait for each other.
//
// The backward recomputes the blend state from the stored final
// transmittance and last contributor: walking back, T_i = T_{i+1}/(1-alpha_i)
// and the colour/depth behind each entry accumulate as B <- B(1-a) + c a.
// Per-Gaussian gradients of the 32 pixels of a warp are summed with warp
// shuffles before one set of global atomics per (warp, Gaussian).
#include "kernels.cuh"

namespace gsr {

namespace {

constexpr int kSubW = 8, kSubH = 4;
constexpr unsigned kFull = 0xffffffffu;

template <int TS>
struct BlendShape {
    static constexpr int WX = TS / kSubW;
    static constexpr int WY = TS / kSubH;
    static constexpr int WARPS = WX * WY;
    static constexpr int THREADS = WARPS * 32;
};

// s = 0.5 log2(e) d^2 of a pixel at offset (dx, dy) from the mean, with the
// Cholesky factor m of 0.5 log2(e) Sigma'^-1.  Round-to-nearest intrinsics:
// the forward and the backward take bit-identical decisions.
__device__ __forceinline__ float pair_s(float dx, float dy, float m00, float m01, float m11, float &p1, float &p2) {
    p1 = __fmaf_rn(m00, dx, __fmul_rn(m01, dy));
    p2 = __fmul_rn(m11, dy);
    return __fmaf_rn(p1, p1, __fmul_rn(p2, p2));
}

// Whether min over the warp's block of pixel centres of s can reach s_max.
// s(dx, dy) = (m00 dx + m01 dy)^2 + (m11 dy)^2; for fixed dy the first term's
// minimum over dx in [dx0, dx1] is max(0, m00 dx0 + m01 dy, -(m00 dx1 + m01 dy))^2,
// a convex function of dy whose minimum over [dy0, dy1] lies at an end or at
// one of three stationary points, all clamped into the interval.
__device__ __forceinline__ bool touches_block(float ur, float vr, float m00, float m01, float m11, float smax) {
    const float dx0 = -ur, dx1 = (float)(kSubW - 1) - ur;
    const float dy0 = -vr, dy1 = (float)(kSubH - 1) - vr;
    const float a0 = m00 * dx0, a1 = m00 * dx1;
    const float inv_den = 1.0f / (m01 * m01 + m11 * m11);
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
    return smin <= smax + 1e-3f * (1.f + smax) + 1e-2f;
}

struct WarpTile {
    int v;
    int X0, Y0;       // pixel of lane 0
    int px, py;       // this lane's pixel
    bool inside;
    uint2 range;
};

template <int TS>
__device__ __forceinline__ WarpTile warp_tile(const ViewTable &vt, const Ws &ws) {
    using S = BlendShape<TS>;
    WarpTile w;
    const uint32_t tile = blockIdx.x;
    w.v = view_of_tile(vt, tile);
    const ViewParams &vp = vt.v[w.v];
    const uint32_t lt = tile - vp.tile_offset;
    const int tx = (int)(lt % (uint32_t)vp.tiles_x), ty = (int)(lt / (uint32_t)vp.tiles_x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    w.X0 = tx * TS + (warp % S::WX) * kSubW;
    w.Y0 = ty * TS + (warp / S::WX) * kSubH;
    w.px = w.X0 + (lane & (kSubW - 1));
    w.py = w.Y0 + lane / kSubW;
    w.inside = w.px < vp.W && w.py < vp.H;
    w.range = ws.ranges[tile];
    return w;
}

// Loads entry idx of the tile list (lane-parallel), tests it against the
// warp's block and compacts the survivors into the warp's slots in list
// order.  Returns the number of survivors.
__device__ __forceinline__ int stage_chunk(const Ws &ws, const uint32_t *vals, size_t vN, uint32_t idx, uint32_t end,
                                           int X0, int Y0, float4 *sA, float4 *sB, float4 *sC) {
    bool keep = false;
    float4 r0, r1;
    float ur = 0.f, vr = 0.f;
    size_t gi = 0;
    const uint32_t g = idx < end ? vals[idx] : 0xffffffffu;
    if (g < ws.N) {  // g >= N only after a reported device error
        gi = vN + g;
        r0 = ws.rec0[gi];
        r1 = ws.rec1[gi];
        ur = __fadd_rn(__fsub_rn(r0.x, (float)X0), r0.z);
        vr = __fadd_rn(__fsub_rn(r0.y, (float)Y0), r0.w);
        keep = touches_block(ur, vr, r1.x, r1.y, r1.z, r1.w);
    }
    const unsigned ballot = __ballot_sync(kFull, keep);
    if (keep) {
        const int slot = __popc(ballot & lanemask_lt());
        const float4 r2 = ws.rec2[gi];
        const float log2o = ws.rec3[gi].x;
        sA[slot] = make_float4(ur, vr, r1.x, r1.y);
        sB[slot] = make_float4(r1.z, r1.w, log2o, r2.w);
        sC[slot] = make_float4(r2.x, r2.y, r2.z, __uint_as_float(idx));
    }
    __syncwarp();
    return __popc(ballot);
}

template <int TS>
__global__ void __launch_bounds__(BlendShape<TS>::THREADS) blend_fwd_kernel(const __grid_constant__ ViewTable vt,
                                                                           const Ws ws) {
    using S = BlendShape<TS>;
    __shared__ float4 sA[S::WARPS][32], sB[S::WARPS][32], sC[S::WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpTile wt = warp_tile<TS>(vt, ws);
    const ViewParams &vp = vt.v[wt.v];
    const uint32_t *vals = ws.vals[ws.passes & 1];
    const size_t vN = (size_t)wt.v * ws.N;
    const float lxf = (float)(lane & (kSubW - 1)), lyf = (float)(lane / kSubW);

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    uint32_t last = 0, ncon = 0;
    bool done = !wt.inside;
    for (uint32_t base = wt.range.x; base < wt.range.y; base += 32) {
        if (__all_sync(kFull, done)) break;
        const int n = stage_chunk(ws, vals, vN, base + lane, wt.range.y, wt.X0, wt.Y0, sA[warp], sB[warp], sC[warp]);
        for (int j = 0; j < n; ++j) {
            const float4 a = sA[warp][j], b = sB[warp][j];
            if (!done) {
                float p1, p2;
                const float s = pair_s(__fsub_rn(lxf, a.x), __fsub_rn(lyf, a.y), a.z, a.w, b.x, p1, p2);
                if (s <= b.y) {
                    const float alpha = fminf(kAlphaMax, ex2_approx(__fsub_rn(b.z, s)));
                    const float Tn = T * (1.f - alpha);
                    if (Tn < kTStop) {
                        done = true;
                    } else {
                        const float4 c = sC[warp][j];
                        const float w = alpha * T;
                        C0 = fmaf(w, c.x, C0);
                        C1 = fmaf(w, c.y, C1);
                        C2 = fmaf(w, c.z, C2);
                        D = fmaf(w, b.w, D);
                        T = Tn;
                        last = __float_as_uint(c.w) + 1u;
                        ++ncon;
                    }
                }
            }
        }
        __syncwarp();
    }
    if (wt.inside) {
        const size_t HW = (size_t)vp.H * vp.W, pix = (size_t)wt.py * vp.W + wt.px;
        vp.color[pix] = C0;
        vp.color[HW + pix] = C1;
        vp.color[2 * HW + pix] = C2;
        if (vp.depth) vp.depth[pix] = D;
        if (vp.alpha) vp.alpha[pix] = 1.f - T;
        ws.T_final[vp.pixel_offset + pix] = T;
        ws.last[vp.pixel_offset + pix] = last;
    }
    const uint32_t tot = __reduce_add_sync(kFull, ncon);
    if (lane == 0 && tot) atomicAdd(&ws.hdr->pairs_contrib, (unsigned long long)tot);
}

template <int TS>
__global__ void __launch_bounds__(BlendShape<TS>::THREADS) blend_bwd_kernel(const __grid_constant__ ViewTable vt,
                                                                           const Ws ws) {
    using S = BlendShape<TS>;
    __shared__ float4 sA[S::WARPS][32], sB[S::WARPS][32], sC[S::WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpTile wt = warp_tile<TS>(vt, ws);
    const ViewParams &vp = vt.v[wt.v];
    const uint32_t *vals = ws.vals[ws.passes & 1];
    const size_t N = ws.N;
    const size_t vN = (size_t)wt.v * N;
    const float lxf = (float)(lane & (kSubW - 1)), lyf = (float)(lane / kSubW);

    float T = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gATf = 0.f;
    uint32_t last = 0;
    if (wt.inside) {
        const size_t HW = (size_t)vp.H * vp.W, pix = (size_t)wt.py * vp.W + wt.px;
        T = ws.T_final[vp.pixel_offset + pix];
        last = ws.last[vp.pixel_offset + pix];
        if (vp.d_color) {
            gC0 = vp.d_color[pix];
            gC1 = vp.d_color[HW + pix];
            gC2 = vp.d_color[2 * HW + pix];
        }
        if (vp.d_depth) gD = vp.d_depth[pix];
        if (vp.d_alpha) gATf = vp.d_alpha[pix] * T;
    }
    const uint32_t wlast = __reduce_max_sync(kFull, last);
    float BC0 = 0.f, BC1 = 0.f, BC2 = 0.f, BD = 0.f;
    float *grads = ws.vg_grads + (size_t)wt.v * kVGGrads * N;

    for (uint32_t end = wlast; end > wt.range.x;) {
        const uint32_t begin = end - wt.range.x > 32u ? end - 32u : wt.range.x;
        const int n = stage_chunk(ws, vals, vN, begin + lane, end, wt.X0, wt.Y0, sA[warp], sB[warp], sC[warp]);
        for (int j = n - 1; j >= 0; --j) {
            const float4 a = sA[warp][j], b = sB[warp][j], c = sC[warp][j];
            const uint32_t eidx = __float_as_uint(c.w);
            float gv[kVGGrads];
#pragma unroll
            for (int k = 0; k < kVGGrads; ++k) gv[k] = 0.f;
            bool contrib = false;
            if (eidx < last) {
                float p1, p2;
                const float dx = __fsub_rn(lxf, a.x), dy = __fsub_rn(lyf, a.y);
                const float s = pair_s(dx, dy, a.z, a.w, b.x, p1, p2);
                if (s <= b.y) {
                    contrib = true;
                    const float raw = ex2_approx(__fsub_rn(b.z, s));
                    const float alpha = fminf(kAlphaMax, raw);
                    const float rom = 1.f / (1.f - alpha);
                    const float Ti = T * rom;
                    const float w = alpha * Ti;
                    gv[6] = gC0 * w;
                    gv[7] = gC1 * w;
                    gv[8] = gC2 * w;
                    gv[9] = gD * w;
                    const float dcr = c.x - BC0, dcg = c.y - BC1, dcb = c.z - BC2, dzz = b.w - BD;
                    const float dA = Ti * (dcr * gC0 + dcg * gC1 + dcb * gC2 + dzz * gD) + gATf * rom;
                    BC0 = fmaf(alpha, dcr, BC0);
                    BC1 = fmaf(alpha, dcg, BC1);
                    BC2 = fmaf(alpha, dcb, BC2);
                    BD = fmaf(alpha, dzz, BD);
                    T = Ti;
                    if (raw <= kAlphaMax) {
                        gv[5] = dA * raw;                      // dL/d ln(sigma)
                        const float ds2 = -2.f * kLn2 * raw * dA;  // 2 dL/ds
                        const float dp1 = p1 * ds2, dp2 = p2 * ds2;
                        gv[2] = dp1 * dx;
                        gv[3] = dp1 * dy;
                        gv[4] = dp2 * dy;
                        gv[0] = -dp1 * a.z;
                        gv[1] = -(dp1 * a.w + dp2 * b.x);
                    }
                }
            }
            if (__any_sync(kFull, contrib)) {
#pragma unroll
                for (int k = 0; k < kVGGrads; ++k) {
                    float x = gv[k];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
                    gv[k] = x;
                }
                const uint32_t g = vals[eidx];
                if (lane == 0 && g < N) {
#pragma unroll
                    for (int k = 0; k < kVGGrads; ++k) atomicAdd(grads + (size_t)k * N + g, gv[k]);
                }
            }
        }
        __syncwarp();
        end = begin;
    }
}

template <int TS>
cudaError_t launch_fwd_t(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    blend_fwd_kernel<TS><<<vt.total_tiles, BlendShape<TS>::THREADS, 0, st>>>(vt, ws);
    return cudaGetLastError();
}

template <int TS>
cudaError_t launch_bwd_t(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    blend_bwd_kernel<TS><<<vt.total_tiles, BlendShape<TS>::THREADS, 0, st>>>(vt, ws);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_fwd(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (vt.total_tiles == 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: return launch_fwd_t<8>(vt, ws, st);
        case 32: return launch_fwd_t<32>(vt, ws, st);
        default: return launch_fwd_t<16>(vt, ws, st);
    }
}

cudaError_t launch_blend_bwd(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (vt.total_tiles == 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: return launch_bwd_t<8>(vt, ws, st);
        case 32: return launch_bwd_t<32>(vt, ws, st);
        default: return launch_bwd_t<16>(vt, ws, st);
    }
}

}  // namespace gsr
