// surfel.cu -- 2-D surfel ("2D Gaussian Splatting") variant of the renderer
// that the paper compares its 3-D Gaussians with (Sec. 3.3, last paragraph;
// Supp. "2D Gaussian Splatting"): each Gaussian is a flat disk, a pixel
// meets it where the pixel's two homogeneous planes cross, and the blend
// also produces a normal map and the depth distortion.
//
// Per (view, Gaussian) the preprocess computes, in the camera frame,
// a = s_u W t_u, b = s_v W t_v, p = W mu + t (compensated) and the normal,
// and bounds the screen region rho <= d2max by the projected disk (dual
// conic) and the low-pass disk.  Records (rec[4i + k], one 64-byte record
// per pair, then two more arrays):
//   k = 0: (u_hi, v_hi, u_lo, v_lo)   projected centre (double-float)
//   k = 1: (a_x, a_y, a_z, b_x)
//   k = 2: (r, g, b, p_z)              p_z: the depth key of the sort
//   k = 3: (log2 sigma, s_max, b_y, b_z)
//   rec4 = (n_x, n_y, n_z, 0)
//   rec5 = (x_lo, y_lo, x_hi, y_hi)    pixel-centre bounds of the cutoff region
// For a pixel (x, y) = (X0 + lx, Y0 + ly) of a warp's 8x8 block the planes
// are h_x = (ax' - lx a_z, bx' - lx b_z, p_z (du - lx)) with
// ax' = fx a_x - (X0 - cx) a_z, du = u_c - X0 (and the same in y), so that
// the large terms cancel exactly before FP32 sees them; (u, v, 1) ~ h_x x h_y.
#include <mutex>

#include "kernels.cuh"
#include "project.cuh"
#include "sh.cuh"

namespace gsr {

namespace {

constexpr int kSubW = 8, kSubH = 8, kPPL = 2, kRowStep = 4;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kSG = 16;   // floats per (Gaussian, view) gradient row
constexpr float kLowPass = 2.0f;   // rho2 = 2 |pixel - centre|^2

template <int TS>
struct Shape {
    // one CTA of one warp per 8x8 block; a tile's blocks are consecutive CTAs
    // (an SM slot is held only while its warp works, as in the Gaussian blends)
    static constexpr int WARPS = 1, THREADS = 32;
    static constexpr int CX = TS / kSubW, CTAS = CX * (TS / kSubH);   // blocks per tile row, per tile
    // resident blocks per SM asked of the backward: three quarters of full occupancy, at least 1
    static constexpr int BWD_BLOCKS = 1024 / THREADS * 3 / 4 > 0 ? 1024 / THREADS * 3 / 4 : 1;
};

// ------------------------------------------------------------------ preprocess forward
// One thread per Gaussian walks the views.
template <int DEG>
__global__ void __launch_bounds__(128) surfel_pre_fwd_kernel(const __grid_constant__ ViewTable vt,
                                                             const GaussianPtrs gp, const Ws ws) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    __shared__ Pose s_pose[GSR_MAX_VIEWS];
    load_poses(vt, s_pose);
    // surfel rows overwrite the Gaussian layout's (rows_known_clean)
    if (blockIdx.x == 0 && threadIdx.x == 0) set_rows_clean(ws, false);
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= gp.N) return;
    const size_t N = (size_t)gp.N;
    GaussPre G;
    gauss_pre(gp, g, G);
    for (int v = 0; v < vt.V; ++v) {
        const ViewParams &vp = vt.v[v];
        const Pose &ps = s_pose[v];
        const size_t i = (size_t)v * N + g;
        uint32_t count = 0;
        if (G.alive) {
            float xh, xl, yh, yl, zh, zl;
            dot3_plus(ps.W[0][0], ps.W[0][1], ps.W[0][2], ps.t[0], G.mx, G.my, G.mz, xh, xl);
            dot3_plus(ps.W[1][0], ps.W[1][1], ps.W[1][2], ps.t[1], G.mx, G.my, G.mz, yh, yl);
            dot3_plus(ps.W[2][0], ps.W[2][1], ps.W[2][2], ps.t[2], G.mx, G.my, G.mz, zh, zl);
            float a[3], b[3], n[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a[k] = G.s[0] * (ps.W[k][0] * G.R[0][0] + ps.W[k][1] * G.R[1][0] + ps.W[k][2] * G.R[2][0]);
                b[k] = G.s[1] * (ps.W[k][0] * G.R[0][1] + ps.W[k][1] * G.R[1][1] + ps.W[k][2] * G.R[2][1]);
                n[k] = ps.W[k][0] * G.R[0][2] + ps.W[k][1] * G.R[1][2] + ps.W[k][2] * G.R[2][2];
            }
            const float z = zh;
            const float zmin = z - 3.f * sqrtf(a[2] * a[2] + b[2] * b[2]);
            if (z > kNearZ && zmin > kNearZ && isfinite(zmin)) {
                float uh, ul, vh, vl;
                const float rzh = rcp_approx(zh);
                project_coord(vp.fx, vp.cx, xh, xl, zh, zl, rzh, uh, ul);
                project_coord(vp.fy, vp.cy, yh, yl, zh, zl, rzh, vh, vl);
                // the screen region rho3 <= d2max: the projected circle u^2 + v^2 = d2max, bounded
                // by its dual conic D = M diag(d2max, d2max, -1) M^T with M taken relative to the
                // projected centre (its first two rows then have no p column)
                const float d2max = G.smax * (1.0f / kHalfLog2e);
                const float tx = xh / z, ty = yh / z;
                const float m00 = vp.fx * (a[0] - tx * a[2]), m01 = vp.fx * (b[0] - tx * b[2]);
                const float m10 = vp.fy * (a[1] - ty * a[2]), m11 = vp.fy * (b[1] - ty * b[2]);
                const float D00 = d2max * (m00 * m00 + m01 * m01), D11 = d2max * (m10 * m10 + m11 * m11);
                const float D02 = d2max * (m00 * a[2] + m01 * b[2]), D12 = d2max * (m10 * a[2] + m11 * b[2]);
                const float D22 = d2max * (a[2] * a[2] + b[2] * b[2]) - z * z;   // < 0: the disk is in front
                const float ex = sqrtf(fmaxf(D02 * D02 - D00 * D22, 0.f)) / -D22;
                const float ey = sqrtf(fmaxf(D12 * D12 - D11 * D22, 0.f)) / -D22;
                const float cxo = D02 / D22, cyo = D12 / D22;
                const float r2 = sqrtf(d2max / kLowPass);
                const float xlo = fminf(cxo - ex, -r2), xhi = fmaxf(cxo + ex, r2);
                const float ylo = fminf(cyo - ey, -r2), yhi = fmaxf(cyo + ey, r2);
                const float ix = 1e-3f * (xhi - xlo) + 0.05f, iy = 1e-3f * (yhi - ylo) + 0.05f;
                const float4 rect = make_float4(uh + ul + xlo - ix, vh + vl + ylo - iy, uh + ul + xhi + ix,
                                                vh + vl + yhi + iy);
                const float px0 = fmaxf(ceilf(rect.x), 0.f), px1 = fminf(floorf(rect.z), (float)(vp.W - 1));
                const float py0 = fmaxf(ceilf(rect.y), 0.f), py1 = fminf(floorf(rect.w), (float)(vp.H - 1));
                if (px0 <= px1 && py0 <= py1 && isfinite(uh + vh + ex + ey)) {
                    const int TS = vt.tile;
                    count = (uint32_t)(((int)px1 / TS - (int)px0 / TS + 1) * ((int)py1 / TS - (int)py0 / TS + 1));
                    if (n[0] * xh + n[1] * yh + n[2] * zh > 0.f) {   // turn the normal towards the camera
                        n[0] = -n[0];
                        n[1] = -n[1];
                        n[2] = -n[2];
                    }
                    float dx, dy, dz, rn;
                    view_dir(G, ps, dx, dy, dz, rn);
                    float Y[K];
                    sh_eval<DEG>(dx, dy, dz, Y);
                    float rgb[3];
#pragma unroll 1
                    for (int c = 0; c < 3; ++c) {
                        const float *shc = gp.sh + (size_t)c * N + g;
                        float acc = 0.5f;
#pragma unroll
                        for (int k = 0; k < K; ++k) acc = fmaf(__ldg(shc + (size_t)k * 3 * N), Y[k], acc);
                        rgb[c] = fmaxf(acc, 0.f);
                    }
                    float4 *rec = ws.rec + 4 * i;
                    rec[0] = make_float4(uh, vh, ul, vl);
                    rec[1] = make_float4(a[0], a[1], a[2], b[0]);
                    rec[2] = make_float4(rgb[0], rgb[1], rgb[2], zh);
                    rec[3] = make_float4(G.log2o, G.smax, b[1], b[2]);
                    ws.rec4[i] = make_float4(n[0], n[1], n[2], 0.f);
                    ws.rec5[i] = rect;
                    float4 *row = reinterpret_cast<float4 *>(ws.vg_grads + ((size_t)g * ws.V + v) * kSG);
#pragma unroll
                    for (int k = 0; k < kSG / 4; ++k) row[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        ws.counts[i] = count;
    }
}

// ------------------------------------------------------------------ blend
// Staged entry of a warp's slot: e0 = (ax', bx', ay', by'), e1 = (a_z, b_z, p_z,
// log2 sigma), e2 = (du, dv, s_max, list index), e3 = (r, g, b, n_x),
// e4 = (n_y, n_z, Gaussian id, -).
constexpr int kQuads = 5;

struct Hit {
    float hx0, hx1, hx2, hy0, hy1, hy2;   // the pixel's planes
    float inv, u, v;                      // 1 / q2 and the disk coordinates
    float dxp, dyp;                       // pixel minus projected centre
    float rho3, rho2, s;                  // s = 0.5 log2(e) min(rho3, rho2)
};

// Round-to-nearest intrinsics only: the forward and the backward take
// bit-identical decisions.
__device__ __forceinline__ void surfel_hit(const float4 &e0, const float4 &e1, const float4 &e2, float lx, float ly,
                                           Hit &h) {
    h.hx0 = __fmaf_rn(-lx, e1.x, e0.x);
    h.hx1 = __fmaf_rn(-lx, e1.y, e0.y);
    h.dxp = __fsub_rn(lx, e2.x);
    h.hx2 = __fmul_rn(-e1.z, h.dxp);
    h.hy0 = __fmaf_rn(-ly, e1.x, e0.z);
    h.hy1 = __fmaf_rn(-ly, e1.y, e0.w);
    h.dyp = __fsub_rn(ly, e2.y);
    h.hy2 = __fmul_rn(-e1.z, h.dyp);
    const float q0 = __fmaf_rn(h.hx1, h.hy2, -__fmul_rn(h.hx2, h.hy1));
    const float q1 = __fmaf_rn(h.hx2, h.hy0, -__fmul_rn(h.hx0, h.hy2));
    const float q2 = __fmaf_rn(h.hx0, h.hy1, -__fmul_rn(h.hx1, h.hy0));
    h.inv = __frcp_rn(q2);
    h.u = __fmul_rn(q0, h.inv);
    h.v = __fmul_rn(q1, h.inv);
    h.rho3 = __fmaf_rn(h.u, h.u, __fmul_rn(h.v, h.v));
    h.rho2 = __fmul_rn(kLowPass, __fmaf_rn(h.dxp, h.dxp, __fmul_rn(h.dyp, h.dyp)));
    h.s = __fmul_rn(kHalfLog2e, fminf(h.rho3, h.rho2));   // a NaN rho3 (q2 = 0) leaves rho2
}

template <typename Write>
__device__ __forceinline__ int stage_surfels(const Ws &ws, const uint32_t *vals, size_t vN, uint32_t idx,
                                             uint32_t end, int X0, int Y0, Write &&write) {
    bool keep = false;
    size_t gi = 0;
    const uint32_t g = idx < end ? vals[idx] : 0xffffffffu;
    if (idx < end) (void)GSR_CHECK(ws.hdr, g < ws.N);
    if (g < ws.N) {
        gi = vN + g;
        const float4 r = ws.rec5[gi];
        keep = r.x <= (float)(X0 + kSubW - 1) && r.z >= (float)X0 && r.y <= (float)(Y0 + kSubH - 1) &&
               r.w >= (float)Y0;
    }
    const unsigned ballot = __ballot_sync(kFull, keep);
    if (keep) write(__popc(ballot & lanemask_lt()), gi, idx, g);
    __syncwarp();
    return __popc(ballot);
}

struct Tile {
    int v, X0, Y0, px, py;
    uint2 range;
};

template <int TS>
__device__ __forceinline__ Tile tile_of(const ViewTable &vt, const Ws &ws) {
    Tile w;
    const uint32_t tile = blockIdx.x / Shape<TS>::CTAS, q = blockIdx.x % Shape<TS>::CTAS;
    w.v = view_of_tile(vt, tile);
    const ViewParams &vp = vt.v[w.v];
    const uint32_t lt = tile - vp.tile_offset;
    const int tx = (int)(lt % (uint32_t)vp.tiles_x), ty = (int)(lt / (uint32_t)vp.tiles_x);
    const int lane = threadIdx.x & 31;
    w.X0 = tx * TS + (int)(q % Shape<TS>::CX) * kSubW;
    w.Y0 = ty * TS + (int)(q / Shape<TS>::CX) * kSubH;
    w.px = w.X0 + (lane & (kSubW - 1));
    w.py = w.Y0 + lane / kSubW;
    w.range = checked_range(ws.ranges, tile, ws.hdr, ws.cap);
    return w;
}

__device__ __forceinline__ void stage_entry(float4 (*sE)[32], const Ws &ws, const ViewParams &vp, int X0, int Y0,
                                            int slot, size_t gi, uint32_t idx, uint32_t g) {
    const float4 *rec = ws.rec + 4 * gi;
    const float4 r0 = rec[0], r1 = rec[1], r2 = rec[2], r3 = rec[3], r4 = ws.rec4[gi];
    const float ox = (float)X0 - vp.cx, oy = (float)Y0 - vp.cy;
    // (a_x, a_y, a_z, b_x) = r1, (b_y, b_z) = r3.zw
    sE[0][slot] = make_float4(vp.fx * r1.x - ox * r1.z, vp.fx * r1.w - ox * r3.w, vp.fy * r1.y - oy * r1.z,
                              vp.fy * r3.z - oy * r3.w);
    sE[1][slot] = make_float4(r1.z, r3.w, r2.w, r3.x);
    sE[2][slot] = make_float4(__fadd_rn(__fsub_rn(r0.x, (float)X0), r0.z), __fadd_rn(__fsub_rn(r0.y, (float)Y0), r0.w),
                              r3.y, __uint_as_float(idx));
    sE[3][slot] = make_float4(r2.x, r2.y, r2.z, r4.x);
    sE[4][slot] = make_float4(r4.y, r4.z, __uint_as_float(g), 0.f);
}

template <int TS>
__global__ void __launch_bounds__(Shape<TS>::THREADS) surfel_blend_fwd_kernel(const __grid_constant__ ViewTable vt,
                                                                             const Ws ws) {
    using S = Shape<TS>;
    __shared__ float4 sE[S::WARPS][kQuads][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile wt = tile_of<TS>(vt, ws);
    const ViewParams &vp = vt.v[wt.v];
    const uint32_t *vals = ws.sorted;
    const size_t vN = (size_t)wt.v * ws.N;
    const float lxf = (float)(lane & (kSubW - 1)), lyf = (float)(lane / kSubW);

    float T[kPPL], C[kPPL][3], Nn[kPPL][3], A[kPPL], D[kPPL], E[kPPL], L[kPPL];
    uint32_t last[kPPL], ncon = 0;
    bool done[kPPL];
#pragma unroll
    for (int q = 0; q < kPPL; ++q) {
        T[q] = 1.f;
        A[q] = D[q] = E[q] = L[q] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) C[q][c] = Nn[q][c] = 0.f;
        last[q] = 0;
        done[q] = !(wt.px < vp.W && wt.py + q * kRowStep < vp.H);
    }
    for (uint32_t base = wt.range.x; base < wt.range.y; base += 32) {
        if (__all_sync(kFull, done[0] && done[1])) break;
        const int n = stage_surfels(ws, vals, vN, base + lane, wt.range.y, wt.X0, wt.Y0,
                                    [&](int slot, size_t gi, uint32_t idx, uint32_t g) {
                                        stage_entry(sE[warp], ws, vp, wt.X0, wt.Y0, slot, gi, idx, g);
                                    });
        for (int j = 0; j < n; ++j) {
            const float4 e0 = sE[warp][0][j], e1 = sE[warp][1][j], e2 = sE[warp][2][j];
#pragma unroll
            for (int q = 0; q < kPPL; ++q) {
                if (done[q]) continue;
                Hit h;
                surfel_hit(e0, e1, e2, lxf, lyf + (float)(q * kRowStep), h);
                if (!(h.s <= e2.z)) continue;
                const float alpha = fminf(kAlphaMax, ex2_approx(__fsub_rn(e1.w, h.s)));
                const float w = alpha * T[q];
                const float Tn = T[q] - w;   // T (1 - alpha)
                if (Tn < kTStop) {
                    done[q] = true;
                    continue;
                }
                const float4 e3 = sE[warp][3][j], e4 = sE[warp][4][j];
                // the intersection's depth where the disk term decides alpha, else the centre's
                const float z = h.rho3 <= h.rho2 ? fmaf(e1.x, h.u, fmaf(e1.y, h.v, e1.z)) : e1.z;
                C[q][0] = fmaf(w, e3.x, C[q][0]);
                C[q][1] = fmaf(w, e3.y, C[q][1]);
                C[q][2] = fmaf(w, e3.z, C[q][2]);
                Nn[q][0] = fmaf(w, e3.w, Nn[q][0]);
                Nn[q][1] = fmaf(w, e4.x, Nn[q][1]);
                Nn[q][2] = fmaf(w, e4.y, Nn[q][2]);
                // distortion: w_i sum_{j<i} w_j (z_i - z_j)^2 = w (z^2 A - 2 z D + E)
                L[q] = fmaf(w, fmaf(z, fmaf(z, A[q], -2.f * D[q]), E[q]), L[q]);
                A[q] += w;
                D[q] = fmaf(w, z, D[q]);
                E[q] = fmaf(w * z, z, E[q]);
                T[q] = Tn;
                last[q] = __float_as_uint(e2.w) + 1u;
                ++ncon;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < kPPL; ++q) {
        const int py = wt.py + q * kRowStep;
        if (wt.px < vp.W && py < vp.H) {
            const size_t HW = (size_t)vp.H * vp.W, pix = (size_t)py * vp.W + wt.px;
#pragma unroll
            for (int c = 0; c < 3; ++c) vp.color[c * HW + pix] = C[q][c];
            if (vp.depth) vp.depth[pix] = D[q];
            if (vp.alpha) vp.alpha[pix] = 1.f - T[q];
            if (vp.normal)
#pragma unroll
                for (int c = 0; c < 3; ++c) vp.normal[c * HW + pix] = Nn[q][c];
            if (vp.distortion) vp.distortion[pix] = L[q];
            const size_t gp = vp.pixel_offset + pix;
            ws.T_final[gp] = T[q];
            ws.last[gp] = last[q];
            ws.aux[gp] = D[q];
            ws.aux[ws.total_pixels + gp] = E[q];
        }
    }
    const uint32_t tot = __reduce_add_sync(kFull, ncon);
    if (lane == 0 && tot) atomicAdd(&ws.hdr->pairs_contrib, (unsigned long long)tot);
}

// Sum of 16 per-lane values over the warp (transposing butterfly): lane l
// ends with component l / 2 (both lanes of a pair).
__device__ __forceinline__ float warp_sum16(const float (&v)[kSG], int lane) {
    float a[8], b[4], c[2], d;
    {
        const bool hi = lane & 16;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float send = hi ? v[i] : v[8 + i];
            a[i] = (hi ? v[8 + i] : v[i]) + __shfl_xor_sync(kFull, send, 16);
        }
    }
    {
        const bool hi = lane & 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float send = hi ? a[i] : a[4 + i];
            b[i] = (hi ? a[4 + i] : a[i]) + __shfl_xor_sync(kFull, send, 8);
        }
    }
    {
        const bool hi = lane & 4;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = hi ? b[i] : b[2 + i];
            c[i] = (hi ? b[2 + i] : b[i]) + __shfl_xor_sync(kFull, send, 4);
        }
    }
    {
        const bool hi = lane & 2;
        const float send = hi ? c[0] : c[1];
        d = (hi ? c[1] : c[0]) + __shfl_xor_sync(kFull, send, 2);
    }
    return d + __shfl_xor_sync(kFull, d, 1);
}

// Three quarters of full occupancy: the register cap this sets (80 at tile 16) trades a few
// spilled bytes for more resident warps, which measured faster than the uncapped 100+.
template <int TS>
__global__ void __launch_bounds__(Shape<TS>::THREADS, Shape<TS>::BWD_BLOCKS)
    surfel_blend_bwd_kernel(const __grid_constant__ ViewTable vt, const Ws ws) {
    using S = Shape<TS>;
    __shared__ float4 sE[S::WARPS][kQuads][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile wt = tile_of<TS>(vt, ws);
    const ViewParams &vp = vt.v[wt.v];
    const uint32_t *vals = ws.sorted;
    const size_t N = ws.N, vN = (size_t)wt.v * N;
    const float lxf = (float)(lane & (kSubW - 1)), lyf = (float)(lane / kSubW);
    const float ox = (float)wt.X0 - vp.cx, oy = (float)wt.Y0 - vp.cy;

    float T[kPPL], Q[kPPL], gC[kPPL][3], gN[kPPL][3], gD[kPPL], gA[kPPL], gL[kPPL], At[kPPL], Dt[kPPL], Et[kPPL];
    uint32_t last[kPPL], lmax = 0;
#pragma unroll
    for (int q = 0; q < kPPL; ++q) {
        T[q] = 1.f;
        Q[q] = gD[q] = gA[q] = gL[q] = At[q] = Dt[q] = Et[q] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) gC[q][c] = gN[q][c] = 0.f;
        last[q] = 0;
        const int py = wt.py + q * kRowStep;
        if (wt.px < vp.W && py < vp.H) {
            const size_t HW = (size_t)vp.H * vp.W, pix = (size_t)py * vp.W + wt.px, gp = vp.pixel_offset + pix;
            T[q] = ws.T_final[gp];
            last[q] = ws.last[gp];
            At[q] = 1.f - T[q];
            Dt[q] = ws.aux[gp];
            Et[q] = ws.aux[ws.total_pixels + gp];
            if (vp.d_color)
#pragma unroll
                for (int c = 0; c < 3; ++c) gC[q][c] = vp.d_color[c * HW + pix];
            if (vp.d_normal)
#pragma unroll
                for (int c = 0; c < 3; ++c) gN[q][c] = vp.d_normal[c * HW + pix];
            if (vp.d_depth) gD[q] = vp.d_depth[pix];
            if (vp.d_alpha) gA[q] = vp.d_alpha[pix];
            if (vp.d_distortion) gL[q] = vp.d_distortion[pix];
        }
        lmax = max(lmax, last[q]);
    }
    const uint32_t wlast = __reduce_max_sync(kFull, lmax);
    float *grads = ws.vg_grads + (size_t)wt.v * kSG;
    const size_t row = (size_t)ws.V * kSG;

    for (uint32_t end = wlast; end > wt.range.x;) {
        const uint32_t begin = end - wt.range.x > 32u ? end - 32u : wt.range.x;
        const int n = stage_surfels(ws, vals, vN, begin + lane, end, wt.X0, wt.Y0,
                                    [&](int slot, size_t gi, uint32_t idx, uint32_t g) {
                                        stage_entry(sE[warp], ws, vp, wt.X0, wt.Y0, slot, gi, idx, g);
                                    });
        for (int j = n - 1; j >= 0; --j) {
            const float4 e0 = sE[warp][0][j], e1 = sE[warp][1][j], e2 = sE[warp][2][j];
            const uint32_t eidx = __float_as_uint(e2.w);
            Hit h[kPPL];
            bool contrib[kPPL], any = false;
#pragma unroll
            for (int q = 0; q < kPPL; ++q) {
                surfel_hit(e0, e1, e2, lxf, lyf + (float)(q * kRowStep), h[q]);
                contrib[q] = eidx < last[q] && h[q].s <= e2.z;
                any |= contrib[q];
            }
            const unsigned cmask = __ballot_sync(kFull, any);
            if (cmask == 0u) continue;
            const float4 e3 = sE[warp][3][j], e4 = sE[warp][4][j];
            // per lane, block-relative: dax', dbx', day', dby', da_z, db_z, dp_z, ddu, ddv,
            // then d ln(sigma), colour, normal
            float acc[kSG];
#pragma unroll
            for (int k = 0; k < kSG; ++k) acc[k] = 0.f;
#pragma unroll
            for (int q = 0; q < kPPL; ++q) {
                if (!contrib[q]) continue;
                const Hit &H = h[q];
                const float raw = ex2_approx(__fsub_rn(e1.w, H.s));
                const float alpha = fminf(kAlphaMax, raw);
                const float Ti = T[q] * rcp_approx(1.f - alpha);
                const float w = alpha * Ti;
                const bool disk = H.rho3 <= H.rho2;   // the disk term decides alpha and the depth
                const float z = disk ? fmaf(e1.x, H.u, fmaf(e1.y, H.v, e1.z)) : e1.z;
                // g = dL/dw of this entry: colour, depth, opacity, normal, distortion
                const float gdist = fmaf(z, fmaf(z, At[q], -2.f * Dt[q]), Et[q]);
                const float g = fmaf(gC[q][0], e3.x, fmaf(gC[q][1], e3.y, fmaf(gC[q][2], e3.z,
                                fmaf(gN[q][0], e3.w, fmaf(gN[q][1], e4.x, fmaf(gN[q][2], e4.y,
                                fmaf(gD[q], z, fmaf(gL[q], gdist, gA[q]))))))));
                const float dA = Ti * (g - Q[q]);
                Q[q] = fmaf(alpha, g - Q[q], Q[q]);
                T[q] = Ti;
                const float dz = w * fmaf(2.f * gL[q], fmaf(z, At[q], -Dt[q]), gD[q]);
                acc[10] = fmaf(w, gC[q][0], acc[10]);
                acc[11] = fmaf(w, gC[q][1], acc[11]);
                acc[12] = fmaf(w, gC[q][2], acc[12]);
                acc[13] = fmaf(w, gN[q][0], acc[13]);
                acc[14] = fmaf(w, gN[q][1], acc[14]);
                acc[15] = fmaf(w, gN[q][2], acc[15]);
                const float glo = raw <= kAlphaMax ? dA * raw : 0.f;   // dL/d ln(sigma)
                acc[9] += glo;
                const float drho = -0.5f * glo;
                acc[6] += dz;
                if (!disk) {   // rho2 = 2 ((x - c_x)^2 + (y - c_y)^2), c_x = X0 + du
                    acc[7] -= 2.f * kLowPass * H.dxp * drho;
                    acc[8] -= 2.f * kLowPass * H.dyp * drho;
                    continue;
                }
                const float du = fmaf(2.f * H.u, drho, dz * e1.x);   // z = a_z u + b_z v + p_z
                const float dv = fmaf(2.f * H.v, drho, dz * e1.y);
                acc[4] = fmaf(dz, H.u, acc[4]);
                acc[5] = fmaf(dz, H.v, acc[5]);
                // (u, v) = (q0, q1) / q2
                const float dq0 = du * H.inv, dq1 = dv * H.inv, dq2 = -(du * H.u + dv * H.v) * H.inv;
                // q = h_x x h_y
                const float dhx0 = H.hy1 * dq2 - H.hy2 * dq1, dhx1 = H.hy2 * dq0 - H.hy0 * dq2;
                const float dhx2 = H.hy0 * dq1 - H.hy1 * dq0;
                const float dhy0 = dq1 * H.hx2 - dq2 * H.hx1, dhy1 = dq2 * H.hx0 - dq0 * H.hx2;
                const float dhy2 = dq0 * H.hx1 - dq1 * H.hx0;
                const float lx = lxf, ly = lyf + (float)(q * kRowStep);
                acc[0] += dhx0;
                acc[1] += dhx1;
                acc[2] += dhy0;
                acc[3] += dhy1;
                acc[4] = fmaf(-lx, dhx0, fmaf(-ly, dhy0, acc[4]));
                acc[5] = fmaf(-lx, dhx1, fmaf(-ly, dhy1, acc[5]));
                // h_x2 = -p_z (x - c_x), h_y2 = -p_z (y - c_y)
                acc[6] = fmaf(-H.dxp, dhx2, fmaf(-H.dyp, dhy2, acc[6]));
                acc[7] = fmaf(e1.z, dhx2, acc[7]);
                acc[8] = fmaf(e1.z, dhy2, acc[8]);
            }
            // block-relative -> global: ax' = fx a_x - ox a_z, bx' = fx b_x - ox b_z (and y)
            float gv[kSG];
            gv[0] = vp.fx * acc[0];                                  // a_x
            gv[1] = vp.fy * acc[2];                                  // a_y
            gv[2] = acc[4] - ox * acc[0] - oy * acc[2];              // a_z
            gv[3] = vp.fx * acc[1];                                  // b_x
            gv[4] = vp.fy * acc[3];                                  // b_y
            gv[5] = acc[5] - ox * acc[1] - oy * acc[3];              // b_z
#pragma unroll
            for (int k = 6; k < kSG; ++k) gv[k] = acc[k];            // p_z, u_c, v_c, ln sigma, rgb, n
            float *gp = grads + (size_t)__float_as_uint(e4.z) * row;   // staged ids are < N
            if (__popc(cmask) <= 4) {
                // up to four lanes: their own atomics are cheaper than a reduction
                if (any) {
#pragma unroll
                    for (int k = 0; k < kSG; ++k) atomicAdd(gp + k, gv[k]);
                }
            } else {
                const float sum = warp_sum16(gv, lane);
                if ((lane & 1) == 0) atomicAdd(gp + (lane >> 1), sum);
            }
        }
        __syncwarp();
        end = begin;
    }
}

// ------------------------------------------------------------------ preprocess backward
// One thread per Gaussian walks the views; the SH gradients gather in
// shared memory, the pose twists are summed per view over the block in a
// fixed order.
constexpr int kPB = 128;

template <int DEG>
__global__ void __launch_bounds__(kPB) surfel_pre_bwd_kernel(const __grid_constant__ ViewTable vt,
                                                             const GaussianPtrs gp, const Ws ws, const GradPtrs out) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    __shared__ Pose s_pose[GSR_MAX_VIEWS];
    __shared__ float s_sh[3 * K][kPB];
    __shared__ float s_red[6][kPB / 32];
    load_poses(vt, s_pose);
    const int g = blockIdx.x * kPB + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool real = g < gp.N;
    const size_t N = (size_t)gp.N;
    GaussPre G;
    if (real) gauss_pre(gp, g, G);
    float dmu[3] = {0.f, 0.f, 0.f}, dR[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float dls0 = 0.f, dls1 = 0.f, dlno = 0.f;
    for (int k = 0; k < 3 * K; ++k) s_sh[k][threadIdx.x] = 0.f;
    for (int v = 0; v < vt.V; ++v) {
        const ViewParams &vp = vt.v[v];
        const Pose &ps = s_pose[v];
        float pose6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (real && ws.counts[(size_t)v * N + g] > 0) {
            float4 *sgp = reinterpret_cast<float4 *>(ws.vg_grads + ((size_t)g * ws.V + v) * kSG);
            float sg[kSG];
#pragma unroll
            for (int k = 0; k < kSG / 4; ++k) {
                const float4 x4 = sgp[k];
                sg[4 * k] = x4.x;
                sg[4 * k + 1] = x4.y;
                sg[4 * k + 2] = x4.z;
                sg[4 * k + 3] = x4.w;
            }
            float xh, xl, yh, yl, zh, zl;
            dot3_plus(ps.W[0][0], ps.W[0][1], ps.W[0][2], ps.t[0], G.mx, G.my, G.mz, xh, xl);
            dot3_plus(ps.W[1][0], ps.W[1][1], ps.W[1][2], ps.t[1], G.mx, G.my, G.mz, yh, yl);
            dot3_plus(ps.W[2][0], ps.W[2][1], ps.W[2][2], ps.t[2], G.mx, G.my, G.mz, zh, zl);
            const float p[3] = {xh, yh, zh};
            float Wt[3][3];   // W t_u, W t_v, W t_w (columns 0..2 of W R)
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    Wt[c][k] = ps.W[k][0] * G.R[0][c] + ps.W[k][1] * G.R[1][c] + ps.W[k][2] * G.R[2][c];
            const float flip = Wt[2][0] * xh + Wt[2][1] * yh + Wt[2][2] * zh > 0.f ? -1.f : 1.f;
            const float da[3] = {sg[0], sg[1], sg[2]}, db[3] = {sg[3], sg[4], sg[5]};
            const float dn[3] = {flip * sg[13], flip * sg[14], flip * sg[15]};   // dL/d(W t_w)
            // projected centre u_c = fx x / z + cx, v_c = fy y / z + cy, and the depth p_z
            const float rz = 1.f / zh;
            float dp[3];
            dp[0] = vp.fx * rz * sg[7];
            dp[1] = vp.fy * rz * sg[8];
            dp[2] = sg[6] - (vp.fx * xh * sg[7] + vp.fy * yh * sg[8]) * rz * rz;
            // a = s_u W t_u, b = s_v W t_v (the normal is flip W t_w)
            float a[3], b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a[k] = G.s[0] * Wt[0][k];
                b[k] = G.s[1] * Wt[1][k];
            }
            dls0 += da[0] * a[0] + da[1] * a[1] + da[2] * a[2];
            dls1 += db[0] * b[0] + db[1] * b[1] + db[2] * b[2];
#pragma unroll
            for (int r = 0; r < 3; ++r) {   // d t_c = W^T (s d a) ...
                const float wa = ps.W[0][r] * da[0] + ps.W[1][r] * da[1] + ps.W[2][r] * da[2];
                const float wb = ps.W[0][r] * db[0] + ps.W[1][r] * db[1] + ps.W[2][r] * db[2];
                const float wn = ps.W[0][r] * dn[0] + ps.W[1][r] * dn[1] + ps.W[2][r] * dn[2];
                dR[r][0] += G.s[0] * wa;
                dR[r][1] += G.s[1] * wb;
                dR[r][2] += wn;
            }
            // colour -> SH coefficients and the view direction
            float dx, dy, dz, rn;
            view_dir(G, ps, dx, dy, dz, rn);
            float Y[K];
            sh_eval<DEG>(dx, dy, dz, Y);
            const float4 rgb = ws.rec[4 * ((size_t)v * N + g) + 2];
            const float dr0 = rgb.x > 0.f ? sg[10] : 0.f, dr1 = rgb.y > 0.f ? sg[11] : 0.f,
                        dr2 = rgb.z > 0.f ? sg[12] : 0.f;
            float wk[K];
            const float *shg = gp.sh + g;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                s_sh[3 * k][threadIdx.x] += dr0 * Y[k];
                s_sh[3 * k + 1][threadIdx.x] += dr1 * Y[k];
                s_sh[3 * k + 2][threadIdx.x] += dr2 * Y[k];
                wk[k] = dr0 * __ldg(shg + (size_t)(k * 3) * N) + dr1 * __ldg(shg + (size_t)(k * 3 + 1) * N) +
                        dr2 * __ldg(shg + (size_t)(k * 3 + 2) * N);
            }
            float gdx, gdy, gdz;
            sh_grad<DEG>(dx, dy, dz, wk, gdx, gdy, gdz);
            const float radial = gdx * dx + gdy * dy + gdz * dz;
            const float dv0 = (gdx - dx * radial) * rn, dv1 = (gdy - dy * radial) * rn, dv2 = (gdz - dz * radial) * rn;
            dmu[0] += dv0;
            dmu[1] += dv1;
            dmu[2] += dv2;
            // the camera centre moves by -W^T rho
            pose6[0] += ps.W[0][0] * dv0 + ps.W[0][1] * dv1 + ps.W[0][2] * dv2;
            pose6[1] += ps.W[1][0] * dv0 + ps.W[1][1] * dv1 + ps.W[1][2] * dv2;
            pose6[2] += ps.W[2][0] * dv0 + ps.W[2][1] * dv1 + ps.W[2][2] * dv2;
            dlno += sg[9];
            // p = W mu + t
#pragma unroll
            for (int j = 0; j < 3; ++j) dmu[j] += ps.W[0][j] * dp[0] + ps.W[1][j] * dp[1] + ps.W[2][j] * dp[2];
            // pose twist of T_cw <- Exp(rho, phi) T_cw: p moves by phi x p + rho, the
            // directions a, b, n by phi x (.)
            pose6[0] += dp[0];
            pose6[1] += dp[1];
            pose6[2] += dp[2];
            // (dn = dL/d(W t_w), so the normal's term is (W t_w) x dn)
            pose6[3] += p[1] * dp[2] - p[2] * dp[1] + a[1] * da[2] - a[2] * da[1] + b[1] * db[2] - b[2] * db[1] +
                        Wt[2][1] * dn[2] - Wt[2][2] * dn[1];
            pose6[4] += p[2] * dp[0] - p[0] * dp[2] + a[2] * da[0] - a[0] * da[2] + b[2] * db[0] - b[0] * db[2] +
                        Wt[2][2] * dn[0] - Wt[2][0] * dn[2];
            pose6[5] += p[0] * dp[1] - p[1] * dp[0] + a[0] * da[1] - a[1] * da[0] + b[0] * db[1] - b[1] * db[0] +
                        Wt[2][0] * dn[1] - Wt[2][1] * dn[0];
            // the row is cleared for the next backward, after every load of this pair
#pragma unroll
            for (int k = 0; k < kSG / 4; ++k) __stcs(sgp + k, make_float4(0.f, 0.f, 0.f, 0.f));
        }
        // this block's pose partial of view v, summed in a fixed order
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float x = pose6[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
            if (lane == 0) s_red[c][warp] = x;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            float x = 0.f;
            for (int w = 0; w < kPB / 32; ++w) x += s_red[threadIdx.x][w];
            ws.pose_partials[((size_t)v * ws.pose_blocks + blockIdx.x) * 6 + threadIdx.x] = x;
        }
        __syncthreads();
    }
    if (!real) return;
    const bool ac = out.accumulate != 0;
    for (int k = 0; k < 3 * K; ++k) {
        float *o = out.sh + (size_t)k * N + g;
        *o = ac ? *o + s_sh[k][threadIdx.x] : s_sh[k][threadIdx.x];
    }
    float dqr[4];
    rot_grad_to_quat(G, dR, dqr);
    const float dls[3] = {dls0, dls1, 0.f};
    const float dlogit = dlno * (1.f - G.o);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float *pm = out.means + (size_t)j * N + g;
        float *pl = out.log_scales + (size_t)j * N + g;
        *pm = ac ? *pm + dmu[j] : dmu[j];
        *pl = ac ? *pl + dls[j] : dls[j];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float *pq = out.quats + (size_t)k * N + g;
        *pq = ac ? *pq + dqr[k] : dqr[k];
    }
    float *po = out.opacity_logits + g;
    *po = ac ? *po + dlogit : dlogit;
}

template <int DEG>
cudaError_t pre_fwd_t(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, cudaStream_t st) {
    surfel_pre_fwd_kernel<DEG><<<(gp.N + 127) / 128, 128, 0, st>>>(vt, gp, ws);
    return cudaGetLastError();
}

template <int DEG>
cudaError_t pre_bwd_t(const ViewTable &vt, const GaussianPtrs &gp, Ws ws, const GradPtrs &out, cudaStream_t st) {
    const int blocks = (gp.N + kPB - 1) / kPB;
    ws.pose_blocks = (uint32_t)blocks;   // at most (N + 31) / 32, the workspace's allotment
    surfel_pre_bwd_kernel<DEG><<<blocks, kPB, 0, st>>>(vt, gp, ws, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pose_reduce(vt, ws, out.accumulate, st);
}

}  // namespace

cudaError_t launch_surfel_preprocess_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, cudaStream_t st) {
    if (gp.N == 0) return cudaSuccess;
    switch (gp.sh_degree) {
        case 0: return pre_fwd_t<0>(vt, gp, ws, st);
        case 1: return pre_fwd_t<1>(vt, gp, ws, st);
        case 2: return pre_fwd_t<2>(vt, gp, ws, st);
        default: return pre_fwd_t<3>(vt, gp, ws, st);
    }
}

cudaError_t launch_surfel_preprocess_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws,
                                         const GradPtrs &out, cudaStream_t st) {
    if (gp.N == 0) return launch_pose_reduce(vt, ws, out.accumulate, st);
    switch (gp.sh_degree) {
        case 0: return pre_bwd_t<0>(vt, gp, ws, out, st);
        case 1: return pre_bwd_t<1>(vt, gp, ws, out, st);
        case 2: return pre_bwd_t<2>(vt, gp, ws, out, st);
        default: return pre_bwd_t<3>(vt, gp, ws, out, st);
    }
}

cudaError_t launch_surfel_blend_fwd(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (vt.total_tiles == 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: surfel_blend_fwd_kernel<8><<<vt.total_tiles * Shape<8>::CTAS, Shape<8>::THREADS, 0, st>>>(vt, ws); break;
        case 32: surfel_blend_fwd_kernel<32><<<vt.total_tiles * Shape<32>::CTAS, Shape<32>::THREADS, 0, st>>>(vt, ws); break;
        default: surfel_blend_fwd_kernel<16><<<vt.total_tiles * Shape<16>::CTAS, Shape<16>::THREADS, 0, st>>>(vt, ws); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_surfel_blend_bwd(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (vt.total_tiles == 0) return cudaSuccess;
    switch (vt.tile) {
        case 8: surfel_blend_bwd_kernel<8><<<vt.total_tiles * Shape<8>::CTAS, Shape<8>::THREADS, 0, st>>>(vt, ws); break;
        case 32: surfel_blend_bwd_kernel<32><<<vt.total_tiles * Shape<32>::CTAS, Shape<32>::THREADS, 0, st>>>(vt, ws); break;
        default: surfel_blend_bwd_kernel<16><<<vt.total_tiles * Shape<16>::CTAS, Shape<16>::THREADS, 0, st>>>(vt, ws); break;
    }
    return cudaGetLastError();
}

}  // namespace gsr
