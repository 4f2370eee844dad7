// preprocess.cu -- forward projection of every (view, Gaussian) pair
// (activation, camera transform, EWA projection, SH colour, exact tile count)
// and its backward (projection/SH chain rule, per-view SE(3) pose reduction).
//
// Forward: persistent warps take work items of 32 Gaussians (one per lane)
// and up to 8 views; each warp projects every pair of an item, queues the
// visible ones in shared memory and gives the expensive part (tile count, SH
// colour, the pair's 64-byte record, per-tile keys) to full warps of visible
// pairs.
// Backward: persistent blocks take groups of Gaussians with all their views;
// a group's visible (view, Gaussian) pairs are compacted Gaussian-major so
// that warps work on visible pairs only, the per-pair gradients are summed
// over views in shared memory in a fixed order (the result does not depend on
// timing), and each pair's screen-gradient row is cleared after it is read.
#include <algorithm>
#include <mutex>

#include "kernels.cuh"
#include "project.cuh"
#include "sh.cuh"
#include "spans.cuh"

namespace gsr {

constexpr int kPreWarps = 8;
constexpr int kPreThreads = 32 * kPreWarps;
// Resident blocks per SM of the forward kernel (its register budget).
constexpr int kPreFwdBlocksPerSM = 3;

// ------------------------------------------------------------------ forward
// Warp-queue forward: persistent warps take batches of 32 Gaussians (one per
// lane, parameters activated once per batch) and walk their views.  Phase A
// projects the 32 pairs of one view; the visible ones are appended, with
// their projected state, to the warp's shared-memory queue.  Whenever 32 are
// queued, phase B gives them to the 32 lanes: tile count, SH colour and
// records.  Warps never wait for each other, and the expensive part runs
// with full warps however few pairs are visible.
constexpr int kQueue = 64;   // a warp's queue: up to 31 waiting + 32 appended
// Views of one forward work item: 8, or kPreSmallItemViews when 8 would leave
// the warps fewer than kPreItemsPerWarp items each (the window, with the
// forward no longer clearing gradient rows: 4-view items 0.0472 ms against
// 0.0487 with 2 and 0.0512 with 8; on the 16- and 32-view workloads 2
// measured 7 % slower than 4, 1 view per item slower still, and 8 faster
// than 4: uneven 0.387 -> 0.372 ms, outdoor 2.406 -> 2.391 ms).
constexpr int kPreItemsPerWarp = 4;
constexpr int kPreItemViews = 8;
constexpr int kPreSmallItemViews = 4;

struct WarpQueue {
    float uh[kQueue], vh[kQueue], ul[kQueue], vl[kQueue];
    float m00[kQueue], m01[kQueue], m11[kQueue];
    float sxx[kQueue], sxy[kQueue], syy[kQueue], zh[kQueue];
    float log2o[kQueue], smax[kQueue];            // the Gaussian's, from the activation of phase A
    float dx[kQueue], dy[kQueue], dz[kQueue];     // unit view direction (camera centre to mean)
    int v[kQueue], g[kQueue];
};

// Phase B for queue entry k of one lane; called by the whole warp, the lanes
// without an entry (a partly filled queue at the end) with active false.
// Returns whether the pair got tile keys and records.
template <int DEG>
__device__ __forceinline__ bool preprocess_fwd_pair(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws,
                                                    const Pose *s_pose, const WarpQueue &q, int k, bool active) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const size_t N = (size_t)gp.N;
    if (!active) k = 0;   // entry 0 is filled whenever a lane is active
    const int pv = q.v[k], pg = q.g[k];
    const ViewParams &vp = vt.v[pv];
    const size_t i = (size_t)pv * N + pg;
    const float puh = q.uh[k], pvh = q.vh[k], m00 = q.m00[k];
    const float sxx = q.sxx[k], sxy = q.sxy[k], syy = q.syy[k];
    const float log2o = q.log2o[k], smax = q.smax[k];
    uint32_t count = 0u;
    if (active) {
        count = visit_tile_spans(puh, pvh, sxx, sxy, syy, m00, smax, vp.W, vp.H, vt.tile, [](int, int, int) {});
        ws.counts[i] = count;
    }
    if (keys_in_preprocess(ws)) {
        // the warp's keys: an inclusive scan of the counts (at most 32 views'
        // worth of tiles, 2^27, so 32 bits hold it) and one reservation
        const int lane = threadIdx.x & 31;
        uint32_t incl = count;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o2);
            if (lane >= o2) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0ull;
        if (lane == 31 && total != 0u) {
            base = atomicAdd(&ws.hdr->keys, (unsigned long long)total);
            if (base + total > ws.cap) set_status(ws.hdr, GSR_ECAPACITY);
        }
        base = __shfl_sync(0xffffffffu, base, 31);
        if (count != 0u) {
            // per-tile key layout: tile id in vals, (depth bits, id) word in keys
            const unsigned long long word = ((unsigned long long)__float_as_uint(q.zh[k]) << 32) | (uint32_t)pg;
            const uint32_t cap = ws.cap;
            unsigned long long pos = base + (incl - count);
            const uint32_t emitted =
                visit_tile_spans(puh, pvh, sxx, sxy, syy, m00, smax, vp.W, vp.H, vt.tile, [&](int ty, int tx0, int tx1) {
                    const uint32_t row = vp.tile_offset + (uint32_t)ty * vp.tiles_x;
                    for (int tx = tx0; tx <= tx1; ++tx, ++pos)
                        if (pos < cap) {
                            ws.vals[0][pos] = row + (uint32_t)tx;
                            ws.keys[0][pos] = word;
                        }
                });
            if (emitted != count) set_status(ws.hdr, GSR_EINTERNAL);
        }
    }
    if (count == 0u) return false;
    float Y[K];
    sh_eval<DEG>(q.dx[k], q.dy[k], q.dz[k], Y);
    float rgb[3];
    // every coefficient load issued before the sums, so that their latencies
    // overlap (one channel at a time: uneven preprocess 0.446 -> 0.491 ms)
    float cf[3][K];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) cf[c][j] = __ldg(gp.sh + ((size_t)j * 3 + c) * N + pg);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.5f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc = fmaf(cf[c][j], Y[j], acc);
        rgb[c] = fmaxf(acc, 0.f);
    }
    float4 *rec = ws.rec + 4 * i;
    rec[0] = make_float4(puh, pvh, q.ul[k], q.vl[k]);
    rec[1] = make_float4(m00, q.m01[k], q.m11[k], smax);
    rec[2] = make_float4(rgb[0], rgb[1], rgb[2], q.zh[k]);
    rec[3] = make_float4(log2o, sxx, sxy, syy);
    return true;
}

// The grid's share of zeroing every (Gaussian, view) gradient row (kept out
// of line: it runs only when a layout's rows are not known clean).
__device__ __noinline__ void clear_rows(const Ws &ws) {
    float2 *rows = reinterpret_cast<float2 *>(ws.vg_grads);
    const size_t n = (size_t)ws.N * ws.V * (kVGGrads / 2);
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        rows[k] = make_float2(0.f, 0.f);
}

template <int DEG>
__global__ void __launch_bounds__(kPreThreads, kPreFwdBlocksPerSM) preprocess_fwd_kernel(const __grid_constant__ ViewTable vt,
                                                                     const GaussianPtrs gp, const Ws ws,
                                                                     int item_views) {
    __shared__ Pose s_pose[GSR_MAX_VIEWS];
    __shared__ WarpQueue s_q[kPreWarps];
    load_poses(vt, s_pose);
    // The blend backward accumulates the visible pairs' screen gradients into
    // rows that must be zero; unless the header records this layout's rows
    // as clean, all blocks clear them first (their last use was the blend
    // backward of another layout, or nothing).  Clearing only the visible
    // pairs' rows in every forward cost the outdoor preprocess 0.55 of 2.4 ms.
    if (!rows_known_clean(ws)) clear_rows(ws);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpQueue &q = s_q[warp];
    const size_t N = (size_t)gp.N;
    // Work items: a batch of 32 Gaussians with up to item_views views.
    // With more views than that, warps take the items in turn from a counter
    // in the workspace header (zeroed by the init kernel), so that warps with
    // light items take more of them (window preprocess 0.066 -> 0.060 ms,
    // 32 views 5.1 -> 4.3 ms); with one item per batch the warps take the
    // batches in a fixed order.
    const int nbatch = (gp.N + 31) / 32, nsplit = (vt.V + item_views - 1) / item_views;
    const int nitems = nbatch * nsplit, nwarps = gridDim.x * kPreWarps;
    const bool dynamic = nsplit > 1;
    int qn = 0;   // queued pairs (the same in every lane)
    uint32_t visible = 0;   // pairs of this lane that got records
    int it = blockIdx.x * kPreWarps + warp;
    if (dynamic) {
        if (lane == 0) it = (int)atomicAdd(&ws.hdr->pre_items, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
    }
    while (it < nitems) {
        const int b = it / nsplit, part = it - b * nsplit;
        const int v0 = part * item_views, v1 = min(vt.V, v0 + item_views);
        const int g = b * 32 + lane;
        const bool real = g < gp.N;
        GaussPre G;
        if (real) gauss_pre(gp, g, G);
        for (int v = v0; v < v1; ++v) {
            // phase A: projection and visibility of (v, the 32 Gaussians)
            bool vis = false;
            float uh = 0.f, ul = 0.f, vh = 0.f, vl = 0.f;
            Proj p;
            if (real) {
                const ViewParams &vp = vt.v[v];
                float rad = 0.f;
                if (G.alive && project_view(G, s_pose[v], vp, p)) {
                    project_coord(vp.fx, vp.cx, p.xh, p.xl, p.zh, p.zl, p.rz, uh, ul);
                    project_coord(vp.fy, vp.cy, p.yh, p.yl, p.zh, p.zl, p.rz, vh, vl);
                    vis = isfinite(uh) && isfinite(vh);
                    // densification visibility: the cutoff ellipse meets the
                    // rectangle of pixel centres.  The same minimum, with the
                    // blend's culling tolerance, drops the pairs that reach no
                    // pixel centre before the tile count and the SH colour.
                    if (vis) {
                        const float u = uh + ul, w = vh + vl;
                        const float dx0 = -u, dx1 = (float)(vp.W - 1) - u, dy0 = -w, dy1 = (float)(vp.H - 1) - w;
                        const float m00 = kSqrtHalfLog2e * p.l00, m01 = kSqrtHalfLog2e * p.l01,
                                    m11 = kSqrtHalfLog2e * p.l11;
                        const float smin = quad_min_over_box(dx0, dx1, dy0, dy1, m00, m01, m11);
                        if (smin <= G.smax) {
                            const float mid = 0.5f * (p.sxx + p.syy);
                            rad = 3.f * sqrtf(mid + sqrtf(fmaxf(mid * mid - p.det, 0.f)));
                        }
                        vis = smin <= G.smax + cull_slack(dx0, dx1, dy0, dy1, m00, m01, m11, G.smax);
                    }
                }
                if (!vis) ws.counts[(size_t)v * N + g] = 0u;
                ws.radius[(size_t)v * N + g] = rad;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, vis);
            if (vis) {
                const int k = qn + __popc(ball & lanemask_lt());
                q.uh[k] = uh;
                q.vh[k] = vh;
                q.ul[k] = ul;
                q.vl[k] = vl;
                q.m00[k] = kSqrtHalfLog2e * p.l00;
                q.m01[k] = kSqrtHalfLog2e * p.l01;
                q.m11[k] = kSqrtHalfLog2e * p.l11;
                q.sxx[k] = p.sxx;
                q.sxy[k] = p.sxy;
                q.syy[k] = p.syy;
                q.zh[k] = p.zh;
                q.log2o[k] = G.log2o;
                q.smax[k] = G.smax;
                // the SH view direction, from the camera centre to the mean
                const Pose &ps = s_pose[v];
                float dx = G.mx - ps.C[0], dy = G.my - ps.C[1], dz = G.mz - ps.C[2];
                const float rn = rsqrt_approx(dx * dx + dy * dy + dz * dz);
                q.dx[k] = dx * rn;
                q.dy[k] = dy * rn;
                q.dz[k] = dz * rn;
                q.v[k] = v;
                q.g[k] = g;
            }
            qn += __popc(ball);
            if (qn >= 32) {   // phase B on the first 32, then move the rest to the front
                __syncwarp();
                visible += preprocess_fwd_pair<DEG>(vt, gp, ws, s_pose, q, lane, true);
                __syncwarp();
                if (lane < qn - 32) {
                    const int k = 32 + lane;
                    q.uh[lane] = q.uh[k];
                    q.vh[lane] = q.vh[k];
                    q.ul[lane] = q.ul[k];
                    q.vl[lane] = q.vl[k];
                    q.m00[lane] = q.m00[k];
                    q.m01[lane] = q.m01[k];
                    q.m11[lane] = q.m11[k];
                    q.sxx[lane] = q.sxx[k];
                    q.sxy[lane] = q.sxy[k];
                    q.syy[lane] = q.syy[k];
                    q.zh[lane] = q.zh[k];
                    q.log2o[lane] = q.log2o[k];
                    q.smax[lane] = q.smax[k];
                    q.dx[lane] = q.dx[k];
                    q.dy[lane] = q.dy[k];
                    q.dz[lane] = q.dz[k];
                    q.v[lane] = q.v[k];
                    q.g[lane] = q.g[k];
                }
                qn -= 32;
                __syncwarp();
            }
        }
        if (dynamic) {
            if (lane == 0) it = (int)atomicAdd(&ws.hdr->pre_items, 1u);
            it = __shfl_sync(0xffffffffu, it, 0);
        } else {
            it += nwarps;
        }
    }
    __syncwarp();
    if (qn > 0) visible += preprocess_fwd_pair<DEG>(vt, gp, ws, s_pose, q, lane, lane < qn);
    // the pairs that got records: one counter add per warp
    visible = __reduce_add_sync(0xffffffffu, visible);
    if (lane == 0 && visible) atomicAdd(&ws.hdr->pairs_visible, visible);
}

// ------------------------------------------------------------------ backward
// A block owns GBT Gaussians and all V views (VW = V rounded up to a power
// of two).  Its candidate (view, Gaussian) pairs are taken Gaussian-major,
// 256 per round; the visible ones are appended, in candidate order, to a
// shared-memory list, so that every Gaussian's visible views form one
// contiguous run, in view order.  The list is then worked through 256 pairs
// at a time with full warps: each pair's partial gradients go to its
// shared-memory column; a Gaussian's run is summed in list order (a run cut
// by the end of a chunk carries its partial sum into the next) and, once
// complete, turned into the parameter gradients.  Per-view pose partials are
// summed in list order.  Deterministic.
template <int DEG>
struct BwdAcc {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    static constexpr int NV = 13 + 3 * K;   // dmu (3), dM (9), d ln(sigma) (1), dSH (3K)
    static constexpr int NS = NV + 1;       // + densification: |(dL/du, dL/dv)|
    static constexpr int NVP = NS | 1;      // odd row stride of the per-pair partials in shared memory
    // shared-memory floats of the partials and of the run totals (one view
    // needs neither: each pair is finished by its own thread)
    __host__ __device__ static constexpr int parts(int VW) { return VW == 1 ? 0 : NVP * kPreThreads; }
    __host__ __device__ static constexpr int tots(int VW, int GBT) { return VW == 1 ? 0 : 13 * GBT; }
};

// Backward of one visible (view, Gaussian) pair; writes its NV partials to
// part[k], its screen-gradient norm |(dL/du, dL/dv)| (densification) to
// part[NV], and its pose twist to pose[c * kPreThreads].
template <int DEG>
__device__ __forceinline__ void pair_backward(const GaussianPtrs &gp, const Ws &ws, const ViewParams &vp,
                                              const Pose &ps, int v, int g, float *part, float *pose) {
    constexpr int K = BwdAcc<DEG>::K;
    const size_t N = (size_t)gp.N;
    const size_t i = (size_t)v * N + g;
    // the forward's colour, loaded first: its latency overlaps the projection
    // (the blend's screen gradients loaded here too: uneven 0.805 -> 0.827 ms)
    const float4 rgb = __ldg(ws.rec + 4 * i + 2);
    GaussPre G;
    gauss_pre(gp, g, G);
    Proj p;
    float pose6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float dmu[3] = {0.f, 0.f, 0.f}, dM[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) dM[k] = 0.f;
    float dlno = 0.f;
    if (!project_view(G, ps, vp, p)) {   // same decision as the forward; kept for safety
        float2 *row = reinterpret_cast<float2 *>(ws.vg_grads + ((size_t)g * ws.V + v) * kVGGrads);
#pragma unroll
        for (int c = 0; c < kVGGrads / 2; ++c) row[c] = make_float2(0.f, 0.f);   // rows stay clean
#pragma unroll
        for (int k = 0; k < BwdAcc<DEG>::NS; ++k) part[k] = 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c) pose[c * kPreThreads] = 0.f;
        return;
    }
    float sg[kVGGrads];
    float2 *row = reinterpret_cast<float2 *>(ws.vg_grads + ((size_t)g * ws.V + v) * kVGGrads);
#pragma unroll
    for (int c = 0; c < kVGGrads / 2; ++c) {   // one 40-byte row, 8-byte aligned
        const float2 x = row[c];
        sg[2 * c] = x.x;
        sg[2 * c + 1] = x.y;
    }
    float dpc[3] = {0.f, 0.f, 0.f};

    // colour -> SH coefficients and the view direction; the forward's stored
    // colour is max(0, raw), so a zero channel was clamped (no gradient)
    float dx, dy, dz, rn;
    view_dir(G, ps, dx, dy, dz, rn);
    float Y[K];
    sh_eval<DEG>(dx, dy, dz, Y);
    const float dr0 = rgb.x > 0.f ? sg[6] : 0.f, dr1 = rgb.y > 0.f ? sg[7] : 0.f, dr2 = rgb.z > 0.f ? sg[8] : 0.f;
    float wk[K];
    const float *shg = gp.sh + g;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        part[13 + k * 3] = dr0 * Y[k];
        part[14 + k * 3] = dr1 * Y[k];
        part[15 + k * 3] = dr2 * Y[k];
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
    // the camera centre moves by -W^T rho: dL/drho gets -W dL/dC with dL/dC = -dv
    pose6[0] += ps.W[0][0] * dv0 + ps.W[0][1] * dv1 + ps.W[0][2] * dv2;
    pose6[1] += ps.W[1][0] * dv0 + ps.W[1][1] * dv1 + ps.W[1][2] * dv2;
    pose6[2] += ps.W[2][0] * dv0 + ps.W[2][1] * dv1 + ps.W[2][2] * dv2;

    // the blend returns dL/d ln(sigma); the logit chain is applied once at the end
    dlno = sg[5];

    // pixel mean and depth: the blend returns the sums of dL/dp1 and dL/dp2
    // (p = m d, d = pixel - mean), so dL/du = -m00 S1, dL/dv = -(m01 S1 + m11 S2)
    const float x = p.xh, y = p.yh, z = p.zh, rz = p.rz;
    // The blend sums dL/dp1, dL/dp2 and their products with the offsets
    // without the factor -2 ln 2 of dL/dp = 2 p dL/ds (dL/ds = -ln 2 dL/d ln
    // sigma, per pixel), which comes in here, once per (view, Gaussian).
    const float du = -kRowScale * p.l00 * sg[0];
    const float dvv = -kRowScale * (p.l01 * sg[0] + p.l11 * sg[1]);
    dpc[0] += du * vp.fx * rz;
    dpc[1] += dvv * vp.fy * rz;
    dpc[2] += -(du * vp.fx * x + dvv * vp.fy * y) * rz * rz + sg[9];

    // Cholesky factor of Sigma'^-1 -> Sigma' = [[A, B], [B, C]]
    const float A = p.sxx, B = p.sxy, C = p.syy, det = p.det, idet = rcp_approx(det), iC = rcp_approx(C);
    const float dl00 = kRowScale * sg[2], dl01 = kRowScale * sg[3], dl11 = kRowScale * sg[4];
    const float rdc = rsqrt_approx(det * C);
    const float dA = -0.5f * C * idet * (dl00 * p.l00 + dl01 * p.l01);
    const float dB = dl00 * p.l00 * B * idet + dl01 * (p.l01 * B * idet - rdc);
    const float dC = dl00 * 0.5f * p.l00 * (iC - A * idet) - dl01 * 0.5f * p.l01 * (A * idet + iC) -
                     dl11 * 0.5f * p.l11 * iC;
    // Sigma' = P P^T + 0.3 I
    float dP[2][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        dP[0][j] = 2.f * dA * p.P[0][j] + dB * p.P[1][j];
        dP[1][j] = dB * p.P[0][j] + 2.f * dC * p.P[1][j];
    }
    // P = T M
    float dT[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) dT[r][k] = dP[r][0] * G.M[k][0] + dP[r][1] * G.M[k][1] + dP[r][2] * G.M[k][2];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) dM[k * 3 + j] += p.T[0][k] * dP[0][j] + p.T[1][k] * dP[1][j];
    // T = J W  (J = [[J00, 0, J02], [0, J11, J12]])
    const float dJ00 = dT[0][0] * ps.W[0][0] + dT[0][1] * ps.W[0][1] + dT[0][2] * ps.W[0][2];
    const float dJ02 = dT[0][0] * ps.W[2][0] + dT[0][1] * ps.W[2][1] + dT[0][2] * ps.W[2][2];
    const float dJ11 = dT[1][0] * ps.W[1][0] + dT[1][1] * ps.W[1][1] + dT[1][2] * ps.W[1][2];
    const float dJ12 = dT[1][0] * ps.W[2][0] + dT[1][1] * ps.W[2][1] + dT[1][2] * ps.W[2][2];
    float dW[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        dW[0][j] = p.J00 * dT[0][j];
        dW[1][j] = p.J11 * dT[1][j];
        dW[2][j] = p.J02 * dT[0][j] + p.J12 * dT[1][j];
    }
    // J(p) with clamped x/z, y/z
    const float rz2 = rz * rz;
    dpc[2] += -(dJ00 * vp.fx + dJ11 * vp.fy) * rz2;
    if (p.clx) {
        dpc[2] += dJ02 * vp.fx * p.txz * rz2;
    } else {
        dpc[0] += -dJ02 * vp.fx * rz2;
        dpc[2] += 2.f * dJ02 * vp.fx * x * rz2 * rz;
    }
    if (p.cly) {
        dpc[2] += dJ12 * vp.fy * p.tyz * rz2;
    } else {
        dpc[1] += -dJ12 * vp.fy * rz2;
        dpc[2] += 2.f * dJ12 * vp.fy * y * rz2 * rz;
    }
    // p = W mu + t
#pragma unroll
    for (int j = 0; j < 3; ++j) dmu[j] += ps.W[0][j] * dpc[0] + ps.W[1][j] * dpc[1] + ps.W[2][j] * dpc[2];
    // pose twist of T_cw <- Exp(rho, phi) T_cw
    pose6[0] += dpc[0];
    pose6[1] += dpc[1];
    pose6[2] += dpc[2];
    pose6[3] += y * dpc[2] - z * dpc[1];
    pose6[4] += z * dpc[0] - x * dpc[2];
    pose6[5] += x * dpc[1] - y * dpc[0];
    float Am[3][3];  // dW W^T
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) Am[r][k] = dW[r][0] * ps.W[k][0] + dW[r][1] * ps.W[k][1] + dW[r][2] * ps.W[k][2];
    pose6[3] += Am[2][1] - Am[1][2];
    pose6[4] += Am[0][2] - Am[2][0];
    pose6[5] += Am[1][0] - Am[0][1];

#pragma unroll
    for (int k = 0; k < 3; ++k) part[k] = dmu[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) part[3 + k] = dM[k];
    part[12] = dlno;
    part[BwdAcc<DEG>::NV] = sqrtf(du * du + dvv * dvv);   // densification
    // the row is cleared for the next backward, after every load of this pair
#pragma unroll
    for (int c = 0; c < kVGGrads / 2; ++c) __stcs(row + c, make_float2(0.f, 0.f));
#pragma unroll
    for (int c = 0; c < 6; ++c) pose[c * kPreThreads] = pose6[c];
}

// Rounds of 256 candidates per block, and Gaussians per block.
template <int VW>
struct BwdShape {
    static constexpr int GB = kPreThreads / VW;                   // Gaussians per round
    // Candidate rounds per group: 6 (192 Gaussians at 8 views, 12 rounds at
    // 16) fill the chunks better than 3 (window backward 0.056 -> 0.045 ms);
    // one view keeps 3 (768 Gaussians, enough groups for the blocks), two
    // views and 32 or more keep 3 rounds per 8 views (so that two blocks'
    // shared memory still fits an SM).
    static constexpr int R = (VW == 4 || VW == 8) ? 6 : (VW == 16 ? 12 : (VW <= 8 ? 3 : 3 * VW / 8));
    static constexpr int GBT = R * GB;
    static constexpr int LC = R * kPreThreads;                    // list capacity
};

// Shared-memory bytes of preprocess_bwd_kernel<DEG, VW>.
template <int DEG, int VW>
static size_t bwd_smem_bytes() {
    using S = BwdShape<VW>;
    constexpr size_t NS = BwdAcc<DEG>::NS;
    return sizeof(unsigned long long) * S::GBT +
           sizeof(float) * (BwdAcc<DEG>::parts(VW) + 6 * kPreThreads + BwdAcc<DEG>::tots(VW, S::GBT) + 2 * NS + 6 * VW) +
           sizeof(int) * (S::LC + 5 * S::GBT);
}

// Densification statistics of Gaussian g: overwritten, or gathered with
// the earlier ones when accumulating (sums for grad and count, max radius).
__device__ __forceinline__ void densify_write(const GradPtrs &out, int g, float grad, float count, float radius) {
    const bool ac = out.accumulate != 0;
    out.densify_grad[g] = ac ? out.densify_grad[g] + grad : grad;
    out.densify_count[g] = ac ? out.densify_count[g] + count : count;
    out.densify_radius[g] = ac ? fmaxf(out.densify_radius[g], radius) : radius;
}

// Parameter gradients of Gaussian g from its view-summed partials (acc:
// dmu (3), dM (9), d ln(sigma) (1)).
__device__ __forceinline__ void bwd_finish(const GaussianPtrs &gp, const GradPtrs &out, int g, const float *acc) {
    const size_t N = (size_t)gp.N;
    const bool ac = out.accumulate != 0;
    GaussPre G;
    gauss_pre(gp, g, G);
    const float *dmu = acc, *dM = acc + 3;
    // M = R diag(s) -> log-scales and the rotation
    float dR[3][3], dls[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float ds = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            ds += dM[r * 3 + j] * G.R[r][j];
            dR[r][j] = dM[r * 3 + j] * G.s[j];
        }
        dls[j] = ds * G.s[j];
    }
    float dqr[4];
    rot_grad_to_quat(G, dR, dqr);
    const float dlogit = acc[12] * (1.f - G.o);   // d ln(sigmoid(l)) / dl = 1 - sigma
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

// One group of GBT Gaussians (group grp: Gaussians grp GBT ...) with all views.
template <int DEG, int VW>
__device__ __forceinline__ void preprocess_bwd_group(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws,
                                                     const GradPtrs &out, const Pose *s_poses, int grp) {
    using S = BwdShape<VW>;
    constexpr int K = BwdAcc<DEG>::K, NV = BwdAcc<DEG>::NV, NS = BwdAcc<DEG>::NS, NVP = BwdAcc<DEG>::NVP;
    constexpr int GB = S::GB, GBT = S::GBT, WARPS = kPreThreads / 32;
    extern __shared__ __align__(16) unsigned long long smem_u64[];
    unsigned long long *s_mask = smem_u64;             // [GBT] visible views of each Gaussian
    float *s_part = reinterpret_cast<float *>(s_mask + GBT);   // [256][NVP] per-pair partials of a chunk
    float *s_pose = s_part + BwdAcc<DEG>::parts(VW);   // [6][256] per-pair pose twists
    float *s_tot = s_pose + 6 * kPreThreads;           // [GBT][13] each Gaussian's view-summed totals
    float *s_carry = s_tot + BwdAcc<DEG>::tots(VW, GBT);   // [2][NS] partial sums of a run cut by a chunk's end
    float *s_vpose = s_carry + 2 * NS;                 // [VW][6] pose partials per view
    int *s_item = reinterpret_cast<int *>(s_vpose + 6 * VW);   // [LC] (Gaussian << 8 | view) per list position
    int *s_first = s_item + S::LC;                     // [GBT] list position of each Gaussian's run
    int *s_cnt = s_first + GBT;                        // [GBT] its length
    float *s_dgrad = reinterpret_cast<float *>(s_cnt + GBT);   // [GBT] densification: summed gradient norms
    int *s_dcount = reinterpret_cast<int *>(s_dgrad + GBT);    // [GBT] visible views
    int *s_drad = s_dcount + GBT;                      // [GBT] max screen radius (bits of a float >= 0)
    __shared__ int s_wcnt[WARPS];
    __shared__ unsigned s_wbal[WARPS];
    __shared__ int s_end[kPreThreads];                 // chunk positions where a run ends
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gbase = grp * GBT;
    const size_t N = (size_t)gp.N;
    const bool ac = out.accumulate != 0, dens = out.densify_grad != nullptr;
    for (int k = tid; k < 6 * VW; k += kPreThreads) s_vpose[k] = 0.f;
    for (int k = tid; k < GBT; k += kPreThreads) {
        s_dgrad[k] = 0.f;
        s_dcount[k] = 0;
        s_drad[k] = 0;
    }
    __syncthreads();

    // The list of visible pairs, Gaussian-major: candidate t of round r is
    // view t % VW of Gaussian r GB + t / VW.  A Gaussian's candidates are VW
    // consecutive lanes of one warp (two whole warps when VW = 64).
    int M = 0;
    for (int r = 0; r < S::R; ++r) {
        const int gl = r * GB + tid / VW, v = tid % VW, g = gbase + gl;
        const bool vis = v < vt.V && g < gp.N && ws.counts[(size_t)v * N + g] > 0;
        const unsigned bal = __ballot_sync(0xffffffffu, vis);
        if (lane == 0) {
            s_wcnt[warp] = __popc(bal);
            s_wbal[warp] = bal;
        }
        __syncthreads();
        int before = 0, nvis = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const int c = s_wcnt[w];
            before += w < warp ? c : 0;
            nvis += c;
        }
        if (vis) s_item[M + before + __popc(bal & lanemask_lt())] = (gl << 8) | v;
        if (dens && v < vt.V && g < gp.N) {   // densification visibility, from the forward
            const float rad = ws.radius[(size_t)v * N + g];
            if (rad > 0.f) {
                atomicAdd(&s_dcount[gl], 1);
                atomicMax(&s_drad[gl], __float_as_int(rad));
            }
        }
        if constexpr (VW <= 32) {
            const int lead = lane & ~(VW - 1);
            if (lane == lead) {
                const unsigned gbits = (bal >> lead) & (VW == 32 ? 0xffffffffu : ((1u << VW) - 1u));
                s_first[gl] = M + before + __popc(bal & ((1u << lead) - 1u));
                s_cnt[gl] = __popc(gbits);
                s_mask[gl] = gbits;
            }
        } else if (lane == 0 && (warp & 1) == 0) {
            s_first[gl] = M + before;
            s_cnt[gl] = s_wcnt[warp] + s_wcnt[warp + 1];
            s_mask[gl] = (unsigned long long)s_wbal[warp] | ((unsigned long long)s_wbal[warp + 1] << 32);
        }
        M += nvis;
        __syncthreads();
    }

    for (int c0 = 0, chunk = 0; c0 < M; c0 += kPreThreads, ++chunk) {
        const int n = min(kPreThreads, M - c0);
        // carries alternate between two buffers: one chunk reads the previous
        // chunk's while it writes its own
        const float *carry_in = s_carry + ((chunk + 1) & 1) * NS;
        float *carry_out = s_carry + (chunk & 1) * NS;
        if constexpr (VW == 1) {
            // one view: every run is one pair, finished by its own thread
            if (tid < n) {
                const int gl = s_item[c0 + tid] >> 8, g = gbase + gl;
                float part[NS];
                pair_backward<DEG>(gp, ws, vt.v[0], s_poses[0], 0, g, part, s_pose + tid);
                for (int k = 13; k < NV; ++k) {
                    float *o = out.sh + (size_t)(k - 13) * N + g;
                    *o = ac ? *o + part[k] : part[k];
                }
                bwd_finish(gp, out, g, part);
                s_dgrad[gl] = part[NV];
            }
            __syncthreads();
            if (warp == 0) {   // the view's pose partial, lanes striding the chunk, then a butterfly
                float pv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int p = lane; p < n; p += 32)
#pragma unroll
                    for (int c = 0; c < 6; ++c) pv[c] += s_pose[c * kPreThreads + p];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) pv[c] += __shfl_xor_sync(0xffffffffu, pv[c], o);
                }
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < 6; ++c) s_vpose[c] += pv[c];
            }
            __syncthreads();
            continue;
        }
        int item = 0;
        bool end = false;
        if (tid < n) {
            item = s_item[c0 + tid];
            const int v = item & 0xff, g = gbase + (item >> 8);
            pair_backward<DEG>(gp, ws, vt.v[v], s_poses[v], v, g, s_part + tid * NVP, s_pose + tid);
            end = tid + 1 == n || (s_item[c0 + tid + 1] >> 8) != (item >> 8);
        }
        // positions where a run ends in this chunk, in order
        const unsigned bal = __ballot_sync(0xffffffffu, end);
        if (lane == 0) s_wcnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, nruns = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const int c = s_wcnt[w];
            before += w < warp ? c : 0;
            nruns += c;
        }
        if (end) s_end[before + __popc(bal & lanemask_lt())] = tid;
        __syncthreads();
        // run sums over this chunk, plus the carry of a run begun earlier: an
        // item is (run, component), components fastest, so that a warp reads
        // consecutive words of a partials row
        const int nk = dens ? NS : NV;   // components summed per run
        for (int idx = tid; idx < nk * nruns; idx += kPreThreads) {
            const int j = idx / nk, k = idx - j * nk;
            const int p = s_end[j], gl = s_item[c0 + p] >> 8;
            const int first = s_first[gl];
            float x = first < c0 ? carry_in[k] : 0.f;
            for (int q = max(first, c0) - c0; q <= p; ++q) x += s_part[q * NVP + k];
            if (c0 + p + 1 < first + s_cnt[gl]) {
                carry_out[k] = x;   // continues in the next chunk
            } else if (k < 13) {
                s_tot[gl * 13 + k] = x;
            } else if (k == NV) {
                s_dgrad[gl] = x;
            } else {
                float *o = out.sh + (size_t)(k - 13) * N + gbase + gl;
                *o = ac ? *o + x : x;
            }
        }
        // pose partials per view, in list order.  With 32 or more views a
        // Gaussian is visible in many of them, so a chunk holds few runs:
        // one thread per view walks them (outdoor, 32 views: 4.54 ms against
        // 5.41 with the warps below); with fewer views the runs are many and
        // the walk would keep most of the block waiting at its barrier
        // (uneven, 16 views: the warps take 0.799 against 0.854 ms).
        if (VW >= 32) {
            // eight lanes per view walk the runs ending in this chunk (lane
            // part of the eight takes runs part, part + 8, ...) and pick
            // their view's entry from the Gaussian's mask; a fixed xor tree
            // adds the eight sums (one thread per view left 7/8 of the block
            // at the barrier: outdoor 4.06 -> 3.76 ms)
            const int part = lane & 7;
            for (int v = tid >> 3; v < VW; v += kPreThreads / 8) {   // the same trip count in a warp
                float pv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (v < vt.V) {
                    for (int j = part; j < nruns; j += 8) {
                        const int gl = s_item[c0 + s_end[j]] >> 8;
                        const unsigned long long m = s_mask[gl];
                        if (!((m >> v) & 1ull)) continue;
                        const int pos = s_first[gl] + __popcll(m & ((1ull << v) - 1ull)) - c0;
                        if (pos < 0 || pos >= n) continue;   // in an earlier or a later chunk
#pragma unroll
                        for (int c = 0; c < 6; ++c) pv[c] += s_pose[c * kPreThreads + pos];
                    }
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    pv[c] += __shfl_xor_sync(0xffffffffu, pv[c], 4);
                    pv[c] += __shfl_xor_sync(0xffffffffu, pv[c], 2);
                    pv[c] += __shfl_xor_sync(0xffffffffu, pv[c], 1);
                }
                if (part == 0 && v < vt.V)
#pragma unroll
                    for (int c = 0; c < 6; ++c) s_vpose[v * 6 + c] += pv[c];
            }
        } else
        // warp w takes views w, w + 8, ...: lanes stride the chunk, then a butterfly
        for (int v = warp; v < vt.V; v += WARPS) {
            float pv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int p = lane; p < n; p += 32) {
                if ((s_item[c0 + p] & 0xff) != v) continue;
#pragma unroll
                for (int c = 0; c < 6; ++c) pv[c] += s_pose[c * kPreThreads + p];
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) pv[c] += __shfl_xor_sync(0xffffffffu, pv[c], o);
            }
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 6; ++c) s_vpose[v * 6 + c] += pv[c];
        }
        __syncthreads();
    }
    // The parameter gradients of every Gaussian visible somewhere, from its
    // totals, once the group's list is done: all threads at once, instead of
    // the few whose Gaussians' runs ended in a chunk while the rest waited at
    // the chunk's barrier.
    if constexpr (VW != 1) {
        for (int gl = tid; gl < GBT; gl += kPreThreads)
            if (gbase + gl < gp.N && s_cnt[gl] != 0) bwd_finish(gp, out, gbase + gl, s_tot + gl * 13);
    }

    // Gaussians visible in no view: zero gradients
    if (!ac) {
        for (int gl = tid; gl < GBT; gl += kPreThreads) {
            const int g = gbase + gl;
            if (g >= gp.N || s_cnt[gl] != 0) continue;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                out.means[(size_t)j * N + g] = 0.f;
                out.log_scales[(size_t)j * N + g] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) out.quats[(size_t)k * N + g] = 0.f;
            out.opacity_logits[g] = 0.f;
            for (int k = 0; k < 3 * K; ++k) out.sh[(size_t)k * N + g] = 0.f;
        }
    }
    for (int i = tid; i < 6 * vt.V; i += kPreThreads) {
        const int v = i / 6, c = i - v * 6;
        ws.pose_partials[((size_t)v * ws.pose_blocks + grp) * 6 + c] = s_vpose[v * 6 + c];
    }
    if (dens)
        for (int gl = tid; gl < GBT; gl += kPreThreads)
            if (gbase + gl < gp.N)
                densify_write(out, gbase + gl, s_dgrad[gl], (float)s_dcount[gl], __int_as_float(s_drad[gl]));
}

// Persistent blocks take the groups in turn from a counter in the workspace
// header (zeroed by the render's init kernel, and again by the pose
// reduction after every backward): no group waits for a wave, whatever N.
// Each group writes its own pose partials, so their sum is deterministic.
template <int DEG, int VW>
__global__ void __launch_bounds__(kPreThreads, 2) preprocess_bwd_kernel(const __grid_constant__ ViewTable vt,
                                                                        const GaussianPtrs gp, const Ws ws,
                                                                        const GradPtrs out) {
    __shared__ Pose s_poses[GSR_MAX_VIEWS];
    __shared__ int s_group;
    load_poses(vt, s_poses);
    const int ngroups = (gp.N + BwdShape<VW>::GBT - 1) / BwdShape<VW>::GBT;
    for (;;) {
        __syncthreads();   // the previous group is done with the shared memory
        if (threadIdx.x == 0) s_group = (int)atomicAdd(&ws.hdr->bwd_groups, 1u);
        __syncthreads();
        const int grp = s_group;
        if (grp >= ngroups) break;
        preprocess_bwd_group<DEG, VW>(vt, gp, ws, out, s_poses, grp);
    }
}

// Sum of the per-block pose partials of each view, in a fixed order.
__global__ void __launch_bounds__(256) pose_reduce_kernel(const __grid_constant__ ViewTable vt, const Ws ws,
                                                          int accumulate) {
    __shared__ float s[256][6];
    const int v = blockIdx.x;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t b = threadIdx.x; b < ws.pose_blocks; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += ws.pose_partials[((size_t)v * ws.pose_blocks + b) * 6 + c];
#pragma unroll
    for (int c = 0; c < 6; ++c) s[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if (threadIdx.x < (unsigned)stride)
#pragma unroll
            for (int c = 0; c < 6; ++c) s[threadIdx.x][c] += s[threadIdx.x + stride][c];
        __syncthreads();
    }
    float *dst = vt.v[v].d_pose;
    if (threadIdx.x < 6 && dst) dst[threadIdx.x] = accumulate ? dst[threadIdx.x] + s[0][threadIdx.x] : s[0][threadIdx.x];
    if (v == 0 && threadIdx.x == 0) {
        ws.hdr->bwd_groups = 0u;   // for the next backward on this workspace
        // the preprocess backward has cleared every row the blend backward wrote
        if (!ws.surfels) set_rows_clean(ws, true);
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_pose_reduce(const ViewTable &vt, const Ws &ws, int accumulate, cudaStream_t st) {
    pose_reduce_kernel<<<vt.V, 256, 0, st>>>(vt, ws, accumulate);
    return cudaGetLastError();
}


template <int DEG>
static cudaError_t launch_pre_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, int sm_count,
                                  cudaStream_t st) {
    const long long batches = ((long long)gp.N + 31) / 32;
    const long long max_warps = (long long)sm_count * kPreFwdBlocksPerSM * kPreWarps;
    const int item_views =
        batches * ((vt.V + kPreItemViews - 1) / kPreItemViews) < kPreItemsPerWarp * max_warps ? kPreSmallItemViews : kPreItemViews;
    const long long items = batches * ((vt.V + item_views - 1) / item_views);
    const long long need = (items + kPreWarps - 1) / kPreWarps;
    const unsigned blocks = (unsigned)std::min<long long>(need, (long long)sm_count * kPreFwdBlocksPerSM);
    preprocess_fwd_kernel<DEG><<<blocks, kPreThreads, 0, st>>>(vt, gp, ws, item_views);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, int sm_count,
                                  cudaStream_t st) {
    if (gp.N == 0) return cudaSuccess;
    switch (gp.sh_degree) {
        case 0: return launch_pre_fwd<0>(vt, gp, ws, sm_count, st);
        case 1: return launch_pre_fwd<1>(vt, gp, ws, sm_count, st);
        case 2: return launch_pre_fwd<2>(vt, gp, ws, sm_count, st);
        default: return launch_pre_fwd<3>(vt, gp, ws, sm_count, st);
    }
}

template <int DEG, int VW>
static cudaError_t launch_pre_bwd_vw(const ViewTable &vt, const GaussianPtrs &gp, Ws ws, const GradPtrs &out,
                                     cudaStream_t st) {
    const size_t smem = bwd_smem_bytes<DEG, VW>();
    // More than 48 KB of dynamic shared memory needs an opt-in, set once per
    // device (the first backward on a device, which should precede capture).
    // The resident blocks (all of them work through the groups) are counted
    // once per device too.
    static std::mutex mu;
    static bool done[64] = {};
    static int resident[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int slots = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        const bool cached = dev >= 0 && dev < 64 && done[dev];
        if (!cached) {
            e = cudaFuncSetAttribute(preprocess_bwd_kernel<DEG, VW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0, sms = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, preprocess_bwd_kernel<DEG, VW>,
                                                                   kPreThreads, smem)) != cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return e;
            slots = std::max(1, per_sm) * std::max(1, sms);
            if (dev >= 0 && dev < 64) {
                resident[dev] = slots;
                done[dev] = true;
            }
        } else {
            slots = resident[dev];
        }
    }
    const int groups = (gp.N + BwdShape<VW>::GBT - 1) / BwdShape<VW>::GBT;
    ws.pose_blocks = (uint32_t)groups;   // one pose partial per group: at most (N + 31) / 32, the allotment
    preprocess_bwd_kernel<DEG, VW><<<std::min(groups, slots), kPreThreads, smem, st>>>(vt, gp, ws, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pose_reduce(vt, ws, out.accumulate, st);
}

template <int DEG>
static cudaError_t launch_pre_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, const GradPtrs &out,
                                  cudaStream_t st) {
    if (vt.V <= 1) return launch_pre_bwd_vw<DEG, 1>(vt, gp, ws, out, st);
    if (vt.V <= 2) return launch_pre_bwd_vw<DEG, 2>(vt, gp, ws, out, st);
    if (vt.V <= 4) return launch_pre_bwd_vw<DEG, 4>(vt, gp, ws, out, st);
    if (vt.V <= 8) return launch_pre_bwd_vw<DEG, 8>(vt, gp, ws, out, st);
    if (vt.V <= 16) return launch_pre_bwd_vw<DEG, 16>(vt, gp, ws, out, st);
    if (vt.V <= 32) return launch_pre_bwd_vw<DEG, 32>(vt, gp, ws, out, st);
    return launch_pre_bwd_vw<DEG, 64>(vt, gp, ws, out, st);
}

cudaError_t launch_preprocess_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, const GradPtrs &out,
                                  cudaStream_t st) {
    if (gp.N == 0) return launch_pose_reduce(vt, ws, out.accumulate, st);   // zero pose gradients
    switch (gp.sh_degree) {
        case 0: return launch_pre_bwd<0>(vt, gp, ws, out, st);
        case 1: return launch_pre_bwd<1>(vt, gp, ws, out, st);
        case 2: return launch_pre_bwd<2>(vt, gp, ws, out, st);
        default: return launch_pre_bwd<3>(vt, gp, ws, out, st);
    }
}

}  // namespace gsr
