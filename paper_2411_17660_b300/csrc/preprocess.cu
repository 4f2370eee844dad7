// preprocess.cu -- forward projection of every (view, Gaussian) pair
// (activation, camera transform, EWA projection, SH colour, exact tile count)
// and its backward (projection/SH chain rule, per-view SE(3) pose reduction).
//
// A block has kPreWarps warps in groups of VW = min(V, kPreWarps) (a power of
// two); each group owns 32 Gaussians (one per lane) and its warps take the
// views round-robin.  The warps of a group read the same Gaussians, so the
// parameters come from DRAM once and from L1 after that, while the
// (view, Gaussian) work is spread over many warps.  The backward sums each
// Gaussian's gradient over the views in shared memory, in a fixed order, so
// the result does not depend on timing.
#include <mutex>

#include "kernels.cuh"
#include "project.cuh"
#include "sh.cuh"
#include "spans.cuh"

namespace gsr {

constexpr int kPreWarps = 8;
constexpr int kPreThreads = 32 * kPreWarps;

__device__ __forceinline__ void load_poses(const ViewTable &vt, Pose *s_pose) {
    for (int i = threadIdx.x; i < vt.V * 12; i += blockDim.x) {
        const int v = i / 12, k = i % 12;
        const float x = vt.v[v].T_cw[k];
        if (k % 4 == 3)
            s_pose[v].t[k / 4] = x;
        else
            s_pose[v].W[k / 4][k % 4] = x;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)vt.V) {
        Pose &p = s_pose[threadIdx.x];
        for (int j = 0; j < 3; ++j) p.C[j] = -(p.W[0][j] * p.t[0] + p.W[1][j] * p.t[1] + p.W[2][j] * p.t[2]);
    }
    __syncthreads();
}

// Unit view direction from the camera centre to the mean and its length.
__device__ __forceinline__ void view_dir(const GaussPre &G, const Pose &ps, float &dx, float &dy, float &dz,
                                         float &rn) {
    dx = G.mx - ps.C[0];
    dy = G.my - ps.C[1];
    dz = G.mz - ps.C[2];
    rn = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= rn;
    dy *= rn;
    dz *= rn;
}

// ------------------------------------------------------------------ forward
template <int DEG>
__global__ void __launch_bounds__(kPreThreads) preprocess_fwd_kernel(const __grid_constant__ ViewTable vt,
                                                                     const GaussianPtrs gp, const Ws ws,
                                                                     int vw_log2) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    __shared__ Pose s_pose[GSR_MAX_VIEWS];
    load_poses(vt, s_pose);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int VW = 1 << vw_log2, slot = warp & (VW - 1);
    const int g = (blockIdx.x * (kPreWarps >> vw_log2) + (warp >> vw_log2)) * 32 + lane;
    if (g >= gp.N) return;
    const size_t N = (size_t)gp.N;
    GaussPre G;
    gauss_pre(gp, g, G);
    for (int v = slot; v < vt.V; v += VW) {
        const ViewParams &vp = vt.v[v];
        const size_t i = (size_t)v * N + g;
        uint32_t count = 0;
        Proj p;
        if (G.alive && project_view(G, s_pose[v], vp, p)) {
            const float m00 = kSqrtHalfLog2e * p.l00, m01 = kSqrtHalfLog2e * p.l01, m11 = kSqrtHalfLog2e * p.l11;
            float uh, ul, vh, vl;
            project_coord(vp.fx, vp.cx, p.xh, p.xl, p.zh, p.zl, uh, ul);
            project_coord(vp.fy, vp.cy, p.yh, p.yl, p.zh, p.zl, vh, vl);
            if (isfinite(uh) && isfinite(vh))
                count = visit_tile_spans(uh, vh, p.sxx, p.sxy, p.syy, m00, G.smax, vp.W, vp.H, vt.tile,
                                         [](int, int, int) {});
            if (count) {
                float dx, dy, dz, rn;
                view_dir(G, s_pose[v], dx, dy, dz, rn);
                float Y[K];
                sh_eval<DEG>(dx, dy, dz, Y);
                float rgb0 = 0.f, rgb1 = 0.f, rgb2 = 0.f;
                // one channel at a time keeps few coefficients live in registers
#pragma unroll 1
                for (int c = 0; c < 3; ++c) {
                    const float *shc = gp.sh + (size_t)c * N + g;
                    float acc = 0.5f;
#pragma unroll
                    for (int k = 0; k < K; ++k) acc = fmaf(__ldg(shc + (size_t)k * 3 * N), Y[k], acc);
                    acc = fmaxf(acc, 0.f);
                    if (c == 0) rgb0 = acc;
                    else if (c == 1) rgb1 = acc;
                    else rgb2 = acc;
                }
                ws.rec0[i] = make_float4(uh, vh, ul, vl);
                ws.rec1[i] = make_float4(m00, m01, m11, G.smax);
                ws.rec2[i] = make_float4(rgb0, rgb1, rgb2, p.zh);
                ws.rec3[i] = make_float4(G.log2o, p.sxx, p.sxy, p.syy);
            }
        }
        ws.counts[i] = count;
    }
}

// ------------------------------------------------------------------ backward
// Per-Gaussian partial gradients summed over views: dmu (3), dM (9, the
// gradient of M = R diag(s)), d ln(sigma) (1), dSH (3K).
template <int DEG>
struct BwdAcc {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    static constexpr int NV = 13 + 3 * K;
};

template <int DEG>
__global__ void __launch_bounds__(kPreThreads, 2) preprocess_bwd_kernel(const __grid_constant__ ViewTable vt,
                                                                     const GaussianPtrs gp, const Ws ws,
                                                                     const GradPtrs out, int vw_log2) {
    constexpr int K = BwdAcc<DEG>::K, NV = BwdAcc<DEG>::NV;
    extern __shared__ float s_red[];   // [kPreWarps][NV][32]
    __shared__ Pose s_pose[GSR_MAX_VIEWS];
    load_poses(vt, s_pose);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int VW = 1 << vw_log2, slot = warp & (VW - 1), group = warp >> vw_log2;
    const uint32_t gblock = blockIdx.x * (kPreWarps >> vw_log2) + group;   // 32-Gaussian group index
    const int g = (int)gblock * 32 + lane;
    const bool active = g < gp.N;
    const size_t N = (size_t)gp.N;
    GaussPre G;
    if (active) gauss_pre(gp, g, G);
    // registers: dmu (3), dM (9), d ln(sigma) (1); the 3K SH gradients live
    // in this warp's shared-memory columns (lane-private, no conflicts)
    float acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.f;
    float *dmu = acc, *dM = acc + 3;
    float *my_red = s_red + warp * NV * 32 + lane;   // element k at my_red[k * 32]
#pragma unroll
    for (int k = 13; k < NV; ++k) my_red[k * 32] = 0.f;

    for (int v = slot; v < vt.V; v += VW) {
        const ViewParams &vp = vt.v[v];
        const Pose &ps = s_pose[v];
        float pose6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const size_t i = (size_t)v * N + g;
        bool vis = active && ws.counts[i] > 0;
        Proj p;
        if (vis) vis = project_view(G, ps, vp, p);
        if (vis) {
            float sg[kVGGrads];
#pragma unroll
            for (int c = 0; c < kVGGrads; ++c) sg[c] = ws.vg_grads[((size_t)v * kVGGrads + c) * N + g];
            float dpc[3] = {0.f, 0.f, 0.f};

            // colour -> SH coefficients and the view direction
            float dx, dy, dz, rn;
            view_dir(G, ps, dx, dy, dz, rn);
            float Y[K];
            sh_eval<DEG>(dx, dy, dz, Y);
            float dr0 = 0.f, dr1 = 0.f, dr2 = 0.f;
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                const float *shc = gp.sh + (size_t)c * N + g;
                float raw = 0.5f;
#pragma unroll
                for (int k = 0; k < K; ++k) raw = fmaf(__ldg(shc + (size_t)k * 3 * N), Y[k], raw);
                const float d = raw > 0.f ? sg[6 + c] : 0.f;   // no gradient through the clamp at 0
                if (c == 0) dr0 = d;
                else if (c == 1) dr1 = d;
                else dr2 = d;
            }
            float wk[K];
            const float *shg = gp.sh + g;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float *r = my_red + (13 + k * 3) * 32;
                r[0] = fmaf(dr0, Y[k], r[0]);
                r[32] = fmaf(dr1, Y[k], r[32]);
                r[64] = fmaf(dr2, Y[k], r[64]);
                wk[k] = dr0 * __ldg(shg + (size_t)(k * 3) * N) + dr1 * __ldg(shg + (size_t)(k * 3 + 1) * N) +
                        dr2 * __ldg(shg + (size_t)(k * 3 + 2) * N);
            }
            float gdx, gdy, gdz;
            sh_grad<DEG>(dx, dy, dz, wk, gdx, gdy, gdz);
            const float radial = gdx * dx + gdy * dy + gdz * dz;
            const float dv0 = (gdx - dx * radial) * rn, dv1 = (gdy - dy * radial) * rn,
                        dv2 = (gdz - dz * radial) * rn;
            dmu[0] += dv0;
            dmu[1] += dv1;
            dmu[2] += dv2;
            // the camera centre moves by -W^T rho: dL/drho gets -W dL/dC with dL/dC = -dv
            pose6[0] += ps.W[0][0] * dv0 + ps.W[0][1] * dv1 + ps.W[0][2] * dv2;
            pose6[1] += ps.W[1][0] * dv0 + ps.W[1][1] * dv1 + ps.W[1][2] * dv2;
            pose6[2] += ps.W[2][0] * dv0 + ps.W[2][1] * dv1 + ps.W[2][2] * dv2;

            // the blend returns dL/d ln(sigma); the logit chain is applied once at the end
            acc[12] += sg[5];

            // pixel mean and depth: the blend returns the sums of dL/dp1 and
            // dL/dp2 (p = m d, d = pixel - mean), so dL/du = -m00 S1 and
            // dL/dv = -(m01 S1 + m11 S2)
            const float x = p.xh, y = p.yh, z = p.zh, rz = 1.0f / z;
            const float du = -kSqrtHalfLog2e * p.l00 * sg[0];
            const float dvv = -kSqrtHalfLog2e * (p.l01 * sg[0] + p.l11 * sg[1]);
            dpc[0] += du * vp.fx * rz;
            dpc[1] += dvv * vp.fy * rz;
            dpc[2] += -(du * vp.fx * x + dvv * vp.fy * y) * rz * rz + sg[9];

            // Cholesky factor of Sigma'^-1 -> Sigma' = [[A, B], [B, C]]
            const float A = p.sxx, B = p.sxy, C = p.syy, det = p.det, idet = 1.0f / det, iC = 1.0f / C;
            const float dl00 = kSqrtHalfLog2e * sg[2], dl01 = kSqrtHalfLog2e * sg[3], dl11 = kSqrtHalfLog2e * sg[4];
            const float rdc = 1.0f / sqrtf(det * C);
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
                for (int k = 0; k < 3; ++k)
                    dT[r][k] = dP[r][0] * G.M[k][0] + dP[r][1] * G.M[k][1] + dP[r][2] * G.M[k][2];
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
                for (int k = 0; k < 3; ++k)
                    Am[r][k] = dW[r][0] * ps.W[k][0] + dW[r][1] * ps.W[k][1] + dW[r][2] * ps.W[k][2];
            pose6[3] += Am[2][1] - Am[1][2];
            pose6[4] += Am[0][2] - Am[2][0];
            pose6[5] += Am[1][0] - Am[0][1];
        }
        // this warp owns view v for its 32 Gaussians: its sum is their partial
        float part[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float x = pose6[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            part[c] = x;
        }
        if (lane < 6) {
            float x = part[0];
#pragma unroll
            for (int c = 1; c < 6; ++c) x = lane == c ? part[c] : x;
            if (gblock < ws.pose_blocks) ws.pose_partials[((size_t)v * ws.pose_blocks + gblock) * 6 + lane] = x;
        }
    }

    // sum each group's per-Gaussian partials over its warps (views) in a
    // fixed order, into the group's first warp
#pragma unroll
    for (int k = 0; k < 13; ++k) my_red[k * 32] = acc[k];
    __syncthreads();
    if (VW > 1) {
        const int groups = kPreWarps >> vw_log2;
        for (int idx = threadIdx.x; idx < groups * NV * 32; idx += kPreThreads) {
            const int grp = idx / (NV * 32), rest = idx - grp * NV * 32;
            float *first = s_red + (grp * VW) * NV * 32 + rest;
            float x = first[0];
            for (int s = 1; s < VW; ++s) x += first[s * NV * 32];
            first[0] = x;
        }
        __syncthreads();
    }
    if (!active) return;
    const float *gsum = s_red + (group * VW) * NV * 32 + lane;   // element k at gsum[k * 32]
    // every warp of the group writes its share of the SH gradient rows
    {
        const bool ac = out.accumulate != 0;
        for (int k = slot; k < 3 * K; k += VW) {
            float *ps2 = out.sh + (size_t)k * N + g;
            const float x = gsum[(13 + k) * 32];
            *ps2 = ac ? *ps2 + x : x;
        }
    }
    if (slot != 0) return;
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = gsum[k * 32];

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
    const float w = G.qw, x = G.qx, y = G.qy, z = G.qz;
    // dR/dq for the unit quaternion (w, x, y, z)
    float dq[4];
    dq[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    dq[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                   w * dR[2][1] - 2.f * x * dR[2][2]);
    dq[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                   z * dR[2][1] - 2.f * y * dR[2][2]);
    dq[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                   y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    const float qu[4] = {w, x, y, z};
    float dqr[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) dqr[k] = (dq[k] - qu[k] * qd) * G.qinv;
    const float dlogit = acc[12] * (1.f - G.o);   // d ln(sigmoid(l)) / dl = 1 - sigma

    const bool ac = out.accumulate != 0;
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
}

// ------------------------------------------------------------------ launchers
// log2 of the warps that share one group of 32 Gaussians: as many as there
// are views, up to the block's kPreWarps (a power of two).
static int views_log2(int V) {
    int l = 0;
    while ((2 << l) <= V && (2 << l) <= kPreWarps) ++l;
    return l;
}

static int pre_blocks(int N, int vw_log2) {
    const int per_block = 32 * (kPreWarps >> vw_log2);
    return (N + per_block - 1) / per_block;
}

template <int DEG>
static cudaError_t launch_pre_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, cudaStream_t st) {
    const int l = views_log2(vt.V);
    preprocess_fwd_kernel<DEG><<<pre_blocks(gp.N, l), kPreThreads, 0, st>>>(vt, gp, ws, l);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, cudaStream_t st) {
    if (gp.N == 0) return cudaSuccess;
    switch (gp.sh_degree) {
        case 0: return launch_pre_fwd<0>(vt, gp, ws, st);
        case 1: return launch_pre_fwd<1>(vt, gp, ws, st);
        case 2: return launch_pre_fwd<2>(vt, gp, ws, st);
        default: return launch_pre_fwd<3>(vt, gp, ws, st);
    }
}

template <int DEG>
static cudaError_t launch_pre_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, const GradPtrs &out,
                                  cudaStream_t st) {
    const int l = views_log2(vt.V);
    const size_t smem = sizeof(float) * kPreWarps * BwdAcc<DEG>::NV * 32;
    // More than 48 KB of dynamic shared memory needs an opt-in, set once per
    // device (the first backward on a device, which should precede capture).
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64 || !done[dev]) {
            e = cudaFuncSetAttribute(preprocess_bwd_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) done[dev] = true;
        }
    }
    preprocess_bwd_kernel<DEG><<<pre_blocks(gp.N, l), kPreThreads, smem, st>>>(vt, gp, ws, out, l);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, const GradPtrs &out,
                                  cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (gp.N > 0) {
        switch (gp.sh_degree) {
            case 0: e = launch_pre_bwd<0>(vt, gp, ws, out, st); break;
            case 1: e = launch_pre_bwd<1>(vt, gp, ws, out, st); break;
            case 2: e = launch_pre_bwd<2>(vt, gp, ws, out, st); break;
            default: e = launch_pre_bwd<3>(vt, gp, ws, out, st); break;
        }
        if (e != cudaSuccess) return e;
    }
    pose_reduce_kernel<<<vt.V, 256, 0, st>>>(vt, ws, out.accumulate);
    return cudaGetLastError();
}

}  // namespace gsr
