// project.cuh -- per (view, Gaussian) projection shared by the forward
// preprocess and its backward: activation and 3-D covariance factor,
// camera transform, EWA projection to the dilated 2-D covariance Sigma', and
// the Cholesky factor of Sigma'^-1 that the blend evaluates (Sec. 3.3,
// alpha_i = sigma_i G(R, t, P_i, r_i, s_i)).
//
// FP32 throughout.  Two choices keep FP32 close to the exact result where the
// textbook formulas lose digits:
//  * det(Sigma') is formed as sum of squared 2x2 minors of P = J W R S
//    (Cauchy-Binet) + 0.3 tr + 0.09, all non-negative terms, instead of
//    a*c - b^2, which cancels for elongated footprints;
//  * the blend evaluates d^2 = (l00 dx + l01 dy)^2 + (l11 dy)^2 with
//    l11 = 1/sqrt(Syy), l00 = sqrt(Syy/det), l01 = -Sxy/sqrt(det Syy), which
//    does not cancel the way a*dx^2 + 2b*dx*dy + c*dy^2 does far along the
//    long axis of a thin ellipse.
#pragma once

#include "common.cuh"

namespace gsr {

struct GaussPre {
    float mx, my, mz;
    float qw, qx, qy, qz, qinv;   // unit quaternion and 1/|q|
    float s[3];
    float R[3][3];
    float M[3][3];                // R diag(s)
    float o, log2o, smax;
    bool alive;                   // 255 o > 1: can pass the alpha skip somewhere
};

__device__ __forceinline__ void gauss_pre(const GaussianPtrs &gp, int g, GaussPre &G) {
    const int N = gp.N;
    G.mx = gp.means[g];
    G.my = gp.means[N + g];
    G.mz = gp.means[2 * N + g];
    const float q0 = gp.quats[g], q1 = gp.quats[N + g], q2 = gp.quats[2 * N + g], q3 = gp.quats[3 * N + g];
    const float qn2 = q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
    G.qinv = 1.0f / sqrtf(qn2);
    G.qw = q0 * G.qinv;
    G.qx = q1 * G.qinv;
    G.qy = q2 * G.qinv;
    G.qz = q3 * G.qinv;
    const float w = G.qw, x = G.qx, y = G.qy, z = G.qz;
    G.R[0][0] = 1.f - 2.f * (y * y + z * z);
    G.R[0][1] = 2.f * (x * y - w * z);
    G.R[0][2] = 2.f * (x * z + w * y);
    G.R[1][0] = 2.f * (x * y + w * z);
    G.R[1][1] = 1.f - 2.f * (x * x + z * z);
    G.R[1][2] = 2.f * (y * z - w * x);
    G.R[2][0] = 2.f * (x * z - w * y);
    G.R[2][1] = 2.f * (y * z + w * x);
    G.R[2][2] = 1.f - 2.f * (x * x + y * y);
    for (int k = 0; k < 3; ++k) G.s[k] = expf(gp.log_scales[k * N + g]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G.M[i][j] = G.R[i][j] * G.s[j];
    const float l = gp.opacity_logits[g];
    G.o = 1.0f / (1.0f + expf(-l));
    G.log2o = log2f(G.o);
    // alpha = o 2^-s >= 1/255  <=>  s <= log2(255 o);  d^2 <= 9  <=>  s <= 9 kHalfLog2e
    G.smax = fminf(kCutoffD2 * kHalfLog2e, G.log2o + kLog2_255);
    G.alive = G.smax >= 0.f && isfinite(G.smax) && isfinite(G.mx + G.my + G.mz) &&
              isfinite(G.s[0] + G.s[1] + G.s[2]) && qn2 > 0.f && isfinite(qn2);
}

// Camera pose in shared memory: W row-major (9), t (3), centre C = -W^T t
// (3), and the view's Jacobian clamp limits on x/z and y/z.
struct Pose {
    float W[3][3];
    float t[3];
    float C[3];
    float limx, limy;
};

// dL/dq of the raw quaternion from dL/dR of R(q / |q|).
__device__ __forceinline__ void rot_grad_to_quat(const GaussPre &G, const float (&dR)[3][3], float (&dqr)[4]) {
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
#pragma unroll
    for (int k = 0; k < 4; ++k) dqr[k] = (dq[k] - qu[k] * qd) * G.qinv;
}

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
        const ViewParams &vp = vt.v[threadIdx.x];
        p.limx = kFovClamp * 0.5f * (float)vp.W / vp.fx;
        p.limy = kFovClamp * 0.5f * (float)vp.H / vp.fy;
    }
    __syncthreads();
}

// Unit view direction from the camera centre to the mean and its length.
__device__ __forceinline__ void view_dir(const GaussPre &G, const Pose &ps, float &dx, float &dy, float &dz,
                                         float &rn) {
    dx = G.mx - ps.C[0];
    dy = G.my - ps.C[1];
    dz = G.mz - ps.C[2];
    rn = rsqrt_approx(dx * dx + dy * dy + dz * dz);
    dx *= rn;
    dy *= rn;
    dz *= rn;
}



struct Proj {
    float xh, yh, zh, xl, yl, zl;  // camera-frame mean, hi + lo
    float rz;                      // 1/zh (rcp.approx)
    bool clx, cly;
    float txz, tyz;                // clamped x/z, y/z
    float J00, J02, J11, J12;
    float T[2][3];                 // J W
    float P[2][3];                 // T M
    float sxx, sxy, syy;           // Sigma' including the dilation
    float det;
    float l00, l01, l11;           // Cholesky factor of Sigma'^-1
};

// Returns false when the Gaussian is culled in this view (near plane, bad
// determinant or non-finite values).
__device__ __forceinline__ bool project_view(const GaussPre &G, const Pose &ps, const ViewParams &vp, Proj &p) {
    dot3_plus(ps.W[0][0], ps.W[0][1], ps.W[0][2], ps.t[0], G.mx, G.my, G.mz, p.xh, p.xl);
    dot3_plus(ps.W[1][0], ps.W[1][1], ps.W[1][2], ps.t[1], G.mx, G.my, G.mz, p.yh, p.yl);
    dot3_plus(ps.W[2][0], ps.W[2][1], ps.W[2][2], ps.t[2], G.mx, G.my, G.mz, p.zh, p.zl);
    const float z = p.zh;
    if (!(z > kNearZ) || !isfinite(z)) return false;
    const float limx = ps.limx, limy = ps.limy;
    const float rz = rcp_approx(z);
    p.rz = rz;
    float tx = p.xh * rz, ty = p.yh * rz;
    p.clx = (tx < -limx) || (tx > limx);
    p.cly = (ty < -limy) || (ty > limy);
    tx = fminf(fmaxf(tx, -limx), limx);
    ty = fminf(fmaxf(ty, -limy), limy);
    p.txz = tx;
    p.tyz = ty;
    p.J00 = vp.fx * rz;
    p.J02 = -vp.fx * tx * rz;      // -fx * xc / z^2 with xc = tx * z
    p.J11 = vp.fy * rz;
    p.J12 = -vp.fy * ty * rz;
    for (int j = 0; j < 3; ++j) {
        p.T[0][j] = p.J00 * ps.W[0][j] + p.J02 * ps.W[2][j];
        p.T[1][j] = p.J11 * ps.W[1][j] + p.J12 * ps.W[2][j];
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) p.P[i][j] = p.T[i][0] * G.M[0][j] + p.T[i][1] * G.M[1][j] + p.T[i][2] * G.M[2][j];
    const float a0 = p.P[0][0] * p.P[0][0] + p.P[0][1] * p.P[0][1] + p.P[0][2] * p.P[0][2];
    const float c0 = p.P[1][0] * p.P[1][0] + p.P[1][1] * p.P[1][1] + p.P[1][2] * p.P[1][2];
    const float b0 = p.P[0][0] * p.P[1][0] + p.P[0][1] * p.P[1][1] + p.P[0][2] * p.P[1][2];
    const float m01 = det2(p.P[0][0], p.P[0][1], p.P[1][0], p.P[1][1]);
    const float m02 = det2(p.P[0][0], p.P[0][2], p.P[1][0], p.P[1][2]);
    const float m12 = det2(p.P[0][1], p.P[0][2], p.P[1][1], p.P[1][2]);
    p.sxx = a0 + kDilation;
    p.sxy = b0;
    p.syy = c0 + kDilation;
    p.det = (m01 * m01 + m02 * m02 + m12 * m12) + kDilation * (a0 + c0) + kDilation * kDilation;
    if (!(p.det > 0.f) || !isfinite(p.det) || !isfinite(p.sxx + p.syy + p.sxy)) return false;
    // l11 = 1/sqrt(Syy), l00 = sqrt(Syy/det) = Syy / sqrt(det Syy),
    // l01 = -Sxy / sqrt(det Syy), from two approximate reciprocal square roots
    // (a few units in the last place)
    const float rds = rsqrt_approx(p.det * p.syy);
    p.l11 = rsqrt_approx(p.syy);
    p.l00 = p.syy * rds;
    p.l01 = -p.sxy * rds;
    return isfinite(p.l00) && isfinite(p.l01);
}

// Minimum over the box dx in [dx0, dx1], dy in [dy0, dy1] of the quadratic
// s = (m00 dx + m01 dy)^2 + (m11 dy)^2 (m00, m11 > 0): for fixed dy the first
// term's minimum over dx is max(0, m00 dx0 + m01 dy, -(m00 dx1 + m01 dy))^2,
// a convex function of dy whose minimum lies at an end of [dy0, dy1] or at
// the stationary point of one of its three pieces.
__device__ __forceinline__ float quad_min_over_box(float dx0, float dx1, float dy0, float dy1, float m00, float m01,
                                                   float m11) {
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
    return smin;
}

// Tolerance of a cull that compares quad_min_over_box with s_max against the
// blend's per-pixel test s <= s_max.  Both evaluate the same linear forms in
// FP32, each with an error of a few units in the last place of
// A = |m00| max|dx| + (|m01| + |m11|) max|dy|; near the cutoff
// (sqrt(s) <= 2.6) that moves s by at most about 2.6 * 2 * 4 eps A, inside
// the 2^-17 A term.  The rest covers the rounding of s_max itself.
__device__ __forceinline__ float cull_slack(float dx0, float dx1, float dy0, float dy1, float m00, float m01,
                                            float m11, float smax) {
    const float A = fabsf(m00) * fmaxf(fabsf(dx0), fabsf(dx1)) +
                    (fabsf(m01) + fabsf(m11)) * fmaxf(fabsf(dy0), fabsf(dy1));
    return 1e-3f * (1.f + smax) + 1e-2f + 0x1p-17f * A;
}

}  // namespace gsr
