// loss.cu -- loss front ends of Eq. "rnd_loss" (Sec. 3.3), with their
// gradients written for the backward: the L1 colour and depth terms alone
// (HBM-bound: one read of rendered and target images, one write of the
// gradients), and the full mixed L1 + SSIM + depth loss.
#include <cmath>
#include <mutex>

#include "kernels.cuh"

namespace gsr {

namespace {

struct L1Table {
    gsr_l1_view t[GSR_MAX_VIEWS];
};

__device__ __forceinline__ float sgn(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(256) l1_loss_kernel(const __grid_constant__ ViewTable vt,
                                                      const __grid_constant__ L1Table lt, float cw, float dw,
                                                      float *loss) {
    __shared__ float s_warp[8];
    const int v = blockIdx.y;
    const ViewParams &vp = vt.v[v];
    const gsr_l1_view &t = lt.t[v];
    const size_t P = (size_t)vp.H * vp.W;
    const float kc = cw / (3.f * (float)P), kd = dw / (float)P;
    const bool depth = t.target_depth != nullptr && vp.depth != nullptr;
    float part = 0.f;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = vp.color[c * P + p] - t.target_color[c * P + p];
            part += fabsf(d) * kc;
            t.d_color[c * P + p] = sgn(d) * kc;
        }
        if (depth) {
            const float d = vp.depth[p] - t.target_depth[p];
            part += fabsf(d) * kd;
            if (t.d_depth) t.d_depth[p] = sgn(d) * kd;
        } else if (t.d_depth) {
            t.d_depth[p] = 0.f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += s_warp[w];
        atomicAdd(loss, s);
    }
}

// ------------------------------------------------------------------ L1 + SSIM
// Eq. "rnd_loss": lambda1 [(1 - lambda2) |I - I*| + lambda2 (1 - SSIM)] +
// (1 - lambda1) |Z - Z*|, per view (means over pixels), summed over views.
// SSIM: 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero
// padding, mean over channels and pixels.
//
// One block produces a 32x32 tile of gradients with no scratch memory: it
// loads the images with a 10-pixel halo, blurs x, y, x^2, y^2, xy (separable,
// horizontal then vertical) over the tile plus a 5-pixel halo, forms there
// the SSIM terms A = dS/dmu_x (through the variances), B = dS/dE[x^2],
// C = dS/dE[xy], and blurs A, B, C again: with the symmetric window,
// d mean(S)/dx_q = (G*A + 2 x_q G*B + y_q G*C)(q) / (3P).
constexpr int kSsimT = 32;                    // output tile edge
constexpr int kSsimR = 5;                     // window radius
constexpr int kSsimE = kSsimT + 4 * kSsimR;   // loaded region edge (two halos)
constexpr int kSsimM = kSsimT + 2 * kSsimR;   // region of the SSIM terms
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;
constexpr size_t kSsimSmem = sizeof(float) * (2 * kSsimE * kSsimE + 5 * kSsimE * kSsimM + 3 * kSsimM * kSsimM);

struct SsimParams {
    float g[2 * kSsimR + 1];   // normalised Gaussian window
    float lambda1, lambda2;
};

__global__ void __launch_bounds__(256) rgbd_loss_kernel(const __grid_constant__ ViewTable vt,
                                                        const __grid_constant__ L1Table lt, const SsimParams sp,
                                                        float *loss) {
    extern __shared__ float sm[];
    float *sx = sm;                          // [E][E] rendered channel
    float *sy = sx + kSsimE * kSsimE;        // [E][E] target channel
    float *h = sy + kSsimE * kSsimE;         // [5][E][M] horizontal blurs; later [3][M][T]
    float *m = h + 5 * kSsimE * kSsimM;      // [3][M][M] A, B, C
    __shared__ float s_warp[8];
    // which view and tile (views concatenated, tiles of kSsimT)
    int v = 0;
    uint32_t t = blockIdx.x, first = 0;
    for (; v < vt.V; ++v) {
        const uint32_t n = (uint32_t)((vt.v[v].W + kSsimT - 1) / kSsimT) * ((vt.v[v].H + kSsimT - 1) / kSsimT);
        if (t < n) break;
        t -= n;
    }
    if (v >= vt.V) return;
    first = t;
    const ViewParams &vp = vt.v[v];
    const gsr_l1_view &tg = lt.t[v];
    const int W = vp.W, H = vp.H, tx = (int)(t % (uint32_t)((W + kSsimT - 1) / kSsimT));
    const int ty = (int)(t / (uint32_t)((W + kSsimT - 1) / kSsimT));
    const int X0 = tx * kSsimT, Y0 = ty * kSsimT;
    const size_t P = (size_t)H * W;
    const float invP3 = 1.f / (3.f * (float)P), invP = 1.f / (float)P;
    const float l1w = sp.lambda1 * (1.f - sp.lambda2), sw = sp.lambda1 * sp.lambda2;
    float part = 0.f;
    for (int c = 0; c < 3; ++c) {
        const float *xc = vp.color + c * P, *yc = tg.target_color + c * P;
        for (int i = threadIdx.x; i < kSsimE * kSsimE; i += blockDim.x) {
            const int r = i / kSsimE, q = i - r * kSsimE;
            const int gy = Y0 - 2 * kSsimR + r, gx = X0 - 2 * kSsimR + q;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            sx[i] = in ? xc[(size_t)gy * W + gx] : 0.f;
            sy[i] = in ? yc[(size_t)gy * W + gx] : 0.f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kSsimE * kSsimM; i += blockDim.x) {
            const int r = i / kSsimM, q = i - r * kSsimM;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * kSsimR; ++j) {
                const float xv = sx[r * kSsimE + q + j], yv = sy[r * kSsimE + q + j], w = sp.g[j];
                a0 = fmaf(w, xv, a0);
                a1 = fmaf(w, yv, a1);
                a2 = fmaf(w * xv, xv, a2);
                a3 = fmaf(w * yv, yv, a3);
                a4 = fmaf(w * xv, yv, a4);
            }
            h[i] = a0;
            h[kSsimE * kSsimM + i] = a1;
            h[2 * kSsimE * kSsimM + i] = a2;
            h[3 * kSsimE * kSsimM + i] = a3;
            h[4 * kSsimE * kSsimM + i] = a4;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kSsimM * kSsimM; i += blockDim.x) {
            const int r = i / kSsimM, q = i - r * kSsimM;
            float b[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j <= 2 * kSsimR; ++j) {
                const int o = (r + j) * kSsimM + q;
#pragma unroll
                for (int k = 0; k < 5; ++k) b[k] = fmaf(sp.g[j], h[k * kSsimE * kSsimM + o], b[k]);
            }
            const int gy = Y0 - kSsimR + r, gx = X0 - kSsimR + q;
            float A = 0.f, B = 0.f, Cc = 0.f;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                const float mx = b[0], my = b[1];
                const float vx = b[2] - mx * mx, vy = b[3] - my * my, cxy = b[4] - mx * my;
                const float n1 = 2.f * mx * my + kSsimC1, n2 = 2.f * cxy + kSsimC2;
                const float d1 = mx * mx + my * my + kSsimC1, d2 = vx + vy + kSsimC2;
                const float id = 1.f / (d1 * d2);
                const float S = n1 * n2 * id;
                const float dS_dmx = 2.f * my * n2 * id - 2.f * mx * S / d1;
                const float dS_dvx = -S / d2;
                const float dS_dcxy = 2.f * n1 * id;
                A = dS_dmx - 2.f * mx * dS_dvx - my * dS_dcxy;
                B = dS_dvx;
                Cc = dS_dcxy;
                if (r >= kSsimR && r < kSsimR + kSsimT && q >= kSsimR && q < kSsimR + kSsimT) part -= sw * S * invP3;
            }
            m[i] = A;
            m[kSsimM * kSsimM + i] = B;
            m[2 * kSsimM * kSsimM + i] = Cc;
        }
        __syncthreads();
        float *h2 = h;   // [3][M][T], the horizontal blurs are no longer needed
        for (int i = threadIdx.x; i < kSsimM * kSsimT; i += blockDim.x) {
            const int r = i / kSsimT, q = i - r * kSsimT;
            float b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * kSsimR; ++j) {
                const int o = r * kSsimM + q + j;
                b0 = fmaf(sp.g[j], m[o], b0);
                b1 = fmaf(sp.g[j], m[kSsimM * kSsimM + o], b1);
                b2 = fmaf(sp.g[j], m[2 * kSsimM * kSsimM + o], b2);
            }
            h2[i] = b0;
            h2[kSsimM * kSsimT + i] = b1;
            h2[2 * kSsimM * kSsimT + i] = b2;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kSsimT * kSsimT; i += blockDim.x) {
            const int r = i / kSsimT, q = i - r * kSsimT;
            const int gy = Y0 + r, gx = X0 + q;
            if (gy >= H || gx >= W) continue;
            float gA = 0.f, gB = 0.f, gC = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * kSsimR; ++j) {
                const int o = (r + j) * kSsimT + q;
                gA = fmaf(sp.g[j], h2[o], gA);
                gB = fmaf(sp.g[j], h2[kSsimM * kSsimT + o], gB);
                gC = fmaf(sp.g[j], h2[2 * kSsimM * kSsimT + o], gC);
            }
            const int e = (r + 2 * kSsimR) * kSsimE + q + 2 * kSsimR;
            const float xq = sx[e], yq = sy[e], d = xq - yq;
            const float dssim = (gA + 2.f * xq * gB + yq * gC) * invP3;
            tg.d_color[c * P + (size_t)gy * W + gx] = l1w * sgn(d) * invP3 - sw * dssim;
            part += l1w * fabsf(d) * invP3;
        }
        __syncthreads();
    }
    // depth term and the constant lambda1 lambda2 of (1 - SSIM), once per view
    const bool depth = tg.target_depth != nullptr && vp.depth != nullptr;
    for (int i = threadIdx.x; i < kSsimT * kSsimT; i += blockDim.x) {
        const int r = i / kSsimT, q = i - r * kSsimT;
        const int gy = Y0 + r, gx = X0 + q;
        if (gy >= H || gx >= W) continue;
        const size_t p = (size_t)gy * W + gx;
        if (depth) {
            const float d = vp.depth[p] - tg.target_depth[p];
            part += (1.f - sp.lambda1) * fabsf(d) * invP;
            if (tg.d_depth) tg.d_depth[p] = (1.f - sp.lambda1) * sgn(d) * invP;
        } else if (tg.d_depth) {
            tg.d_depth[p] = 0.f;
        }
    }
    if (first == 0 && threadIdx.x == 0) part += sw;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += s_warp[w];
        atomicAdd(loss, s);
    }
}

}  // namespace

cudaError_t launch_rgbd_loss(const ViewTable &vt, const gsr_l1_view *targets, float lambda1, float lambda2,
                             float *loss, cudaStream_t st) {
    L1Table lt;
    uint32_t tiles = 0;
    for (int v = 0; v < vt.V; ++v) {
        lt.t[v] = targets[v];
        tiles += (uint32_t)((vt.v[v].W + kSsimT - 1) / kSsimT) * ((vt.v[v].H + kSsimT - 1) / kSsimT);
    }
    SsimParams sp;
    double g[2 * kSsimR + 1], s = 0.0;
    for (int k = 0; k <= 2 * kSsimR; ++k) {
        const double x = k - kSsimR;
        g[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k <= 2 * kSsimR; ++k) sp.g[k] = (float)(g[k] / s);
    sp.lambda1 = lambda1;
    sp.lambda2 = lambda2;
    // more than 48 KB of dynamic shared memory needs an opt-in, once per device
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64 || !done[dev]) {
            e = cudaFuncSetAttribute(rgbd_loss_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimSmem);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) done[dev] = true;
        }
    }
    e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    rgbd_loss_kernel<<<tiles, 256, kSsimSmem, st>>>(vt, lt, sp, loss);
    return cudaGetLastError();
}

cudaError_t launch_l1_loss(const ViewTable &vt, const gsr_l1_view *targets, float color_weight, float depth_weight,
                           float *loss, cudaStream_t st) {
    L1Table lt;
    uint32_t maxP = 0;
    for (int v = 0; v < vt.V; ++v) {
        lt.t[v] = targets[v];
        maxP = max(maxP, (uint32_t)(vt.v[v].H * vt.v[v].W));
    }
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    const unsigned bx = min(1024u, (maxP + 255u) / 256u);
    l1_loss_kernel<<<dim3(bx, vt.V), 256, 0, st>>>(vt, lt, color_weight, depth_weight, loss);
    return cudaGetLastError();
}

}  // namespace gsr
