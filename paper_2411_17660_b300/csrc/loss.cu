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

// 16-byte loads and stores over the pixels whose groups of four are aligned
// (all of them when H W is a multiple of 4 and the images are 16-byte
// aligned), plain ones for the rest.
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
    auto aligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool vec = (P & 3) == 0 && aligned(vp.color) && aligned(t.target_color) && aligned(t.d_color) &&
                     (!depth || (aligned(vp.depth) && aligned(t.target_depth))) && (!t.d_depth || aligned(t.d_depth));
    const size_t n4 = vec ? P / 4 : 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    float part = 0.f;
    auto l1 = [&](float d, float k, float &g) {
        part += fabsf(d) * k;
        g = sgn(d) * k;
    };
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 x = reinterpret_cast<const float4 *>(vp.color + c * P)[q];
            const float4 y = reinterpret_cast<const float4 *>(t.target_color + c * P)[q];
            float4 g;
            l1(x.x - y.x, kc, g.x);
            l1(x.y - y.y, kc, g.y);
            l1(x.z - y.z, kc, g.z);
            l1(x.w - y.w, kc, g.w);
            reinterpret_cast<float4 *>(t.d_color + c * P)[q] = g;
        }
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (depth) {
            const float4 x = reinterpret_cast<const float4 *>(vp.depth)[q];
            const float4 y = reinterpret_cast<const float4 *>(t.target_depth)[q];
            l1(x.x - y.x, kd, g.x);
            l1(x.y - y.y, kd, g.y);
            l1(x.z - y.z, kd, g.z);
            l1(x.w - y.w, kd, g.w);
        }
        if (t.d_depth) reinterpret_cast<float4 *>(t.d_depth)[q] = g;
    }
    for (size_t p = 4 * n4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
#pragma unroll
        for (int c = 0; c < 3; ++c) l1(vp.color[c * P + p] - t.target_color[c * P + p], kc, t.d_color[c * P + p]);
        float g = 0.f;
        if (depth) l1(vp.depth[p] - t.target_depth[p], kd, g);
        if (t.d_depth) t.d_depth[p] = g;
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
// Each 1-D blur is register-blocked: a thread reads a strip of K + 10 inputs
// once and writes K outputs.  Maps that take the same blur are stored as
// pairs (x, y), (x^2, y^2), (A, B) and blurred with packed FP32 FMAs.  Row
// strides are odd, so that the lanes of a warp, which walk down a column of
// strips, hit distinct banks.
constexpr int kSsimT = 32;                    // output tile edge
constexpr int kSsimR = 5;                     // window radius
constexpr int kSsimTaps = 2 * kSsimR + 1;
constexpr int kSsimE = kSsimT + 4 * kSsimR;   // loaded region edge (two halos)
constexpr int kSsimM = kSsimT + 2 * kSsimR;   // region of the SSIM terms
constexpr int kSsimEp = kSsimE + 1, kSsimMp = kSsimM + 1, kSsimTp = kSsimT + 1;   // padded strides
constexpr int kSsimThreads = 256;
constexpr int kSsimLoads = (kSsimE * kSsimE + kSsimThreads - 1) / kSsimThreads;   // input pixels per thread
// outputs per thread of the four blurs (each divides its extent)
constexpr int kH1 = 6, kV1 = 7, kH2 = 8, kV2 = 4;
static_assert(kSsimM % kH1 == 0 && kSsimM % kV1 == 0 && kSsimT % kH2 == 0 && kSsimT % kV2 == 0, "strips");
static_assert(kSsimM * (kSsimM / kV1) <= kSsimThreads && kSsimT * (kSsimT / kV2) <= kSsimThreads, "one round");
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;
constexpr int kSsimPlane = kSsimE * kSsimEp;  // one [E][Ep] map
// smem, in floats: (x, y) and (x^2, y^2) pairs and xy [E][Ep] (later (A, B)
// pairs and C [M][Mp]), then their horizontal blurs [E][Mp] (later the blurs
// of (A, B) and C [M][Tp])
constexpr size_t kSsimSmem = sizeof(float) * (5 * kSsimPlane + 5 * kSsimE * kSsimMp);
static_assert(kSsimPlane % 2 == 0 && (kSsimE * kSsimMp) % 2 == 0 && (kSsimM * kSsimMp) % 2 == 0 &&
              (kSsimM * kSsimTp) % 2 == 0, "float2 alignment");
static_assert(3 * kSsimM * kSsimMp <= 3 * kSsimPlane && 3 * kSsimM * kSsimTp <= 5 * kSsimE * kSsimMp, "alias");

struct SsimParams {
    float g[kSsimTaps];   // normalised Gaussian window
    float lambda1, lambda2;
};

__device__ __forceinline__ float fma_g(float g, float v, float a) { return fmaf(g, v, a); }
__device__ __forceinline__ float2 fma_g(float g, float2 v, float2 a) { return __ffma2_rn(make_float2(g, g), v, a); }

// K outputs of a 1-D blur along a strip: in[i * step], i < K + 10, to
// out[o * ostep], o < K (or to registers).
template <int K, typename T>
__device__ __forceinline__ void blur_strip_reg(const T *in, int step, T (&out)[K], const float (&g)[kSsimTaps]) {
    T v[K + 2 * kSsimR];
#pragma unroll
    for (int i = 0; i < K + 2 * kSsimR; ++i) v[i] = in[i * step];
#pragma unroll
    for (int o = 0; o < K; ++o) {
        T a{};
#pragma unroll
        for (int j = 0; j < kSsimTaps; ++j) a = fma_g(g[j], v[o + j], a);
        out[o] = a;
    }
}

template <int K, typename T>
__device__ __forceinline__ void blur_strip(const T *in, int step, T *out, int ostep, const float (&g)[kSsimTaps]) {
    T r[K];
    blur_strip_reg<K, T>(in, step, r, g);
#pragma unroll
    for (int o = 0; o < K; ++o) out[o * ostep] = r[o];
}

__global__ void __launch_bounds__(kSsimThreads, 2) rgbd_loss_kernel(const __grid_constant__ ViewTable vt,
                                                                    const __grid_constant__ L1Table lt,
                                                                    const __grid_constant__ SsimParams sp,
                                                                    float *loss) {
    extern __shared__ __align__(16) float sm[];
    float2 *sxy = reinterpret_cast<float2 *>(sm);              // [E][Ep] (rendered, target) channel
    float2 *ssq = sxy + kSsimPlane;                            // [E][Ep] squares
    float *spr = reinterpret_cast<float *>(ssq + kSsimPlane);  // [E][Ep] products
    float2 *hxy = reinterpret_cast<float2 *>(spr + kSsimPlane);   // [E][Mp] horizontal blurs
    float2 *hsq = hxy + kSsimE * kSsimMp;
    float *hpr = reinterpret_cast<float *>(hsq + kSsimE * kSsimMp);
    float2 *mAB = ssq;                                         // [M][Mp] (A, B), over the squares
    float *mC = reinterpret_cast<float *>(mAB + kSsimM * kSsimMp);
    float2 *gAB = hxy;                                         // [M][Tp] blurs of (A, B) and C
    float *gC = reinterpret_cast<float *>(gAB + kSsimM * kSsimTp);
    __shared__ float s_warp[kSsimThreads / 32];
    // which view and tile (views concatenated, tiles of kSsimT)
    int v = 0;
    uint32_t t = blockIdx.x;
    for (; v < vt.V; ++v) {
        const uint32_t n = (uint32_t)((vt.v[v].W + kSsimT - 1) / kSsimT) * ((vt.v[v].H + kSsimT - 1) / kSsimT);
        if (t < n) break;
        t -= n;
    }
    if (v >= vt.V) return;
    const ViewParams &vp = vt.v[v];
    const gsr_l1_view &tg = lt.t[v];
    const int W = vp.W, H = vp.H, tilesx = (W + kSsimT - 1) / kSsimT;
    const int X0 = (int)(t % (uint32_t)tilesx) * kSsimT, Y0 = (int)(t / (uint32_t)tilesx) * kSsimT;
    const size_t P = (size_t)H * W;
    const float invP3 = 1.f / (3.f * (float)P), invP = 1.f / (float)P;
    const float l1w = sp.lambda1 * (1.f - sp.lambda2), sw = sp.lambda1 * sp.lambda2;
    const int tid = threadIdx.x;
    float part = 0.f;
    // a channel's inputs are all fetched into registers before any is stored,
    // so that the block waits on global memory once per channel
    float px[kSsimLoads], py[kSsimLoads];
    auto fetch = [&](int c) {
        const float *xc = vp.color + c * P, *yc = tg.target_color + c * P;
#pragma unroll
        for (int k = 0; k < kSsimLoads; ++k) {
            const int i = tid + k * kSsimThreads;
            const int r = i / kSsimE, q = i - r * kSsimE;
            const int gy = Y0 - 2 * kSsimR + r, gx = X0 - 2 * kSsimR + q;
            const bool in = i < kSsimE * kSsimE && gy >= 0 && gy < H && gx >= 0 && gx < W;
            px[k] = in ? xc[(size_t)gy * W + gx] : 0.f;
            py[k] = in ? yc[(size_t)gy * W + gx] : 0.f;
        }
    };
    for (int c = 0; c < 3; ++c) {
        fetch(c);
#pragma unroll
        for (int k = 0; k < kSsimLoads; ++k) {
            const int i = tid + k * kSsimThreads;
            if (i < kSsimE * kSsimE) {
                const int r = i / kSsimE, q = i - r * kSsimE;
                const int o = r * kSsimEp + q;
                const float xv = px[k], yv = py[k];
                sxy[o] = make_float2(xv, yv);
                ssq[o] = make_float2(xv * xv, yv * yv);
                spr[o] = xv * yv;
            }
        }
        __syncthreads();
        // horizontal blur of the five maps: rows [0, E), columns [0, M)
        for (int it = tid; it < kSsimE * (kSsimM / kH1); it += kSsimThreads) {
            const int r = it % kSsimE, q0 = (it / kSsimE) * kH1;
            const int src = r * kSsimEp + q0, dst = r * kSsimMp + q0;
            blur_strip<kH1>(sxy + src, 1, hxy + dst, 1, sp.g);
            blur_strip<kH1>(ssq + src, 1, hsq + dst, 1, sp.g);
            blur_strip<kH1>(spr + src, 1, hpr + dst, 1, sp.g);
        }
        __syncthreads();
        // vertical blur and the SSIM terms over [M][M]
        if (tid < kSsimM * (kSsimM / kV1)) {
            const int q = tid % kSsimM, r0 = (tid / kSsimM) * kV1;
            float2 bxy[kV1], bsq[kV1];
            float bpr[kV1];
            blur_strip_reg<kV1>(hxy + r0 * kSsimMp + q, kSsimMp, bxy, sp.g);
            blur_strip_reg<kV1>(hsq + r0 * kSsimMp + q, kSsimMp, bsq, sp.g);
            blur_strip_reg<kV1>(hpr + r0 * kSsimMp + q, kSsimMp, bpr, sp.g);
            const int gx = X0 - kSsimR + q;
#pragma unroll
            for (int o = 0; o < kV1; ++o) {
                const int r = r0 + o, gy = Y0 - kSsimR + r;
                float A = 0.f, B = 0.f, Cc = 0.f;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const float mx = bxy[o].x, my = bxy[o].y;
                    const float vx = bsq[o].x - mx * mx, vy = bsq[o].y - my * my, cxy = bpr[o] - mx * my;
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
                    if (r >= kSsimR && r < kSsimR + kSsimT && q >= kSsimR && q < kSsimR + kSsimT)
                        part -= sw * S * invP3;
                }
                mAB[r * kSsimMp + q] = make_float2(A, B);
                mC[r * kSsimMp + q] = Cc;
            }
        }
        __syncthreads();
        // horizontal blur of A, B, C: rows [0, M), columns [0, T)
        for (int it = tid; it < kSsimM * (kSsimT / kH2); it += kSsimThreads) {
            const int r = it % kSsimM, q0 = (it / kSsimM) * kH2;
            blur_strip<kH2>(mAB + r * kSsimMp + q0, 1, gAB + r * kSsimTp + q0, 1, sp.g);
            blur_strip<kH2>(mC + r * kSsimMp + q0, 1, gC + r * kSsimTp + q0, 1, sp.g);
        }
        __syncthreads();
        // vertical blur of A, B, C over the tile and the colour gradient
        {
            const int q = tid % kSsimT, r0 = (tid / kSsimT) * kV2;
            float2 fAB[kV2];
            float fC[kV2];
            blur_strip_reg<kV2>(gAB + r0 * kSsimTp + q, kSsimTp, fAB, sp.g);
            blur_strip_reg<kV2>(gC + r0 * kSsimTp + q, kSsimTp, fC, sp.g);
            const int gx = X0 + q;
#pragma unroll
            for (int o = 0; o < kV2; ++o) {
                const int gy = Y0 + r0 + o;
                if (gy < H && gx < W) {
                    const float2 xy = sxy[(r0 + o + 2 * kSsimR) * kSsimEp + q + 2 * kSsimR];
                    const float d = xy.x - xy.y;
                    const float dssim = (fAB[o].x + 2.f * xy.x * fAB[o].y + xy.y * fC[o]) * invP3;
                    tg.d_color[c * P + (size_t)gy * W + gx] = l1w * sgn(d) * invP3 - sw * dssim;
                    part += l1w * fabsf(d) * invP3;
                }
            }
        }
        __syncthreads();
    }
    // depth term and the constant lambda1 lambda2 of (1 - SSIM), once per view
    const bool depth = tg.target_depth != nullptr && vp.depth != nullptr;
    constexpr int kDepthLoads = kSsimT * kSsimT / kSsimThreads;
    float dz[kDepthLoads];
#pragma unroll
    for (int k = 0; k < kDepthLoads; ++k) {   // all loads first, then the stores
        const int i = tid + k * kSsimThreads, gy = Y0 + i / kSsimT, gx = X0 + i % kSsimT;
        const size_t p = (size_t)gy * W + gx;
        dz[k] = depth && gy < H && gx < W ? vp.depth[p] - tg.target_depth[p] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kDepthLoads; ++k) {
        const int i = tid + k * kSsimThreads, gy = Y0 + i / kSsimT, gx = X0 + i % kSsimT;
        if (gy >= H || gx >= W) continue;
        part += (1.f - sp.lambda1) * fabsf(dz[k]) * invP;
        if (tg.d_depth) tg.d_depth[(size_t)gy * W + gx] = depth ? (1.f - sp.lambda1) * sgn(dz[k]) * invP : 0.f;
    }
    if (t == 0 && tid == 0) part += sw;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) s_warp[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < kSsimThreads / 32; ++w) s += s_warp[w];
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
    rgbd_loss_kernel<<<tiles, kSsimThreads, kSsimSmem, st>>>(vt, lt, sp, loss);
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
    const unsigned bx = max(1u, min(1024u, (maxP / 4 + 255u) / 256u));
    l1_loss_kernel<<<dim3(bx, vt.V), 256, 0, st>>>(vt, lt, color_weight, depth_weight, loss);
    return cudaGetLastError();
}

}  // namespace gsr
