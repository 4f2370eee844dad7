// loss.cu -- L1 loss front end: the L1 colour and depth terms of Eq.
// "rnd_loss" (Sec. 3.3), mean over each view's pixels, with their gradients
// written for the backward.  HBM-bound: one read of rendered and target
// images, one write of the gradients.
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

}  // namespace

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
