// noalloc.cu -- gsr_render_noalloc: the forward render for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: plug-ins and
// callbacks that run inside another framework's execution phase, where only
// the host framework owns the device allocator, and real-time loops that must
// not allocate because an allocation can synchronise the device and has no
// bounded latency.  They still own their inputs and outputs; what they cannot
// provide is the render's scratch workspace.  This entry point gives them one
// that already exists: a file-scope static device array, loaded with the
// library, so every GPU that loads the library holds it until the process
// exits.  The render itself is gsr_render, unchanged, pointed at that array.
// Each build of the library (libgsr.so, libgsr_checked.so) links its own copy
// of this file and so holds its own array: a process that loads both holds
// two, and the two builds never share one.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "kernels.cuh"

namespace {

// The workspace of every gsr_render_noalloc call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GSR_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol's name is only a host-side stand-in, never a device
// address, so the address must come from cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_addr[kMaxDevices] = {};

__global__ void copy_status_kernel(const gsr::WsHeader *h, int32_t *out) { *out = h->status; }

gsr_status cuda_error(gsr_ctx *ctx, cudaError_t e, const char *what) {
    char msg[256];
    snprintf(msg, sizeof msg, "gsr_render_noalloc: %s: %s", what, cudaGetErrorString(e));
    gsr::set_ctx_error(ctx, msg);
    return GSR_ECUDA;
}

}  // namespace

extern "C" gsr_status gsr_render_noalloc(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V,
                                         int32_t *status, gsr_stream stream) {
    if (!ctx || !gs || !views) return GSR_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(ctx, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        gsr::set_ctx_error(ctx, "gsr_render_noalloc: device index beyond the 64 this entry point tracks");
        return GSR_ECUDA;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            // set-up, once per device, with that device current
            e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return cuda_error(ctx, e, "cudaGetSymbolAddress of the static scratch");
            }
        }
        scratch = g_addr[dev];
    }
    // The smallest useful workspace holds one sort tile of keys; if even that
    // is larger than the static scratch, this scene is too big for this path.
    size_t need = 0;
    gsr_status s = gsr_workspace_size(ctx, gs->N, views, V, 1, &need);
    if (s != GSR_OK) return s;
    if (need > (size_t)GSR_NOALLOC_SCRATCH_BYTES) {
        gsr::set_ctx_error(ctx, "gsr_render_noalloc: this scene needs a larger workspace than the "
                                "static scratch of GSR_NOALLOC_SCRATCH_BYTES; use gsr_render");
        return GSR_EINVAL;
    }
    s = gsr_render(ctx, gs, views, V, scratch, (size_t)GSR_NOALLOC_SCRATCH_BYTES, stream);
    if (s != GSR_OK || !status) return s;
    // launched with cudaLaunchKernel, whose return is this launch's own error
    // (cudaGetLastError could return one that the caller left behind)
    const gsr::WsHeader *hdr = static_cast<const gsr::WsHeader *>(scratch);
    void *args[] = {&hdr, &status};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(&copy_status_kernel), dim3(1), dim3(1), args, 0,
                         reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GSR_OK : cuda_error(ctx, e, "status copy launch");
}
