// kernels.cuh -- launch wrappers of the rasteriser stages (host side).
#pragma once

#include "common.cuh"

namespace gsr {

struct GradPtrs {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
    int accumulate;
    float *densify_grad, *densify_count, *densify_radius;   // all NULL or all set
};

// preprocess.cu
cudaError_t launch_preprocess_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, int sm_count,
                                  cudaStream_t st);
cudaError_t launch_preprocess_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, const GradPtrs &out,
                                  cudaStream_t st);

cudaError_t launch_pose_reduce(const ViewTable &vt, const Ws &ws, int accumulate, cudaStream_t st);

// surfel.cu
cudaError_t launch_surfel_preprocess_fwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws, cudaStream_t st);
cudaError_t launch_surfel_preprocess_bwd(const ViewTable &vt, const GaussianPtrs &gp, const Ws &ws,
                                         const GradPtrs &out, cudaStream_t st);
cudaError_t launch_surfel_blend_fwd(const ViewTable &vt, const Ws &ws, cudaStream_t st);
cudaError_t launch_surfel_blend_bwd(const ViewTable &vt, const Ws &ws, cudaStream_t st);

// binning.cu
cudaError_t launch_scan_duplicate(const ViewTable &vt, const Ws &ws, cudaStream_t st);
cudaError_t launch_sort(const Ws &ws, int sm_count, cudaStream_t st);
cudaError_t launch_ranges(const Ws &ws, int sm_count, cudaStream_t st);

// density.cu
size_t density_workspace_bytes(int N);
cudaError_t launch_densify_adc(const GaussianPtrs &gp, const float *grad, const float *count, const float *radius,
                               const float *normals, const gsr_adc_params &prm, const gsr_gaussians_out &out,
                               int *out_count, void *ws, cudaStream_t st);
cudaError_t launch_mcmc_relocate(const GaussianPtrs &gp, const uint32_t *draws, float min_opacity,
                                 const gsr_gaussians_out &out, int *relocated, void *ws, cudaStream_t st);
cudaError_t launch_mcmc_noise(const GaussianPtrs &gp, const float *eta, float scale, float *means_out,
                              cudaStream_t st);

// blend.cu
cudaError_t launch_blend_fwd(const ViewTable &vt, const Ws &ws, cudaStream_t st);
cudaError_t launch_blend_bwd(const ViewTable &vt, const Ws &ws, cudaStream_t st);

// api.cu: sets the message gsr_last_error returns
void set_ctx_error(gsr_ctx *ctx, const char *msg);

// loss.cu
cudaError_t launch_rgbd_loss(const ViewTable &vt, const gsr_l1_view *targets, float lambda1, float lambda2,
                             float *loss, cudaStream_t st);
cudaError_t launch_l1_loss(const ViewTable &vt, const gsr_l1_view *targets, float color_weight, float depth_weight,
                           float *loss, cudaStream_t st);

}  // namespace gsr
