/*
 * gsr.h -- C ABI of the B300 (sm_103a) differentiable Gaussian rasteriser.
 *
 * The library renders anisotropic 3-D Gaussians into a batch of keyframes and
 * differentiates the result, following the rendering equation of
 * DROID-Splat (arXiv 2411.17660), Sec. 3.3, Eq. "rendering":
 *     C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j),   alpha_i = sigma_i G_i,
 * where c_i is the colour converted from the spherical harmonics and G_i the
 * Gaussian projected with the keyframe pose (R, t).  gsr_render produces the
 * image I', the depth Z' and the opacity of every keyframe of a batch;
 * gsr_render_backward backpropagates dL/d(images) to every Gaussian parameter
 * (Sec. 3.3: "optimized via backpropagation") and to each keyframe pose
 * (Sec. 3.3, pose finetuning; Supp. Sec. 1.3 "Feedback").
 *
 * Memory: every pointer in the structs below is a DEVICE pointer owned by the
 * caller, except where marked "host".  The library allocates no device
 * memory: the caller provides one workspace buffer per render (size from
 * gsr_workspace_size) and must pass the same workspace, Gaussians and views
 * to gsr_render_backward as to the gsr_render it differentiates.  A
 * workspace may start with any content and may be reused for other scenes;
 * between iterations on one layout it keeps its per-pair gradient rows zero
 * (the backward clears them after use, and its header records the layout
 * whose rows are clean, so that the next gsr_render need not clear them;
 * on any other layout or content gsr_render clears them all).  All calls
 * enqueue work on the given stream and return without synchronising, except
 * gsr_read_info, which waits for the stream.
 *
 * Errors: argument errors are returned synchronously (GSR_EINVAL, with a
 * message in gsr_last_error).  Launch failures return GSR_ECUDA.  Errors
 * found on the device (key capacity exceeded, a bounded wait that ran out)
 * are recorded in the workspace and reported by gsr_read_info; the outputs of
 * such a call are undefined.
 *
 * Parameter layout is planar ("[K][N]": component k of Gaussian g at k*N+g).
 * Conventions (readings of the paper, which inherits them from 3DGS):
 * pinhole camera with pixel centres at integer (x, y), u = fx x/z + cx;
 * T_cw = [W | t] maps world to camera (camera looks down +z); quaternions are
 * (w, x, y, z) and need not be normalised; scales are log-scales; opacity is
 * sigmoid(logit); colour = max(0, sum_k SH_k Y_k(dir) + 0.5) with real SH of
 * degree <= 3 (Condon-Shortley phase), dir from the camera centre to the mean.
 * Rules: cull z <= 0.2; Sigma' = J W Sigma W^T J^T + 0.3 I (J with x/z, y/z
 * clamped to 1.3x the half field of view); per pixel, Gaussians with
 * Mahalanobis d^2 <= 9 in depth order; alpha = min(0.99, sigma exp(-d^2/2));
 * alpha < 1/255 skipped; stop before the Gaussian that would take the
 * transmittance below 1e-4.  Depth output = sum_i w_i z_i, opacity output =
 * 1 - T_final.  Everything is computed in FP32.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSR_ABI_VERSION 7
#define GSR_MAX_VIEWS 64

typedef enum {
    GSR_OK = 0,
    GSR_EINVAL = -1,     /* bad argument (synchronous) */
    GSR_ECAPACITY = -2,  /* device: more tile keys than the workspace holds */
    GSR_ECUDA = -3,      /* a CUDA call or launch failed */
    GSR_ETIMEOUT = -4,   /* device: a bounded inter-block wait gave up */
    GSR_ENOTREADY = -5,  /* backward called without a matching forward */
    GSR_EINTERNAL = -6   /* device: an internal consistency check failed */
} gsr_status;

/* Same handle type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *gsr_stream;

typedef struct gsr_ctx gsr_ctx;

/* Library configuration of a context (gsr_autotune may replace tile,
 * binning, batch and fwd_rows with the fastest it measured). */
typedef struct {
    int tile;              /* screen tile edge in pixels: 8, 16 or 32 (0 = 16) */
    uint32_t spin_limit;   /* iterations before a bounded device wait gives up (0 = default) */
    int flags;             /* 0, or GSR_TEST_STALL_SORT (test hook, see below) */
    int binning;           /* GSR_BIN_TILE (0, default) or GSR_BIN_RADIX */
    int batch;             /* depth-sorted list entries a blend warp stages per round: 32 or 64
                              (0 = 32); 64 needs a tile of 8 or 16 (GSR_EINVAL otherwise).
                              The images do not depend on it, only the speed. */
    int fwd_rows;          /* pixel rows of a forward blend warp's block (8 columns wide): 8 or
                              16 (0 = 16, or 8 at tile 8); 16 needs a tile of 16 or 32
                              (GSR_EINVAL otherwise).  Taller blocks share each staged entry
                              among more pixels, shorter ones evaluate fewer entries that do
                              not reach a pixel; the images do not depend on it. */
} gsr_config;

/* Test hook for the bounded-wait path: the first tile of the first radix-sort
 * pass never publishes its digit counts, so the next tile's look-back wait
 * runs out after spin_limit iterations and the call reports GSR_ETIMEOUT
 * (outputs undefined).  Only the onesweep passes wait on other blocks: all of
 * GSR_BIN_RADIX's, and GSR_BIN_TILE's beyond 32,768 tiles.  Never set outside
 * tests. */
#define GSR_TEST_STALL_SORT 1

/* Tile binning strategies; both give the same list order (by tile, then
 * depth, then Gaussian index) and so bit-identical results.
 * GSR_BIN_TILE: the preprocess emits each pair's (tile, depth, index) keys
 *   (one slot reservation per warp); with up to 32,768 tiles a count kernel
 *   counts them per tile (shared-memory counts per block, one atomic per
 *   block and tile, the last block scans the counts into the ranges) and a
 *   scatter kernel groups them by tile; beyond, onesweep passes over the tile
 *   bits group them; then each tile's (depth, index) words are sorted in
 *   registers or shared memory.
 * GSR_BIN_RADIX: a scan of the per-pair tile counts and a duplication kernel
 *   emit the keys, then one stable onesweep LSD radix sort of all (tile,
 *   depth) keys, 8 bits per pass, with a bounded decoupled look-back. */
#define GSR_BIN_TILE 0
#define GSR_BIN_RADIX 1

/* The Gaussian map (Sec. 3.3: position P, rotation r, scale s, density
 * sigma, SH coefficients).  Device pointers, float32, planar. */
typedef struct {
    int N;                        /* number of Gaussians, >= 0 */
    int sh_degree;                /* 0..3 */
    const float *means;           /* [3][N] world position */
    const float *log_scales;      /* [3][N] log of the axis scales */
    const float *quats;           /* [4][N] (w, x, y, z), unnormalised */
    const float *opacity_logits;  /* [N] sigma = sigmoid(logit) */
    const float *sh;              /* [(deg+1)^2 * 3][N], row = coeff*3 + channel */
} gsr_gaussians;

/* One keyframe: intrinsics (host values), pose and outputs (device). */
typedef struct {
    int H, W;                 /* image size, 1..16384 each */
    float fx, fy, cx, cy;     /* pinhole intrinsics (host values) */
    const float *T_cw;        /* device, 12 floats, row-major [W | t] world->camera */
    float *color;             /* device out [3][H][W] */
    float *depth;             /* device out [H][W] (may be NULL) */
    float *alpha;             /* device out [H][W] (may be NULL) */
    float *median_depth;      /* device out [H][W] (may be NULL): the median depth of Sec. 3.3, read
                                 as the z of the last contributor entered with transmittance above
                                 0.5 (the Gaussian during which the accumulated opacity passes 0.5,
                                 or the last contributor if it never does), 0 without contributors */
} gsr_view;

/* Upstream gradients of one keyframe (device; NULL means zero) and the
 * output pose gradient: dL/dxi for the left perturbation T_cw <- Exp(xi) T_cw,
 * xi = (rho, phi), at xi = 0. */
typedef struct {
    const float *d_color;     /* [3][H][W] or NULL */
    const float *d_depth;     /* [H][W] or NULL */
    const float *d_alpha;     /* [H][W] or NULL */
    const float *d_median_depth; /* [H][W] or NULL; needs a forward that rendered median_depth
                                    (of any view) on the same workspace, else GSR_ENOTREADY */
    float *d_pose;            /* out [6] or NULL */
} gsr_view_grad;

/* Output parameter gradients (device, same layouts as gsr_gaussians),
 * summed over the views of the batch.  accumulate != 0 adds into the arrays
 * (also for d_pose); otherwise they are overwritten. */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
    int accumulate;
    /* Densification statistics of the batch (adaptive density control of
     * 3DGS, used by the paper's mapper), [N] each, all NULL or all set.  A
     * Gaussian is visible in a view when it is not culled and its cutoff
     * ellipse (d^2 <= min(9, 2 ln(255 sigma))) meets the rectangle
     * [0, W-1] x [0, H-1] spanned by the pixel centres (decided in FP32 from
     * the exact minimum of d^2 over that rectangle).  With accumulate != 0,
     * grad and count add and radius takes the maximum, so the arrays can
     * gather several batches. */
    float *densify_grad;      /* sum over visible views of |(dL/du, dL/dv)|, pixels */
    float *densify_count;     /* number of visible views */
    float *densify_radius;    /* max over visible views of 3 sqrt(lambda_max(Sigma')), pixels */
} gsr_grads;

/* Device-side state of the last call on a workspace (gsr_read_info). */
typedef struct {
    int32_t status;              /* first device error (gsr_status), 0 = none */
    uint32_t keys;               /* (Gaussian, tile) keys the last render produced */
    uint32_t key_capacity;       /* keys the workspace holds */
    uint32_t tiles;              /* screen tiles over all views */
    uint64_t pairs_contributing; /* (pixel, Gaussian) pairs composited by the last render */
    uint32_t pairs_visible;      /* (view, Gaussian) pairs of the last Gaussian render that reach a
                                    pixel centre and got tile keys (0 for surfels) */
    uint32_t pairs_backward;     /* checked build (libgsr_checked.so) only, else 0: the (pixel,
                                    Gaussian) pairs the backward since that render took as
                                    contributors, saturated at 2^32 - 1; equal to
                                    pairs_contributing after one backward, as the two kernels take
                                    the same decisions */
} gsr_info;

/* Target images for the L1 loss front end (device). */
typedef struct {
    const float *target_color;   /* [3][H][W] */
    const float *target_depth;   /* [H][W] or NULL (no depth term) */
    float *d_color;              /* out [3][H][W] dL/dcolor */
    float *d_depth;              /* out [H][W] dL/ddepth, or NULL */
} gsr_l1_view;

/* Creates a context (host memory only).  cfg may be NULL for defaults.
 * Returns GSR_EINVAL for an unsupported tile size, binning, batch or fwd_rows. */
gsr_status gsr_create(const gsr_config *cfg, gsr_ctx **out);

/* Frees a context.  NULL is ignored. */
gsr_status gsr_destroy(gsr_ctx *ctx);

/* Bytes of workspace for N Gaussians, these V views and room for
 * key_capacity (Gaussian, tile) keys (0 = a default estimate of 8 keys per
 * (view, Gaussian) pair, at least 1M).  Host only. */
gsr_status gsr_workspace_size(gsr_ctx *ctx, int N, const gsr_view *views, int V,
                              size_t key_capacity, size_t *bytes);

/* Forward render of V keyframes (1..GSR_MAX_VIEWS) in one batched pass:
 * projection (EWA, SH colour), tile binning with a depth-keyed radix sort,
 * front-to-back compositing (Sec. 3.3, Eq. "rendering").  Writes each view's
 * color/depth/alpha and keeps in the workspace what the backward needs.
 * ws must be 256-byte aligned and ws_bytes >= gsr_workspace_size(..., cap)
 * for some cap; the key capacity is derived from ws_bytes.  The first render
 * on a device also raises some binning kernels' shared-memory limit (a
 * host-side setting), so make one render call before capturing the stream
 * into a CUDA graph. */
gsr_status gsr_render(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V,
                      void *ws, size_t ws_bytes, gsr_stream stream);

/* Backward of the last gsr_render on ws: back-to-front replay from the stored
 * final transmittance and contributor index, then projection/SH backward and
 * the per-view SE(3) pose reduction.  grads[v] gives view v's upstream
 * gradients and pose output.  Returns GSR_ENOTREADY if ws was not rendered
 * with the same N, views and tile size.  The first backward on a device also
 * raises a kernel's shared-memory limit (a host-side setting), so make one
 * backward call before capturing the stream into a CUDA graph. */
gsr_status gsr_render_backward(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views,
                               const gsr_view_grad *grads, int V, const gsr_grads *out,
                               void *ws, size_t ws_bytes, gsr_stream stream);

/* Waits for stream, then copies the workspace's device state into *info
 * (host).  Use it to detect GSR_ECAPACITY (grow key_capacity to info->keys
 * and render again) or GSR_ETIMEOUT. */
gsr_status gsr_read_info(gsr_ctx *ctx, const void *ws, size_t ws_bytes, gsr_info *info,
                         gsr_stream stream);

/* The device status word of ws alone: waits for stream and returns the first
 * device error that the calls on ws recorded (GSR_ECAPACITY, GSR_ETIMEOUT,
 * GSR_EINTERNAL), or GSR_OK; the same value as gsr_read_info's info.status.
 * Its own failures are GSR_EINVAL (bad arguments) and GSR_ECUDA, with a
 * message in gsr_last_error. */
gsr_status gsr_get_status(gsr_ctx *ctx, const void *ws, size_t ws_bytes, gsr_stream stream);

/* One configuration timed by gsr_autotune. */
typedef struct {
    int tile, binning, batch, fwd_rows;   /* the candidate (see gsr_config) */
    float ms;                   /* best of reps forward + backward times (CUDA events), or -1 */
    int32_t status;             /* GSR_OK, or why it was not timed (GSR_ECAPACITY: its keys
                                   exceed the workspace; a synchronous error code) */
} gsr_tune_entry;

/* Autotuner of the batched render (the paper's mapper renders a batch of
 * keyframes every iteration, Supp. Sec. 1.2; tile size and per-warp entry
 * batch trade sort work against blend work differently for every scene and
 * set of views).  Times forward + backward on the caller's own Gaussians,
 * views and workspace for every candidate (tile 8, 16, 32) x (GSR_BIN_TILE,
 * GSR_BIN_RADIX) x (batch 32, 64; 64 not at tile 32) x (fwd_rows 16, 8; 16
 * not at tile 8), best of reps (1..100)
 * after one warm-up run, the rendered colour serving as the upstream
 * gradient, and leaves the fastest configuration in ctx (ties: the earlier
 * candidate in that order).  The candidates' results are identical images;
 * only their speed differs.
 * - views' color/depth/alpha receive renders and grads (all arrays, pose
 *   outputs not used) receives gradients: pass scratch buffers.
 * - ws must be large enough for the candidate with the most keys (tile 8):
 *   a candidate whose keys do not fit is skipped with status GSR_ECAPACITY.
 *   After tuning, size workspaces again with gsr_workspace_size: the tile
 *   size changes the layout.
 * - entries (host, may be NULL when max_entries is 0) receives up to
 *   max_entries candidates in the order above, *n_entries (may be NULL)
 *   their number.
 * - It synchronises the stream after every run (it reads the device status
 *   and the event times), so it cannot be captured in a CUDA graph.
 * Returns GSR_OK when at least one candidate ran; otherwise the first
 * candidate's failure (the context keeps its configuration).  A context
 * created with test flags is rejected (GSR_EINVAL). */
gsr_status gsr_autotune(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V,
                        const gsr_grads *grads, void *ws, size_t ws_bytes, int reps,
                        gsr_tune_entry *entries, int max_entries, int *n_entries, gsr_stream stream);

/* L1 loss front end (the L1 terms of Eq. "rnd_loss"): for each view,
 * loss += color_weight * mean|C - C*| + depth_weight * mean|D - D*| over its
 * pixels (colour mean over 3 channels), and writes dL/dC, dL/dD.  Reads the
 * rendered color/depth of views[v].  loss: device float, overwritten. */
gsr_status gsr_l1_loss(gsr_ctx *ctx, const gsr_view *views, const gsr_l1_view *targets, int V,
                       float color_weight, float depth_weight, float *loss, gsr_stream stream);

/* gsr_render and gsr_l1_loss in one pass: the forward blend takes the L1
 * terms of each pixel it has just composited, so the rendered images are not
 * read back and no loss kernel runs.  Arguments are those of gsr_render and
 * gsr_l1_loss; the depth term is on wherever targets[v].target_depth is
 * non-NULL (views[v].depth may then be NULL).  d_color and d_depth equal
 * gsr_l1_loss's bit for bit; loss (device float, overwritten) equals it up to
 * the order of the FP32 sum.  Errors: those of gsr_render, and GSR_EINVAL for
 * a NULL targets, loss, target_color or d_color. */
gsr_status gsr_render_l1(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V,
                         const gsr_l1_view *targets, float color_weight, float depth_weight, float *loss,
                         void *ws, size_t ws_bytes, gsr_stream stream);

/* Mixed rendering loss of Eq. "rnd_loss" (Sec. 3.3), summed over views:
 *   lambda1 [(1 - lambda2) mean|C - C*| + lambda2 (1 - SSIM(C, C*))]
 *   + (1 - lambda1) mean|D - D*|,
 * SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2,
 * zero padding, averaged over the 3 channels and the pixels; the paper uses
 * lambda2 = 0.2 and lambda1 = 0.9 (TUM-RGBD) or 0.8 (Replica).  Reads each
 * view's rendered color/depth, writes dL/dC and dL/dD into targets[v]
 * (d_depth may be NULL; without target_depth the depth term is 0).  loss:
 * device float, overwritten.  Needs no workspace. */
gsr_status gsr_rgbd_loss(gsr_ctx *ctx, const gsr_view *views, const gsr_l1_view *targets, int V, float lambda1,
                         float lambda2, float *loss, gsr_stream stream);

/* ------------------------------------------------------------------ */
/* 2-D surfels (the "2D Gaussian Splatting" primitives the paper compares
 * its 3-D Gaussians with, Sec. 3.3 last paragraph, Supp. "2D Gaussian
 * Splatting"): each Gaussian is a flat disk with tangents t_u, t_v (first
 * two columns of R(q)) scaled by exp(log_scales[0..1]) (log_scales[2] is
 * unused and gets zero gradient) and normal t_w.  A pixel meets the disk
 * where its two homogeneous planes h_x = M_0 - x M_2, h_y = M_1 - y M_2 cross
 * (M = K [s_u W t_u | s_v W t_v | W mu + t]): (u, v, 1) ~ h_x x h_y;
 * rho = min(u^2 + v^2, 2 |pixel - projected centre|^2) (screen-space
 * low-pass), alpha = min(0.99, sigma exp(-rho/2)) with the 3-D path's cutoff
 * (rho <= 9), skip (1/255) and stop (1e-4) rules; sorted by the depth of
 * the centre.  Culled: centre depth <= 0.2 or the cutoff disk reaching
 * depth 0.2.  Extra outputs: the normal map sum w n (n = W t_w turned
 * towards the camera, camera frame) and the depth distortion
 * sum_{i>j} w_i w_j (z_i - z_j)^2 with z the depth of the ray-disk
 * intersection (the colour/depth/alpha outputs of gsr_view use the same
 * weights and z). */
typedef struct {
    float *normal;            /* device out [3][H][W] or NULL */
    float *distortion;        /* device out [H][W] or NULL */
} gsr_surfel_out;

typedef struct {
    const float *d_normal;    /* [3][H][W] or NULL */
    const float *d_distortion; /* [H][W] or NULL */
} gsr_surfel_grad;

/* Forward render of surfels, batched like gsr_render; views[v].median_depth
 * must be NULL; extra[v] holds view v's normal and distortion outputs
 * (extra may be NULL: neither is written).  Same workspace rules. */
gsr_status gsr_render_surfels(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views,
                              const gsr_surfel_out *extra, int V, void *ws, size_t ws_bytes, gsr_stream stream);

/* Backward of the last gsr_render_surfels on ws: grads[v] (d_median_depth
 * must be NULL) and extra[v] (may be NULL) give the upstream gradients;
 * parameter and pose gradients as for gsr_render_backward (densification
 * statistics are not produced for surfels: their pointers must be NULL).
 * Returns GSR_ENOTREADY unless ws holds a surfel forward of the same
 * Gaussians and views. */
gsr_status gsr_render_surfels_backward(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views,
                                       const gsr_view_grad *grads, const gsr_surfel_grad *extra, int V,
                                       const gsr_grads *out, void *ws, size_t ws_bytes, gsr_stream stream);

/* Stage events (a profiling aid).  events holds GSR_STAGE_EVENTS cudaEvent_t
 * handles created by the caller (copied at this call), or is NULL to stop.
 * While set, gsr_render records events[0] on its stream before its first
 * launch and events[1+k] after forward stage k (0 preprocess, 1 scan + key
 * duplication, 2 radix sort, 3 tile ranges, 4 blend); gsr_render_backward
 * records events[6] before its first launch and events[7+k] after backward
 * stage k (0 empty: the gradient rows are already zero, 1 blend backward, 2
 * preprocess backward with the pose reduction).  Elapsed times between consecutive events are the stage
 * durations on the device. */
#define GSR_STAGE_EVENTS 10
gsr_status gsr_set_stage_events(gsr_ctx *ctx, void *const *events);

/* Forward render without a caller-provided workspace.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory (plug-ins running inside another framework's execution
 * phase, where only that framework owns the allocator, and real-time loops
 * that must not allocate).  It renders exactly as gsr_render, but its scratch
 * is a static device array of GSR_NOALLOC_SCRATCH_BYTES inside the library,
 * held on every device that loads the library until the process exits.  No
 * device memory is allocated by the call.  Each build of the library
 * (libgsr.so, libgsr_checked.so) holds its own array; a process that loads
 * both holds both, and the builds never share one.
 * - Scenes whose smallest workspace (gsr_workspace_size with key_capacity 1)
 *   exceeds GSR_NOALLOC_SCRATCH_BYTES are rejected with GSR_EINVAL.  The key
 *   capacity is whatever fits in the rest of the array.
 * - status: device pointer to one int32 that receives the call's device-side
 *   status (0, or GSR_ECAPACITY when the tile keys did not fit); may be NULL.
 * - The first call on a device looks up the array's device address; make it
 *   before any stream capture on that device.
 * - All calls share the one array and each leaves its contents behind; calls
 *   that can overlap on the GPU (different streams, or threads) race.
 * - There is no backward for this render: use gsr_render when gradients are
 *   needed. */
#define GSR_NOALLOC_SCRATCH_BYTES (64u << 20)
gsr_status gsr_render_noalloc(gsr_ctx *ctx, const gsr_gaussians *gs, const gsr_view *views, int V,
                              int32_t *status, gsr_stream stream);

/* ------------------------------------------------------------------ */
/* Density control of the map between optimisation steps (Sec. 3.3, last
 * paragraph; Supp. "Monte Carlo Markov Chain Gaussian Splatting"): the 3DGS
 * adaptive density control driven by the statistics of gsr_grads.densify_*,
 * and the MCMC strategy's relocation and position noise.  Every random draw
 * is an input, so the results are deterministic.  All pointers are device
 * pointers; parameter arrays are planar like gsr_gaussians. */

/* Thresholds of the adaptive density control. */
typedef struct {
    float grad_threshold;      /* densify when densify_grad >= grad_threshold * densify_count (count > 0) */
    float split_scale;         /* a densifying Gaussian whose largest scale exceeds this is split, else cloned */
    float min_opacity;         /* prune below this opacity, > 0 and < 1 */
    float max_screen_radius;   /* prune above this densify_radius (pixels); 0 = no such test */
    float max_world_scale;     /* prune above this largest scale; 0 = no such test */
} gsr_adc_params;

/* Writable Gaussian arrays with room for N Gaussians (planar with stride N;
 * sh has 3 (deg+1)^2 rows for the degree of the input). */
typedef struct {
    int N;
    float *means, *log_scales, *quats, *opacity_logits, *sh;
} gsr_gaussians_out;

/* Scratch bytes the density calls need for N Gaussians (caller-allocated,
 * 256-byte aligned, passed as ws). */
gsr_status gsr_density_workspace_size(gsr_ctx *ctx, int N, size_t *bytes);

/* Adaptive density control.  In the input's order, Gaussian g becomes:
 * nothing if pruned (opacity < min_opacity, or densify_radius above
 * max_screen_radius, or largest scale above max_world_scale); two children
 * if it densifies and its largest scale exceeds split_scale, at
 * mean + R diag(scale) eps_c (eps_c = split_normals rows [3c, 3c+3), c = 0,
 * 1, each [N]) with log-scales - ln 1.6 and everything else copied; itself
 * and an exact copy if it densifies otherwise; else itself.  grad, count,
 * radius: [N] as gathered by gsr_render_backward.  *out_count (device int)
 * receives the number of output Gaussians, which may exceed out->N: only the
 * first out->N are written.  out must not overlap the input. */
gsr_status gsr_densify_adc(gsr_ctx *ctx, const gsr_gaussians *gs, const float *grad, const float *count,
                           const float *radius, const float *split_normals, const gsr_adc_params *params,
                           const gsr_gaussians_out *out, int *out_count, void *ws, size_t ws_bytes,
                           gsr_stream stream);

/* MCMC relocation.  Gaussians of opacity <= min_opacity are dead; dead slot
 * g takes a live source drawn with probability proportional to opacity by
 * the uniform 32-bit draws[g] (integer weights floor(sigmoid(logit) 2^24),
 * the first source whose inclusive weight sum exceeds floor(draws[g] W /
 * 2^32)).  A source drawn n times and its n copies get opacity
 * o' = 1 - (1 - o)^(1/k) and scales times
 * o / sum_{i=1..k} sum_{j<i} C(i-1, j) (-1)^j o'^(j+1) / sqrt(j+1),
 * k = min(n + 1, 51), o' within [min_opacity, 1 - 2^-23].  out (room for at
 * least gs->N, not overlapping the input) receives all N Gaussians;
 * *relocated (device int) the number of dead slots filled (0 when no
 * Gaussian is live). */
gsr_status gsr_mcmc_relocate(gsr_ctx *ctx, const gsr_gaussians *gs, const uint32_t *draws, float min_opacity,
                             const gsr_gaussians_out *out, int *relocated, void *ws, size_t ws_bytes,
                             gsr_stream stream);

/* MCMC position noise: means_out = mean + scale sigmoid(-100 (o - 0.005))
 * Sigma eta, Sigma = R diag(scale^2) R^T the Gaussian's covariance, eta
 * [3][N] standard-normal draws, scale = lr_noise (1e4 in the paper) times
 * the position learning rate.  means_out ([3][N]) may be gs->means. */
gsr_status gsr_mcmc_noise(gsr_ctx *ctx, const gsr_gaussians *gs, const float *eta, float scale,
                          float *means_out, gsr_stream stream);

/* Message of the last synchronous error on ctx (host string owned by ctx). */
const char *gsr_last_error(const gsr_ctx *ctx);

/* Name of a status code. */
const char *gsr_status_string(gsr_status s);

/* GSR_ABI_VERSION of the built library. */
int gsr_abi_version(void);

/* sizeof of the ABI structs, for binding checks: 0 gsr_config, 1
 * gsr_gaussians, 2 gsr_view, 3 gsr_view_grad, 4 gsr_grads, 5 gsr_info,
 * 6 gsr_l1_view, 7 gsr_surfel_out, 8 gsr_surfel_grad, 9 gsr_adc_params,
 * 10 gsr_gaussians_out, 11 gsr_tune_entry; 0 for other values. */
size_t gsr_abi_sizeof(int which);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H */
