// density.cu -- density control of the Gaussian map between optimisation
// steps (Sec. 3.3, last paragraph; Supp. "Monte Carlo Markov Chain Gaussian
// Splatting"): the 3DGS adaptive density control (clone, split, prune from
// the densification statistics the backward gathers) and the MCMC strategy's
// relocation of low-opacity Gaussians and its position noise.
//
// Every decision that selects or counts Gaussians is exact: thresholds are
// compared in FP64 (FP32 inputs, exact products) or, for the MCMC draws, on
// integer weights made from an FP32 sigmoid built only from correctly rounded
// operations (exp by Cody-Waite reduction and a degree-7 Taylor polynomial),
// so the result does not depend on the compiler or the GPU.  Output order is
// the input order (device-wide scans), so the results are deterministic.
#include <cmath>

#include "kernels.cuh"
#include "project.cuh"

namespace gsr {

namespace {

constexpr int kDThreads = 256;
constexpr int kDItems = 16;
constexpr int kDChunk = kDThreads * kDItems;   // values per scan block
// The scans' first passes take a chunk with 1024 threads, 4 coalesced rounds
// of 32 per warp: enough warps in flight to hide the loads of each round.
constexpr int kDScanThreads = 1024;
constexpr int kDScanRounds = kDChunk / kDScanThreads;
constexpr int kMaxCopies = 51;
constexpr float kSplitLog = 0.47000362924573558f;   // ln 1.6
constexpr float kNoiseK = 100.f, kNoiseT = 0.005f;

// ---------------------------------------------------------------- device-wide scan of u64 values
// Block b scans values [b kDChunk, (b + 1) kDChunk), each warp a run of
// kDScanRounds * 32 of them in coalesced rounds; the block totals are scanned by
// one block; a last pass adds each block's offset.
template <int THREADS>
__device__ __forceinline__ unsigned long long block_scan_ex(unsigned long long x, unsigned long long *s_warp,
                                                            unsigned long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int W = THREADS / 32;
        unsigned long long w = lane < W ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < W) s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned long long before = warp > 0 ? s_warp[warp - 1] : 0ull;
    total = s_warp[THREADS / 32 - 1];
    __syncthreads();
    return before + incl - x;
}

// vals[i] := exclusive (or inclusive) prefix of vals within its block; block
// totals to partials.
// Warp w of block b takes the kDScanRounds * 32 values from b kDChunk + w kDScanRounds 32,
// in kDScanRounds coalesced rounds of 32 with a warp scan each: v[k] holds the
// value of index rounds_base() + 32 k + lane and becomes its block-local
// (inclusive or exclusive) prefix; returns the block total.
__device__ __forceinline__ size_t rounds_base() {
    return (size_t)blockIdx.x * kDChunk + (size_t)(threadIdx.x >> 5) * (32 * kDScanRounds);
}

__device__ __forceinline__ unsigned long long block_rounds_scan(unsigned long long (&v)[kDScanRounds], bool inclusive,
                                                                unsigned long long *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long run = 0;
#pragma unroll
    for (int k = 0; k < kDScanRounds; ++k) {
        unsigned long long incl = v[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned long long x = v[k];
        v[k] = run + (inclusive ? incl : incl - x);   // warp-local prefix
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) s_warp[warp] = run;
    __syncthreads();
    unsigned long long before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kDScanThreads / 32; ++w) {
        const unsigned long long c = s_warp[w];
        before += w < warp ? c : 0ull;
        total += c;
    }
#pragma unroll
    for (int k = 0; k < kDScanRounds; ++k) v[k] += before;
    return total;
}

// partials := exclusive prefix of the block totals; *total := their sum.
__global__ void __launch_bounds__(1024) scan_partials_kernel(unsigned long long *partials, uint32_t blocks,
                                                             unsigned long long *total) {
    __shared__ unsigned long long s_warp[32];
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < blocks; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long x = i < blocks ? partials[i] : 0ull;
        unsigned long long t;
        const unsigned long long ex = block_scan_ex<1024>(x, s_warp, t);
        if (i < blocks) partials[i] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kDThreads) scan_add_kernel(unsigned long long *vals, size_t n,
                                                             const unsigned long long *partials) {
    const size_t i = (size_t)blockIdx.x * kDThreads + threadIdx.x;
    if (i < n) vals[i] += partials[i / kDChunk];
}

// ---------------------------------------------------------------- shared per-Gaussian helpers
struct DensityPtrs {
    GaussianPtrs in;
    int C;   // SH rows
    float *om, *ols, *oq, *oo, *osh;   // outputs, planar with capacity cap
    uint32_t cap;
};

// rows values of column g of a planar source to columns k .. k + copies - 1
// (those below cap) of a planar destination, loaded kCopyBatch at a time
// ahead of their stores (one load in flight per thread otherwise: the stores
// may alias the source)
constexpr int kCopyBatch = 16;
__device__ __forceinline__ void copy_rows(const float *src, size_t sstride, float *dst, size_t dstride, int rows,
                                          size_t g, size_t k, int copies, size_t cap) {
    for (int j0 = 0; j0 < rows; j0 += kCopyBatch) {
        float v[kCopyBatch];
#pragma unroll
        for (int c = 0; c < kCopyBatch; ++c) v[c] = j0 + c < rows ? __ldg(src + (j0 + c) * sstride + g) : 0.f;
        for (int r = 0; r < copies; ++r) {
            if (k + r >= cap) break;
#pragma unroll
            for (int c = 0; c < kCopyBatch; ++c)
                if (j0 + c < rows) dst[(j0 + c) * dstride + k + r] = v[c];
        }
    }
}

// Copies Gaussian g of the input to output slots k .. k + copies - 1 (those below the capacity).
__device__ __forceinline__ void copy_gaussian(const DensityPtrs &d, int g, uint32_t k, int copies = 1) {
    const size_t N = (size_t)d.in.N, cap = d.cap;
    copy_rows(d.in.means, N, d.om, cap, 3, (size_t)g, k, copies, cap);
    copy_rows(d.in.log_scales, N, d.ols, cap, 3, (size_t)g, k, copies, cap);
    copy_rows(d.in.quats, N, d.oq, cap, 4, (size_t)g, k, copies, cap);
    copy_rows(d.in.opacity_logits, N, d.oo, cap, 1, (size_t)g, k, copies, cap);
    copy_rows(d.in.sh, N, d.osh, cap, d.C, (size_t)g, k, copies, cap);
}

// ---------------------------------------------------------------- adaptive density control
struct AdcParams {
    float grad_threshold, max_screen_radius;
    double log_split, logit_min, log_world;   // ln(split_scale), logit(min_opacity), ln(max_world_scale) or +inf
    // The same thresholds for FP32 compares of FP32 inputs: x > t <=> x > the
    // largest float <= t, x < t <=> x < the smallest float >= t.
    float log_split_f, logit_min_f, log_world_f;
    int screen_on;
};

// 0: pruned, 1: kept, 2: kept and cloned, 3: split into two.  Every compare
// is exact (the decisions of the FP64 oracle): FP32 inputs against FP64
// thresholds through their FP32 bounds, and grad >= threshold count -- a
// product exact in FP64 -- as grad against the rounded product p and its
// exact error e = fma(threshold, count, -p) (grad > p, or grad == p and
// e <= 0).  e is exact while p lies in [2^-80, 2^100] (its lowest bit, at
// most 47 binades below p, stays above the smallest subnormal); other
// products take FP64, whose rate on this part is low.
__device__ __forceinline__ int adc_decide(const GaussianPtrs &gp, const float *grad, const float *count,
                                          const float *radius, const AdcParams &p, int g) {
    const size_t N = (size_t)gp.N;
    const float ls = fmaxf(gp.log_scales[g], fmaxf(gp.log_scales[N + g], gp.log_scales[2 * N + g]));
    const float cnt = count[g], gr = grad[g];
    const float prod = __fmul_rn(p.grad_threshold, cnt);
    bool dense;
    if (prod >= 0x1p-80f && prod <= 0x1p100f) {
        const float err = __fmaf_rn(p.grad_threshold, cnt, -prod);
        dense = cnt > 0.f && (gr > prod || (gr == prod && err <= 0.f));
    } else {
        dense = cnt > 0.f && (double)gr >= (double)p.grad_threshold * (double)cnt;
    }
    const bool big = ls > p.log_split_f;
    bool pruned = gp.opacity_logits[g] < p.logit_min_f || ls > p.log_world_f;
    if (p.screen_on) pruned |= radius[g] > p.max_screen_radius;
    return pruned ? 0 : (dense ? (big ? 3 : 2) : 1);
}

// The decisions and the in-block exclusive prefix of their output counts,
// in one pass: block b takes Gaussians [b kDChunk, (b + 1) kDChunk), warp w
// the 32 kDScanRounds from b kDChunk + 32 kDScanRounds w, in kDScanRounds coalesced
// rounds of 32 with a warp scan each.  code[g] = in-block output offset << 2
// | decision; the block's output count goes to partials[b].
__global__ void __launch_bounds__(kDScanThreads) adc_decide_scan_kernel(const GaussianPtrs gp, const float *grad,
                                                                    const float *count, const float *radius,
                                                                    const AdcParams p, uint32_t *code,
                                                                    unsigned long long *partials) {
    __shared__ uint32_t s_wsum[kDScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t base = (size_t)blockIdx.x * kDChunk + (size_t)warp * (32 * kDScanRounds);
    uint32_t oc[kDScanRounds], run = 0;   // warp-exclusive offset << 2 | decision
#pragma unroll
    for (int r = 0; r < kDScanRounds; ++r) {
        const size_t g = base + (size_t)r * 32 + lane;
        const int c = g < (size_t)gp.N ? adc_decide(gp, grad, count, radius, p, (int)g) : 0;
        const uint32_t n = c == 0 ? 0u : (c == 1 ? 1u : 2u);
        uint32_t incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        oc[r] = ((run + incl - n) << 2) | (uint32_t)c;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) s_wsum[warp] = run;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kDScanThreads / 32; ++w) {
        const uint32_t c = s_wsum[w];
        before += w < warp ? c : 0u;
        total += c;
    }
#pragma unroll
    for (int r = 0; r < kDScanRounds; ++r) {
        const size_t g = base + (size_t)r * 32 + lane;
        if (g < (size_t)gp.N) code[g] = oc[r] + (before << 2);
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// Output slot of Gaussian g from its code and its block's exclusive prefix.
__device__ __forceinline__ unsigned long long adc_slot(const uint32_t *code, const unsigned long long *partials,
                                                       size_t g, int &c) {
    const uint32_t v = code[g];
    c = (int)(v & 3u);
    return partials[g / kDChunk] + (v >> 2);
}

// Every kept Gaussian to its output slots (a split one to both children's).
__global__ void __launch_bounds__(kDThreads) adc_write_kernel(const DensityPtrs d, const uint32_t *code,
                                                              const unsigned long long *partials,
                                                              const unsigned long long *total, int *out_count) {
    const int g = blockIdx.x * kDThreads + threadIdx.x;
    if (g == 0) *out_count = *total > 0x7fffffffull ? 0x7fffffff : (int)*total;
    if (g >= d.in.N) return;
    int c;
    const unsigned long long k0 = adc_slot(code, partials, (size_t)g, c);
    if (c != 0 && k0 < d.cap) copy_gaussian(d, g, (uint32_t)k0, c == 1 ? 1 : 2);
}

// The children of the split Gaussians (already copied there): means
// mu + R diag(s) eps_c and log-scales - ln 1.6.
__global__ void __launch_bounds__(kDThreads) adc_split_kernel(const DensityPtrs d, const float *normals,
                                                              const uint32_t *code,
                                                              const unsigned long long *partials) {
    const int g = blockIdx.x * kDThreads + threadIdx.x;
    if (g >= d.in.N) return;
    int c;
    const unsigned long long k0 = adc_slot(code, partials, (size_t)g, c);
    if (c != 3) return;
    GaussPre G;
    gauss_pre(d.in, g, G);
    const size_t N = (size_t)d.in.N, cap = d.cap;
    for (int r = 0; r < 2; ++r) {
        if (k0 + r >= d.cap) break;
        const uint32_t k = (uint32_t)(k0 + r);
        const float e0 = normals[(size_t)(r * 3 + 0) * N + g], e1 = normals[(size_t)(r * 3 + 1) * N + g];
        const float e2 = normals[(size_t)(r * 3 + 2) * N + g];
        const float mu[3] = {G.mx, G.my, G.mz};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            d.om[j * cap + k] = mu[j] + (G.M[j][0] * e0 + G.M[j][1] * e1 + G.M[j][2] * e2);
            d.ols[j * cap + k] = d.in.log_scales[j * N + g] - kSplitLog;
        }
    }
}

// ---------------------------------------------------------------- MCMC relocation
// FP32 exp and sigmoid from correctly rounded operations only (no fused
// multiply-add, no approximate instructions): x = n ln2 + f with ln 2 split
// into an exactly representable high part and a low part, e^f by its
// degree-7 Taylor polynomial, then 2^n by exponent scaling.
__device__ __forceinline__ float exp_rn(float x) {
    // FP32 constants, written with the digits that round to them exactly
    const float ln2_hi = 0.693145751953125f, ln2_lo = 1.428606765330187e-06f;
    const float log2e = 1.4426950216293335f;
    x = fminf(fmaxf(x, -87.f), 88.f);
    const float n = rintf(__fmul_rn(x, log2e));
    const float f = __fsub_rn(__fsub_rn(x, __fmul_rn(n, ln2_hi)), __fmul_rn(n, ln2_lo));
    const float c[8] = {1.f, 1.f, 0.5f, 0.16666667f, 0.041666668f, 0.008333334f, 0.0013888889f, 0.0001984127f};
    float p = c[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) p = __fadd_rn(__fmul_rn(p, f), c[k]);
    return ldexpf(p, (int)n);
}

__device__ __forceinline__ float sigmoid_rn(float l) { return __fdiv_rn(1.f, __fadd_rn(1.f, exp_rn(-l))); }

// The sampling weights floor(o 2^24) of the live Gaussians (0 for dead
// ones) and the dead flags, formed in the first pass of the weights'
// inclusive scan (block-local prefix to w, block totals to partials); also
// clears the draw counters.
__global__ void __launch_bounds__(kDScanThreads) mcmc_weight_scan_kernel(const GaussianPtrs gp, float min_opacity,
                                                                     unsigned long long *w, uint32_t *dead,
                                                                     uint32_t *drawn, unsigned long long *partials) {
    __shared__ unsigned long long s_warp[kDScanThreads / 32];
    const int lane = threadIdx.x & 31;
    const size_t base = rounds_base(), N = (size_t)gp.N;
    unsigned long long v[kDScanRounds];
#pragma unroll
    for (int k = 0; k < kDScanRounds; ++k) {
        const size_t g = base + (size_t)k * 32 + lane;
        v[k] = 0ull;
        if (g < N) {
            const float o = sigmoid_rn(gp.opacity_logits[g]);
            const bool d = o <= min_opacity;
            dead[g] = d ? 1u : 0u;
            drawn[g] = 0u;
            v[k] = d ? 0ull : (unsigned long long)(o * 16777216.f);   // exact scaling; truncation = floor
        }
    }
    const unsigned long long total = block_rounds_scan(v, true, s_warp);
#pragma unroll
    for (int k = 0; k < kDScanRounds; ++k) {
        const size_t g = base + (size_t)k * 32 + lane;
        if (g < N) w[g] = v[k];
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// Each dead slot draws its source: the first Gaussian whose inclusive weight
// sum exceeds floor(r W / 2^32).  src[g] = source, or 0xffffffff.
__global__ void __launch_bounds__(kDThreads) mcmc_draw_kernel(int N, const uint32_t *draws,
                                                              const unsigned long long *cum,
                                                              const unsigned long long *W_total,
                                                              const uint32_t *dead, uint32_t *src, uint32_t *drawn,
                                                              int *relocated) {
    const int g = blockIdx.x * kDThreads + threadIdx.x;
    if (g >= N) return;
    const unsigned long long W = *W_total;
    uint32_t s = 0xffffffffu;
    if (dead[g] && W > 0) {
        const unsigned long long r = draws[g];
        const unsigned long long lo = r * W, hi = __umul64hi(r, W);
        const unsigned long long t = (hi << 32) | (lo >> 32);   // floor(r W / 2^32), r W < 2^77
        int a = 0, b = N;   // first index with cum > t: in [a, b)
        while (a < b) {
            const int m = (a + b) >> 1;
            if (cum[m] > t)
                b = m;
            else
                a = m + 1;
        }
        s = (uint32_t)a;
        atomicAdd(&drawn[s], 1u);
        atomicAdd(relocated, 1);
    }
    src[g] = s;
}

// Opacity logit and log-scale shift of a source drawn n times.
__device__ __forceinline__ void relocation_rule(float logit, uint32_t n, float min_opacity, float &new_logit,
                                                float &dls) {
    const int k = min((int)n + 1, kMaxCopies);
    const double o = 1.0 / (1.0 + exp(-(double)logit));
    double on = 1.0 - pow(1.0 - o, 1.0 / (double)k);
    on = fmin(fmax(on, (double)min_opacity), 1.0 - 1.0 / 8388608.0);
    double den = 0.0;
    for (int i = 1; i <= k; ++i) {
        double binom = 1.0, pw = on;   // C(i-1, j), on^(j+1)
        for (int j = 0; j < i; ++j) {
            den += ((j & 1) ? -1.0 : 1.0) * binom * pw / sqrt((double)(j + 1));
            binom = binom * (double)(i - 1 - j) / (double)(j + 1);
            pw *= on;
        }
    }
    new_logit = (float)log(on / (1.0 - on));
    dls = (float)log(o / den);
}

__global__ void __launch_bounds__(kDThreads) mcmc_write_kernel(const DensityPtrs d, float min_opacity,
                                                               const uint32_t *src, const uint32_t *drawn) {
    const int g = blockIdx.x * kDThreads + threadIdx.x;
    if (g >= d.in.N) return;
    const uint32_t s = src[g] != 0xffffffffu ? src[g] : (uint32_t)g;
    copy_gaussian(d, (int)s, (uint32_t)g);
    const uint32_t n = drawn[s];
    if (n == 0) return;
    float new_logit, dls;
    relocation_rule(d.in.opacity_logits[s], n, min_opacity, new_logit, dls);
    const size_t N = (size_t)d.in.N, cap = d.cap;
    d.oo[g] = new_logit;
#pragma unroll
    for (int j = 0; j < 3; ++j) d.ols[j * cap + g] = d.in.log_scales[j * N + s] + dls;
}

// ---------------------------------------------------------------- MCMC noise
__global__ void __launch_bounds__(kDThreads) mcmc_noise_kernel(const GaussianPtrs gp, const float *eta, float scale,
                                                               float *means_out) {
    const int g = blockIdx.x * kDThreads + threadIdx.x;
    if (g >= gp.N) return;
    GaussPre G;
    gauss_pre(gp, g, G);
    const size_t N = (size_t)gp.N;
    const float o = 1.f / (1.f + expf(-gp.opacity_logits[g]));
    const float gate = 1.f / (1.f + expf(kNoiseK * (o - kNoiseT)));
    const float e[3] = {eta[g], eta[N + g], eta[2 * N + g]};
    // Sigma eta = M (M^T eta), M = R diag(s)
    float t[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) t[j] = G.M[0][j] * e[0] + G.M[1][j] * e[1] + G.M[2][j] * e[2];
    const float mu[3] = {G.mx, G.my, G.mz};
#pragma unroll
    for (int j = 0; j < 3; ++j)
        means_out[j * N + g] = mu[j] + scale * gate * (G.M[j][0] * t[0] + G.M[j][1] * t[1] + G.M[j][2] * t[2]);
}

unsigned blocks_of(size_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

size_t density_workspace_bytes(int N) {
    const size_t n = (size_t)(N > 0 ? N : 1), nb = (n + kDChunk - 1) / kDChunk;
    auto a = [](size_t b) { return (b + 255) & ~size_t(255); };
    return a(8 * n) + a(4 * n) + a(4 * n) + a(4 * n) + a(8 * nb) + a(64);
}

namespace {
struct DensityWs {
    unsigned long long *vals;
    uint32_t *dead, *src, *drawn;
    unsigned long long *partials, *total;
};

DensityWs density_ws(void *base, int N) {
    const size_t n = (size_t)(N > 0 ? N : 1), nb = (n + kDChunk - 1) / kDChunk;
    auto a = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(base);
    DensityWs w;
    w.vals = reinterpret_cast<unsigned long long *>(p);
    p += a(8 * n);
    w.dead = reinterpret_cast<uint32_t *>(p);
    p += a(4 * n);
    w.src = reinterpret_cast<uint32_t *>(p);
    p += a(4 * n);
    w.drawn = reinterpret_cast<uint32_t *>(p);
    p += a(4 * n);
    w.partials = reinterpret_cast<unsigned long long *>(p);
    p += a(8 * nb);
    w.total = reinterpret_cast<unsigned long long *>(p);
    return w;
}

DensityPtrs density_ptrs(const GaussianPtrs &gp, const gsr_gaussians_out &out) {
    DensityPtrs d;
    d.in = gp;
    d.C = 3 * (gp.sh_degree + 1) * (gp.sh_degree + 1);
    d.om = out.means;
    d.ols = out.log_scales;
    d.oq = out.quats;
    d.oo = out.opacity_logits;
    d.osh = out.sh;
    d.cap = (uint32_t)out.N;
    return d;
}
}  // namespace

cudaError_t launch_densify_adc(const GaussianPtrs &gp, const float *grad, const float *count, const float *radius,
                               const float *normals, const gsr_adc_params &prm, const gsr_gaussians_out &out,
                               int *out_count, void *ws, cudaStream_t st) {
    const DensityWs w = density_ws(ws, gp.N);
    AdcParams p;
    p.grad_threshold = prm.grad_threshold;
    p.max_screen_radius = prm.max_screen_radius;
    p.screen_on = prm.max_screen_radius > 0.f;
    p.log_split = std::log((double)prm.split_scale);
    const double m = (double)prm.min_opacity;
    p.logit_min = std::log(m / (1.0 - m));
    p.log_world = prm.max_world_scale > 0.f ? std::log((double)prm.max_world_scale) : HUGE_VAL;
    auto below = [](double t) {   // the largest float <= t
        float f = (float)t;
        if ((double)f > t) f = std::nextafter(f, -HUGE_VALF);
        return f;
    };
    auto above = [](double t) {   // the smallest float >= t
        float f = (float)t;
        if ((double)f < t) f = std::nextafter(f, HUGE_VALF);
        return f;
    };
    p.log_split_f = below(p.log_split);
    p.logit_min_f = above(p.logit_min);
    p.log_world_f = below(p.log_world);
    if (gp.N == 0) return cudaMemsetAsync(out_count, 0, sizeof(int), st);
    // the decision codes use the first half of the scan buffer
    uint32_t *code = reinterpret_cast<uint32_t *>(w.vals);
    const unsigned nc = blocks_of((size_t)gp.N, kDChunk), nb = blocks_of((size_t)gp.N, kDThreads);
    adc_decide_scan_kernel<<<nc, kDScanThreads, 0, st>>>(gp, grad, count, radius, p, code, w.partials);
    scan_partials_kernel<<<1, 1024, 0, st>>>(w.partials, nc, w.total);
    const DensityPtrs d = density_ptrs(gp, out);
    adc_write_kernel<<<nb, kDThreads, 0, st>>>(d, code, w.partials, w.total, out_count);
    adc_split_kernel<<<nb, kDThreads, 0, st>>>(d, normals, code, w.partials);
    return cudaGetLastError();
}

cudaError_t launch_mcmc_relocate(const GaussianPtrs &gp, const uint32_t *draws, float min_opacity,
                                 const gsr_gaussians_out &out, int *relocated, void *ws, cudaStream_t st) {
    const DensityWs w = density_ws(ws, gp.N);
    cudaError_t e = cudaMemsetAsync(relocated, 0, sizeof(int), st);
    if (e != cudaSuccess || gp.N == 0) return e;
    const unsigned nb = blocks_of((size_t)gp.N, kDThreads), nc = blocks_of((size_t)gp.N, kDChunk);
    mcmc_weight_scan_kernel<<<nc, kDScanThreads, 0, st>>>(gp, min_opacity, w.vals, w.dead, w.drawn, w.partials);
    scan_partials_kernel<<<1, 1024, 0, st>>>(w.partials, nc, w.total);
    scan_add_kernel<<<nb, kDThreads, 0, st>>>(w.vals, (size_t)gp.N, w.partials);
    mcmc_draw_kernel<<<nb, kDThreads, 0, st>>>(gp.N, draws, w.vals, w.total, w.dead, w.src, w.drawn, relocated);
    mcmc_write_kernel<<<nb, kDThreads, 0, st>>>(density_ptrs(gp, out), min_opacity, w.src, w.drawn);
    return cudaGetLastError();
}

cudaError_t launch_mcmc_noise(const GaussianPtrs &gp, const float *eta, float scale, float *means_out,
                              cudaStream_t st) {
    if (gp.N == 0) return cudaSuccess;
    mcmc_noise_kernel<<<blocks_of((size_t)gp.N, kDThreads), kDThreads, 0, st>>>(gp, eta, scale, means_out);
    return cudaGetLastError();
}

}  // namespace gsr
