// binning.cu -- tile binning of the projected Gaussians: exclusive scan of the
// per-(view, Gaussian) tile counts, key duplication (key = global tile id in
// the high 32 bits, FP32 depth bits in the low 32), a hand-written onesweep
// LSD radix sort of the (key, Gaussian id) pairs, and the [start, end) range
// of every tile in the sorted list.  All sizes the host cannot know (the key
// count) are read on the device, so the sequence needs no host sync and can
// be captured in a CUDA graph.
#include "kernels.cuh"
#include "spans.cuh"

namespace gsr {

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;

__device__ __forceinline__ uint32_t key_count(const Ws &ws) { return min(ws.hdr->keys, ws.cap); }

// Block-wide exclusive scan of one value per thread (blockDim.x = 32 * W).
template <typename T, int THREADS>
__device__ __forceinline__ T block_exclusive_scan(T x, T *s_warp, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int W = THREADS / 32;
        T w = lane < W ? s_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < W) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const T before = warp > 0 ? s_warp[warp - 1] : T(0);
    total = s_warp[THREADS / 32 - 1];
    __syncthreads();
    return before + incl - x;
}

// ------------------------------------------------------------------ scan
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const Ws ws) {
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const size_t base = (size_t)blockIdx.x * kScanChunk;
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const size_t i = base + (size_t)k * kScanThreads + threadIdx.x;
        if (i < ws.VN) sum += ws.counts[i];
    }
    unsigned long long total;
    block_exclusive_scan<unsigned long long, kScanThreads>(sum, s_warp, total);
    if (threadIdx.x == 0) ws.scan_partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_partials_kernel(const Ws ws) {
    __shared__ unsigned long long s_warp[32];
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < ws.scan_blocks; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long x = i < ws.scan_blocks ? ws.scan_partials[i] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_exclusive_scan<unsigned long long, 1024>(x, s_warp, total);
        if (i < ws.scan_blocks) ws.scan_partials[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        ws.hdr->keys = carry > 0xffffffffull ? 0xffffffffu : (uint32_t)carry;
        if (carry > ws.cap) set_status(ws.hdr, GSR_ECAPACITY);
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const Ws ws) {
    __shared__ uint32_t s_val[kScanChunk];
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const size_t base = (size_t)blockIdx.x * kScanChunk;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int j = k * kScanThreads + threadIdx.x;
        const size_t i = base + j;
        s_val[j] = i < ws.VN ? ws.counts[i] : 0u;
    }
    __syncthreads();
    unsigned long long run = 0;
    uint32_t mine[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        mine[k] = s_val[threadIdx.x * kScanItems + k];
        run += mine[k];
    }
    unsigned long long total;
    unsigned long long ex = block_exclusive_scan<unsigned long long, kScanThreads>(run, s_warp, total);
    ex += ws.scan_partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        s_val[threadIdx.x * kScanItems + k] = ex > 0xffffffffull ? 0xffffffffu : (uint32_t)ex;
        ex += mine[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int j = k * kScanThreads + threadIdx.x;
        const size_t i = base + j;
        if (i < ws.VN) ws.offsets[i] = s_val[j];
    }
}

// ------------------------------------------------------------------ duplicate
// A block takes 256 consecutive (view, Gaussian) pairs, compacts those with
// keys (most pairs have none) and has full warps emit them along the exact
// tile spans.
__global__ void __launch_bounds__(256) duplicate_kernel(const __grid_constant__ ViewTable vt, const Ws ws) {
    __shared__ int s_wcount[8];
    __shared__ uint32_t s_pair[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t i0 = (size_t)blockIdx.x * 256 + threadIdx.x;
    const bool has = i0 < ws.VN && ws.counts[i0] != 0u;
    const unsigned ball = __ballot_sync(0xffffffffu, has);
    if (lane == 0) s_wcount[warp] = __popc(ball);
    __syncthreads();
    int off = 0, n = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int c = s_wcount[w];
        off += w < warp ? c : 0;
        n += c;
    }
    if (has) s_pair[off + __popc(ball & lanemask_lt())] = threadIdx.x;
    __syncthreads();
    if ((int)threadIdx.x >= n) return;
    const size_t i = (size_t)blockIdx.x * 256 + s_pair[threadIdx.x];
    const uint32_t cnt = ws.counts[i];
    const uint32_t off_k = ws.offsets[i];
    const uint32_t v = (uint32_t)(i / ws.N), g = (uint32_t)(i - (size_t)v * ws.N);
    const ViewParams &vp = vt.v[v];
    const float4 r0 = ws.rec0[i], r1 = ws.rec1[i], r3 = ws.rec3[i];
    const unsigned long long zbits = __float_as_uint(ws.rec2[i].w);
    unsigned long long *keys = ws.keys[0];
    uint32_t *vals = ws.vals[0];
    const uint32_t cap = ws.cap;
    uint32_t k = off_k;
    if (ws.surfels) {   // surfels: every tile of the pixel bounds
        const float4 r = ws.rec5[i];
        const int TS = vt.tile;
        const int px0 = (int)fmaxf(ceilf(r.x), 0.f), px1 = (int)fminf(floorf(r.z), (float)(vp.W - 1));
        const int py0 = (int)fmaxf(ceilf(r.y), 0.f), py1 = (int)fminf(floorf(r.w), (float)(vp.H - 1));
        uint32_t emitted = 0;
        for (int ty = py0 / TS; ty <= py1 / TS; ++ty) {
            const uint32_t row = vp.tile_offset + (uint32_t)ty * vp.tiles_x;
            for (int tx = px0 / TS; tx <= px1 / TS; ++tx, ++k, ++emitted)
                if (k < cap) {
                    keys[k] = ((unsigned long long)(row + tx) << 32) | zbits;
                    vals[k] = g;
                }
        }
        if (emitted != cnt) set_status(ws.hdr, GSR_EINTERNAL);
        return;
    }
    const uint32_t emitted = visit_tile_spans(r0.x, r0.y, r3.y, r3.z, r3.w, r1.x, r1.w, vp.W, vp.H, vt.tile,
                                              [&](int ty, int tx0, int tx1) {
                                                  const uint32_t row = vp.tile_offset + (uint32_t)ty * vp.tiles_x;
                                                  for (int tx = tx0; tx <= tx1; ++tx, ++k) {
                                                      if (k < cap) {
                                                          keys[k] = ((unsigned long long)(row + tx) << 32) | zbits;
                                                          vals[k] = g;
                                                      }
                                                  }
                                              });
    if (emitted != cnt) set_status(ws.hdr, GSR_EINTERNAL);
}

// ------------------------------------------------------------------ sort
// One read of the keys gives the digit histogram of every pass; it also
// clears the look-back flags of the first pass and the tile counters.
__global__ void __launch_bounds__(256) sort_hist_kernel(const Ws ws) {
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    const uint32_t n = key_count(ws);
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t i = tid; i < (size_t)ntiles * kRadix; i += stride) ws.lookback[i] = 0u;
    if (tid < kMaxPasses) ws.hdr->sort_counter[tid] = 0u;
    __syncthreads();
    const unsigned long long *keys = ws.keys[0];
    constexpr int U = 4;   // keys loaded ahead of their shared-memory atomics
    for (size_t i = tid; i < n; i += U * stride) {
        unsigned long long k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) k[u] = i + u * stride < n ? keys[i + u * stride] : 0ull;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i + u * stride < n)
                for (int p = 0; p < ws.passes; ++p) atomicAdd(&s_hist[p][(k[u] >> (8 * p)) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ws.passes * kRadix; i += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&ws.hist[i], c);
    }
}

// One round of a digit's decoupled look-back over tiles hi-1, hi-2, ...,
// hi-W (col: the digit's column of the [tile][digit] flags): adds the
// published counts down to the first inclusive flag or to the first flag not
// yet published, and returns the new hi.  Below tile 0 reads as an
// inclusive zero.
constexpr int kLookNear = 16;
constexpr int kSortBlocksPerSM = 3;   // resident onesweep CTAs per SM (registers and shared memory allow 3)
constexpr int kLookAll = 0, kLookFound = 1, kLookWaiting = 2;
template <int W>
__device__ __forceinline__ int lookback_round(const uint32_t *col, int hi, uint32_t &prefix, int &state) {
    uint32_t f[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const int u = hi - 1 - q;
        f[q] = u >= 0 ? ld_relaxed_gpu(col + (size_t)u * kRadix) : kFlagInc;
    }
    state = kLookAll;
#pragma unroll
    for (int q = 0; q < W; ++q) {
        if (state != kLookAll) continue;
        const uint32_t flag = f[q] & ~kCountMask;
        if (flag == 0u) {
            state = kLookWaiting;
            continue;
        }
        prefix += f[q] & kCountMask;
        --hi;
        if (flag == kFlagInc) state = kLookFound;
    }
    return hi;
}

// One stable LSD pass over 8 bits: tiles of kSortTile keys are taken in order
// from an atomic counter; each tile ranks its keys per digit (warp match +
// per-warp counters), publishes its digit counts, places its keys in shared
// memory in digit order, resolves its global digit offsets by a bounded
// decoupled look-back over earlier tiles, then writes them out, so that
// global writes are runs of equal digits.  One thread per digit walks the
// look-back; a round first reads the 16 nearest predecessors (while they are
// still being ranked, polling them is cheap) and, once those are all
// published, kLookBatch at a time, so that one round trip to L2 advances the
// walk by up to kLookBatch tiles.
__global__ void __launch_bounds__(kSortThreads, kSortBlocksPerSM) onesweep_kernel(const Ws ws, int pass) {
    constexpr int WARPS = kSortThreads / 32;
    __shared__ uint32_t s_whist[WARPS][kRadix];
    __shared__ uint32_t s_hist_ex[kRadix];
    __shared__ uint32_t s_tile_ex[kRadix];
    __shared__ uint32_t s_glob[kRadix];
    __shared__ uint32_t s_scan[WARPS];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, d_own = threadIdx.x;
    const uint32_t n = key_count(ws);
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int shift = 8 * pass;
    const unsigned long long *keys_in = ws.keys[pass & 1];
    const uint32_t *vals_in = ws.vals[pass & 1];
    unsigned long long *keys_out = ws.keys[(pass + 1) & 1];
    uint32_t *vals_out = ws.vals[(pass + 1) & 1];
    // this thread's digit column of the flags of this pass and of the next ([tile][digit])
    uint32_t *col = ws.lookback + (size_t)(pass & 1) * ws.lb_tiles * kRadix + d_own;
    uint32_t *col_next = ws.lookback + (size_t)((pass + 1) & 1) * ws.lb_tiles * kRadix + d_own;

    {   // global exclusive digit offsets of this pass
        uint32_t total;
        s_hist_ex[d_own] = block_exclusive_scan<uint32_t, kSortThreads>(ws.hist[pass * kRadix + d_own], s_scan, total);
    }

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ws.hdr->sort_counter[pass], 1u);
        for (int d = lane; d < kRadix; d += 32) s_whist[warp][d] = 0u;
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= ntiles) break;
        col_next[(size_t)t * kRadix] = 0u;   // the next pass's flag of this tile (its array is idle now)

        const uint32_t base = t * kSortTile + warp * (kSortItems * 32);
        uint32_t rank[kSortItems];
        unsigned long long k[kSortItems];
        uint32_t val[kSortItems];
        // all loads first: the warp barriers of the ranking below would
        // otherwise serialise them
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const uint32_t idx = base + it * 32 + lane;
            k[it] = idx < n ? keys_in[idx] : 0ull;
            val[it] = idx < n ? vals_in[idx] : 0u;
        }
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const bool valid = base + it * 32 + lane < n;
            const uint32_t d = valid ? (uint32_t)((k[it] >> shift) & 0xff) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (valid && lane == leader) {
                old = s_whist[warp][d];
                s_whist[warp][d] = old + __popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[it] = old + __popc(peers & lanemask_lt());
            __syncwarp();
        }
        __syncthreads();

        // per digit: exclusive offsets across warps and the tile's count
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = s_whist[w][d_own];
            s_whist[w][d_own] = cnt;
            cnt += c;
        }
        const bool stalled = t == 0 && pass == 0 && (ws.test_flags & GSR_TEST_STALL_SORT);
        if (!stalled) st_relaxed_gpu(col + (size_t)t * kRadix, (t == 0 ? kFlagInc : kFlagAgg) | cnt);
        uint32_t tile_total;
        const uint32_t tile_ex = block_exclusive_scan<uint32_t, kSortThreads>(cnt, s_scan, tile_total);
        s_tile_ex[d_own] = tile_ex;
        __syncthreads();
        // the tile in digit order in shared memory (frees the registers
        // before the look-back)
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const uint32_t idx = base + it * 32 + lane;
            if (idx < n) {
                const uint32_t d = (uint32_t)((k[it] >> shift) & 0xff);
                const uint32_t local = s_tile_ex[d] + s_whist[warp][d] + rank[it];
                s_keys[local] = k[it];
                s_vals[local] = val[it];
            }
        }

        // bounded decoupled look-back: sums the counts of earlier tiles down
        // to the first inclusive flag; a flag not yet published means
        // another round trip
        uint32_t prefix = 0;
        if (t > 0) {
            int hi = (int)t;   // tiles [0, hi) not yet summed
            uint32_t spins = 0;
            bool wide = false;
            for (;;) {
                int state;
                hi = wide ? lookback_round<kLookBatch>(col, hi, prefix, state)
                          : lookback_round<kLookNear>(col, hi, prefix, state);
                if (state == kLookFound) break;
                wide = state == kLookAll;
                if (state == kLookWaiting && ++spins > ws.spin_limit) {  // waited on a flag that never came
                    set_status(ws.hdr, GSR_ETIMEOUT);
                    break;
                }
            }
            st_relaxed_gpu(col + (size_t)t * kRadix, kFlagInc | ((prefix + cnt) & kCountMask));
        }
        s_glob[d_own] = s_hist_ex[d_own] + prefix - tile_ex;
        __syncthreads();

        const uint32_t tile_n = min((uint32_t)kSortTile, n - t * kSortTile);
        for (uint32_t j = threadIdx.x; j < tile_n; j += kSortThreads) {
            const unsigned long long key = s_keys[j];
            const uint32_t d = (uint32_t)((key >> shift) & 0xff);
            const uint32_t o = s_glob[d] + j;
            if (o < n) {
                keys_out[o] = key;
                vals_out[o] = s_vals[j];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ ranges
__global__ void __launch_bounds__(256) ranges_kernel(const Ws ws, const unsigned long long *keys) {
    const uint32_t n = key_count(ws);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t tile = (uint32_t)(keys[i] >> 32);
        if (tile >= ws.total_tiles) {  // only after a reported device error
            set_status(ws.hdr, GSR_EINTERNAL);
            continue;
        }
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ws.ranges[tile].x = (uint32_t)i;
        if (i + 1 == n || (uint32_t)(keys[i + 1] >> 32) != tile) ws.ranges[tile].y = (uint32_t)(i + 1);
    }
}

}  // namespace

cudaError_t launch_scan_duplicate(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (ws.VN == 0) return cudaSuccess;
    scan_reduce_kernel<<<ws.scan_blocks, kScanThreads, 0, st>>>(ws);
    scan_partials_kernel<<<1, 1024, 0, st>>>(ws);
    scan_down_kernel<<<ws.scan_blocks, kScanThreads, 0, st>>>(ws);
    cudaError_t e = cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * kMaxPasses * kRadix, st);
    if (e != cudaSuccess) return e;
    duplicate_kernel<<<(unsigned)((ws.VN + 255) / 256), 256, 0, st>>>(vt, ws);
    return cudaGetLastError();
}

cudaError_t launch_sort(const Ws &ws, int sm_count, cudaStream_t st) {
    if (ws.VN == 0) return cudaSuccess;
    sort_hist_kernel<<<sm_count * 4, 256, 0, st>>>(ws);
    for (int p = 0; p < ws.passes; ++p) onesweep_kernel<<<sm_count * kSortBlocksPerSM, kSortThreads, 0, st>>>(ws, p);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const Ws &ws, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * ws.total_tiles, st);
    if (e != cudaSuccess || ws.VN == 0) return e;
    ranges_kernel<<<sm_count * 4, 256, 0, st>>>(ws, ws.keys[ws.passes & 1]);
    return cudaGetLastError();
}

}  // namespace gsr
