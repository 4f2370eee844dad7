// binning.cu -- tile binning of the projected Gaussians: every (view,
// Gaussian) pair becomes one key per screen tile it touches, the keys are put
// in (global tile, FP32 depth, Gaussian id) order, and every tile gets its
// [start, end) range of the sorted list.  Two strategies, with the same
// result:
//
// radix: an exclusive scan of the per-pair tile counts places each pair's
//   keys, a duplication kernel emits them as (tile << 32 | depth bits) with
//   the Gaussian id as value, one stable hand-written onesweep LSD radix sort
//   runs over all used bits (8 per pass; equal depths keep the pair order,
//   i.e. the id order), and a boundary pass gives the ranges.
// per-tile (default): the preprocess emits u32 tile keys with (depth bits <<
//   32 | id) words as values, grouped here by tile, after which each tile's
//   words -- unique, since a Gaussian meets a tile once -- are sorted in
//   registers (a warp) or shared memory (a block), which orders them by depth
//   and then id.  Grouping: with up to 32,768 tiles a count kernel counts
//   each block's slice of the keys per tile in shared memory and adds them
//   with one atomic per (block, tile), its last block scans the counts into
//   the ranges, and a scatter kernel places each key in its tile's slots
//   (bucket_binning); beyond, the onesweep sort runs over the tile bits only
//   and the boundary pass gives the ranges.
//
// All sizes the host cannot know (the key count) are read on the device, so
// either sequence needs no host sync and can be captured in a CUDA graph.
#include <algorithm>
#include <mutex>

#include "kernels.cuh"
#include "spans.cuh"

namespace gsr {

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;

__device__ __forceinline__ uint32_t key_count(const Ws &ws) {
    return (uint32_t)min(ws.hdr->keys, (unsigned long long)ws.cap);
}

constexpr unsigned long long kNoKey = ~0ull;   // padding, after every real (depth, id) word

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
        ws.hdr->keys = carry;
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
    const bool by_tile = ws.bin_tile != 0;
    const uint32_t off_k = ws.offsets[i];
    const uint32_t v = (uint32_t)(i / ws.N), g = (uint32_t)(i - (size_t)v * ws.N);
    const ViewParams &vp = vt.v[v];
    const float4 *rec = ws.rec + 4 * i;
    const float4 r0 = rec[0], r1 = rec[1], r3 = rec[3];
    const unsigned long long zbits = __float_as_uint(rec[2].w);
    unsigned long long *keys = ws.keys[0];
    uint32_t *vals = ws.vals[0];
    const uint32_t cap = ws.cap;
    uint32_t k = off_k;
    // the pair's next key: tile t
    auto emit = [&](uint32_t t) {
        if (k < cap) {
            if (by_tile) {
                vals[k] = t;
                keys[k] = (zbits << 32) | g;
            } else {
                keys[k] = ((unsigned long long)t << 32) | zbits;
                vals[k] = g;
            }
        }
        ++k;
    };
    if (ws.surfels) {   // surfels: every tile of the pixel bounds
        const float4 r = ws.rec5[i];
        const int TS = vt.tile;
        const int px0 = (int)fmaxf(ceilf(r.x), 0.f), px1 = (int)fminf(floorf(r.z), (float)(vp.W - 1));
        const int py0 = (int)fmaxf(ceilf(r.y), 0.f), py1 = (int)fminf(floorf(r.w), (float)(vp.H - 1));
        uint32_t emitted = 0;
        for (int ty = py0 / TS; ty <= py1 / TS; ++ty) {
            const uint32_t row = vp.tile_offset + (uint32_t)ty * vp.tiles_x;
            for (int tx = px0 / TS; tx <= px1 / TS; ++tx, ++emitted) emit(row + tx);
        }
        if (emitted != cnt) set_status(ws.hdr, GSR_EINTERNAL);
        return;
    }
    const uint32_t emitted = visit_tile_spans(r0.x, r0.y, r3.y, r3.z, r3.w, r1.x, r1.w, vp.W, vp.H, vt.tile,
                                              [&](int ty, int tx0, int tx1) {
                                                  const uint32_t row = vp.tile_offset + (uint32_t)ty * vp.tiles_x;
                                                  for (int tx = tx0; tx <= tx1; ++tx) emit(row + tx);
                                              });
    if (emitted != cnt) set_status(ws.hdr, GSR_EINTERNAL);
}

// ------------------------------------------------------------------ sort
// Keys and values of the two strategies (radix: u64 (tile, depth) keys, u32
// ids; per-tile: u32 tile keys, u64 (depth, id) words), double-buffered.
template <typename K, typename V>
struct SortBufs {
    K *k[2];
    V *v[2];
};

template <typename K, typename V>
SortBufs<K, V> sort_bufs(const Ws &ws);
template <>
SortBufs<unsigned long long, uint32_t> sort_bufs(const Ws &ws) {
    return {{ws.keys[0], ws.keys[1]}, {ws.vals[0], ws.vals[1]}};
}
template <>
SortBufs<uint32_t, unsigned long long> sort_bufs(const Ws &ws) {
    return {{ws.vals[0], ws.vals[1]}, {ws.keys[0], ws.keys[1]}};
}

// One read of the keys gives the digit histogram of every pass; it also
// clears the look-back flags of the first pass and the tile counters.
template <typename K>
__global__ void __launch_bounds__(256) sort_hist_kernel(const Ws ws, const K *keys) {
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
    const uint32_t n = key_count(ws);
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t i = tid; i < (size_t)ntiles * kRadix; i += stride) ws.lookback[i] = 0u;
    if (tid < kMaxPasses) ws.hdr->sort_counter[tid] = 0u;
    __syncthreads();
    constexpr int U = 4;   // keys loaded ahead of their shared-memory atomics
    for (size_t i = tid; i < n; i += U * stride) {
        K k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) k[u] = i + u * stride < n ? keys[i + u * stride] : K(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i + u * stride < n)
                for (int p = 0; p < ws.passes; ++p) atomicAdd(&s_hist[p][(uint32_t)(k[u] >> (8 * p)) & 0xff], 1u);
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
template <typename K, typename V>
__global__ void __launch_bounds__(kSortThreads, kSortBlocksPerSM) onesweep_kernel(const Ws ws, int pass,
                                                                              const SortBufs<K, V> b) {
    constexpr int WARPS = kSortThreads / 32;
    __shared__ uint32_t s_whist[WARPS][kRadix];
    __shared__ uint32_t s_hist_ex[kRadix];
    __shared__ uint32_t s_tile_ex[kRadix];
    __shared__ uint32_t s_glob[kRadix];
    __shared__ uint32_t s_scan[WARPS];
    __shared__ uint32_t s_tile;
    __shared__ K s_keys[kSortTile];
    __shared__ V s_vals[kSortTile];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, d_own = threadIdx.x;
    const uint32_t n = key_count(ws);
    const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int shift = 8 * pass;
    const K *keys_in = b.k[pass & 1];
    const V *vals_in = b.v[pass & 1];
    K *keys_out = b.k[(pass + 1) & 1];
    V *vals_out = b.v[(pass + 1) & 1];
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
        K k[kSortItems];
        V val[kSortItems];
        // all loads first: the warp barriers of the ranking below would
        // otherwise serialise them
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const uint32_t idx = base + it * 32 + lane;
            k[it] = idx < n ? keys_in[idx] : K(0);
            val[it] = idx < n ? vals_in[idx] : V(0);
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
            const K key = s_keys[j];
            const uint32_t d = (uint32_t)((key >> shift) & 0xff);
            const uint32_t o = s_glob[d] + j;
            if (GSR_CHECK(ws.hdr, o < n)) {
                keys_out[o] = key;
                vals_out[o] = s_vals[j];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ ranges
__device__ __forceinline__ uint32_t tile_of(unsigned long long key) { return (uint32_t)(key >> 32); }
__device__ __forceinline__ uint32_t tile_of(uint32_t key) { return key; }

template <typename K>
__global__ void __launch_bounds__(256) ranges_kernel(const Ws ws, const K *keys) {
    const uint32_t n = key_count(ws);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t tile = tile_of(keys[i]);
        if (tile >= ws.total_tiles) {  // only after a reported device error
            set_status(ws.hdr, GSR_EINTERNAL);
            continue;
        }
        if (i == 0 || tile_of(keys[i - 1]) != tile) ws.ranges[tile].x = (uint32_t)i;
        if (i + 1 == n || tile_of(keys[i + 1]) != tile) ws.ranges[tile].y = (uint32_t)(i + 1);
    }
}

// ------------------------------------------------------------------ per-tile: bucket grouping
// A block per SM takes one contiguous slice of the unsorted keys and counts
// them per tile in shared memory (a counter per tile), so that a crowded tile
// costs one global atomic per block instead of one per key:
//   count:   tile_cursor[t] += the slice's keys of tile t; the last block to
//            finish scans the counts into the ranges [start, end) and sets
//            tile_cursor[t] = start;
//   scatter: the block reserves its keys' slots of every tile with one
//            atomic each, then places each key at the next reserved slot.
// The order within a tile depends on timing; the per-tile sort below makes
// it (depth, id).
constexpr int kBucketThreads = 1024;
constexpr int kBucketScanItems = kBucketMaxTiles / kBucketThreads;   // tiles per thread in the scan
constexpr int kBucketReserve = 8;                                     // reservations in flight per thread
constexpr int kBucketLoads = 4;                                       // keys loaded ahead per thread

__device__ __forceinline__ void bucket_slice(uint32_t n, uint32_t &b0, uint32_t &b1) {
    const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
    b0 = min(n, blockIdx.x * per);
    b1 = min(n, b0 + per);
}

// Counts of the slice's keys per tile in s_bins (zeroed here).
__device__ __forceinline__ void bucket_block_counts(const Ws &ws, uint32_t *s_bins, uint32_t b0, uint32_t b1) {
    const uint32_t T = ws.total_tiles;
    const uint32_t *tiles = ws.vals[0];
    for (uint32_t i = threadIdx.x; i < T; i += kBucketThreads) s_bins[i] = 0u;
    __syncthreads();
    for (uint32_t i0 = b0 + threadIdx.x; i0 < b1; i0 += kBucketThreads * kBucketLoads) {
        uint32_t t[kBucketLoads];
#pragma unroll
        for (int u = 0; u < kBucketLoads; ++u) {
            const uint32_t i = i0 + u * kBucketThreads;
            t[u] = i < b1 ? tiles[i] : T;
        }
#pragma unroll
        for (int u = 0; u < kBucketLoads; ++u) {
            if (t[u] < T)
                atomicAdd(s_bins + t[u], 1u);
            else if (i0 + u * kBucketThreads < b1)
                (void)GSR_CHECK(ws.hdr, false);
        }
    }
    __syncthreads();
}

// Tile t's word in the scan's staging buffer: one word of padding after
// every 32, so that a thread walking its kBucketScanItems consecutive tiles
// and a warp reading 32 consecutive ones both meet 32 different banks.
__device__ __forceinline__ uint32_t bucket_pad(uint32_t t) { return t + (t >> 5); }
constexpr size_t kBucketSmemMax = 4ull * (kBucketMaxTiles + kBucketMaxTiles / 32 + 1);
__host__ __device__ constexpr size_t bucket_smem(uint32_t T) { return 4ull * (T + T / 32 + 1); }

// Exclusive scan of the T <= kBucketMaxTiles tile counts (complete in
// tile_cursor) by one block, staged in s (bucket_smem(T) bytes): ranges and
// first slots.
__device__ __forceinline__ void bucket_scan(const Ws &ws, uint32_t *s, uint32_t *s_warp) {
    const uint32_t T = ws.total_tiles;
    {   // all of a thread's loads in flight at once
        uint32_t c[kBucketScanItems];
#pragma unroll
        for (int k = 0; k < kBucketScanItems; ++k) {
            const uint32_t i = threadIdx.x + k * kBucketThreads;
            c[k] = i < T ? __ldcg(ws.tile_cursor + i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kBucketScanItems; ++k) {
            const uint32_t i = threadIdx.x + k * kBucketThreads;
            if (i < T) s[bucket_pad(i)] = c[k];
        }
    }
    __syncthreads();
    const uint32_t t0 = threadIdx.x * kBucketScanItems;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kBucketScanItems; ++k) sum += t0 + k < T ? s[bucket_pad(t0 + k)] : 0u;
    uint32_t total;
    uint32_t at = block_exclusive_scan<uint32_t, kBucketThreads>(sum, s_warp, total);
#pragma unroll
    for (int k = 0; k < kBucketScanItems; ++k) {
        if (t0 + k < T) {
            const uint32_t c = s[bucket_pad(t0 + k)];
            s[bucket_pad(t0 + k)] = at;
            at += c;
        }
    }
    __syncthreads();
    // the counts add up to the key count, which is at most the capacity
    (void)GSR_CHECK(ws.hdr, total <= ws.cap);
    // the blends' launch order: tiles by decreasing key count, bucketed by
    // the count's bit length (so that the heaviest tiles start first and do
    // not trail the last wave)
    __shared__ uint32_t s_ob[2 * 33];
    for (uint32_t i = threadIdx.x; i < 2 * 33; i += kBucketThreads) s_ob[i] = 0u;
    __syncthreads();
    // (a warp's lanes of one bucket add to it with one shared-memory atomic:
    // 33 counters for thousands of tiles otherwise serialise)
    auto bits = [](uint32_t c) { return c == 0u ? 0u : 32u - (uint32_t)__clz(c); };
    const int lane = threadIdx.x & 31;
    for (uint32_t i0 = 0; i0 < T; i0 += kBucketThreads) {   // whole warps in every round
        const uint32_t i = i0 + threadIdx.x;
        uint32_t b = 33u;   // none
        if (i < T) {
            const uint32_t a = s[bucket_pad(i)], e = i + 1 < T ? s[bucket_pad(i + 1)] : total;
            ws.ranges[i] = make_uint2(min(a, ws.cap), min(e, ws.cap));
            ws.tile_cursor[i] = a;
            b = bits(e - a);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (b < 33u && lane == __ffs(peers) - 1) atomicAdd(s_ob + b, (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t at = 0;
        for (int b = 32; b >= 0; --b) {
            s_ob[33 + b] = at;
            at += s_ob[b];
        }
    }
    __syncthreads();
    for (uint32_t i0 = 0; i0 < T; i0 += kBucketThreads) {
        const uint32_t i = i0 + threadIdx.x;
        uint32_t b = 33u;
        if (i < T) {
            const uint32_t a = s[bucket_pad(i)], e = i + 1 < T ? s[bucket_pad(i + 1)] : total;
            b = bits(e - a);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0u;
        if (b < 33u && lane == leader) base = atomicAdd(s_ob + 33 + b, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b < 33u) ws.tile_order[base + __popc(peers & ((1u << lane) - 1u))] = i;
    }
}

__global__ void __launch_bounds__(kBucketThreads) bucket_count_kernel(const Ws ws) {
    extern __shared__ uint32_t s_bins[];
    __shared__ uint32_t s_warp[kBucketThreads / 32];
    __shared__ bool s_last;
    uint32_t b0, b1;
    bucket_slice(key_count(ws), b0, b1);
    bucket_block_counts(ws, s_bins, b0, b1);
    for (uint32_t t = threadIdx.x; t < ws.total_tiles; t += kBucketThreads)
        if (s_bins[t]) atomicAdd(ws.tile_cursor + t, s_bins[t]);
    // the last block to finish (its counts and every other block's are in
    // tile_cursor once each block has fenced them) scans
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ws.hdr->sort_counter[0], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bucket_scan(ws, s_bins, s_warp);
}

__global__ void __launch_bounds__(kBucketThreads) bucket_scatter_kernel(const Ws ws) {
    extern __shared__ uint32_t s_bins[];
    uint32_t b0, b1;
    bucket_slice(key_count(ws), b0, b1);
    bucket_block_counts(ws, s_bins, b0, b1);
    // the block's first slot of every tile it has keys of; kBucketReserve
    // atomics in flight per thread
    for (uint32_t t0 = threadIdx.x; t0 < ws.total_tiles; t0 += kBucketThreads * kBucketReserve) {
        uint32_t c[kBucketReserve], at[kBucketReserve];
#pragma unroll
        for (int k = 0; k < kBucketReserve; ++k) {
            const uint32_t t = t0 + k * kBucketThreads;
            c[k] = t < ws.total_tiles ? s_bins[t] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kBucketReserve; ++k)
            if (c[k]) at[k] = atomicAdd(ws.tile_cursor + t0 + k * kBucketThreads, c[k]);
#pragma unroll
        for (int k = 0; k < kBucketReserve; ++k)
            if (c[k]) s_bins[t0 + k * kBucketThreads] = at[k];
    }
    __syncthreads();
    const uint32_t *tiles = ws.vals[0];
    const unsigned long long *words = ws.keys[0];
    unsigned long long *out = ws.keys[1];
    for (uint32_t i0 = b0 + threadIdx.x; i0 < b1; i0 += kBucketThreads * kBucketLoads) {
        uint32_t t[kBucketLoads];
        unsigned long long w[kBucketLoads];
#pragma unroll
        for (int u = 0; u < kBucketLoads; ++u) {
            const uint32_t i = i0 + u * kBucketThreads;
            t[u] = i < b1 ? tiles[i] : ws.total_tiles;
            w[u] = i < b1 ? words[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kBucketLoads; ++u) {
            if (t[u] >= ws.total_tiles) continue;   // past the slice, or reported by the count
            const uint32_t pos = atomicAdd(s_bins + t[u], 1u);
            if (GSR_CHECK(ws.hdr, pos < ws.cap)) out[pos] = w[u];
        }
    }
}

// ------------------------------------------------------------------ per-tile: sort within each tile
// After the tile-key passes, tile t's (depth bits << 32 | id) words sit in
// words[start, end) in pair order; ascending words are the list order.  Up to
// kWarpSortMax words a warp sorts them in registers (a bitonic network over
// 32 E words, word e * 32 + lane in lane's x[e]); beyond, a block with
// kBlockSortCap words of shared memory sorts them by a radix sort of the
// depth bits, as runs merged pairwise through the free word buffer when there
// are more.  (Tiles of 513 to 2,048 words sorted by the block of the tile's
// warp held that block's other warps until they were done: window sort
// 0.0498 -> 0.0473 ms with those tiles in the big-tile kernel and blocks of
// two warps instead of eight.)  The ids go to ws.sorted.
constexpr int kWarpSortMax = 512;
constexpr int kTilesPerSortBlock = 2;   // one warp each
constexpr int kBlockSortCap = 16384;
constexpr int kBigSortThreads = 1024;
constexpr size_t kBigSortSmem = kBlockSortCap * sizeof(unsigned long long) + (kBigSortThreads / 32) * kRadix * 4;
constexpr int kMergeItems = 16;         // outputs per thread per merge-path step

__device__ __forceinline__ unsigned long long shfl_xor64(unsigned long long x, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[E], int lane) {
    constexpr int M = 32 * E;
#pragma unroll
    for (int k = 2; k <= M; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const bool up = ((e * 32 + lane) & k) == 0;   // this pair sorts ascending
                if (j >= 32) {   // partner word in the same lane
                    const int f = e ^ (j >> 5);
                    if (f > e) {
                        const unsigned long long a = x[e], b = x[f];
                        const bool sw = (a > b) == up;
                        x[e] = sw ? b : a;
                        x[f] = sw ? a : b;
                    }
                } else {         // partner word in lane ^ j
                    const unsigned long long y = shfl_xor64(x[e], j);
                    x[e] = ((lane & j) == 0) == up ? min(x[e], y) : max(x[e], y);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_tile(const unsigned long long *in, uint32_t *out, uint32_t n, int lane) {
    unsigned long long x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)(e * 32 + lane);
        x[e] = i < n ? in[i] : kNoKey;
    }
    warp_bitonic<E>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)(e * 32 + lane);
        if (i < n) out[i] = (uint32_t)x[e];
    }
}

// One stable 8-bit LSD pass (digit at bit shift) over the n <= THREADS *
// ITEMS words in s.  Ranking as in onesweep_kernel: warp w takes words
// [w 32 ITEMS, (w + 1) 32 ITEMS) in order, ranks them per digit with
// __match_any_sync and per-warp counters, and the (digit, warp) offsets come
// from one scan.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void block_radix_pass(unsigned long long *s, uint32_t n, int shift,
                                                 uint32_t (*s_whist)[kRadix], uint32_t *s_red) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t base = (uint32_t)warp * (ITEMS * 32);
    unsigned long long x[ITEMS];
    uint32_t rank[ITEMS];
    for (int d = lane; d < kRadix; d += 32) s_whist[warp][d] = 0u;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t idx = base + it * 32 + lane;
        x[it] = idx < n ? s[idx] : 0ull;
    }
    __syncthreads();   // all words are in registers before the scatter overwrites s
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const bool valid = base + it * 32 + lane < n;
        const uint32_t d = valid ? (uint32_t)(x[it] >> shift) & 0xffu : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = s_whist[warp][d];
            s_whist[warp][d] = old + __popc(peers);
        }
        rank[it] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lanemask_lt());
        __syncwarp();
    }
    __syncthreads();
    // offsets: digit-major, then warp order
    uint32_t cnt = 0;
    if (threadIdx.x < kRadix)
        for (int w = 0; w < WARPS; ++w) cnt += s_whist[w][threadIdx.x];
    uint32_t total;
    const uint32_t start = block_exclusive_scan<uint32_t, THREADS>(cnt, s_red, total);
    if (threadIdx.x < kRadix) {
        uint32_t c = start;
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t t = s_whist[w][threadIdx.x];
            s_whist[w][threadIdx.x] = c;
            c += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        if (base + it * 32 + lane < n) {
            const uint32_t d = (uint32_t)(x[it] >> shift) & 0xffu;
            s[s_whist[warp][d] + rank[it]] = x[it];
        }
    }
    __syncthreads();
}

// Sorts the n <= THREADS * ITEMS (depth bits << 32 | id) words in s, which
// arrive in any order, ascending.  Passes skip the digits that are the same
// in every word.  The depth digits leave only equal depths out of order (the
// words are unique); in big tiles some equal depths are all but certain, in
// short runs, so odd-even transposition rounds over neighbours of equal depth
// put them in id order (a depth-sorted array whose equal-depth neighbours are
// in order is sorted).  Runs too long for kTieRounds rounds (many Gaussians
// at one depth) get a full LSD sort from the id digits up.
constexpr int kTieRounds = 8;
template <int THREADS, int ITEMS>
__device__ __forceinline__ void block_radix_depth(unsigned long long *s, uint32_t n, uint32_t (*s_whist)[kRadix],
                                                  uint32_t *s_red) {
    static_assert(THREADS >= kRadix, "one thread per digit");
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long vor = 0ull, vand = ~0ull;
    for (uint32_t i = threadIdx.x; i < n; i += THREADS) {
        vor |= s[i];
        vand &= s[i];
    }
    uint32_t olo = __reduce_or_sync(0xffffffffu, (uint32_t)vor), ohi = __reduce_or_sync(0xffffffffu, (uint32_t)(vor >> 32));
    uint32_t alo = __reduce_and_sync(0xffffffffu, (uint32_t)vand), ahi = __reduce_and_sync(0xffffffffu, (uint32_t)(vand >> 32));
    if (lane == 0) {
        s_red[warp] = olo;
        s_red[WARPS + warp] = alo;
    }
    __syncthreads();
    uint32_t o = 0u, a = ~0u;
    for (int w = 0; w < WARPS; ++w) {
        o |= s_red[w];
        a &= s_red[WARPS + w];
    }
    const uint32_t differ_id = o ^ a;
    __syncthreads();
    if (lane == 0) {
        s_red[warp] = ohi;
        s_red[WARPS + warp] = ahi;
    }
    __syncthreads();
    o = 0u;
    a = ~0u;
    for (int w = 0; w < WARPS; ++w) {
        o |= s_red[w];
        a &= s_red[WARPS + w];
    }
    const uint32_t differ_depth = o ^ a;
    __syncthreads();
    // steps 0-3: depth digits; then, only with ties the transposition rounds
    // leave out of order, 4-7: id digits and 8-11: depth digits again (one
    // call site keeps the pass inlined once)
#pragma unroll 1
    for (int step = 0; step < 12; ++step) {
        if (step == 4) {
            bool sorted = false;
#pragma unroll 1
            for (int round = 0; round < kTieRounds && !sorted; ++round) {
                bool swapped = false;
#pragma unroll 1
                for (uint32_t phase = 0; phase < 2; ++phase) {
                    for (uint32_t i = 2 * threadIdx.x + phase; i + 1 < n; i += 2 * THREADS) {
                        const unsigned long long a = s[i], b = s[i + 1];
                        if ((a >> 32) == (b >> 32) && a > b) {
                            s[i] = b;
                            s[i + 1] = a;
                            swapped = true;
                        }
                    }
                    __syncthreads();
                }
                sorted = !__syncthreads_or(swapped);
            }
            if (sorted) break;
        }
        const bool depth = step < 4 || step >= 8;
        const int pass = step & 3;
        if ((((depth ? differ_depth : differ_id) >> (8 * pass)) & 0xffu) == 0u) continue;
        block_radix_pass<THREADS, ITEMS>(s, n, (depth ? 32 : 0) + 8 * pass, s_whist, s_red);
    }
}

// Sorts the m words of src (m <= THREADS * ITEMS) with the whole block and
// writes them to dst (words) or, if ids is set, their ids to ids.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void block_sort_run(const unsigned long long *src, uint32_t m, unsigned long long *s,
                                               uint32_t (*s_whist)[kRadix], uint32_t *s_red,
                                               unsigned long long *dst, uint32_t *ids) {
    for (uint32_t i = threadIdx.x; i < m; i += THREADS) s[i] = src[i];
    __syncthreads();
    block_radix_depth<THREADS, ITEMS>(s, m, s_whist, s_red);
    for (uint32_t i = threadIdx.x; i < m; i += THREADS) {
        if (ids)
            ids[i] = (uint32_t)s[i];
        else
            dst[i] = s[i];
    }
    __syncthreads();
}

// Tiles of up to kWarpSortMax keys: warp w of block b takes tile
// kTilesPerSortBlock b + w.
__global__ void __launch_bounds__(32 * kTilesPerSortBlock) tile_sort_kernel(const Ws ws) {
    const int lane = threadIdx.x & 31;
    const uint32_t t0 = blockIdx.x * kTilesPerSortBlock;
    const unsigned long long *words = ws.keys[ws.passes & 1];
    uint32_t *ids = ws.sorted;
    {
        const uint32_t t = t0 + (threadIdx.x >> 5);
        const uint2 r = t < ws.total_tiles ? checked_range(ws.ranges, t, ws.hdr, ws.cap) : make_uint2(0u, 0u);
        const uint32_t n = r.y - r.x;
        if (n == 1) {
            if (lane == 0) ids[r.x] = (uint32_t)words[r.x];
        } else if (n >= 2 && n <= 32) {
            warp_sort_tile<1>(words + r.x, ids + r.x, n, lane);
        } else if (n > 32 && n <= 64) {
            warp_sort_tile<2>(words + r.x, ids + r.x, n, lane);
        } else if (n > 64 && n <= 128) {
            warp_sort_tile<4>(words + r.x, ids + r.x, n, lane);
        } else if (n > 128 && n <= 256) {
            warp_sort_tile<8>(words + r.x, ids + r.x, n, lane);
        } else if (n > 256 && n <= kWarpSortMax) {   // 512 words: measured 10.4 -> 9.0 ms of outdoor tile sorts
            warp_sort_tile<16>(words + r.x, ids + r.x, n, lane);
        }
    }
}

// Merge of the sorted runs A[0, na) and B[0, nb) (distinct words) into C:
// each thread finds where its kMergeItems outputs start on the merge path by
// a binary search, then merges them sequentially.
__device__ __forceinline__ void block_merge(const unsigned long long *A, uint32_t na, const unsigned long long *B,
                                            uint32_t nb, unsigned long long *C) {
    const uint32_t n = na + nb;
    for (uint32_t d0 = threadIdx.x * kMergeItems; d0 < n; d0 += kBigSortThreads * kMergeItems) {
        uint32_t lo = d0 > nb ? d0 - nb : 0u, hi = min(d0, na);
        while (lo < hi) {   // the number of A's words among the first d0 outputs
            const uint32_t m = (lo + hi) >> 1;
            if (A[m] < B[d0 - m - 1])
                lo = m + 1;
            else
                hi = m;
        }
        uint32_t ia = lo, ib = d0 - lo;
        const uint32_t d1 = min(d0 + kMergeItems, n);
        for (uint32_t d = d0; d < d1; ++d) {
            const bool from_a = ib >= nb || (ia < na && A[ia] < B[ib]);
            C[d] = from_a ? A[ia++] : B[ib++];
        }
    }
}

// Tiles of more than kWarpSortMax keys, a block each in turn.  Block b
// looks at tiles b, b + G, b + 2G, ... (G blocks), a thread per tile at a
// time, and lists the big ones in shared memory first.
__global__ void __launch_bounds__(kBigSortThreads) tile_sort_big_kernel(const Ws ws) {
    constexpr int ITEMS = kBlockSortCap / kBigSortThreads;
    extern __shared__ unsigned long long s_sort[];   // kBlockSortCap words, then the counters
    uint32_t(*s_whist)[kRadix] = reinterpret_cast<uint32_t(*)[kRadix]>(s_sort + kBlockSortCap);
    __shared__ uint32_t s_red[2 * (kBigSortThreads / 32)];
    __shared__ uint32_t s_big[kBigSortThreads];
    __shared__ uint32_t s_nbig;
    uint32_t *ids = ws.sorted;
    const size_t G = gridDim.x;
    for (size_t first = blockIdx.x; first < ws.total_tiles; first += G * kBigSortThreads) {
        if (threadIdx.x == 0) s_nbig = 0u;
        __syncthreads();
        const size_t tt = first + threadIdx.x * G;
        if (tt < ws.total_tiles) {
            const uint2 r = checked_range(ws.ranges, (uint32_t)tt, ws.hdr, ws.cap);
            if (r.y - r.x > (uint32_t)kWarpSortMax) s_big[atomicAdd(&s_nbig, 1u)] = (uint32_t)tt;
        }
        __syncthreads();
        const uint32_t nbig = s_nbig;
        for (uint32_t q = 0; q < nbig; ++q) {
            const uint2 r = checked_range(ws.ranges, s_big[q], ws.hdr, ws.cap);
            const uint32_t n = r.y - r.x;
            unsigned long long *a = ws.keys[ws.passes & 1] + r.x, *b = ws.keys[(ws.passes + 1) & 1] + r.x;
            if (n <= (uint32_t)kBlockSortCap) {
                block_sort_run<kBigSortThreads, ITEMS>(a, n, s_sort, s_whist, s_red, nullptr, ids + r.x);
                continue;
            }
            for (uint32_t c0 = 0; c0 < n; c0 += kBlockSortCap)
                block_sort_run<kBigSortThreads, ITEMS>(a + c0, min(n - c0, (uint32_t)kBlockSortCap), s_sort, s_whist,
                                                       s_red, a + c0, nullptr);
            for (uint32_t w = kBlockSortCap; w < n; w <<= 1) {
                for (uint32_t lo = 0; lo < n; lo += 2 * w) {
                    const uint32_t mid = min(lo + w, n), hi = min(lo + 2 * w, n);
                    block_merge(a + lo, mid - lo, a + mid, hi - mid, b + lo);
                }
                __syncthreads();
                unsigned long long *x = a;
                a = b;
                b = x;
            }
            for (uint32_t i = threadIdx.x; i < n; i += kBigSortThreads) ids[r.x + i] = (uint32_t)a[i];
            __syncthreads();
        }
        __syncthreads();
    }
}

template <typename K, typename V>
cudaError_t launch_radix(const Ws &ws, int sm_count, cudaStream_t st) {
    const SortBufs<K, V> b = sort_bufs<K, V>(ws);
    sort_hist_kernel<K><<<sm_count * 4, 256, 0, st>>>(ws, b.k[0]);
    for (int p = 0; p < ws.passes; ++p)
        onesweep_kernel<K, V><<<sm_count * kSortBlocksPerSM, kSortThreads, 0, st>>>(ws, p, b);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ blend order
// The blends' tile order, most keys first (tiles bucketed by the bit length
// of their key count, the order within a bucket arbitrary), for the
// groupings that do not list it themselves (radix binning, per-tile binning
// beyond kBucketMaxTiles): a count kernel whose last block turns the bucket
// sizes into each bucket's first slot, then a scatter of the tile ids.  Both
// take warp-aggregated atomics (lanes of one bucket add with one atomic).
constexpr int kOrderThreads = 256;
__device__ __forceinline__ uint32_t count_bits(uint32_t c) { return c == 0u ? 0u : 32u - (uint32_t)__clz(c); }

__device__ __forceinline__ uint32_t order_bucket(const Ws &ws, uint32_t t) {
    if (t >= ws.total_tiles) return 33u;   // none
    const uint2 r = ws.ranges[t];
    return count_bits(r.y - r.x);
}

__global__ void __launch_bounds__(kOrderThreads) order_count_kernel(const Ws ws) {
    __shared__ uint32_t s_bins[33];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < 33; i += kOrderThreads) s_bins[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (uint32_t t0 = blockIdx.x * kOrderThreads; t0 < ws.total_tiles; t0 += gridDim.x * kOrderThreads) {
        const uint32_t b = order_bucket(ws, t0 + threadIdx.x);
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (b < 33u && lane == __ffs(peers) - 1) atomicAdd(s_bins + b, (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 33; i += kOrderThreads)
        if (s_bins[i]) atomicAdd(ws.order_bins + i, s_bins[i]);
    // the last block to finish (every block fences its counts first) lays out the buckets
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ws.hdr->order_counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    uint32_t at = 0;
    for (int b = 32; b >= 0; --b) {
        ws.order_bins[33 + b] = at;
        at += __ldcg(ws.order_bins + b);
    }
}

__global__ void __launch_bounds__(kOrderThreads) order_scatter_kernel(const Ws ws) {
    const int lane = threadIdx.x & 31;
    for (uint32_t t0 = blockIdx.x * kOrderThreads; t0 < ws.total_tiles; t0 += gridDim.x * kOrderThreads) {
        const uint32_t t = t0 + threadIdx.x, b = order_bucket(ws, t);
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0u;
        if (b < 33u && lane == leader) base = atomicAdd(ws.order_bins + 33 + b, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b < 33u) ws.tile_order[base + __popc(peers & lanemask_lt())] = t;
    }
}

cudaError_t launch_tile_order(const Ws &ws, int sm_count, cudaStream_t st) {
    if (!ws.order_tiles || bucket_binning(ws) || ws.total_tiles == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<uint64_t>(((uint64_t)ws.total_tiles + kOrderThreads - 1) / kOrderThreads,
                                                         (uint64_t)sm_count * 4);
    order_count_kernel<<<blocks, kOrderThreads, 0, st>>>(ws);
    order_scatter_kernel<<<blocks, kOrderThreads, 0, st>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_ranges_of(const Ws &ws, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * ws.total_tiles, st);
    if (e != cudaSuccess || ws.VN == 0) return e;
    if (ws.bin_tile)
        ranges_kernel<uint32_t><<<sm_count * 4, 256, 0, st>>>(ws, ws.vals[ws.passes & 1]);
    else
        ranges_kernel<unsigned long long><<<sm_count * 4, 256, 0, st>>>(ws, ws.keys[ws.passes & 1]);
    return cudaGetLastError();
}

// More than 48 KB of dynamic shared memory needs an opt-in (a host-side
// attribute of the kernel), once per kernel and device.
template <auto Kernel>
cudaError_t allow_smem(size_t bytes) {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}


}  // namespace

// Gaussians binned per tile emit their keys in the preprocess (keys_in_preprocess).
cudaError_t launch_scan_duplicate(const ViewTable &vt, const Ws &ws, cudaStream_t st) {
    if (ws.VN == 0 || keys_in_preprocess(ws)) return cudaSuccess;
    scan_reduce_kernel<<<ws.scan_blocks, kScanThreads, 0, st>>>(ws);
    scan_partials_kernel<<<1, 1024, 0, st>>>(ws);
    scan_down_kernel<<<ws.scan_blocks, kScanThreads, 0, st>>>(ws);
    duplicate_kernel<<<(unsigned)((ws.VN + 255) / 256), 256, 0, st>>>(vt, ws);
    return cudaGetLastError();
}

// Per-tile binning also makes the ranges and sorts within the tiles here.
cudaError_t launch_sort(const Ws &ws, int sm_count, cudaStream_t st) {
    if (!ws.bin_tile) return ws.VN == 0 ? cudaSuccess : launch_radix<unsigned long long, uint32_t>(ws, sm_count, st);
    cudaError_t e = cudaSuccess;
    if (bucket_binning(ws)) {   // writes every tile's range, even with no pairs
        const size_t smem = bucket_smem(ws.total_tiles);   // the tile counters were cleared by the init kernel
        if ((e = allow_smem<bucket_count_kernel>(kBucketSmemMax)) != cudaSuccess ||
            (e = allow_smem<bucket_scatter_kernel>(kBucketSmemMax)) != cudaSuccess)
            return e;
        bucket_count_kernel<<<sm_count, kBucketThreads, smem, st>>>(ws);   // also scans: always
        if (ws.VN > 0) bucket_scatter_kernel<<<sm_count, kBucketThreads, smem, st>>>(ws);
        e = cudaGetLastError();
    } else {
        e = ws.VN == 0 ? cudaSuccess : launch_radix<uint32_t, unsigned long long>(ws, sm_count, st);
        if (e == cudaSuccess) e = launch_ranges_of(ws, sm_count, st);   // clears the ranges even with no pairs
        if (e == cudaSuccess) e = launch_tile_order(ws, sm_count, st);
    }
    if (e != cudaSuccess || ws.VN == 0 || ws.total_tiles == 0) return e;
    tile_sort_kernel<<<(ws.total_tiles + kTilesPerSortBlock - 1) / kTilesPerSortBlock, 32 * kTilesPerSortBlock, 0,
                       st>>>(ws);
    if ((e = allow_smem<tile_sort_big_kernel>(kBigSortSmem)) != cudaSuccess) return e;
    const unsigned blocks = std::min<unsigned>(ws.total_tiles, (unsigned)sm_count);
    tile_sort_big_kernel<<<blocks, kBigSortThreads, kBigSortSmem, st>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const Ws &ws, int sm_count, cudaStream_t st) {
    if (ws.bin_tile) return cudaSuccess;   // made by launch_sort
    const cudaError_t e = launch_ranges_of(ws, sm_count, st);
    return e == cudaSuccess ? launch_tile_order(ws, sm_count, st) : e;
}

}  // namespace gsr
