// K2-K5: duplication into (tile id | depth) keys, LSD radix sort, tile
// ranges.  Depth ordering of the splats that cover a pixel (Sec. 3.1) is
// realised per screen tile: keys are ((tile id) << 32 | fp32 depth bits), and
// every tile's list comes out ordered by depth, ties by Gaussian index.
//
// Depth first (the key buffers hold at least one entry per Gaussian):
//   depth_min, depth_keys (keys and digit histograms) + 4 radix passes:
//        the Gaussians sorted by depth (the 32 bits of (depth bits - the
//        smallest) << 32 | index keys, stable; a pass whose digit is the
//        same for every key is a copy), into buffer 1;
//   scan_emit: single-pass exclusive scan of the tile counts in that order
//        (decoupled look-back) fused with key emission, into buffer 0: the
//        CTA's keys are emitted by all its threads together (key k of the
//        CTA by thread k mod 256, its position found by a binary search of
//        the positions' running counts), so that the stores coalesce;
//   1-2 radix passes on the tile bits only (stable), so each tile keeps the
//        depth order of emission.  Two passes over the tile keys instead of
//        six: the depth digits are sorted once per Gaussian, not per key.
// Otherwise: emission in index order and passes over all 32 + tile bits.
//
// K4 radix pass: a global digit histogram pass, then one kernel per 8-bit
//        digit: stable warp-level multisplit ranking in shared memory,
//        decoupled look-back across tiles for the digit offsets, and a
//        shared-memory staged scatter so that writes are runs of equal digit.
// K5     tile_ranges: [start, end) of every tile in the sorted keys.
//
// All device waits are bounded (kSpinLimit); a wait that gives up writes
// P2E_ERR_TIMEOUT to the status word and the kernel finishes without
// further waiting.
#include "common.cuh"

namespace p2e {

// look-back waits: spin (one L2 round trip per try) before sleeping
__device__ __forceinline__ void backoff_lb(uint32_t it) {
    if (it > 64) __nanosleep(it < 1024 ? 32 : 256);
}

// ---------------------------------------------------------------------------
// scratch layout (see sort_scratch_bytes)
// ---------------------------------------------------------------------------
constexpr int kScanItems = 4;
constexpr int kScanThreads = 256;
constexpr int kScanTile = kScanItems * kScanThreads;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;

struct SortScratch {
    uint32_t *hist;        // [kMaxPasses][256] digit totals
    uint32_t *tickets;     // [16]: [0] scan, [1 + p] sort pass p
    int64_t *n_depth;      // number of Gaussians in the depth sort
    uint32_t *zmin_inv;    // ~(smallest depth bits of a Gaussian that covers a tile)
    uint64_t *scan_state;  // [scan tiles] look-back words (flag << 62 | value)
    uint32_t *sort_state;  // [kMaxPasses][sort tiles][256] (flag << 30 | count)
    int64_t scan_tiles, sort_tiles;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t sort_scratch_bytes(int64_t n_total, int64_t capacity) {
    const int64_t st = (n_total + kScanTile - 1) / kScanTile;
    const int64_t kt = (capacity + kSortTile - 1) / kSortTile;
    return align256(kMaxPasses * kRadix * 4) + align256(16 * 4) + align256(16) + align256((size_t)(st + 1) * 8) +
           align256((size_t)kMaxPasses * (size_t)(kt + 1) * kRadix * 4);
}

static SortScratch carve(void *base, int64_t n_total, int64_t capacity) {
    SortScratch s;
    char *p = (char *)base;
    s.scan_tiles = (n_total + kScanTile - 1) / kScanTile;
    s.sort_tiles = (capacity + kSortTile - 1) / kSortTile;
    s.hist = (uint32_t *)p;
    p += align256(kMaxPasses * kRadix * 4);
    s.tickets = (uint32_t *)p;
    p += align256(16 * 4);
    s.n_depth = (int64_t *)p;
    s.zmin_inv = (uint32_t *)(p + 8);
    p += align256(16);
    s.scan_state = (uint64_t *)p;
    p += align256((size_t)(s.scan_tiles + 1) * 8);
    s.sort_state = (uint32_t *)p;
    return s;
}

// ---------------------------------------------------------------------------
// K2+K3: scan of tile counts fused with key emission
// ---------------------------------------------------------------------------
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagPre = 2ull << 62, kValMask = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// A look-back word is read for its own value only (no data published with
// it), so several can be in flight at once.
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Block-wide exclusive sum of one value per thread (256 threads).
template <int NT>
__device__ __forceinline__ uint64_t block_excl_sum(uint64_t v, uint64_t &total, uint64_t *sm /*NT/32*/) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    uint64_t wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const uint64_t s = sm[w];
        if (w < wid) wpre += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_emit_kernel(
    const uint32_t *__restrict__ ntiles, const ushort4 *__restrict__ rect,
    const float4 *__restrict__ xy_depth, const uint32_t *__restrict__ order, int64_t n_total,
    uint64_t *__restrict__ keys,
    uint32_t *__restrict__ vals, int64_t capacity, SortScratch S, int64_t *n_keys_dev,
    int32_t *status, uint32_t spin_limit, __grid_constant__ const Views P) {
    __shared__ uint64_t sm[kScanThreads / 32];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(&S.tickets[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t cnt[kScanItems], src[kScanItems];
    uint64_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t r = base + i;  // position in emission order: Gaussian order[r] (or r)
        src[i] = r < n_total ? (order ? __ldg(order + r) : (uint32_t)r) : 0u;
        cnt[i] = r < n_total ? __ldg(ntiles + src[i]) : 0u;
        local += cnt[i];
    }
    uint64_t total;
    const uint64_t texcl = block_excl_sum<kScanThreads>(local, total, sm);
    // decoupled look-back by warp 0, 32 predecessors per round trip
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        uint64_t prefix = 0;
        if (tile == 0) {
            if (lane == 0) st_release_u64(&S.scan_state[0], kFlagPre | total);
        } else {
            if (lane == 0) st_release_u64(&S.scan_state[tile], kFlagAgg | total);
            int64_t p = tile - 1;  // lane l reads p - l
            uint32_t spins = 0;
            while (true) {
                const int64_t idx = p - lane;
                const uint64_t w = idx >= 0 ? ld_acquire_u64(&S.scan_state[idx]) : kFlagPre;
                const uint32_t flag = (uint32_t)(w >> 62);
                const unsigned pre = __ballot_sync(0xffffffffu, flag == 2u);
                const unsigned notready = __ballot_sync(0xffffffffu, flag == 0u);
                const int first = pre ? __ffs(pre) - 1 : 32;
                const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
                if (notready & need) {
                    if (++spins > spin_limit) {
                        if (lane == 0) atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
                        break;
                    }
                    backoff_lb(spins);
                    continue;
                }
                uint64_t add = lane <= first ? (w & kValMask) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
                prefix += add;
                if (first < 32) break;
                p -= 32;
            }
            if (lane == 0) st_release_u64(&S.scan_state[tile], kFlagPre | (prefix + total));
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (tile == S.scan_tiles - 1) *n_keys_dev = (int64_t)(prefix + total);
        }
    }
    // the tile's positions: running key counts (inclusive, from the tile's
    // start) and Gaussians, so that the threads can emit the tile's keys
    // together, key k by thread k mod kScanThreads (coalesced stores)
    __shared__ uint32_t s_incl[kScanTile], s_src[kScanTile];
    {
        uint32_t run = (uint32_t)texcl;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            run += cnt[i];
            s_incl[threadIdx.x * kScanItems + i] = run;
            s_src[threadIdx.x * kScanItems + i] = src[i];
        }
    }
    __syncthreads();
    const uint64_t base_off = s_prefix;
    const int B = P.tile;
    for (uint32_t k = threadIdx.x; k < (uint32_t)total; k += kScanThreads) {
        int lo = 0, hi = kScanTile - 1;  // the first position whose running count exceeds k
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_incl[mid] > k) hi = mid;
            else lo = mid + 1;
        }
        const uint32_t j = k - (lo > 0 ? s_incl[lo - 1] : 0u);  // the key's rank in its Gaussian's tiles
        const int64_t e = s_src[lo];
        const int vi = (int)(e / P.n);
        const View &V = P.v[vi];
        const int64_t g = e - (int64_t)vi * P.n;
        const ushort4 r = __ldg(rect + e);  // pixel rectangle -> tiles
        const int tx0 = r.x / B, ty0 = r.y / B, w = r.z / B - tx0 + 1;
        const int ty = ty0 + (int)(j / (uint32_t)w), tx = tx0 + (int)(j % (uint32_t)w);
        const uint32_t zb = __float_as_uint(__ldg(&xy_depth[e].z));
        const uint64_t o = base_off + k;
        if ((int64_t)o < capacity) {
            keys[o] = ((uint64_t)(V.tile_base + (int64_t)ty * V.tiles_x + tx) << 32) | zb;
            vals[o] = (uint32_t)g;
        }
    }
}

// Smallest depth bits over the Gaussians that cover a tile (as a maximum of
// the complements, so that the zeroed scratch is the identity).
__global__ void __launch_bounds__(256) depth_min_kernel(const uint32_t *__restrict__ ntiles,
                                                        const float4 *__restrict__ xy_depth, int64_t n_total,
                                                        uint32_t *zmin_inv) {
    uint32_t best = 0u;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_total;
         e += (int64_t)gridDim.x * blockDim.x)
        if (__ldg(ntiles + e)) best = max(best, ~__float_as_uint(__ldg(&xy_depth[e].z)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(zmin_inv, best);
}

// Depth keys of all Gaussians (every view): ((depth bits - smallest) << 32
// | e), value e (positive fp32 depths order as their bits, so the offset
// keeps the order and a narrow depth range leaves the top byte 0, a pass the
// radix sort then skips); a Gaussian that covers no tile takes key 0 (it
// emits nothing, so its place is irrelevant).  The histograms of the four
// depth bytes (the depth passes' digits) are counted on the way.
__global__ void __launch_bounds__(256) depth_keys_kernel(const uint32_t *__restrict__ ntiles,
                                                         const float4 *__restrict__ xy_depth, int64_t n_total,
                                                         uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                         int64_t *n_depth, const uint32_t *zmin_inv,
                                                         uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[4 * kRadix];
    const uint32_t zmin = ~*zmin_inv;
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_depth = n_total;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_total; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < n_total;
        uint32_t zb = 0u;
        if (valid) {
            if (__ldg(ntiles + e)) zb = __float_as_uint(__ldg(&xy_depth[e].z)) - zmin;
            keys[e] = ((uint64_t)zb << 32) | (uint64_t)e;
            vals[e] = (uint32_t)e;
        }
        // the low bytes spread over the bins; the high ones (sign, exponent)
        // crowd a few, so equal digits of a warp are added once
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (valid) atomicAdd(&sh[b * kRadix + ((zb >> (8 * b)) & 255u)], 1u);
#pragma unroll
        for (int b = 2; b < 4; ++b) {
            const uint32_t d = valid ? (zb >> (8 * b)) & 255u : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == 31 - __clz(peers)) atomicAdd(&sh[b * kRadix + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// ---------------------------------------------------------------------------
// K4: radix sort
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t sort_count(const int64_t *n_keys_dev, int64_t capacity) {
    const int64_t k = *n_keys_dev;
    return k < capacity ? k : capacity;
}

__global__ void __launch_bounds__(256) digit_hist_kernel(const uint64_t *__restrict__ keys,
                                                         const int64_t *n_keys_dev, int64_t capacity,
                                                         int shift0, int passes, uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[kMaxPasses * kRadix];
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t K = sort_count(n_keys_dev, capacity);
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < K; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < K;
        const uint64_t k = valid ? keys[i] : 0ull;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? (uint32_t)(k >> (shift0 + 8 * p)) & 255u : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == 31 - __clz(peers)) atomicAdd(&sh[p * kRadix + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

constexpr uint32_t kSFlagAgg = 1u << 30, kSFlagPre = 2u << 30, kSValMask = (1u << 30) - 1;
constexpr int kLookWindow = 16;  // predecessors read per look-back round trip

struct __align__(16) SortSmem {
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t block_excl[kRadix];
    uint64_t digit_out[kRadix];  // global position of the digit's first key in this tile
    uint64_t scan_tmp[kSortThreads / 32];
    uint32_t tile;
};

__global__ void __launch_bounds__(kSortThreads) radix_pass_kernel(
    const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const int64_t *n_keys_dev,
    int64_t capacity, int shift, const uint32_t *__restrict__ hist, uint32_t *sort_state,
    uint32_t *ticket, int32_t *status, uint32_t spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_raw);
    const int64_t K = sort_count(n_keys_dev, capacity);
    const int64_t ntiles = (K + kSortTile - 1) / kSortTile;
    if (threadIdx.x == 0) sm.tile = atomicAdd(ticket, 1u);
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&sm.warp_hist[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile = sm.tile;
    if (tile >= ntiles) return;
    if (__syncthreads_or(threadIdx.x < kRadix && (int64_t)hist[threadIdx.x] == K)) {
        // every key has the same digit: the stable pass is the identity
        const int64_t t0 = tile * kSortTile, t1 = min(K, t0 + kSortTile);
        for (int64_t i = t0 + threadIdx.x; i < t1; i += kSortThreads) {
            keys_out[i] = keys_in[i];
            vals_out[i] = vals_in[i];
        }
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t wbase = tile * kSortTile + (int64_t)wid * (32 * kSortItems);

    uint64_t k[kSortItems];
    uint32_t v[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t idx = wbase + j * 32 + lane;
        const bool valid = idx < K;
        k[j] = valid ? keys_in[idx] : 0ull;
        v[j] = valid ? vals_in[idx] : 0u;
        rank[j] = valid ? 0u : 0xffffffffu;
    }
    // stable warp-level multisplit: element order within a warp is (j, lane)
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = rank[j] != 0xffffffffu;
        const uint32_t d = valid ? (uint32_t)(k[j] >> shift) & 255u : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (valid) before = sm.warp_hist[wid][d];
        __syncwarp();
        if (valid) {
            rank[j] = before + __popc(peers & lt_mask);
            if (lane == 31 - __clz(peers)) sm.warp_hist[wid][d] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets across warps, tile count, look-back
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = sm.warp_hist[w][d];
        sm.warp_hist[w][d] = cnt;
        cnt += c;
    }
    uint64_t tot;
    const uint64_t bexcl = block_excl_sum<kSortThreads>(cnt, tot, sm.scan_tmp);
    sm.block_excl[d] = (uint32_t)bexcl;
    uint64_t gtot;
    const uint64_t gexcl = block_excl_sum<kSortThreads>(hist[d], gtot, sm.scan_tmp);
    uint32_t *st = sort_state + (size_t)tile * kRadix + d;
    uint64_t prefix = 0;
    if (tile == 0) {
        st_release_u32(st, kSFlagPre | cnt);
    } else {
        st_release_u32(st, kSFlagAgg | cnt);
        // the predecessors' words kLookWindow at a time (one round trip):
        // add aggregates up to the first inclusive prefix, or up to the
        // first tile not yet published and read again from there
        int64_t p = tile - 1;
        uint32_t spins = 0;
        while (p >= 0) {
            uint32_t w[kLookWindow];
#pragma unroll
            for (int i = 0; i < kLookWindow; ++i)
                w[i] = p - i >= 0 ? ld_relaxed_u32(sort_state + (size_t)(p - i) * kRadix + d) : kSFlagPre;
            int used = kLookWindow;
            bool done = false;
#pragma unroll
            for (int i = kLookWindow - 1; i >= 0; --i) {  // find the first stop in window order
                const uint32_t f = w[i] >> 30;
                if (f != 1u) {
                    used = i;
                    done = f == 2u;
                }
            }
            // w[0 .. used) are aggregates; w[used] (if done) the inclusive prefix
#pragma unroll
            for (int i = 0; i < kLookWindow; ++i)
                if (i < used || (done && i == used)) prefix += w[i] & kSValMask;
            if (done) break;
            p -= used;
            if (used < kLookWindow) {  // stopped at a tile not yet published
                if (++spins > spin_limit) { atomicExch(status, (int32_t)P2E_ERR_TIMEOUT); break; }
                backoff_lb(spins);
            }
        }
        st_release_u32(st, kSFlagPre | (uint32_t)(prefix + cnt));
    }
    sm.digit_out[d] = gexcl + prefix;
    __syncthreads();
    // stage in shared memory in block-sorted order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        if (rank[j] != 0xffffffffu) {
            const uint32_t dd = (uint32_t)(k[j] >> shift) & 255u;
            const uint32_t pos = sm.block_excl[dd] + sm.warp_hist[wid][dd] + rank[j];
            sm.keys[pos] = k[j];
            sm.vals[pos] = v[j];
        }
    }
    __syncthreads();
    const int64_t tcount = (K - tile * kSortTile) < kSortTile ? (K - tile * kSortTile) : kSortTile;
    for (int i = threadIdx.x; i < tcount; i += kSortThreads) {
        const uint64_t kk = sm.keys[i];
        const uint32_t dd = (uint32_t)(kk >> shift) & 255u;
        const uint64_t o = sm.digit_out[dd] + (uint64_t)(i - sm.block_excl[dd]);
        if (o < (uint64_t)K) {  // always true unless a look-back gave up
            keys_out[o] = kk;
            vals_out[o] = sm.vals[i];
        }
    }
}

// ---------------------------------------------------------------------------
// K5: tile ranges
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint64_t *__restrict__ keys,
                                                          const int64_t *n_keys_dev, int64_t capacity,
                                                          int64_t total_tiles, uint2 *__restrict__ ranges) {
    const int64_t K = sort_count(n_keys_dev, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t t = keys[i] >> 32;
        if (t >= (uint64_t)total_tiles) continue;
        if (i == 0 || (keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
        if (i == K - 1 || (keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

// Non-empty tiles, longest list first (by power-of-two length class), for
// the persistent compositing kernel: work[0] = count, work[1] = counter
// (zeroed here and by p2e_render), work[2..] = tile ids.
__global__ void __launch_bounds__(1024) tile_work_kernel(const uint2 *__restrict__ ranges,
                                                         int64_t total_tiles, uint32_t *work) {
    __shared__ uint32_t cnt[33], base[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < total_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x;
        if (len) atomicAdd(&cnt[31 - __clz(len)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 31; b >= 0; --b) {
            base[b] = acc;
            acc += cnt[b];
        }
        work[0] = acc;
        work[1] = 0;
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < total_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x;
        if (len) work[2 + atomicAdd(&base[31 - __clz(len)], 1u)] = (uint32_t)t;
    }
}

// The radix pass takes more than the default 48 KB of dynamic shared
// memory; the attribute is per device, so it is set once on each.
static cudaError_t configure_radix_pass() {
    static int configured[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (configured[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(radix_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
    if (e == cudaSuccess) configured[dev] = 1;
    return e;
}

int sort_passes(int64_t total_tiles) {
    int tb = 0;
    while ((int64_t(1) << tb) < total_tiles) ++tb;
    return (32 + tb + 7) / 8;
}

cudaError_t launch_sort_bin(const p2e_projected *proj, const Views &P, p2e_bins *io,
                            int num_sms, cudaStream_t st) {
    const int64_t n_total = P.n * P.n_views;
    SortScratch S = carve(io->scratch, n_total, io->capacity);
    const int passes = sort_passes(P.total_tiles);
    cudaError_t e;
    // one memset clears histograms, tickets and every look-back word
    e = cudaMemsetAsync(io->scratch, 0, sort_scratch_bytes(n_total, io->capacity), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(io->ranges, 0, (size_t)P.total_tiles * sizeof(uint2), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(io->n_keys_dev, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(SortSmem);
    if ((e = configure_radix_pass()) != cudaSuccess) return e;
    const unsigned sort_grid = (unsigned)(S.sort_tiles > 0 ? S.sort_tiles : 1);
    auto pass = [&](int slot, int src, int shift, const int64_t *count, unsigned grid) {
        radix_pass_kernel<<<grid, kSortThreads, smem, st>>>(
            io->keys[src], io->vals[src], io->keys[src ^ 1], io->vals[src ^ 1], count, io->capacity, shift,
            S.hist + slot * kRadix, S.sort_state + (size_t)slot * (S.sort_tiles + 1) * kRadix,
            S.tickets + 1 + slot, io->status_dev, kSpinLimit);
        return cudaGetLastError();
    };
    const unsigned scan_grid = (unsigned)S.scan_tiles;
    if (n_total > 0 && n_total <= io->capacity) {
        // depth first: sort the Gaussians by depth (four passes over n_total
        // keys, into buffer 1), emit the tile keys in that order, then sort
        // them stably by tile only
        const int tpasses = passes - 4;
        depth_min_kernel<<<num_sms * 2, 256, 0, st>>>(proj->ntiles, (const float4 *)proj->xy_depth, n_total,
                                                      S.zmin_inv);
        depth_keys_kernel<<<num_sms * 2, 256, 0, st>>>(proj->ntiles, (const float4 *)proj->xy_depth, n_total,
                                                       io->keys[1], io->vals[1], S.n_depth, S.zmin_inv, S.hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const unsigned dgrid = (unsigned)((n_total + kSortTile - 1) / kSortTile);
        for (int p = 0; p < 4; ++p)
            if ((e = pass(p, (p & 1) ? 0 : 1, 32 + 8 * p, S.n_depth, dgrid)) != cudaSuccess) return e;
        scan_emit_kernel<<<scan_grid, kScanThreads, 0, st>>>(proj->ntiles, (const ushort4 *)proj->rect,
                                                             (const float4 *)proj->xy_depth, io->vals[1], n_total,
                                                             io->keys[0], io->vals[0], io->capacity, S,
                                                             io->n_keys_dev, io->status_dev, kSpinLimit, P);
        digit_hist_kernel<<<num_sms * 4, 256, 0, st>>>(io->keys[0], io->n_keys_dev, io->capacity, 32, tpasses,
                                                       S.hist + 4 * kRadix);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (int p = 0; p < tpasses; ++p)
            if ((e = pass(4 + p, p & 1, 32 + 8 * p, io->n_keys_dev, sort_grid)) != cudaSuccess) return e;
        io->result = tpasses & 1;
    } else {
        // all key bits, least significant first
        if (n_total > 0) {
            scan_emit_kernel<<<scan_grid, kScanThreads, 0, st>>>(proj->ntiles, (const ushort4 *)proj->rect,
                                                                 (const float4 *)proj->xy_depth, nullptr, n_total,
                                                                 io->keys[0], io->vals[0], io->capacity, S,
                                                                 io->n_keys_dev, io->status_dev, kSpinLimit, P);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        digit_hist_kernel<<<num_sms * 4, 256, 0, st>>>(io->keys[0], io->n_keys_dev, io->capacity, 0, passes,
                                                       S.hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (int p = 0; p < passes; ++p)
            if ((e = pass(p, p & 1, 8 * p, io->n_keys_dev, sort_grid)) != cudaSuccess) return e;
        io->result = passes & 1;
    }

    tile_ranges_kernel<<<num_sms * 8, 256, 0, st>>>(io->keys[io->result], io->n_keys_dev, io->capacity,
                                                    P.total_tiles, (uint2 *)io->ranges);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tile_work_kernel<<<1, 1024, 0, st>>>((const uint2 *)io->ranges, P.total_tiles, io->tile_work);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Timeout self-test: one radix pass over two tiles of keys whose work
// tickets start at 1, so the only CTA takes tile 1 and its look-back waits
// on tile 0's state, which no CTA ever publishes.  The wait gives up after
// `spin_limit` tries, records P2E_ERR_TIMEOUT and the pass finishes (its
// writes stay inside the buffers).
// ---------------------------------------------------------------------------
__global__ void selftest_sort_init_kernel(uint32_t *ticket, int64_t *n_keys, int64_t k) {
    if (threadIdx.x == 0) {
        *ticket = 1u;
        *n_keys = k;
    }
}

size_t selftest_sort_bytes() {
    const size_t k = 2 * kSortTile;
    return align256(2 * k * 8) + align256(2 * k * 4) + align256(kRadix * 4) + align256(3 * kRadix * 4) +
           align256(16) + align256(16);
}

cudaError_t launch_selftest_sort(void *scratch, int32_t *status, uint32_t spin_limit, cudaStream_t st) {
    const int64_t k = 2 * kSortTile;
    char *p = (char *)scratch;
    uint64_t *keys = (uint64_t *)p;
    p += align256(2 * k * 8);
    uint32_t *vals = (uint32_t *)p;
    p += align256(2 * k * 4);
    uint32_t *hist = (uint32_t *)p;  // all zero: no digit holds every key, so the pass ranks
    p += align256(kRadix * 4);
    uint32_t *state = (uint32_t *)p;
    p += align256(3 * kRadix * 4);
    uint32_t *ticket = (uint32_t *)p;
    p += align256(16);
    int64_t *n_keys = (int64_t *)p;
    cudaError_t e = cudaMemsetAsync(scratch, 0, selftest_sort_bytes(), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    if ((e = configure_radix_pass()) != cudaSuccess) return e;
    selftest_sort_init_kernel<<<1, 32, 0, st>>>(ticket, n_keys, k);
    radix_pass_kernel<<<1, kSortThreads, sizeof(SortSmem), st>>>(keys, vals, keys + k, vals + k, n_keys, k, 0, hist,
                                                                 state, ticket, status, spin_limit);
    return cudaGetLastError();
}

}  // namespace p2e
