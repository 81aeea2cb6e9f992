// K6: front-to-back alpha compositing (Sec. 3.1, Eq. 1-2), with the normal
// and depth images obtained by substituting n_k and z_k for c_k.
//
// Work decomposition.  A compact subject covers few tiles (a 1 m figure at
// 2.5 m fills ~150 of 4096 16-px tiles at 1024^2) with long depth lists
// (up to ~40K splats), so neither a CTA per tile nor a thread per pixel
// keeps the GPU busy.  Here one WARP owns an 8 x 4 pixel block (lane =
// pixel) of one binning tile, and a tile's list is cut into SEGMENTS of 128
// splats per block of the tile (1024 for 16-px tiles).  Warps are fully
// independent (no block-wide barrier, no waiting) and pull (tile, segment,
// block) items from a global counter, tiles in work-list order (longest
// first).
//
// Per segment the warp streams the list in steps of 128 splats: every lane
// loads four indices (one step ahead) and pixel rectangles; the warp keeps
// (ballot) the splats whose rectangle meets a live pixel of the block; their
// records are copied (cp.async) in list order into one of two shared-memory
// stage buffers while the previous chunk of 32 is composited from the other
// (broadcast reads, one splat per step for all 32 pixels).
//
// Segments are combined under the associative "over" operator:
//   segment 0   composited from T = 1 with the stop rule: exactly the
//               sequential recurrence;
//   segment s   its aggregate: composited from T = 1 without stopping.  The
//               state after it is fold(state before, aggregate):
//               C = C_in + T_in C_s, T = T_in T_s, unless the stop falls
//               inside the segment (T_in T_s < t_min, T non-increasing):
//               then the segment is re-walked from the true state with the
//               stop rule, which reproduces the sequential result.
// Chained schedule: the aggregate and the predecessor's state are stored in
// the free half of the key double buffer; whichever of the two arrives
// second (an acquire-release counter) computes the segment's state and
// carries the chain on while successors' aggregates are already there; the
// last segment's state is the pixel.  While it speculates, a warp polls the
// predecessor's state: pixels it shows done, or whose stop it shows to lie
// in the part already walked, drop out (their aggregate is not used; the
// latter publish T = 0).  The states take 8 bytes per key of the segments
// they cover; the longest tiles take them first, and where the free buffers
// run out (small capacities) one warp runs the same segments of a (tile,
// block) in turn, tile by tile.  Which rule
// gives a pixel's result depends only on its tile's list: results are
// bit-identical across schedules, batches and runs.
//
// Sub-pixel accuracy: the pixel offset is formed as
//   (x - (floor(u) - x0)) + (0.5 - frac(u)),
// an exact small integer plus an exact fraction, so it keeps ~1e-7 px at
// any image size.
#include <algorithm>

#include "splat.cuh"

namespace p2e {

constexpr int kBW = 8, kBH = 4;    // pixel block of one warp
constexpr int kWarps = 8;          // warps per CTA
constexpr int kStateFloats = 8;    // T, C0..2, N0..2, D (and a word last | deferred << 30 | done << 31 apart)
constexpr uint32_t kDoneBit = 1u << 31;
constexpr uint32_t kIncl = 2u;  // segment flag: inclusive state published

__host__ __device__ constexpr int blocks_of(int tile) { return (tile / kBW) * (tile / kBH); }
// Segment length: 128 splats per pixel block of the tile (1024 for 16-px
// tiles).  It is fixed, so a pixel's arithmetic depends only on its tile's
// list, never on the capacity, the other views of the call, or timing.
// (Longer segments leave too few items: with 2048 nearly every segment of
// a frame starts at once and is speculated in full before its predecessor
// publishes; measured 2.7x the evaluated pairs.)
__host__ __device__ constexpr uint32_t seg_len(int tile) { return 128u * (uint32_t)blocks_of(tile); }

struct StageBuf {          // one chunk of staged splats (raw records)
    float4 xy[32];         // xy_depth record
    float4 co[32];         // (A, B, C, o)
    float4 cc[32];         // rgb
    float4 nr[32];         // (nx, ny, nz, -)
    float4 off[32];        // block-relative offset of the centre (splat_offset), per splat
    uint32_t pos[32];      // list position
};
struct StageRec {          // per warp: two buffers, filled by cp.async in turn
    StageBuf b[2];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

struct PixState {
    float T, c0, c1, c2, n0, n1, n2, D;
    uint32_t last;
    bool done;
    bool deferred;  // done, its output written by a deferred re-walk
};
constexpr uint32_t kDeferBit = 1u << 30;  // list positions stay below 2^30 when chained

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Layout of the free half of the key double buffer while p2e_render runs
// (n_work work entries, NB pixel blocks per tile, one state slot per
// segment of a chained tile):
//   vals[1 - result] (uint32 words):
//     [0]                          1 when the chained schedule is in use
//     [1, n_work + 1]              item_base: first item of work entry w, then the total
//     [n_work + 2, 2 n_work + 2]   slot_base: first state slot of entry w (kNoSlot for a
//                                  tile whose blocks each run in one warp), then the
//                                  slots in use
//     [2 n_work + 3]               multi-segment tiles run without chaining
//     [2 n_work + 4]               max_slots: the slots the two buffers hold
//     from tbl_words(n_work)       per (slot, block) 32 words 'last | deferred << 30
//                                  | done << 31', then max_slots x NB arrival
//                                  counters and as many ready flags
//   keys[1 - result] (floats):     per (slot, block) kStateFloats x 32 state floats
//                                  (word-major)
// A slot costs NB x 1 KB of the key buffer, i.e. 8 bytes per key of its
// segment: the key buffer holds the states of every key it can hold.
constexpr uint32_t kNoSlot = 0xffffffffu;
__host__ __device__ inline int64_t tbl_words(uint32_t n_work) { return (2 * (int64_t)n_work + 5 + 31) & ~int64_t(31); }
constexpr int kSlotWords = 32 + 1 + 1;  // value-buffer words per (slot, block)

// Item table (one CTA).  Over the work list (longest tiles first), the
// multi-segment tiles take state slots while they fit (a prefix of the
// list): each of their segments is an item per block, chained across
// warps.  A multi-segment tile past the prefix is one item per block whose
// warp runs the same segments in turn (same arithmetic, same result); a
// one-segment tile is one item per block in either case.  Chaining needs
// the key count within the capacity and the table within the value buffer;
// otherwise every (tile, block) is one item and nothing else is written.
__global__ void __launch_bounds__(1024) render_items_kernel(const uint2 *__restrict__ ranges,
                                                            const uint32_t *__restrict__ work,
                                                            const int64_t *__restrict__ n_keys_dev,
                                                            int64_t capacity, int allow_chain, int tile,
                                                            uint32_t *__restrict__ table) {
    __shared__ uint32_t s_sum[32], s_off[32];
    __shared__ uint32_t s_carry, s_carry2, s_tot, s_used, s_alone;
    const uint32_t n_work = work[0];
    const uint32_t nb = (uint32_t)blocks_of(tile), S = seg_len(tile);
    const int64_t tbl = tbl_words(n_work);
    const bool fits = allow_chain && *n_keys_dev <= capacity && tbl <= capacity && capacity < (int64_t(1) << 30);
    if (!fits) {
        if (threadIdx.x == 0 && capacity > 0) table[0] = 0u;
        return;
    }
    const int64_t ms = min(capacity * 8 / ((int64_t)nb * 32 * kStateFloats * 4),  // key buffer (bytes)
                           (capacity - tbl) / ((int64_t)nb * kSlotWords));        // value buffer (words)
    const uint32_t max_slots = (uint32_t)min(ms, (int64_t)0x7fffffff);
    uint32_t *item_base = table + 1, *slot_base = table + 2 + n_work;
    if (threadIdx.x == 0) s_carry = s_carry2 = s_used = s_alone = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5);
    // exclusive block scan of one value per thread (and the block's total)
    auto block_scan = [&](uint32_t v, uint32_t &excl, uint32_t &tot) {
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const uint32_t s = lane < nw ? s_sum[lane] : 0u;
            uint32_t t = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_off[lane] = t - s;
            if (lane == 31) s_tot = t;
        }
        __syncthreads();
        excl = s_off[wid] + x - v;
        tot = s_tot;
        __syncthreads();
    };
    for (uint32_t b0 = 0; b0 < n_work; b0 += blockDim.x) {
        const uint32_t w = b0 + threadIdx.x;
        uint32_t v = 0;
        if (w < n_work) {
            const uint2 r = ranges[work[2 + w]];
            v = (r.y - r.x + S - 1) / S;  // segments of the tile
        }
        const uint32_t vs = v > 1 ? v : 0u;  // slots a chained tile takes
        uint32_t e1, t1, e0, t0;
        block_scan(vs, e1, t1);
        const uint64_t first = (uint64_t)s_carry2 + e1;
        const bool chain = vs > 0 && first + vs <= max_slots;
        const uint32_t vi = (vs > 0 && !chain) ? 1u : v;  // items per block
        block_scan(vi, e0, t0);
        const uint32_t carry = s_carry;
        if (w < n_work) {
            item_base[w] = (carry + e0) * nb;
            slot_base[w] = chain ? (uint32_t)first : (vs > 0 ? kNoSlot : 0u);
            if (chain) atomicMax(&s_used, (uint32_t)(first + vs));
            if (vs > 0 && !chain) atomicAdd(&s_alone, 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry = carry + t0;
            s_carry2 = s_carry2 + t1;
        }
        __syncthreads();
    }
    const uint32_t used = s_used;
    if (threadIdx.x == 0) {
        item_base[n_work] = s_carry * nb;
        slot_base[n_work] = used;
        table[2 * n_work + 3] = s_alone;
        table[2 * n_work + 4] = max_slots;
        table[0] = 1u;
    }
    // arrival counters and ready flags of the slots in use
    uint32_t *counters = table + tbl + (size_t)max_slots * nb * 32, *ready = counters + (size_t)max_slots * nb;
    for (uint32_t t = threadIdx.x; t < used * nb; t += blockDim.x) {
        counters[t] = 0u;
        ready[t] = 0u;
    }
}

__device__ __forceinline__ void fresh_state(PixState &s, bool inside) {
    s.T = 1.f;
    s.c0 = s.c1 = s.c2 = s.n0 = s.n1 = s.n2 = s.D = 0.f;
    s.last = 0u;
    s.done = !inside;
    s.deferred = false;
}

// per-lane state words, word-major ([word][lane]: coalesced), through L2:
// the floats in fs, the word 'last | done << 31' in ls
__device__ __forceinline__ void load_state(const float *fs, const uint32_t *ls, int lane, PixState &s) {
    s.T = __ldcg(fs + 0 * 32 + lane);
    s.c0 = __ldcg(fs + 1 * 32 + lane);
    s.c1 = __ldcg(fs + 2 * 32 + lane);
    s.c2 = __ldcg(fs + 3 * 32 + lane);
    s.n0 = __ldcg(fs + 4 * 32 + lane);
    s.n1 = __ldcg(fs + 5 * 32 + lane);
    s.n2 = __ldcg(fs + 6 * 32 + lane);
    s.D = __ldcg(fs + 7 * 32 + lane);
    const uint32_t w = __ldcg(ls + lane);
    s.last = w & ~(kDoneBit | kDeferBit);
    s.done = (w & kDoneBit) != 0u;
    s.deferred = (w & kDeferBit) != 0u;
}
__device__ __forceinline__ void store_state(float *fs, uint32_t *ls, int lane, const PixState &s) {
    __stcg(fs + 0 * 32 + lane, s.T);
    __stcg(fs + 1 * 32 + lane, s.c0);
    __stcg(fs + 2 * 32 + lane, s.c1);
    __stcg(fs + 3 * 32 + lane, s.c2);
    __stcg(fs + 4 * 32 + lane, s.n0);
    __stcg(fs + 5 * 32 + lane, s.n1);
    __stcg(fs + 6 * 32 + lane, s.n2);
    __stcg(fs + 7 * 32 + lane, s.D);
    __stcg(ls + lane, s.last | (s.done ? kDoneBit : 0u) | (s.deferred ? kDeferBit : 0u));
}

// Bits of the 8 x 4 block (bit 8y + x) covered by the block-relative
// rectangle [rx0, rx1] x [ry0, ry1] (non-empty, inside the block).
__device__ __forceinline__ uint32_t rect_bits(int rx0, int rx1, int ry0, int ry1) {
    const uint32_t row = (0xffu >> (kBW - 1 - (rx1 - rx0))) << rx0;
    const uint32_t rows = (0xfu >> (kBH - 1 - (ry1 - ry0))) << ry0;
    const uint32_t spread = (rows & 1u) | ((rows & 2u) << 7) | ((rows & 4u) << 14) | ((rows & 8u) << 21);
    return row * spread;
}

// Shared-memory staging of every warp of a CTA (declared at namespace
// scope so that the out-of-line segment walk addresses it directly).
__shared__ StageRec g_stage[kWarps];

// What every segment walk of one (tile, pixel block) item shares.
struct SegArgs {
    const uint32_t *vals;
    const float4 *xy_depth, *conic_op;
    const ushort4 *rect;
    const float4 *rgb, *normal;
    int64_t gbase;
    int x0, y0;
    float lxf, lyf;
    uint32_t n;
    float pw_min, amax, afloor, tmin;
};

// Composites the nh staged splats of one buffer for the lane's pixel, in
// list order.  kStop: the stop rule of the sequential recurrence;
// otherwise a pure product from the given state.  `pairs` counts the
// (pixel, splat) pairs evaluated.
// The splat's block-relative offset (the same for every pixel of the
// block) was formed once per splat when the chunk was staged.
template <bool kStop>
__device__ __forceinline__ void composite_chunk(const StageBuf &sb, int nh, const SegArgs &a, PixState &st,
                                                uint32_t &pairs) {
    if (st.done) return;
    int j = 0;
    for (; j < nh; ++j) {
        const float4 o = sb.off[j], co = sb.co[j];
        const float power = splat_power(o, co, a.lxf, a.lyf);
        if (power < a.pw_min) continue;
        float e;
        bool fr;
        const float alpha = splat_alpha(co.w, power, a.amax, e, fr);
        if (alpha < a.afloor) continue;
        const float Tn = st.T * (1.f - alpha);
        if (kStop && Tn < a.tmin) {
            st.done = true;
            ++j;  // the stopping splat was evaluated too
            break;
        }
        const float wgt = alpha * st.T;
        const float4 cc = sb.cc[j], nr = sb.nr[j];
        st.c0 = fmaf(wgt, cc.x, st.c0);
        st.c1 = fmaf(wgt, cc.y, st.c1);
        st.c2 = fmaf(wgt, cc.z, st.c2);
        st.n0 = fmaf(wgt, nr.x, st.n0);
        st.n1 = fmaf(wgt, nr.y, st.n1);
        st.n2 = fmaf(wgt, nr.z, st.n2);
        st.D = fmaf(wgt, sb.xy[j].z, st.D);
        st.T = Tn;
        st.last = sb.pos[j] + 1u;
    }
    pairs += (uint32_t)j;
}

// Streams list positions [s0, s1) for the warp's block.  Every lane
// screens four splats per step of 128 (independent loads; the next step's
// indices are fetched one step ahead); the hits of each chunk of 32 are
// copied (cp.async) into one of two stage buffers in list order while the
// previous chunk is composited from the other.  `stop`: the stop rule of
// the sequential recurrence, else the pure product (an aggregate).  With a
// poll flag, returns early (the position reached, a multiple of 128 splats
// past s0) as soon as the flag is set; otherwise returns s1.
//
// Out of line: the kernel walks segments from several places (the exact
// first segment, aggregates, catch-ups and re-walks); one copy of this loop
// keeps the kernel's code within the instruction caches.  The state is
// copied in and out once per call; the loop runs on registers.
__device__ __noinline__ uint32_t composite_segment(bool stop, uint32_t s0, uint32_t s1, const SegArgs &args,
                                                   PixState &state, uint32_t &pair_count, const uint32_t *poll) {
    constexpr int kAhead = 4;  // chunks of 32 screened per step
    const SegArgs a = args;
    PixState st = state;
    uint32_t pairs = 0;
    const int lane = threadIdx.x & 31;
    StageRec &sg = g_stage[threadIdx.x >> 5];
    const uint32_t lt = (1u << lane) - 1u;
    int cur = 0;               // buffer the next chunk is copied into
    int pend = 0;              // splats staged in buffer cur ^ 1, not yet composited
    uint32_t gk[kAhead];
    auto fetch = [&](uint32_t b, uint32_t (&g)[kAhead]) {
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            const uint32_t idx = b + 32u * k + (uint32_t)lane;
            g[k] = idx < s1 ? __ldg(a.vals + idx) : 0xffffffffu;
        }
    };
    auto composite = [&](StageBuf &sb, int nh) {
        // one lane per staged splat: its offset from the block's origin
        if (lane < nh) sb.off[lane] = splat_offset(sb.xy[lane], a.x0, a.y0);
        __syncwarp();
        if (stop) composite_chunk<true>(sb, nh, a, st, pairs);
        else composite_chunk<false>(sb, nh, a, st, pairs);
    };
    fetch(s0, gk);
    uint32_t reached = s1;
    for (uint32_t base = s0; base < s1; base += 32 * kAhead) {
        if (poll) {
            uint32_t ready = 0;
            if (lane == 0) ready = ld_acquire_u32(poll) & kIncl;
            if (__shfl_sync(0xffffffffu, ready, 0)) {
                reached = base;
                break;
            }
        }
        const uint32_t live = __ballot_sync(0xffffffffu, !st.done);
        if (!live) break;
        bool hk[kAhead];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            hk[k] = false;
            if (gk[k] != 0xffffffffu) {
                if (gk[k] >= a.n) gk[k] = 0;  // only reachable with corrupted bins
                const ushort4 rc = __ldg(a.rect + a.gbase + gk[k]);
                const int rx0 = max(0, (int)rc.x - a.x0), rx1 = min(kBW - 1, (int)rc.z - a.x0);
                const int ry0 = max(0, (int)rc.y - a.y0), ry1 = min(kBH - 1, (int)rc.w - a.y0);
                if (rx0 <= rx1 && ry0 <= ry1) hk[k] = (rect_bits(rx0, rx1, ry0, ry1) & live) != 0u;
            }
        }
        uint32_t gcur[kAhead];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) gcur[k] = gk[k];
        if (base + 32 * kAhead < s1) fetch(base + 32 * kAhead, gk);  // next step's indices, in flight
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            const uint32_t hits = __ballot_sync(0xffffffffu, hk[k]);
            if (!hits) continue;
            StageBuf &sb = sg.b[cur];
            if (hk[k]) {
                const int q = __popc(hits & lt);
                const uint32_t g = gcur[k];
                cp_async16(&sb.xy[q], a.xy_depth + a.gbase + g);
                cp_async16(&sb.co[q], a.conic_op + a.gbase + g);
                cp_async16(&sb.cc[q], a.rgb + g);
                cp_async16(&sb.nr[q], a.normal + g);
                sb.pos[q] = base + 32u * k + (uint32_t)lane;
            }
            cp_async_commit();
            if (pend) {
                cp_async_wait_all_but_one();
                __syncwarp();
                composite(sg.b[cur ^ 1], pend);
                __syncwarp();  // buffer cur ^ 1 is free again
            }
            pend = __popc(hits);
            cur ^= 1;
        }
    }
    if (pend) {
        cp_async_wait_all();
        __syncwarp();
        composite(sg.b[cur ^ 1], pend);
        __syncwarp();
    }
    state = st;
    pair_count += pairs;
    return reached;
}

// C = C_a + T_a C_b, T = T_a T_b: segment b composited after state a.
__device__ __forceinline__ PixState fold(const PixState &a, const PixState &b) {
    PixState o;
    o.c0 = fmaf(a.T, b.c0, a.c0);
    o.c1 = fmaf(a.T, b.c1, a.c1);
    o.c2 = fmaf(a.T, b.c2, a.c2);
    o.n0 = fmaf(a.T, b.n0, a.n0);
    o.n1 = fmaf(a.T, b.n1, a.n1);
    o.n2 = fmaf(a.T, b.n2, a.n2);
    o.D = fmaf(a.T, b.D, a.D);
    o.T = a.T * b.T;
    o.last = b.last ? b.last : a.last;
    o.done = false;
    return o;
}

__device__ __forceinline__ uint32_t atomic_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Publication of a state by the whole warp: every lane's stores, a fence by
// every lane, then one arrival on `counter` (lane 0, acquire-release).
// Returns the counter's previous value (uniform); a caller that sees 1
// arrived second and may read the other party's state.
__device__ __forceinline__ uint32_t arrive(uint32_t *counter, int lane) {
    __threadfence();
    __syncwarp();
    uint32_t old = 0;
    if (lane == 0) old = atomic_add_acq_rel(counter, 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    __syncwarp();
    __threadfence();
    return old;
}

// Deferred re-walks.  Where the stop of some pixels of a block falls
// inside a segment, the chained schedule does not re-walk the segment on
// the chain (whose links are then serial re-walks through most of a long
// list of faint splats): the pixels are marked done and deferred, the
// chain carries on, and the re-walk goes to its CTA's task queue, which the
// CTA's warps drain once the items run out.  A task re-walks the segment with the stop rule from the
// predecessor's inclusive state (kept in its slot) and writes its pixels'
// outputs: the same arithmetic as a re-walk on the chain.  Only a pixel
// whose stop falls inside for certain is deferred (T_in T_s below t_min by
// a 0.1 % margin, far above the rounding of the products of one segment),
// so the re-walk stops inside the segment.  The queue lives in shared
// memory (no global polling); its lock is held for a few instructions and
// every wait on it is bounded.
constexpr float kDeferMargin = 0.999f;
constexpr int kCtaTasks = 64;
struct CtaQueue {
    uint32_t lock, head, tail, busy;  // busy: warps of the CTA inside an item
    uint4 task[kCtaTasks];            // work entry, segment, block, pixel mask
};

__device__ __forceinline__ bool cq_lock(CtaQueue *q, uint32_t limit) {
    uint32_t s = 0;
    while (atomicCAS(&q->lock, 0u, 1u) != 0u) {
        if (++s > limit) return false;
        __nanosleep(32);
    }
    __threadfence_block();
    return true;
}
__device__ __forceinline__ void cq_unlock(CtaQueue *q) {
    __threadfence_block();
    atomicExch(&q->lock, 0u);
}
// lane 0 only; false when the queue is full (or the lock was not had)
__device__ __forceinline__ bool cq_push(CtaQueue *q, uint4 t, uint32_t limit) {
    if (!cq_lock(q, limit)) return false;
    volatile CtaQueue *v = q;
    const bool ok = v->tail - v->head < (uint32_t)kCtaTasks;
    if (ok) {
        v->task[v->tail % kCtaTasks].x = t.x;
        v->task[v->tail % kCtaTasks].y = t.y;
        v->task[v->tail % kCtaTasks].z = t.z;
        v->task[v->tail % kCtaTasks].w = t.w;
        v->tail = v->tail + 1u;
    }
    cq_unlock(q);
    return ok;
}
// lane 0 only: 1 a task taken, 0 the queue empty, -1 the lock was not had.
// An empty queue is seen without the lock.
__device__ __forceinline__ int cq_pop(CtaQueue *q, uint4 &t, uint32_t limit) {
    if (((volatile CtaQueue *)q)->head == ((volatile CtaQueue *)q)->tail) return 0;
    if (!cq_lock(q, limit)) return -1;
    volatile CtaQueue *v = q;
    const bool ok = v->head < v->tail;
    if (ok) {
        t = make_uint4(v->task[v->head % kCtaTasks].x, v->task[v->head % kCtaTasks].y,
                       v->task[v->head % kCtaTasks].z, v->task[v->head % kCtaTasks].w);
        v->head = v->head + 1u;
    }
    cq_unlock(q);
    return ok ? 1 : 0;
}

// Runs the CTA's queued re-walks (take: 1 one was run, 0 none queued, -1
// the queue's lock was not had) until none is queued and no warp of the
// CTA is inside an item (only those queue re-walks).  Every wait is
// bounded: after `limit` rounds it records P2E_ERR_TIMEOUT and returns.
template <typename Take>
__device__ __forceinline__ void drain_queue(CtaQueue *q, uint32_t limit, int32_t *status, Take &&take) {
    const int lane = threadIdx.x & 31;
    uint32_t spins = 0;
    for (;;) {
        const int got = take();
        if (got > 0) {
            spins = 0;
            continue;
        }
        if (got < 0) break;
        uint32_t idle = 0;
        if (lane == 0) idle = atomicAdd(&q->busy, 0u) == 0u ? 1u : 0u;
        if (__shfl_sync(0xffffffffu, idle, 0)) {
            if (take() > 0) continue;  // queued before the last item ended
            break;
        }
        if (++spins > limit) {
            if (lane == 0) atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
            break;
        }
        __nanosleep(spins < 5 ? 32u << spins : 1024u);
    }
}

// The inclusive state after a segment, from the state before it (cur) and
// the segment's aggregate (ag: composited from T = 1 without stopping):
// fold C = C_in + T_in C_s, T = T_in T_s, unless the stop falls inside the
// segment (T_in T_s < t_min; T is non-increasing): then the segment is
// re-walked from the true state with the stop rule, here or (q != NULL,
// when the CTA's queue has room) by a deferred task for work entry w,
// segment seg, block blk.  An aggregate with T = 0 marks a pixel whose stop is
// already known to fall inside.
__device__ __forceinline__ void combine(PixState &cur, const PixState &ag, uint32_t s0, uint32_t s1,
                                        const SegArgs &a, uint32_t &pairs, CtaQueue *q, uint32_t limit,
                                        uint32_t w, uint32_t seg, int blk) {
    const int lane = threadIdx.x & 31;
    bool rw = false, df = false;
    if (!cur.done) {
        const float tt = cur.T * ag.T;
        if (tt >= a.tmin) cur = fold(cur, ag);
        else if (q && tt < a.tmin * kDeferMargin) df = true;
        else rw = true;
    }
    const uint32_t dm = __ballot_sync(0xffffffffu, df);
    if (dm) {
        uint32_t ok = 0;
        if (lane == 0) ok = cq_push(q, make_uint4(w, seg, (uint32_t)blk, dm), limit) ? 1u : 0u;
        if (__shfl_sync(0xffffffffu, ok, 0)) {
            if (df) {
                cur.done = true;
                cur.deferred = true;
            }
        } else {
            rw = rw || df;  // no room in the queue: re-walk here
        }
    }
    if (__any_sync(0xffffffffu, rw)) {
        PixState x = cur;
        x.done = !rw;  // only the re-walking pixels take part
        composite_segment(true, s0, s1, a, x, pairs, nullptr);
        if (rw) cur = x;
    }
}

template <int BT>
__global__ void __launch_bounds__(kWarps * 32, 3) blend_kernel(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ work,
    uint32_t *__restrict__ work_counter, uint32_t *__restrict__ table, char *__restrict__ store,
    const float4 *__restrict__ xy_depth, const float4 *__restrict__ conic_op, const ushort4 *__restrict__ rect,
    const float4 *__restrict__ rgb, const float4 *__restrict__ normal, float *__restrict__ out_rgb,
    float *__restrict__ out_nrm, float *__restrict__ out_depth, float *__restrict__ out_alpha,
    uint32_t *__restrict__ out_last, unsigned long long *__restrict__ pair_count, int32_t *__restrict__ status,
    uint32_t spin_limit, __grid_constant__ const Views P) {
    constexpr int NBX = BT / kBW, NB = blocks_of(BT);
    constexpr int SW = kStateFloats * 32;  // state floats of one (slot, block)
    const int lane = threadIdx.x & 31;
    const int lx = lane % kBW, ly = lane / kBW;
    const float lxf = (float)lx, lyf = (float)ly;
    const float tmin = P.t_min;
    const uint32_t n_work = work[0];
    constexpr uint32_t S = seg_len(BT);
    // chained: one item per (tile, segment, block) of the tiles with state
    // slots, one per (tile, block) of the others; otherwise one per
    // (tile, block), whose warp runs the same segments in turn
    const bool chained = table && table[0] == 1u;
    const uint32_t *item_base = chained ? table + 1 : nullptr;
    const uint32_t *slot_base = chained ? table + 2 + n_work : nullptr;
    const uint32_t total = chained ? item_base[n_work] : n_work * (uint32_t)NB;
    const uint32_t max_slots = chained ? table[2 * n_work + 4] : 0u;
    float *states = (float *)store;
    uint32_t *lastw = chained ? table + tbl_words(n_work) : nullptr;
    uint32_t *counters = chained ? lastw + (size_t)max_slots * NB * 32 : nullptr;
    uint32_t *ready = chained ? counters + (size_t)max_slots * NB : nullptr;
    __shared__ CtaQueue s_q;  // this CTA's deferred re-walks
    if (threadIdx.x == 0) s_q.lock = s_q.head = s_q.tail = s_q.busy = 0u;
    __syncthreads();
    CtaQueue *const cq = &s_q;
    uint32_t pairs = 0;  // (pixel, splat) pairs this lane evaluated

    // what one (work entry, pixel block) needs
    struct Block {
        const View *V;
        int px, py;
        bool inside;
        uint2 r;
        uint32_t nseg;
        SegArgs sa;
    };
    auto block_of = [&](uint32_t w, int blk, Block &b) {
        const int64_t tile = work[2 + w];
        const int vi = view_of_tile(P, tile);
        const View &V = P.v[vi];
        const int64_t ltile = tile - V.tile_base;
        const int ty = (int)(ltile / V.tiles_x), tx = (int)(ltile - (int64_t)ty * V.tiles_x);
        const int x0 = tx * BT + (blk % NBX) * kBW, y0 = ty * BT + (blk / NBX) * kBH;
        b.V = &V;
        b.px = x0 + lx;
        b.py = y0 + ly;
        b.inside = b.px < V.W && b.py < V.H;
        b.r = ranges[tile];
        b.nseg = (b.r.y - b.r.x + S - 1) / S;
        SegArgs &sa = b.sa;
        sa.vals = vals;
        sa.xy_depth = xy_depth;
        sa.conic_op = conic_op;
        sa.rect = rect;
        sa.rgb = rgb;
        sa.normal = normal;
        sa.gbase = (int64_t)vi * P.n;
        sa.x0 = x0;
        sa.y0 = y0;
        sa.lxf = lxf;
        sa.lyf = lyf;
        sa.n = (uint32_t)P.n;
        sa.pw_min = -0.5f * P.sigma_mult * P.sigma_mult;
        sa.amax = P.alpha_max;
        sa.afloor = P.alpha_floor;
        sa.tmin = P.t_min;
    };
    auto write_pixel = [&](const Block &b, const PixState &cur) {
        const View &V = *b.V;
        const int64_t HW = (int64_t)V.H * V.W;
        const int64_t p = (int64_t)b.py * V.W + b.px;
        if (out_rgb) {
            float *o = out_rgb + 3 * V.pix_base + p;
            o[0] = fmaf(cur.T, P.bg[0], cur.c0);
            o[HW] = fmaf(cur.T, P.bg[1], cur.c1);
            o[2 * HW] = fmaf(cur.T, P.bg[2], cur.c2);
        }
        if (out_nrm) {
            float *o = out_nrm + 3 * V.pix_base + p;
            o[0] = cur.n0;
            o[HW] = cur.n1;
            o[2 * HW] = cur.n2;
        }
        if (out_depth) out_depth[V.pix_base + p] = cur.D;
        if (out_alpha) out_alpha[V.pix_base + p] = 1.f - cur.T;
        if (out_last) out_last[V.pix_base + p] = cur.last;
    };

    // Takes one re-walk from the CTA's queue and runs it: 1 done, 0 none
    // queued, -1 the queue's lock was not had (status recorded).
    auto take_task = [&]() -> int {
        uint4 tk = make_uint4(0u, 0u, 0u, 0u);
        int got = 0;
        if (lane == 0) got = cq_pop(cq, tk, spin_limit);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got <= 0) {
            if (got < 0 && lane == 0) atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
            return got;
        }
        const uint32_t w = __shfl_sync(0xffffffffu, tk.x, 0), seg = __shfl_sync(0xffffffffu, tk.y, 0);
        const int blk = (int)__shfl_sync(0xffffffffu, tk.z, 0);
        const uint32_t mask = __shfl_sync(0xffffffffu, tk.w, 0);
        Block b;
        block_of(w, blk, b);
        const size_t pi = ((size_t)__ldg(slot_base + w) + seg - 1) * NB + blk;
        PixState x;
        load_state(states + pi * SW, lastw + pi * 32, lane, x);
        const bool mine = ((mask >> lane) & 1u) != 0u;
        x.done = !mine;
        x.deferred = false;
        composite_segment(true, b.r.x + seg * S, min(b.r.y, b.r.x + (seg + 1) * S), b.sa, x, pairs, nullptr);
        if (mine && b.inside) write_pixel(b, x);
        return 1;
    };

    // one item: a (tile, segment, block), or a (tile, block) run alone
    auto do_item = [&](uint32_t item) {
        uint32_t w, local;
        if (chained) {  // last work entry whose first item is <= item
            uint32_t lo = 0, hi = n_work;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(item_base + mid) <= item) lo = mid;
                else hi = mid;
            }
            w = lo;
            local = item - __ldg(item_base + w);
        } else {
            w = item / (uint32_t)NB;
            local = item % (uint32_t)NB;
        }
        // the tile's first state slot; kNoSlot: its blocks run alone
        const uint32_t sbase = chained ? __ldg(slot_base + w) : kNoSlot;
        const bool tch = sbase != kNoSlot;
        const uint32_t seg = tch ? local / (uint32_t)NB : 0u;
        const int blk = (int)(tch ? local % (uint32_t)NB : local);
        Block b;
        block_of(w, blk, b);
        const SegArgs &sa = b.sa;
        const uint32_t nseg = b.nseg;
        const bool inside = b.inside;
        auto seg_lo = [&](uint32_t si) { return b.r.x + si * S; };
        auto seg_hi = [&](uint32_t si) { return min(b.r.y, b.r.x + (si + 1) * S); };
        // (state slot, block) index of the chain's bookkeeping (tiles of
        // two or more segments only)
        auto sidx = [&](uint32_t si) -> size_t { return ((size_t)sbase + si) * NB + blk; };
        CtaQueue *q = chained ? cq : nullptr;

        PixState cur;  // the inclusive state through segment m
        uint32_t m = seg;
        fresh_state(cur, inside);
        if (!tch) {
            // the chain in one warp: segment 0 exact, every later one
            // speculated from T = 1 and combined, as the chained schedule does
            composite_segment(true, seg_lo(0), seg_hi(0), sa, cur, pairs, nullptr);
            for (m = 1; m < nseg; ++m) {
                PixState ag;
                fresh_state(ag, inside);
                ag.done = ag.done || cur.done;
                composite_segment(false, seg_lo(m), seg_hi(m), sa, ag, pairs, nullptr);
                combine(cur, ag, seg_lo(m), seg_hi(m), sa, pairs, nullptr, spin_limit, w, m, blk);
            }
            m = nseg - 1;
        } else if (seg == 0) {
            composite_segment(true, seg_lo(0), seg_hi(0), sa, cur, pairs, nullptr);
        } else {
            // speculate: the segment from T = 1 without stopping (its aggregate)
            const size_t pi = sidx(seg - 1);
            PixState pr;
            fresh_state(pr, inside);
            bool known = __all_sync(0xffffffffu, ld_acquire_u32(ready + pi) != 0u);
            if (known) load_state(states + pi * SW, lastw + pi * 32, lane, pr);
            // pixels the predecessor shows done, or whose stop it shows to lie
            // in the part already walked (with the deferral margin), drop out
            // (their result no longer depends on this aggregate; the latter
            // publish T = 0)
            bool rewalk = false;
            PixState ag;
            fresh_state(ag, inside);
            if (known) ag.done = ag.done || pr.done;
            const uint32_t s0 = seg_lo(seg), s1 = seg_hi(seg);
            const uint32_t reached = composite_segment(false, s0, s1, sa, ag, pairs, known ? nullptr : ready + pi);
            if (!known && reached < s1) {
                (void)ld_acquire_u32(ready + pi);
                load_state(states + pi * SW, lastw + pi * 32, lane, pr);
                rewalk = !pr.done && !ag.done && pr.T * ag.T < tmin * kDeferMargin;
                ag.done = ag.done || pr.done || rewalk;
                composite_segment(false, reached, s1, sa, ag, pairs, nullptr);
            }
            if (rewalk) ag.T = 0.f;
            const size_t si = sidx(seg);
            store_state(states + si * SW, lastw + si * 32, lane, ag);
            // the second to arrive (this aggregate or the predecessor's
            // inclusive state) continues the chain
            if (arrive(counters + si, lane) == 0u) return;
            load_state(states + pi * SW, lastw + pi * 32, lane, cur);  // the predecessor's inclusive state
            combine(cur, ag, s0, s1, sa, pairs, q, spin_limit, w, seg, blk);
        }
        // publish the chain forward: while the successor's aggregate is
        // already stored, combine it too
        while (tch && m + 1 < nseg) {
            const size_t mi = sidx(m);
            store_state(states + mi * SW, lastw + mi * 32, lane, cur);
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_u32(ready + mi, kIncl);  // polled by the successor
            const size_t ni = sidx(m + 1);
            if (arrive(counters + ni, lane) == 0u) break;  // the successor continues
            PixState ag;
            load_state(states + ni * SW, lastw + ni * 32, lane, ag);
            ++m;
            combine(cur, ag, seg_lo(m), seg_hi(m), sa, pairs, q, spin_limit, w, m, blk);
        }
        if (m + 1 == nseg && inside && !cur.deferred) write_pixel(b, cur);  // the last state is the pixel
    };

    // (the CTA's queued re-walks wait until its warps run out of items: a
    // check of the queue before each item measured 0.15 ms slower per frame)
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) {
            if (chained) atomicAdd(&cq->busy, 1u);
            item = atomicAdd(work_counter, 1u);
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item < total) do_item(item);
        __syncwarp();
        if (chained && lane == 0) atomicSub(&cq->busy, 1u);  // after any re-walk it queued
        if (item >= total) break;
    }

    if (chained) drain_queue(cq, spin_limit, status, take_task);
    if (pair_count) {  // one atomic per warp (every lane reaches here)
        unsigned long long t = pairs;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t) atomicAdd(pair_count, t);
    }
}

// Timeout self-test of the re-walk queue's waits, one warp: which 0 drains
// a queue whose CTA never leaves its item (busy stays 1), which 1 pops from
// a non-empty queue whose lock is never released.  Both give up after
// `spin_limit` rounds and record P2E_ERR_TIMEOUT; no task is ever run.
__global__ void selftest_queue_kernel(int which, uint32_t spin_limit, int32_t *status) {
    __shared__ CtaQueue q;
    if (threadIdx.x == 0) {
        q.head = 0u;
        q.tail = which == 1 ? 1u : 0u;
        q.lock = which == 1 ? 1u : 0u;
        q.busy = which == 0 ? 1u : 0u;
        q.task[0] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncwarp();
    drain_queue(&q, spin_limit, status, [&]() -> int {
        int got = 0;
        uint4 t;
        if ((threadIdx.x & 31) == 0) {
            got = cq_pop(&q, t, spin_limit);
            if (got < 0) atomicExch(status, (int32_t)P2E_ERR_TIMEOUT);
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        return got > 0 ? 0 : got;  // a popped task is not run
    });
}

cudaError_t launch_selftest_queue(int which, int32_t *status, uint32_t spin_limit, cudaStream_t st) {
    selftest_queue_kernel<<<1, 32, 0, st>>>(which, spin_limit, status);
    return cudaGetLastError();
}

// Background for every pixel of a tile with an empty list.
__global__ void __launch_bounds__(256) fill_empty_kernel(const uint2 *__restrict__ ranges,
                                                         int64_t total_pix, float *__restrict__ out_rgb,
                                                         float *__restrict__ out_nrm,
                                                         float *__restrict__ out_depth,
                                                         float *__restrict__ out_alpha,
                                                         uint32_t *__restrict__ out_last,
                                                         __grid_constant__ const Views P) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total_pix;
         q += (int64_t)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < P.n_views && P.v[v + 1].pix_base <= q) ++v;
        const View &V = P.v[v];
        const int64_t p = q - V.pix_base;
        const int y = (int)(p / V.W), x = (int)(p - (int64_t)y * V.W);
        const int64_t tile = V.tile_base + (int64_t)(y / P.tile) * V.tiles_x + x / P.tile;
        const uint2 r = ranges[tile];
        if (r.y > r.x) continue;
        const int64_t HW = (int64_t)V.H * V.W;
        if (out_rgb) {
            float *o = out_rgb + 3 * V.pix_base + p;
            o[0] = P.bg[0];
            o[HW] = P.bg[1];
            o[2 * HW] = P.bg[2];
        }
        if (out_nrm) {
            float *o = out_nrm + 3 * V.pix_base + p;
            o[0] = 0.f;
            o[HW] = 0.f;
            o[2 * HW] = 0.f;
        }
        if (out_depth) out_depth[q] = 0.f;
        if (out_alpha) out_alpha[q] = 0.f;
        if (out_last) out_last[q] = 0u;
    }
}

int device_sms();

template <int BT>
static cudaError_t launch_blend(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                                const Views &P, float *rgb, float *nrm, float *depth, float *alpha,
                                uint32_t *last, cudaStream_t st) {
    static int per_sm[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    const int slot = (dev >= 0 && dev < 64) ? dev : 0;
    if (!per_sm[slot]) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, blend_kernel<BT>, kWarps * 32, 0) != cudaSuccess)
            nb = 0;
        per_sm[slot] = nb > 0 ? nb : 1;
    }
    cudaError_t e = cudaMemsetAsync(bins->tile_work + 1, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int64_t total_pix = P.v[P.n_views - 1].pix_base +
                              (int64_t)P.v[P.n_views - 1].W * P.v[P.n_views - 1].H;
    const int sms = device_sms();
    fill_empty_kernel<<<sms * 8, 256, 0, st>>>((const uint2 *)bins->ranges, total_pix, rgb, nrm, depth,
                                               alpha, last, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // segment chaining: the item table, the state words 'last | done',
    // counters and flags in vals[1 - result], the state floats in
    // keys[1 - result] (decided on the device by the item table)
    const int other = 1 - bins->result;
    // (its re-walk queue's bounded waits report through status_dev)
    const bool allow = bins->capacity > 0 && bins->keys[other] && bins->vals[other] && bins->status_dev;
    uint32_t *table = allow ? bins->vals[other] : nullptr;
    char *store = allow ? (char *)bins->keys[other] : nullptr;
    if (allow) {
        render_items_kernel<<<1, 1024, 0, st>>>((const uint2 *)bins->ranges, bins->tile_work, bins->n_keys_dev,
                                                bins->capacity, P.schedule == P2E_SCHEDULE_AUTO ? 1 : 0, BT, table);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t grid = (int64_t)sms * per_sm[slot];
    const p2e_kernel_probe *pr = kernel_probe(P2E_PROBE_BLEND);
    probe_start(pr, st);
    blend_kernel<BT><<<(unsigned)grid, kWarps * 32, 0, st>>>(
        (const uint2 *)bins->ranges, bins->vals[bins->result], bins->tile_work, bins->tile_work + 1, table, store,
        (const float4 *)proj->xy_depth, (const float4 *)proj->conic_op, (const ushort4 *)proj->rect,
        (const float4 *)g->rgb, (const float4 *)g->normal, rgb, nrm, depth, alpha, last,
        pr ? (unsigned long long *)pr->count_dev : nullptr, bins->status_dev, kSpinLimit, P);
    probe_stop(pr, st);
    return cudaGetLastError();
}

cudaError_t launch_render(const p2e_gaussians *g, const p2e_projected *proj, const p2e_bins *bins,
                          const Views &P, float *rgb, float *nrm, float *depth, float *alpha,
                          uint32_t *last, cudaStream_t st) {
    if (P.total_tiles == 0) return cudaSuccess;
    switch (P.tile) {
        case 8: return launch_blend<8>(g, proj, bins, P, rgb, nrm, depth, alpha, last, st);
        case 16: return launch_blend<16>(g, proj, bins, P, rgb, nrm, depth, alpha, last, st);
        case 32: return launch_blend<32>(g, proj, bins, P, rgb, nrm, depth, alpha, last, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace p2e
